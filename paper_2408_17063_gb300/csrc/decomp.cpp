// Client-side Decomp (Alg. 6) on decrypted answer slots, host C++.
//
// Per record group: the power sums w_1..w_s' (row 0) give, by Newton's
// identity (Lem. 1, Alg. 1 step 1), the coefficients of
// f(X) = prod_{nodes}(X - node) * X^{s' - #nodes}; the factors of X are
// stripped and the roots among the nodes 1..G_sz are found (Alg. 1 step 2):
// by evaluating the stripped polynomial at every node where that is the
// cheaper, else by Cantor-Zassenhaus root finding as the paper suggests
// (Sec. 3.1), whose cost grows with log t instead of t; the root set is
// unique, so both give the same nodes.  The values solve
// sum_l node_l^{j} x_l = e_j, j = 1..l (Alg. 4); this system is node-scaled
// transposed Vandermonde, solved in O(l^2) through the Lagrange basis of the
// nodes, and rows l+1..s' must agree.  Record groups are independent and
// decoded in parallel on the host cores.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "pdq_internal.h"
#include "pdq_ops.h"

namespace pdq {
namespace {

struct Zt {
    u64 t;
    u64 mul(u64 a, u64 b) const { return a * b % t; }
    u64 add(u64 a, u64 b) const { u64 s = a + b; return s >= t ? s - t : s; }
    u64 sub(u64 a, u64 b) const { return a >= b ? a - b : a + t - b; }
    u64 pow(u64 a, u64 e) const {
        u64 r = 1;
        a %= t;
        while (e) {
            if (e & 1) r = mul(r, a);
            a = mul(a, a);
            e >>= 1;
        }
        return r;
    }
    u64 inv(u64 a) const { return pow(a, t - 2); }
};

unsigned host_threads() {
    return std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
}

// roots of g (coefficients low to high) among 1..hi, evaluated on nt threads
std::vector<u64> roots_among(const std::vector<u64>& g, u64 hi, const Zt& z, unsigned nt) {
    if (nt <= 1) {
        std::vector<u64> r;
        for (u64 x = 1; x <= hi; ++x) {
            u64 acc = 0;
            for (size_t i = g.size(); i-- > 0;) acc = (acc * x + g[i]) % z.t;
            if (acc == 0) r.push_back(x);
        }
        return r;
    }
    std::vector<std::vector<u64>> part(nt);
    std::vector<std::thread> th;
    const u64 chunk = (hi + nt - 1) / nt;
    for (unsigned w = 0; w < nt; ++w) {
        th.emplace_back([&, w] {
            const u64 lo = 1 + w * chunk, up = std::min(hi, (w + 1) * chunk);
            for (u64 x = lo; x <= up; ++x) {
                u64 acc = 0;
                for (size_t i = g.size(); i-- > 0;) acc = (acc * x + g[i]) % z.t;
                if (acc == 0) part[w].push_back(x);
            }
        });
    }
    for (auto& t : th) t.join();
    std::vector<u64> r;
    for (auto& p : part) r.insert(r.end(), p.begin(), p.end());
    return r;
}

// Polynomials over Z_t, coefficients low to high, trimmed (no zero leading
// coefficient; the zero polynomial is empty).
using Poly = std::vector<u64>;

void trim(Poly& a) {
    while (!a.empty() && a.back() == 0) a.pop_back();
}

// a mod m (m trimmed, nonzero)
void poly_rem(Poly& a, const Poly& m, const Zt& z) {
    trim(a);
    const size_t dm = m.size() - 1;
    const u64 il = z.inv(m.back());
    while (a.size() > dm) {
        const u64 c = z.mul(a.back(), il);
        const size_t sh = a.size() - 1 - dm;
        for (size_t i = 0; i < dm; ++i) a[sh + i] = z.sub(a[sh + i], z.mul(c, m[i]));
        a.pop_back();                    // its coefficient is now zero
    }
    trim(a);
}

// a / m for m dividing a
Poly poly_div_exact(Poly a, const Poly& m, const Zt& z) {
    trim(a);
    const size_t dm = m.size() - 1;
    if (a.size() < m.size()) return {};
    Poly q(a.size() - dm, 0);
    const u64 il = z.inv(m.back());
    while (a.size() > dm) {
        const u64 c = z.mul(a.back(), il);
        const size_t sh = a.size() - 1 - dm;
        q[sh] = c;
        for (size_t i = 0; i < dm; ++i) a[sh + i] = z.sub(a[sh + i], z.mul(c, m[i]));
        a.pop_back();
    }
    trim(q);
    return q;
}

Poly mul_mod(const Poly& a, const Poly& b, const Poly& m, const Zt& z) {
    if (a.empty() || b.empty()) return {};
    Poly r(a.size() + b.size() - 1, 0);
    for (size_t i = 0; i < a.size(); ++i) {
        if (a[i] == 0) continue;
        for (size_t j = 0; j < b.size(); ++j) r[i + j] = (r[i + j] + a[i] * b[j]) % z.t;
    }
    poly_rem(r, m, z);
    return r;
}

// (X + a)^e mod m
Poly pow_linear(u64 a, u64 e, const Poly& m, const Zt& z) {
    Poly base{a % z.t, 1}, r{1};
    poly_rem(base, m, z);
    poly_rem(r, m, z);
    while (e) {
        if (e & 1) r = mul_mod(r, base, m, z);
        e >>= 1;
        if (e) base = mul_mod(base, base, m, z);
    }
    return r;
}

// monic gcd
Poly poly_gcd(Poly a, Poly b, const Zt& z) {
    trim(a);
    trim(b);
    while (!b.empty()) {
        poly_rem(a, b, z);
        std::swap(a, b);
    }
    if (!a.empty()) {
        const u64 il = z.inv(a.back());
        for (u64& c : a) c = z.mul(c, il);
    }
    return a;
}

// Roots of f, a product of distinct linear factors over Z_t with f(0) != 0,
// by equal-degree splitting (Cantor and Zassenhaus, 1981): for a = 0, 1, ...
// gcd(g, (X + a)^((t-1)/2) - 1) keeps the roots r of g with r + a a nonzero
// square, which splits g as soon as g has roots on both sides.
int split_roots(const Poly& f, const Zt& z, std::vector<u64>& out) {
    std::vector<Poly> work{f};
    u64 a = 0, tries = 0;
    while (!work.empty()) {
        Poly g = std::move(work.back());
        work.pop_back();
        trim(g);
        if (g.size() <= 1) continue;
        if (g.size() == 2) {
            out.push_back(z.mul(z.sub(0, g[0]), z.inv(g[1])));
            continue;
        }
        const size_t d = g.size() - 1;
        for (;;) {
            if (++tries > 4 * z.t) return fail(PDQ_E_DECODE, "decomp: root splitting did not converge");
            Poly h = pow_linear(a, (z.t - 1) / 2, g, z);
            a = (a + 1) % z.t;
            if (h.empty()) h.push_back(0);
            h[0] = z.sub(h[0], 1);
            Poly c = poly_gcd(g, h, z);
            if (c.size() > 1 && c.size() - 1 < d) {
                work.push_back(poly_div_exact(g, c, z));
                work.push_back(std::move(c));
                break;
            }
        }
    }
    std::sort(out.begin(), out.end());
    return PDQ_OK;
}

// The roots of g (g(0) != 0) among the nodes 1..hi: every node evaluated
// (Horner, on all host cores) when that is the cheaper, else the distinct
// roots of g in Z_t as gcd(g, X^t - X), split into linear factors (the
// Cantor-Zassenhaus root finding of Sec. 3.1), at a cost that grows with
// log t instead of t.  Both give the same set.
// (nt: threads for the node evaluation.  The two costs in the same unit:
// one node evaluation per Horner step, and for the gcd route about d^2 log t
// products per polynomial power, log d + 2 powers, each product about an
// eighth of a Horner step's cost, as measured on the host.)
int find_roots(const Poly& g, u64 hi, const Zt& z, unsigned nt, std::vector<u64>& roots) {
    const double d = (double)(g.size() - 1);
    const double by_nodes = (double)hi * (d + 1) / nt;
    const double by_gcd = d * d * std::log2((double)z.t) * (std::log2(d) + 2) / 8;
    if (by_nodes <= by_gcd) {
        roots = roots_among(g, hi, z, nt);
        return PDQ_OK;
    }
    Poly xt = pow_linear(0, z.t, g, z);          // X^t mod g
    if (xt.size() < 2) xt.resize(2, 0);
    xt[1] = z.sub(xt[1], 1);
    const Poly f = poly_gcd(g, xt, z);           // the distinct roots of g in Z_t
    roots.clear();
    if (f.size() != g.size()) return PDQ_OK;     // fewer roots than the degree: the caller refuses
    PDQ_TRY(split_roots(f, z, roots));
    std::vector<u64> in;
    for (u64 r : roots)
        if (r >= 1 && r <= hi) in.push_back(r);
    roots.swap(in);
    return PDQ_OK;
}

int decode_group(const u32* w, const u32* e, u32 sp, u64 G_sz, const Zt& z, unsigned nt,
                 std::vector<u64>& nodes, std::vector<u64>& vals) {
    // Newton's identity
    std::vector<u64> a(sp + 1, 0);
    a[0] = 1;
    for (u32 k = 1; k <= sp; ++k) {
        u64 acc = 0;
        for (u32 i = 1; i <= k; ++i) {
            const u64 term = z.mul(a[k - i], w[i - 1] % z.t);
            acc = (i % 2 == 1) ? z.add(acc, term) : z.sub(acc, term);
        }
        a[k] = z.mul(acc, z.inv(k % z.t));
    }
    // f(X) = sum_k (-1)^k a_k X^{s'-k}, lowest degree first
    std::vector<u64> f(sp + 1);
    for (u32 k = 0; k <= sp; ++k) f[sp - k] = (k % 2 == 0) ? a[k] : z.sub(0, a[k]);
    u32 zlow = 0;
    while (zlow < sp && f[zlow] == 0) ++zlow;
    std::vector<u64> g(f.begin() + zlow, f.end());
    const u32 deg = (u32)g.size() - 1;
    nodes.clear();
    vals.clear();
    if (deg == 0) {
        for (u32 j = 0; j < sp; ++j)
            if (e[j] % z.t) return fail(PDQ_E_DECODE, "decomp: values without indices");
        return PDQ_OK;
    }
    PDQ_TRY(find_roots(g, G_sz, z, nt, nodes));
    if (nodes.size() != deg) return fail(PDQ_E_DECODE, "decomp: root count differs from the degree");
    const u32 l = deg;
    // M(X) = prod (X - node)
    std::vector<u64> M(1, 1);
    for (u64 r : nodes) {
        std::vector<u64> nm(M.size() + 1, 0);
        for (size_t i = 0; i < M.size(); ++i) {
            nm[i + 1] = z.add(nm[i + 1], M[i]);
            nm[i] = z.sub(nm[i], z.mul(M[i], r));
        }
        M.swap(nm);
    }
    vals.resize(l);
    std::vector<u64> num(l);
    for (u32 k = 0; k < l; ++k) {
        // num = M / (X - node_k) by synthetic division (degree l-1)
        const u64 r = nodes[k];
        u64 carry = 0;
        for (int i = (int)l; i >= 1; --i) {
            carry = z.add(M[i], z.mul(carry, r));
            num[i - 1] = carry;
        }
        u64 den = 0;
        for (int i = (int)l - 1; i >= 0; --i) den = z.add(z.mul(den, r), num[i]);
        u64 y = 0;
        for (u32 j = 0; j < l; ++j) y = z.add(y, z.mul(num[j], e[j] % z.t));
        // y_k = node_k x_k
        vals[k] = z.mul(y, z.inv(z.mul(den, r)));
    }
    for (u32 j = l; j < sp; ++j) {
        u64 s = 0;
        for (u32 k = 0; k < l; ++k) s = z.add(s, z.mul(z.pow(nodes[k], j + 1), vals[k]));
        if (s != e[j] % z.t) return fail(PDQ_E_DECODE, "decomp: inconsistent compressed values");
    }
    return PDQ_OK;
}

// Decomp over every record group of the plan's output ciphertexts; only the
// ring and t of c are read (c may be a host ring without device tables).
// The groups are independent: with several, min(G, threads) workers each
// decode every nw-th group, a group's node evaluation (where chosen) on the
// threads left over per worker; with one, that evaluation runs on every
// thread.  An error is reported as the first failing group (in group order)
// raised it.
int decomp_run(const Ctx& c, const pdq_plan* plan, const uint32_t* slots, uint64_t* idx_out,
               uint32_t* val_out, uint64_t cap, uint64_t* count) {
    if (!plan || !slots || !count) return fail(PDQ_E_PARAM, "decomp: null argument");
    if (!valid_plan(c, plan)) return fail(PDQ_E_PARAM, "decomp: invalid plan");
    const Zt z{c.t};
    const u32 sp = plan->s_prime, G = plan->G;
    std::vector<std::vector<u64>> nodes(G), vals(G);
    std::vector<int> rc(G, PDQ_OK);
    std::vector<std::string> err(G);
    auto one = [&](u32 gamma, unsigned nt) {
        const u32 cidx = G > 1 ? gamma / plan->per_out : 0;
        const u32 o = G > 1 ? gamma % plan->per_out : 0;
        const u32* s = slots + (u64)cidx * c.N;
        rc[gamma] = decode_group(s + (u64)o * sp, s + c.m + (u64)o * sp, sp, plan->G_sz, z, nt,
                                 nodes[gamma], vals[gamma]);
        if (rc[gamma] != PDQ_OK) err[gamma] = pdq_last_error();   // this thread's message
    };
    const unsigned hw = host_threads();
    if (G == 1 || hw == 1) {
        for (u32 gamma = 0; gamma < G; ++gamma) one(gamma, hw);
    } else {
        const unsigned nw = std::min<unsigned>(hw, G), per = std::max(1u, hw / nw);
        std::vector<std::thread> th;
        for (unsigned w = 0; w < nw; ++w)
            th.emplace_back([&, w] {
                for (u32 gamma = w; gamma < G; gamma += nw) one(gamma, per);
            });
        for (auto& t : th) t.join();
    }
    for (u32 gamma = 0; gamma < G; ++gamma)
        if (rc[gamma] != PDQ_OK) return fail(rc[gamma], err[gamma]);
    u64 total = 0;
    for (u32 gamma = 0; gamma < G; ++gamma) {
        for (size_t k = 0; k < nodes[gamma].size(); ++k) {
            if (total < cap) {
                if (idx_out) idx_out[total] = (u64)gamma * plan->G_sz + nodes[gamma][k] - 1;
                if (val_out) val_out[total] = (u32)vals[gamma][k];
            }
            ++total;
        }
    }
    *count = total;
    if (total > cap) return fail(PDQ_E_NOMEM, "decomp: output capacity too small");
    return PDQ_OK;
}

}  // namespace
}  // namespace pdq

using namespace pdq;

extern "C" int pdq_decomp(const pdq_ctx* ctx, const pdq_plan* plan, const uint32_t* slots,
                          uint64_t* idx_out, uint32_t* val_out, uint64_t cap, uint64_t* count) {
    if (!ctx) return fail(PDQ_E_PARAM, "decomp: null argument");
    return decomp_run(*reinterpret_cast<const Ctx*>(ctx), plan, slots, idx_out, val_out, cap,
                      count);
}

extern "C" int pdq_decomp_client(uint64_t t, uint32_t log_n, const pdq_plan* plan,
                                 const uint32_t* slots, uint64_t* idx_out, uint32_t* val_out,
                                 uint64_t cap, uint64_t* count) {
    Ctx c;
    PDQ_TRY(host_ring(t, log_n, &c));
    return decomp_run(c, plan, slots, idx_out, val_out, cap, count);
}
