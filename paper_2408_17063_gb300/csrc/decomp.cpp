// Client-side Decomp (Alg. 6) on decrypted answer slots, host C++.
//
// Per record group: the power sums w_1..w_s' (row 0) give, by Newton's
// identity (Lem. 1, Alg. 1 step 1), the coefficients of
// f(X) = prod_{nodes}(X - node) * X^{s' - #nodes}; the factors of X are
// stripped and the roots among the nodes 1..G_sz are found by evaluating the
// stripped polynomial at every node (Alg. 1 step 2; the paper suggests
// Cantor-Zassenhaus, any exact root finder gives the same set).  The values
// solve sum_l node_l^{j} x_l = e_j, j = 1..l (Alg. 4); this system is
// node-scaled transposed Vandermonde, solved in O(l^2) through the Lagrange
// basis of the nodes, and rows l+1..s' must agree.
#include <algorithm>
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

// roots of g (coefficients low to high) among 1..hi, evaluated in parallel
std::vector<u64> roots_among(const std::vector<u64>& g, u64 hi, const Zt& z) {
    const unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
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

int decode_group(const u32* w, const u32* e, u32 sp, u64 G_sz, const Zt& z,
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
    nodes = roots_among(g, G_sz, z);
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
int decomp_run(const Ctx& c, const pdq_plan* plan, const uint32_t* slots, uint64_t* idx_out,
               uint32_t* val_out, uint64_t cap, uint64_t* count) {
    if (!plan || !slots || !count) return fail(PDQ_E_PARAM, "decomp: null argument");
    if (!valid_plan(c, plan)) return fail(PDQ_E_PARAM, "decomp: invalid plan");
    const Zt z{c.t};
    const u32 sp = plan->s_prime;
    u64 total = 0;
    std::vector<u64> nodes, vals;
    for (u32 gamma = 0; gamma < plan->G; ++gamma) {
        const u32 cidx = plan->G > 1 ? gamma / plan->per_out : 0;
        const u32 o = plan->G > 1 ? gamma % plan->per_out : 0;
        const u32* s = slots + (u64)cidx * c.N;
        PDQ_TRY(decode_group(s + (u64)o * sp, s + c.m + (u64)o * sp, sp, plan->G_sz, z, nodes, vals));
        for (size_t k = 0; k < nodes.size(); ++k) {
            if (total < cap) {
                if (idx_out) idx_out[total] = (u64)gamma * plan->G_sz + nodes[k] - 1;
                if (val_out) val_out[total] = (u32)vals[k];
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
