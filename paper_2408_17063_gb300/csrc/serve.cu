// Batched answers and a continuous-batching server around pdq_answer.
//
// Batch: the queries of one call are dealt round-robin onto `lanes` CUDA
// streams owned by the context; the lanes fork from the caller's stream and
// join back into it with events, so a batch can be captured into one CUDA
// graph together with the caller's work.
//
// Server: requests (possibly for different parameter sets) are queued in
// arrival order; one worker thread per lane takes the oldest request whose
// workspace fits into the free part of the caller's device arena (the
// admission budget), launches Mask+Comp on its own stream and waits for it,
// so requests that arrive while others run are admitted as soon as a lane
// and memory free up, and their kernels overlap on the device.  With
// stacking on, the worker also takes queued requests of the oldest one's
// shape and answers them all with one stacked call.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "pdq_internal.h"
#include "pdq_ops.h"

namespace pdq {

static u64 now_ns() {
    return (u64)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

int lanes_ensure(const Ctx& c, u32 lanes) {
    std::lock_guard<std::mutex> lock(c.lanes_mu);
    Ctx::Lanes& L = c.lanes;
    if (!L.fork) {
        if (cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming) != cudaSuccess)
            return fail(PDQ_E_CUDA, "batch: event creation failed");
    }
    while (L.streams.size() < lanes) {
        cudaStream_t s;
        cudaEvent_t e;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
            return fail(PDQ_E_CUDA, "batch: stream creation failed");
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaStreamDestroy(s);
            return fail(PDQ_E_CUDA, "batch: event creation failed");
        }
        L.streams.push_back(s);
        L.joins.push_back(e);
    }
    return PDQ_OK;
}

void lanes_release(Ctx* c) {
    Ctx::Lanes& L = c->lanes;
    for (auto s : L.streams) cudaStreamDestroy(s);
    for (auto e : L.joins) cudaEventDestroy(e);
    if (L.fork) cudaEventDestroy(L.fork);
    L.streams.clear();
    L.joins.clear();
    L.fork = nullptr;
}

}  // namespace pdq

using namespace pdq;

extern "C" int pdq_answer_batch(const pdq_ctx* ctx, const pdq_query* queries, uint32_t nq,
                                void* const* lane_ws, const size_t* lane_ws_bytes,
                                uint32_t lanes, void* stream) {
    if (!ctx || (!queries && nq) || !lane_ws || !lane_ws_bytes)
        return fail(PDQ_E_PARAM, "answer_batch: null argument");
    if (lanes == 0 || lanes > 32) return fail(PDQ_E_PARAM, "answer_batch: 1..32 lanes");
    if (nq == 0) return PDQ_OK;
    const Ctx& c = *reinterpret_cast<const Ctx*>(ctx);
    for (uint32_t i = 0; i < nq; ++i) {
        const pdq_query& q = queries[i];
        if (!q.plan) return fail(PDQ_E_PARAM, "answer_batch: query without plan");
        const size_t need = pdq_answer_workspace_bytes(ctx, q.plan);
        if (need == 0) return fail(PDQ_E_PARAM, "answer_batch: invalid plan in query " + std::to_string(i));
        if (lane_ws_bytes[i % lanes] < need)
            return fail(PDQ_E_NOMEM, "answer_batch: lane workspace too small for query " + std::to_string(i));
    }
    PDQ_TRY(lanes_ensure(c, lanes));
    cudaStream_t st = (cudaStream_t)stream;
    Ctx::Lanes& L = c.lanes;
    const bool prof = c.prof.on;
    c.prof.on = false;             // stage events would interleave across lanes
    int rc = PDQ_OK;
    if (cudaEventRecord(L.fork, st) != cudaSuccess) rc = fail(PDQ_E_CUDA, "answer_batch: fork record failed");
    for (uint32_t k = 0; k < lanes && rc == PDQ_OK; ++k)
        if (cudaStreamWaitEvent(L.streams[k], L.fork, 0) != cudaSuccess)
            rc = fail(PDQ_E_CUDA, "answer_batch: fork wait failed");
    for (uint32_t i = 0; i < nq && rc == PDQ_OK; ++i) {
        const pdq_query& q = queries[i];
        const uint32_t k = i % lanes;
        rc = pdq_answer(ctx, q.plan, q.v_cts, q.db, q.keys, q.galois, q.nkeys, q.consts, q.out,
                        lane_ws[k], lane_ws_bytes[k], L.streams[k]);
    }
    // join every lane back into the caller's stream, also after an error
    for (uint32_t k = 0; k < lanes; ++k) {
        if (cudaEventRecord(L.joins[k], L.streams[k]) != cudaSuccess ||
            cudaStreamWaitEvent(st, L.joins[k], 0) != cudaSuccess) {
            if (rc == PDQ_OK) rc = fail(PDQ_E_CUDA, "answer_batch: join failed");
        }
    }
    c.prof.on = prof;
    return rc;
}

// --------------------------------------------------------------- server ----

namespace {

struct Request {
    u64 ticket;
    const pdq_ctx* ctx;
    pdq_plan plan;
    pdq_query q;
    std::vector<u64> galois;
    size_t ws_bytes;
};

struct Ticket {
    int state = PDQ_REQ_QUEUED;
    int status = PDQ_OK;
    u64 t_submit = 0, t_start = 0, t_done = 0;
    u32 stacked = 0;
    std::string error;
};

// Requests that one stacked call can answer: the same context, database,
// plan constants and Galois list, and plans equal in every field but the
// record and match counts (the Answer's kernels never read those; the
// client's Decomp does).
bool stackable(const Request& r) { return !r.plan.plain_db && r.plan.ring_ratio <= 1; }

bool same_shape(const Request& a, const Request& b) {
    if (a.ctx != b.ctx || a.q.db != b.q.db || a.q.consts != b.q.consts || a.galois != b.galois)
        return false;
    pdq_plan x = a.plan, y = b.plan;
    x.n = y.n = 0;
    x.s = y.s = 0;
    return std::memcmp(&x, &y, sizeof x) == 0;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// arena bytes of Q stacked requests: the stacked workspace, then the
// gathered index ciphertexts and the outputs
size_t stacked_bytes(const Request& r, u32 Q) {
    const Ctx& c = *reinterpret_cast<const Ctx*>(r.ctx);
    const size_t cts = ct_elems(c) * sizeof(u64);
    return align256(pdq_answer_stacked_workspace_bytes(r.ctx, &r.plan, Q)) +
           align256((size_t)Q * r.plan.J * cts) + align256((size_t)Q * r.plan.n_out * cts);
}

// first-fit allocator over the caller's arena (offsets aligned to 256 bytes)
struct Arena {
    char* base = nullptr;
    size_t size = 0;
    std::list<std::pair<size_t, size_t>> free_list;   // (offset, bytes), sorted
    void init(void* b, size_t s) {
        base = reinterpret_cast<char*>(b);
        size = s & ~(size_t)255;
        free_list.clear();
        free_list.emplace_back(0, size);
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_list.begin(); it != free_list.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                it->first += bytes;
                it->second -= bytes;
                if (it->second == 0) free_list.erase(it);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        auto it = free_list.begin();
        while (it != free_list.end() && it->first < off) ++it;
        it = free_list.insert(it, {off, bytes});
        // merge with the next and the previous block
        auto nx = std::next(it);
        if (nx != free_list.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_list.erase(nx);
        }
        if (it != free_list.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_list.erase(it);
            }
        }
    }
};

}  // namespace

struct pdq_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    std::unordered_map<u64, Ticket> tickets;
    Arena arena;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    int device = 0;
    u32 max_queue = 0;
    u32 max_stack = 1;
    u64 next_ticket = 1;
    u64 inflight = 0;
    bool stop = false;

    void worker(u32 lane) {
        cudaSetDevice(device);
        cudaStream_t st = streams[lane];
        for (;;) {
            std::vector<Request> batch;          // batch[0]: the oldest admitted request
            size_t off = 0, bytes = 0;
            {
                std::unique_lock<std::mutex> lock(mu);
                cv_work.wait(lock, [&] {
                    return stop || (!queue.empty() && arena.alloc(queue.front().ws_bytes, &off));
                });
                if (stop) return;
                batch.push_back(std::move(queue.front()));
                queue.pop_front();
                bytes = batch[0].ws_bytes;
                if (max_stack > 1 && stackable(batch[0])) {
                    // queued requests of the same shape, in arrival order, as
                    // many as a stacked workspace the arena can hold
                    std::vector<size_t> idx;
                    for (size_t i = 0; i < queue.size() && idx.size() + 1 < max_stack; ++i)
                        if (same_shape(batch[0], queue[i])) idx.push_back(i);
                    if (!idx.empty()) {
                        arena.release(off, bytes);
                        bool got = false;
                        while (!idx.empty() && !got) {
                            const size_t need = stacked_bytes(batch[0], (u32)idx.size() + 1);
                            if (arena.alloc(need, &off)) { bytes = need; got = true; }
                            else idx.pop_back();
                        }
                        // alone: the space it was admitted with is free again
                        if (!got && !arena.alloc(bytes, &off)) {
                            queue.push_front(std::move(batch[0]));
                            continue;
                        }
                    }
                    for (auto it = idx.rbegin(); it != idx.rend(); ++it) {
                        batch.push_back(std::move(queue[*it]));
                        queue.erase(queue.begin() + (long)*it);
                    }
                    std::reverse(batch.begin() + 1, batch.end());
                }
                for (const Request& r : batch) {
                    Ticket& t = tickets[r.ticket];
                    t.state = PDQ_REQ_RUNNING;
                    t.t_start = now_ns();
                    t.stacked = (u32)batch.size();
                }
                inflight += batch.size();
            }
            cv_work.notify_all();   // the next request may fit too
            int rc = run(batch, arena.base + off, st);
            std::string err = rc == PDQ_OK ? std::string() : std::string(pdq_last_error());
            if (cudaStreamSynchronize(st) != cudaSuccess && rc == PDQ_OK) {
                rc = PDQ_E_CUDA;
                err = "server: stream synchronisation failed";
            }
            {
                std::lock_guard<std::mutex> lock(mu);
                const u64 t_done = now_ns();
                for (const Request& r : batch) {
                    Ticket& t = tickets[r.ticket];
                    t.t_done = t_done;
                    t.state = PDQ_REQ_DONE;
                    t.status = rc;
                    t.error = err;
                }
                arena.release(off, bytes);
                inflight -= batch.size();
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
    }

    // Answer the requests of `batch` (one, or several of one shape stacked)
    // with the workspace at ws on stream st.
    static int run(std::vector<Request>& batch, char* ws, cudaStream_t st) {
        Request& r0 = batch[0];
        for (Request& r : batch) {
            r.q.plan = &r.plan;
            r.q.galois = r.galois.data();
        }
        if (batch.size() == 1)
            return pdq_answer(r0.ctx, &r0.plan, r0.q.v_cts, r0.q.db, r0.q.keys, r0.q.galois,
                              r0.q.nkeys, r0.q.consts, r0.q.out, ws, r0.ws_bytes, st);
        const u32 Q = (u32)batch.size();
        const Ctx& c = *reinterpret_cast<const Ctx*>(r0.ctx);
        const size_t cts = ct_elems(c) * sizeof(u64);
        const size_t wsb = align256(pdq_answer_stacked_workspace_bytes(r0.ctx, &r0.plan, Q));
        const size_t vb = (size_t)r0.plan.J * cts, ob = (size_t)r0.plan.n_out * cts;
        char* vstage = ws + wsb;
        char* ostage = vstage + align256((size_t)Q * vb);
        const uint64_t* keys[kMaxStack];
        for (u32 q = 0; q < Q; ++q) {
            if (cudaMemcpyAsync(vstage + q * vb, batch[q].q.v_cts, vb, cudaMemcpyDeviceToDevice,
                                st) != cudaSuccess)
                return fail(PDQ_E_CUDA, "server: gathering a stacked query failed");
            keys[q] = batch[q].q.keys;
        }
        PDQ_TRY(pdq_answer_stacked(r0.ctx, &r0.plan, Q, reinterpret_cast<const uint64_t*>(vstage),
                                   r0.q.db, keys, r0.q.galois, r0.q.nkeys, r0.q.consts,
                                   reinterpret_cast<uint64_t*>(ostage), ws, wsb, st));
        for (u32 q = 0; q < Q; ++q)
            if (cudaMemcpyAsync(batch[q].q.out, ostage + q * ob, ob, cudaMemcpyDeviceToDevice,
                                st) != cudaSuccess)
                return fail(PDQ_E_CUDA, "server: copying a stacked answer failed");
        return PDQ_OK;
    }
};

extern "C" {

int pdq_server_create(void* arena, size_t arena_bytes, uint32_t lanes, uint32_t max_queue,
                      pdq_server** out) {
    if (!out || !arena || arena_bytes < 4096) return fail(PDQ_E_PARAM, "server: need an arena");
    if (lanes == 0 || lanes > 32) return fail(PDQ_E_PARAM, "server: 1..32 lanes");
    *out = nullptr;
    pdq_server* s = new pdq_server();
    s->arena.init(arena, arena_bytes);
    s->max_queue = max_queue;
    cudaGetDevice(&s->device);
    for (u32 k = 0; k < lanes; ++k) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (auto x : s->streams) cudaStreamDestroy(x);
            delete s;
            return fail(PDQ_E_CUDA, "server: stream creation failed");
        }
        s->streams.push_back(st);
    }
    for (u32 k = 0; k < lanes; ++k) s->workers.emplace_back([s, k] { s->worker(k); });
    *out = s;
    return PDQ_OK;
}

int pdq_server_submit(pdq_server* s, const pdq_ctx* ctx, const pdq_query* q, uint64_t* ticket) {
    if (!s || !ctx || !q || !q->plan || !ticket) return fail(PDQ_E_PARAM, "server_submit: null argument");
    const size_t need = pdq_answer_workspace_bytes(ctx, q->plan);
    if (need == 0) return fail(PDQ_E_PARAM, "server_submit: invalid plan");
    if (!q->galois && q->nkeys) return fail(PDQ_E_PARAM, "server_submit: null Galois list");
    Request r;
    r.ctx = ctx;
    r.plan = *q->plan;
    r.q = *q;
    r.galois.assign(q->galois, q->galois + q->nkeys);
    r.ws_bytes = need;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (((need + 255) & ~(size_t)255) > s->arena.size)
            return fail(PDQ_E_NOMEM, "server_submit: workspace larger than the whole budget");
        if (s->max_queue && s->queue.size() >= s->max_queue)
            return fail(PDQ_E_BUSY, "server_submit: queue full");
        r.ticket = s->next_ticket++;
        Ticket& t = s->tickets[r.ticket];
        t.t_submit = now_ns();
        *ticket = r.ticket;
        s->queue.push_back(std::move(r));
    }
    s->cv_work.notify_all();
    return PDQ_OK;
}

int pdq_server_status(pdq_server* s, uint64_t ticket, pdq_ticket_info* info) {
    if (!s || !info) return fail(PDQ_E_PARAM, "server_status: null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(PDQ_E_PARAM, "server_status: unknown ticket");
    info->state = it->second.state;
    info->status = it->second.status;
    info->t_submit_ns = it->second.t_submit;
    info->t_start_ns = it->second.t_start;
    info->t_done_ns = it->second.t_done;
    info->stacked = it->second.stacked;
    info->reserved = 0;
    if (it->second.status != PDQ_OK) set_error(it->second.error);
    return PDQ_OK;
}

int pdq_server_set_stacking(pdq_server* s, uint32_t max_stack) {
    if (!s) return fail(PDQ_E_PARAM, "server_set_stacking: null server");
    if (max_stack > kMaxStack) return fail(PDQ_E_PARAM, "server_set_stacking: at most 64");
    std::lock_guard<std::mutex> lock(s->mu);
    s->max_stack = max_stack < 1 ? 1 : max_stack;
    return PDQ_OK;
}

int pdq_server_wait(pdq_server* s, uint64_t ticket, uint32_t timeout_ms) {
    if (!s) return fail(PDQ_E_PARAM, "server_wait: null server");
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(PDQ_E_PARAM, "server_wait: unknown ticket");
    const bool ok = s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), [&] {
        return s->tickets[ticket].state == PDQ_REQ_DONE;
    });
    if (!ok) return fail(PDQ_E_TIMEOUT, "server_wait: timed out");
    const Ticket& t = s->tickets[ticket];
    if (t.status != PDQ_OK) return fail(t.status, t.error);
    return PDQ_OK;
}

int pdq_server_drain(pdq_server* s, uint32_t timeout_ms) {
    if (!s) return fail(PDQ_E_PARAM, "server_drain: null server");
    std::unique_lock<std::mutex> lock(s->mu);
    const bool ok = s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms),
                                        [&] { return s->queue.empty() && s->inflight == 0; });
    return ok ? PDQ_OK : fail(PDQ_E_TIMEOUT, "server_drain: timed out");
}

int pdq_server_destroy(pdq_server* s) {
    if (!s) return PDQ_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& w : s->workers) w.join();
    for (auto st : s->streams) cudaStreamDestroy(st);
    delete s;
    return PDQ_OK;
}

}  // extern "C"
