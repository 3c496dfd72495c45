"""Benchmark: Mask+Comp queries/s and p50/p99 latency of the private database
query answer at N = 2^15 (8 x 60-bit ciphertext primes + 2 special primes, 4
key-switching digits), n = 2^20 records, s = 256 clustered matches: one query
per step on one GPU, database plaintexts, diagonals and rotation keys
resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pdq|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank answers its own
queries (replicas; the method has no cross-GPU exchange), rank 0 prints.
``--impl reference`` times the CPU oracle on the host cores instead (a
bounded sample per step, see ``oracle.baseline``).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mask+Comp queries/sec and p50/p99 latency at N=2^15, batched vs plain"
WORKLOAD = "c3"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pdq", choices=["pdq", "reference"])
    ap.add_argument("--config", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--n", type=int, default=0, help="override the record count")
    ap.add_argument("--L", type=int, default=0, help="override the ciphertext primes")
    ap.add_argument("--K", type=int, default=0, help="override the special primes")
    ap.add_argument("--dnum", type=int, default=0, help="override the key-switching digits")
    ap.add_argument("--B", type=int, default=0, help="baby-step count of the plan (0: the library's choice)")
    ap.add_argument("--lane-budget-gb", type=float, default=100.0,
                    help="cap on the batched lanes' workspaces (fewer lanes for the largest ring beyond)")
    ap.add_argument("--clients", type=int, default=4,
                    help="second batched run with this many clients sharing key sets (0: skip)")
    ap.add_argument("--s", type=int, default=0, help="override the sparsity")
    ap.add_argument("--mix", type=int, default=64, help="queries of the batched/served mix (0: skip)")
    ap.add_argument("--paper-shapes", type=int, default=1,
                    help="also time the paper's Table II/III shapes (N=2^13, 2x54-bit primes; 0: skip)")
    ap.add_argument("--switch-L", type=int, default=2,
                    help="also time the Answer with Comp on this many primes after modulus "
                         "switching (0: skip)")
    ap.add_argument("--ring-log-n", type=int, default=13,
                    help="also time the Answer with Comp in the subring of this log2 dimension "
                         "after ring switching (with --switch-L primes; 0: skip)")
    ap.add_argument("--plain-db", type=int, default=1,
                    help="also time the Answer on an unencrypted database (0: skip)")
    ap.add_argument("--plain-db-B", type=int, default=0,
                    help="baby-step count of the unencrypted-database plan (0: its cost rule)")
    ap.add_argument("--stacked", type=int, default=1,
                    help="queries of one plan answered together (0: skip)")
    ap.add_argument("--stacked-configs", default="",
                    help="comma-separated configurations of the stacked leg (default: all)")
    ap.add_argument("--tune", type=int, default=1,
                    help="also run the batched mix with autotuned plans (0: skip)")
    ap.add_argument("--tune-cache", default="", help="JSON file of tuned plans (read and written)")
    ap.add_argument("--tune-schedule", type=int, default=1,
                    help="autotune the context's launch schedule on the benchmark's shape first")
    ap.add_argument("--rotation-budget-gib", type=float, default=2.0,
                    help="also time the Answer holding at most this many GiB of baby-step "
                         "rotations (0: skip)")
    ap.add_argument("--lanes", type=int, default=4)
    ap.add_argument("--rates", default="50,200,500,1000,2000", help="served arrival rates, queries/s")
    ap.add_argument("--served-requests", type=int, default=2000)
    ap.add_argument("--served-stack", type=int, default=16,
                    help="served again with up to this many requests of one shape stacked (<= 1: skip)")
    ap.add_argument("--stack-rates", default="2000",
                    help="arrival rates of the stacked served run, queries/s")
    ap.add_argument("--latency-steps", type=int, default=200,
                    help="steps of the plain path timed one by one for its p50/p99")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="served HBM budget")
    return ap.parse_args()


def config_dict(cfg, extra=None):
    d = {"workload": f"{cfg.name}: plain single query, BFV N=2^{cfg.log_n}, t={cfg.t}, "
                     f"{cfg.L}x{cfg.prime_bits}-bit + {cfg.K} special primes (dnum={cfg.dnum}), "
                     f"n={cfg.n} records, s={cfg.s} {cfg.pattern} matches",
         "N": cfg.N, "n": cfg.n, "s": cfg.s, "L": cfg.L, "K": cfg.K, "dnum": cfg.dnum,
         "t": cfg.t, "queries_per_step": 1, "mode": "plain (one query at a time)"}
    d.update(extra or {})
    return d


# ------------------------------------------------------------- replicas -----

def max_over_ranks(value: float, dist=None, device="cuda") -> float:
    """The slowest rank's value (each rank answers its own queries; the job
    takes as long as its slowest replica)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(total_ms: float, steps: int, world: int, queries_per_step: int = 1) -> float:
    """Whole-job queries/s: all ranks' queries over the slowest rank's time."""
    return world * steps * queries_per_step / (total_ms / 1000.0)


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------- CPU oracle sample --

def run_reference(args, cfg, rank: int):
    """The reference arm: the CPU oracle on every host core, one bounded
    sample of the workload per step (oracle.baseline.all_cores)."""
    if rank != 0:
        return
    from oracle import baseline
    procs, rounds = baseline.all_cores(cfg, rounds=args.warmup + args.steps)
    timed = rounds[args.warmup:]
    vals = [1.0 / r["seconds_per_query"] for r in timed]
    wall = sum(r["round_wall_s"] for r in timed)
    v = statistics.median(vals)
    sample = (f"each step: the oracle (untuned) times one full-size raise, rotation with "
              f"ModDown, extended-basis rotation, polynomial ModDown, Mask product and two "
              f"diagonal products over Q u P in each of {procs} processes at once "
              f"({timed[-1]['sampled_s_per_process']:.1f} s per process), weighted by the "
              f"oracle's operation counts per Answer and divided over the {procs} cores "
              f"(the operations are independent across half-blocks, giant steps and groups)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "queries/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * wall / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64 (exact modular integers)",
            "data": "synthetic", "config": config_dict(cfg),
            "cpu_baseline": {"value": v, "unit": "queries/s", "cores": procs, "kind": "oracle",
                             "cpu_model": baseline.cpu_model(), "sample": sample},
            "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_e2e(args, ctx, plan, v_cts, db, keys, galois, consts, ws, stream, dist, world):
    """queries/s through pdq_answer_host: H2D of the query, Mask+Comp, D2H of
    the answer inside the timed region (pinned host buffers)."""
    import torch
    vc = v_cts.clone()
    ctx.ntt_inverse(vc, 2 * plan.J, ctx.L)
    v_host = vc.cpu().pin_memory()
    del vc
    out_host = torch.empty(plan.n_out * ctx.ct_elems, dtype=torch.int64).pin_memory()
    ws_host = ctx.answer_host_workspace(plan)
    for _ in range(2):
        ctx.answer_host(plan, v_host, db, keys, galois, consts, out_host, ws=ws_host, stream=stream)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        ctx.answer_host(plan, v_host, db, keys, galois, consts, out_host, ws=ws_host, stream=stream)
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
    e2e = {"value": world * args.e2e_steps / e2e_s, "unit": "queries/s",
           "h2d_bytes_per_step": v_host.numel() * 8, "d2h_bytes_per_step": out_host.numel() * 8,
           "steps": args.e2e_steps, "entry_point": "pdq_answer_host"}
    return e2e



# ------------------------------------------------------ batched / served ----

class Mix:
    """The batched workload: independent queries with mixed ring dimension,
    record count and sparsity; one resident database of 2^20 records (values
    uniform in [0, 2^16)) per ring size; diagonal constants shared by queries
    with the same plan.  clients = 0: every query has its own secret and key
    set; clients = c > 0: query i belongs to client i mod c, whose secret and
    rotation keys (every element its queries of that ring need) all its
    queries share."""

    def __init__(self, nq: int, lanes: int, clients: int = 0, tuner=None):
        import numpy as np
        import torch
        import workloads as W
        from paper_2408_17063_gb300 import pdq

        self.pdq = pdq
        self.specs = W.batched_mix(nq)
        self.lanes = lanes
        self.ctx, self.db, self.dbvals = {}, {}, {}
        for ln in sorted({q.log_n for q in self.specs}):
            ctx = pdq.Context(**W.RING_PARAMS[ln])
            vals = W.rng_for(0xDB, ln).integers(0, 1 << 16, size=1 << 20).astype(np.uint32)
            self.ctx[ln] = ctx
            self.dbvals[ln] = vals
            self.db[ln] = ctx.db_encode(torch.from_numpy(vals.astype(np.int32)).cuda())
        consts = {}
        self.items = []
        self.clients = clients
        # plans: the library's cost model, or the autotuner's timed choice
        plans = [self.ctx[q.log_n].plan(q.n, q.s, tuner.best(self.ctx[q.log_n], q.n, q.s)
                                        if tuner else 0) for q in self.specs]
        self.tuned = tuner is not None

        def make_keys(ctx, sk, galois, seed):
            keys = ctx._u64(len(galois) * ctx.key_elems)
            kv = keys.view(len(galois), -1)
            kr = W.rotation_key_randomness(ctx.moduli, ctx.N, ctx.ndigits, galois, seed)
            for i, k in enumerate(galois):
                a, e = kr[k]
                ctx.rotkey_gen(sk, k, torch.from_numpy(a.view(np.int64)).cuda(),
                               torch.from_numpy(e).cuda(), out=kv[i])
            return keys

        shared = {}
        if clients:
            need = {}
            for i, (q, plan) in enumerate(zip(self.specs, plans)):
                need.setdefault((i % clients, q.log_n), set()).update(
                    self.ctx[q.log_n].plan_galois(plan))
            for (c, ln), ks in sorted(need.items()):
                ctx = self.ctx[ln]
                seed = 0xC1E0 + 16 * c + ln
                sk = ctx.secret_prepare(torch.from_numpy(W.draw_ternary(ctx.N, W.rng_for(seed, 3))))
                galois = sorted(ks)
                shared[(c, ln)] = (sk, galois, make_keys(ctx, sk, galois, seed))
        for qi, (q, plan) in enumerate(zip(self.specs, plans)):
            ctx = self.ctx[q.log_n]
            key = (q.log_n, plan.s_prime, plan.B, plan.hclass, plan.G > 1)
            if key not in consts:
                consts[key] = ctx.plan_constants(plan)
            pos = W.draw_matches_uniform(q.n, q.s, W.rng_for(q.seed, 2))
            if clients:
                sk, galois, keys = shared[(qi % clients, q.log_n)]
            else:
                sk = ctx.secret_prepare(torch.from_numpy(W.draw_ternary(ctx.N, W.rng_for(q.seed, 3))))
                galois = ctx.plan_galois(plan)
                keys = make_keys(ctx, sk, galois, q.seed)
            v = np.zeros(plan.J * ctx.N, dtype=np.int32)
            v[pos] = 1
            a, e = W.encryption_randomness(ctx.moduli[:ctx.L], ctx.N, plan.J, q.seed)
            v_cts = ctx.encrypt(sk, torch.from_numpy(v).cuda(),
                                torch.from_numpy(a.view(np.int64)).cuda(), torch.from_numpy(e).cuda())
            truth = [(int(i), int(self.dbvals[q.log_n][i])) for i in pos]
            self.items.append(dict(spec=q, ctx=ctx, plan=plan, galois=galois, keys=keys,
                                   consts=consts[key], v_cts=v_cts, sk=sk, truth=truth))
            torch.cuda.synchronize()
        self.n_consts = len(consts)

    def handle(self, it, out=None):
        ctx = it["ctx"]
        out = ctx._u64(it["plan"].n_out * ctx.ct_elems) if out is None else out
        return ctx.query(it["plan"], it["v_cts"], self.db[it["spec"].log_n], it["keys"],
                         it["galois"], it["consts"], out)

    def ws_bytes(self, it):
        return self.pdq.load().pdq_answer_workspace_bytes(it["ctx"].h, it["plan"])

    def check(self, it, out) -> bool:
        ctx = it["ctx"]
        slots = ctx.decrypt(it["sk"], out.view(it["plan"].n_out, 2, ctx.L, ctx.N)).cpu().numpy()
        return ctx.decomp(it["plan"], slots) == it["truth"]


def run_batched(args, mix) -> dict:
    """All queries of the mix: one pdq_answer_batch per ring size on its own
    stream (lanes per context), captured in CUDA graphs and replayed, against
    the plain path (the same queries one at a time on one stream)."""
    import torch
    by_ring = {}
    for it in mix.items:
        by_ring.setdefault(it["spec"].log_n, []).append(it)
    handles = {ln: [mix.handle(it) for it in its] for ln, its in by_ring.items()}
    # lanes per ring, fewer where the lanes' workspaces would pass the budget
    def lane_need(its, lanes):
        need = [0] * lanes
        for i, it in enumerate(its):
            need[i % lanes] = max(need[i % lanes], mix.ws_bytes(it))
        return need
    lanes = {ln: min(args.lanes, len(its)) for ln, its in by_ring.items()}
    budget = int(args.lane_budget_gb * (1 << 30))
    while sum(sum(lane_need(by_ring[ln], k)) for ln, k in lanes.items()) > budget:
        big = max((ln for ln in lanes if lanes[ln] > 1),
                  key=lambda ln: max(lane_need(by_ring[ln], lanes[ln])), default=None)
        if big is None:
            break
        lanes[big] -= 1
    lane_ws = {ln: [torch.empty(max(b, 8), dtype=torch.uint8, device="cuda")
                    for b in lane_need(by_ring[ln], lanes[ln])] for ln in by_ring}
    streams = {ln: torch.cuda.Stream() for ln in by_ring}
    for ln in by_ring:
        streams[ln].wait_stream(torch.cuda.current_stream())

    def launch_all():
        for ln in by_ring:
            mix.ctx[ln].answer_batch(handles[ln], lane_ws[ln], stream=streams[ln])

    launch_all()
    torch.cuda.synchronize()
    ok = all(mix.check(it, h.out) for ln in by_ring for it, h in zip(by_ring[ln], handles[ln]))
    graphs = {}
    for ln in by_ring:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=streams[ln]):
            mix.ctx[ln].answer_batch(handles[ln], lane_ws[ln], stream=streams[ln])
        graphs[ln] = g
    torch.cuda.synchronize()

    def replay():
        for ln, g in graphs.items():
            with torch.cuda.stream(streams[ln]):
                g.replay()

    for _ in range(2):
        replay()
    torch.cuda.synchronize()
    reps = 3
    t0 = time.perf_counter()
    for _ in range(reps):
        replay()
    torch.cuda.synchronize()
    t_graph = (time.perf_counter() - t0) / reps
    ok = ok and all(mix.check(it, h.out) for ln in by_ring for it, h in zip(by_ring[ln], handles[ln]))
    # the lanes' workspaces go before the plain run allocates its own
    del graphs, lane_ws
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    # plain: one query at a time on one stream, no graph
    ws_plain = {ln: torch.empty(max(max(mix.ws_bytes(it) for it in its), 8), dtype=torch.uint8,
                                device="cuda") for ln, its in by_ring.items()}
    outs = [mix.handle(it) for it in mix.items]

    def plain():
        for it, h in zip(mix.items, outs):
            it["ctx"].answer(it["plan"], it["v_cts"], mix.db[it["spec"].log_n], it["keys"],
                             it["galois"], it["consts"], ws=ws_plain[it["spec"].log_n], out=h.out)

    plain()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain()
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    # device time of each query alone (events around each call)
    qev = [torch.cuda.Event(enable_timing=True) for _ in range(len(mix.items) + 1)]
    qev[0].record()
    for i, (it, h) in enumerate(zip(mix.items, outs)):
        it["ctx"].answer(it["plan"], it["v_cts"], mix.db[it["spec"].log_n], it["keys"],
                         it["galois"], it["consts"], ws=ws_plain[it["spec"].log_n], out=h.out)
        qev[i + 1].record()
    torch.cuda.synchronize()
    per_query = [qev[i].elapsed_time(qev[i + 1]) for i in range(len(mix.items))]
    nq = len(mix.items)
    return {"queries": nq, "rings": {str(1 << ln): len(v) for ln, v in by_ring.items()},
            "lanes_per_ring": {str(1 << ln): k for ln, k in lanes.items()}, "cuda_graph": True, "distinct_plan_constants": mix.n_consts,
            "batched_qps": nq / t_graph, "plain_qps": nq / t_plain,
            "batched_ms_per_batch": 1000 * t_graph, "plain_ms_per_batch": 1000 * t_plain,
            "speedup": t_plain / t_graph, "all_decompress_exactly": bool(ok),
            "peak_device_gib": torch.cuda.max_memory_allocated() / 2**30,
            "plans": "autotuned (timed choice of B per shape)" if mix.tuned else
                     "the library's cost model",
            "plain_ms_by_ring": {str(1 << ln): sum(per_query[i] for i, it in enumerate(mix.items)
                                                   if it["spec"].log_n == ln)
                                 for ln in by_ring},
            "mix": "64 queries, N uniform in {2^13, 2^14, 2^15}, log2 n uniform in 12..20, "
                   "s uniform in [1, min(1024, n/16)], "
                   + (f"{mix.clients} clients sharing secret and keys per ring" if mix.clients
                      else "own key set per query")}


def run_served(args, mix, stack: int = 1, rates: str = "") -> list:
    """Poisson arrivals of the mix against resident databases and keys; the
    continuous-batching server admits requests by the HBM budget (stack > 1:
    and answers up to `stack` queued requests of one shape together)."""
    import numpy as np
    import torch
    import workloads as W
    pdq = mix.pdq
    free, total = torch.cuda.mem_get_info()
    resident = torch.cuda.memory_allocated()
    budget = int(args.budget_gb * (1 << 30))
    arena_bytes = max(budget - resident, 1 << 30)
    arena_bytes = min(arena_bytes, free - (4 << 30))
    arena = torch.empty(arena_bytes, dtype=torch.uint8, device="cuda")
    # every query's answer alone, checked once (decrypts and decompresses to
    # its matches); a served answer is exact iff it equals it bit for bit
    # (the Answer is deterministic)
    reference = []
    for it in mix.items:
        h = mix.handle(it)
        it["ctx"].answer(it["plan"], it["v_cts"], mix.db[it["spec"].log_n], it["keys"],
                         it["galois"], it["consts"], out=h.out)
        torch.cuda.synchronize()
        if not mix.check(it, h.out):
            raise SystemExit("served reference answer does not decompress")
        reference.append(h.out)
    out = []
    for r_i, rate in enumerate(float(x) for x in (rates or args.rates).split(",") if x):
        nreq = args.served_requests
        arrivals = W.poisson_arrivals(rate, nreq, 0x5E + r_i)
        order = [mix.items[i % len(mix.items)] for i in range(nreq)]
        handles = [mix.handle(it) for it in order]
        srv = pdq.Server(arena, lanes=8)
        if stack > 1:
            srv.set_stacking(stack)
        tickets = []
        t0 = time.perf_counter()
        for ta, h in zip(arrivals, handles):
            delay = t0 + ta - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(h))
        srv.drain()
        infos = [srv.status(t) for t in tickets]
        srv.close()
        lat = np.array([(i.t_done_ns - i.t_submit_ns) / 1e6 for i in infos])
        span = (max(i.t_done_ns for i in infos) - min(i.t_submit_ns for i in infos)) / 1e9
        ok = all(i.status == 0 for i in infos)
        exact = all(torch.equal(h.out, reference[i % len(mix.items)])
                    for i, h in enumerate(handles))
        out.append({"rate_qps": rate, "requests": nreq, "p50_ms": float(np.percentile(lat, 50)),
                    "p99_ms": float(np.percentile(lat, 99)), "served_qps": nreq / span,
                    "offered_s": float(arrivals[-1]), "all_ok": bool(ok),
                    "stacking": stack,
                    "mean_requests_per_launch": float(np.mean([i.stacked for i in infos])),
                    "all_decompress_exactly": bool(exact),
                    "check": "every result equal bit for bit to its query's answer alone, "
                             "which decrypts and decompresses to the query's matches"})
        del handles
        torch.cuda.empty_cache()
    del arena
    return out

# ------------------------------------------------------------------ GPU arm --

# Peak of 60-bit modular multiply-accumulates on the integer multiply-add
# pipe: 152 SMs x 2070 MHz x 32 IMAD.WIDE per clock per SM (a 64-bit-result
# multiply-add issues at half the 32-bit rate of 64 per clock) / 4 for the
# four 32x32-bit products of the schoolbook form = 2.52e12/s.  The kernel's
# Karatsuba form (three products, each a mad.lo.cc/madc.hi.cc/addc chain)
# runs 8.1 per SM per clock at a fully busy pipe (a register-only loop at
# 92% fmaheavy: 2.35e12/s, microbench/ceilings.cu), i.e. 2.55e12/s: the same
# bound.
MAC_PEAK_PER_S = 152 * 2070e6 * 32 / 4
MAC_CEILING_MEASURED = 2.35e12
# DRAM bytes of one k_diag_mac launch from ncu (dram__bytes_read.sum +
# dram__bytes_write.sum) on the same plan (B=32, 8 giant steps) with 3 primes
# (L=2, K=1), scaled by 10/3 to the 10 primes of Q u P (every CTA works on
# one prime); None when the kernel has changed since the capture.  Capture:
# 4.065 GB read + 0.214 GB written per launch with 3 primes.
MAC_TRAFFIC_BYTES = round((4.064706e9 + 0.213533e9) * 10 / 3)
MAC_TRAFFIC_PLAN = (2**15, 10, 64, 32, 8)       # N, primes, H, B, giant steps


def mac_roofline(ctx, plan, ms):
    E, N = ctx.E, ctx.N
    macs = plan.H * plan.B * plan.giants * 2 * E * N
    # algorithmic bytes: every rotated operand, diagonal and accumulator once
    algo_bytes = 8 * N * E * (plan.H * plan.B * 2 + plan.hclass * plan.giants * plan.B
                              + plan.G * plan.giants * 2)
    achieved = macs / (ms / 1e3)
    return {"kernel": "k_diag_mac", "bound": "alu", "achieved": achieved / 1e12,
            "peak": MAC_PEAK_PER_S / 1e12, "unit": "T modmac/s", "frac": achieved / MAC_PEAK_PER_S,
            "frac_of_measured_ceiling": achieved / MAC_CEILING_MEASURED,
            "traffic": MAC_TRAFFIC_BYTES if (N, E, plan.H, plan.B, plan.giants) == MAC_TRAFFIC_PLAN
            else None, "algorithmic_bytes": algo_bytes,
            "macs_per_launch": macs, "ms_per_launch": ms,
            "timing": "CUDA events recorded on the launching stream around each launch",
            "peak_source": "derived: 152 SMs x 2070 MHz x 32 IMAD.WIDE/clk/SM / 4 per modmac; "
                           "measured ceiling: register-only Karatsuba loop"}


def run_switched(args, cfg, ctx, plan, q, v_cts, stream, rank: int) -> dict:
    """The Answer with Comp on smaller parameters: the resident query (over
    the configuration's L primes) is switched to the first L' primes
    (pdq_mod_switch) and answered there with keys, database and diagonals
    made for L' primes; one step = switch + Answer."""
    import dataclasses
    import numpy as np
    import torch
    import workloads as W
    from paper_2408_17063_gb300 import pdq

    L2 = args.switch_L
    lcfg = dataclasses.replace(cfg, L=L2, dnum=-(-L2 // cfg.K))
    lo = pdq.Context.from_config(lcfg)
    lplan = lo.plan(cfg.n, cfg.s, args.B)
    galois = lo.plan_galois(lplan)
    sk = lo.secret_prepare(torch.from_numpy(q.sk))
    keys = lo._u64(len(galois) * lo.key_elems)
    kv = keys.view(len(galois), -1)
    kr = W.rotation_key_randomness(lo.moduli, lo.N, lo.ndigits, galois, cfg.seed + rank + 1)
    for i, k in enumerate(galois):
        a, e = kr[k]
        lo.rotkey_gen(sk, k, torch.from_numpy(a.view(np.int64)).cuda(),
                      torch.from_numpy(e).cuda(), out=kv[i])
    db = lo.db_encode(torch.from_numpy(q.db.astype(np.int32)).cuda())
    consts = lo.plan_constants(lplan)
    sw = lo._u64(plan.J * lo.ct_elems)
    sws = ctx._ws(pdq.load().pdq_mod_switch_workspace_bytes(ctx.h, plan.J))
    ws = lo.answer_workspace(lplan)
    out = lo._u64(lplan.n_out * lo.ct_elems)
    # the answer switched once more, to one prime, before it leaves the server
    one = pdq.Context.from_config(dataclasses.replace(cfg, L=1, dnum=1)) if L2 > 1 else None
    out1 = one._u64(lplan.n_out * one.ct_elems) if one else None
    ws1 = lo._ws(pdq.load().pdq_mod_switch_workspace_bytes(lo.h, lplan.n_out)) if one else None
    torch.cuda.synchronize()

    def step():
        ctx.mod_switch(lo, v_cts, out=sw, ws=sws, stream=stream)
        lo.answer(lplan, sw, db, keys, galois, consts, ws=ws, out=out, stream=stream)
        if one:
            lo.mod_switch(one, out, out=out1, ws=ws1, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    truth = [(int(i), int(q.db[i])) for i in q.positions]
    ok = lo.decomp(lplan, lo.decrypt(sk, out).cpu().numpy()) == truth
    if one:
        sk1 = one.secret_prepare(torch.from_numpy(q.sk))
        ok = ok and lo.decomp(lplan, one.decrypt(sk1, out1).cpu().numpy()) == truth
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    lo.profile_enable(True)
    launches0 = pdq.pdq_launch_count()
    torch.cuda.nvtx.range_push("switched")
    ev[0].record(stream)
    for i in range(args.steps):
        step()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    launches = pdq.pdq_launch_count() - launches0
    stages = {k: v[0] / args.steps for k, v in lo.profile_read().items()}
    lo.profile_enable(False)
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total = ev[0].elapsed_time(ev[-1])
    stages["switches"] = total / args.steps - sum(stages.values())
    return {"value": args.steps / (total / 1000.0), "unit": "queries/s",
            "ms_per_query": total / args.steps, "p50_ms": statistics.median(per),
            "stages_ms_per_query": stages,
            "comp_primes": L2, "special_primes": lcfg.K, "dnum": lcfg.dnum,
            "query_primes": cfg.L,
            "answer_bytes": lplan.n_out * (one or lo).ct_elems * 8,
            "answer_primes": 1 if one else L2,
            "rotation_keys_mib": keys.numel() * 8 / 2**20,
            "gpu_launches_per_step": int(launches) / args.steps,
            "all_decompress_exactly": bool(ok),
            "what": (f"the query over {cfg.L} primes switched to {L2} (pdq_mod_switch) and "
                     f"answered there (Mask + Comp, keys and diagonals for {L2} primes, "
                     f"{lcfg.K} special primes, dnum {lcfg.dnum}), the answer switched to "
                     f"{1 if one else L2} prime(s); one step = the switches + Answer")}


def run_ring_switched(args, cfg, ctx, plan, q, v_cts, stream, rank: int) -> dict:
    """The Answer with Comp in a subring (Sec. 5.3): the resident query over
    the configuration's primes is switched to L' primes (pdq_mod_switch),
    masked in the big ring (pdq_mask), switched to R = 2^(log_n - log_small)
    ciphertexts of the subring each (pdq_ring_switch), compressed there
    (pdq_comp with a switched plan and subring keys) and the answer switched
    to one prime.  One step = all of these."""
    import dataclasses
    import numpy as np
    import torch
    import workloads as W
    from paper_2408_17063_gb300 import pdq

    L2, ls = args.switch_L, args.ring_log_n
    lcfg = dataclasses.replace(cfg, L=L2, dnum=-(-L2 // cfg.K))
    lo = pdq.Context.from_config(lcfg)
    small = lo.subring(ls)
    one = pdq.Context.from_config(dataclasses.replace(cfg, L=1, dnum=1)).subring(ls)
    bplan = lo.plan(cfg.n, cfg.s)                    # the big-ring Mask only needs J
    splan = small.plan_switched(cfg.log_n, cfg.n, cfg.s, args.B)
    seed = cfg.seed + rank + 2
    sk = lo.secret_prepare(torch.from_numpy(q.sk))
    s_small = W.draw_ternary(small.N, W.rng_for(seed, 11))
    ka, ke = W.rotation_key_randomness(lo.moduli, lo.N, lo.ndigits, [1], seed, stream=12)[1]
    rsk = lo.ring_switch_key_gen(small, sk, torch.from_numpy(s_small),
                                 torch.from_numpy(ka.view(np.int64)).cuda(), torch.from_numpy(ke))
    galois = small.plan_galois(splan)
    ssk = small.secret_prepare(torch.from_numpy(s_small))
    keys = small._u64(len(galois) * small.key_elems)
    kv = keys.view(len(galois), -1)
    kr = W.rotation_key_randomness(small.moduli, small.N, small.ndigits, galois, seed, stream=13)
    for i, k in enumerate(galois):
        a, e = kr[k]
        small.rotkey_gen(ssk, k, torch.from_numpy(a.view(np.int64)).cuda(),
                         torch.from_numpy(e).cuda(), out=kv[i])
    db = lo.db_encode(torch.from_numpy(q.db.astype(np.int32)).cuda())
    consts = small.plan_constants(splan)
    lib = pdq.load()
    sw = lo._u64(bplan.J * lo.ct_elems)
    sws = ctx._ws(lib.pdq_mod_switch_workspace_bytes(ctx.h, bplan.J))
    masked = lo._u64(4 * bplan.J * lo.ct_elems)
    R = lo.N // small.N
    ms = small._u64(4 * bplan.J * R * small.ct_elems)
    rws = lo._ws(lib.pdq_ring_switch_workspace_bytes(lo.h, 4 * bplan.J))
    cws = small.comp_workspace(splan)
    out = small._u64(splan.n_out * small.ct_elems)
    out1 = one._u64(splan.n_out * one.ct_elems)
    ws1 = small._ws(lib.pdq_mod_switch_workspace_bytes(small.h, splan.n_out))
    torch.cuda.synchronize()
    ev = {}

    def step(mark=False):
        def rec(name):
            if mark:
                ev.setdefault(name, []).append(torch.cuda.Event(enable_timing=True))
                ev[name][-1].record(stream)
        rec("start")
        ctx.mod_switch(lo, v_cts, out=sw, ws=sws, stream=stream)
        rec("mod_switch")
        lo.mask(bplan, sw, db, out=masked, stream=stream)
        rec("mask")
        lo.ring_switch(small, masked, rsk, group=4, out=ms, ws=rws, stream=stream)
        rec("ring_switch")
        small.comp(splan, ms, keys, galois, consts, ws=cws, out=out, stream=stream)
        rec("comp")
        small.mod_switch(one, out, out=out1, ws=ws1, stream=stream)
        rec("answer_mod_switch")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    truth = [(int(i), int(q.db[i])) for i in q.positions]
    ok = small.decomp(splan, small.decrypt(ssk, out).cpu().numpy()) == truth
    ssk1 = one.secret_prepare(torch.from_numpy(s_small))
    ok = ok and one.decomp(splan, one.decrypt(ssk1, out1).cpu().numpy()) == truth
    launches0 = pdq.pdq_launch_count()
    torch.cuda.nvtx.range_push("ring_switched")
    for _ in range(args.steps):
        step(mark=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    launches = pdq.pdq_launch_count() - launches0
    names = ["mod_switch", "mask", "ring_switch", "comp", "answer_mod_switch"]
    stages = {}
    prev = "start"
    for nm in names:
        stages[nm] = sum(a.elapsed_time(b) for a, b in zip(ev[prev], ev[nm])) / args.steps
        prev = nm
    per = [a.elapsed_time(b) for a, b in zip(ev["start"], ev["answer_mod_switch"])]
    total = sum(per)
    return {"value": args.steps / (total / 1000.0), "unit": "queries/s",
            "ms_per_query": total / args.steps, "p50_ms": statistics.median(per),
            "stages_ms_per_query": stages, "ring_ratio": R, "small_N": small.N,
            "comp_primes": L2, "special_primes": lcfg.K, "dnum": lcfg.dnum,
            "plan": {k: getattr(splan, k) for k in ("B", "giants", "J", "H", "G", "n_out")},
            "answer_bytes_u64": splan.n_out * one.ct_elems * 8,
            "answer_bytes_packed_60bit": splan.n_out * 2 * one.N * 60 // 8,
            "rotation_keys_mib": keys.numel() * 8 / 2**20,
            "gpu_launches_per_step": int(launches) / args.steps,
            "all_decompress_exactly": bool(ok),
            "what": (f"the query over {cfg.L} primes switched to {L2} (pdq_mod_switch), Mask in "
                     f"the ring 2^{cfg.log_n} (pdq_mask), every masked ciphertext ring-switched to "
                     f"{R} ciphertexts of the ring 2^{ls} (pdq_ring_switch), Comp there "
                     f"(pdq_comp, switched plan), the answer switched to one prime; one step = "
                     f"all of these")}


def run_plain_db(args, cfg, ctx, q, v_cts, sk, stream, rank: int) -> dict:
    """The Answer on an unencrypted database (Sec. 5.2 remark): the resident
    index ciphertexts compressed with [C; C diag(DB)] (pdq_answer_plain_db),
    no Mask; the database-specific diagonals resident in HBM."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2408_17063_gb300 import pdq

    plan = ctx.plan_plain_db(cfg.n, cfg.s, args.plain_db_B)
    galois = ctx.plan_galois(plan)
    keys = ctx._u64(len(galois) * ctx.key_elems)
    kv = keys.view(len(galois), -1)
    kr = W.rotation_key_randomness(ctx.moduli, ctx.N, ctx.ndigits, galois, cfg.seed + rank)
    for i, k in enumerate(galois):
        a, e = kr[k]
        ctx.rotkey_gen(sk, k, torch.from_numpy(a.view(np.int64)).cuda(),
                       torch.from_numpy(e).cuda(), out=kv[i])
    t0 = time.perf_counter()
    consts = ctx.db_diagonals(plan, torch.from_numpy(q.db.astype(np.int32)))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    ws = ctx.answer_plain_db_workspace(plan)
    out = ctx._u64(plan.n_out * ctx.ct_elems)

    def step():
        ctx.answer_plain_db(plan, v_cts, keys, galois, consts, ws=ws, out=out, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    truth = [(int(i), int(q.db[i])) for i in q.positions]
    ok = ctx.decomp(plan, ctx.decrypt(sk, out).cpu().numpy()) == truth
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ctx.profile_enable(True)
    launches0 = pdq.pdq_launch_count()
    ev[0].record(stream)
    for i in range(args.steps):
        step()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    launches = pdq.pdq_launch_count() - launches0
    stages = {k: v[0] / args.steps for k, v in ctx.profile_read().items() if v[1]}
    ctx.profile_enable(False)
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total = ev[0].elapsed_time(ev[-1])
    diag_bytes = consts.numel() * 8
    mac_ms = stages.get("mac")
    res = {"value": args.steps / (total / 1000.0), "unit": "queries/s",
           "ms_per_query": total / args.steps, "p50_ms": statistics.median(per),
           "stages_ms_per_query": stages,
           "plan": {k: getattr(plan, k) for k in ("B", "giants", "J", "G", "n_out")},
           "db_diagonals_gib": diag_bytes / 2**30, "db_diagonals_build_s": build_s,
           "rotation_keys": len(galois), "gpu_launches_per_step": int(launches) / args.steps,
           "all_decompress_exactly": bool(ok),
           "what": "the index ciphertexts compressed with [C; C diag(DB)] (no Mask), "
                   "database-specific diagonals resident; one step = pdq_answer_plain_db"}
    if mac_ms:
        res["mac_dram_gbs"] = diag_bytes / (mac_ms / 1e3) / 1e9
    del consts, ws, keys
    torch.cuda.empty_cache()
    return res


# The paper's Table II (n = 16384, s = 8..128) and Table III (s = 16,
# n = 2^13..2^17) shapes: ring 2^13, t = 65537, two 54-bit ciphertext primes;
# its Comp times (single-thread Xeon Silver 4114, seconds) for context.
PAPER_SHAPES = [(16384, 8, 1.17), (16384, 16, 2.06), (16384, 32, 3.80), (16384, 64, 7.06),
                (16384, 128, 13.40), (1 << 13, 16, 1.09), (1 << 14, 16, 2.06), (1 << 15, 16, 4.01),
                (1 << 16, 16, 7.92), (1 << 17, 16, 15.75)]


def run_paper_shapes(args, rank: int) -> list:
    """Comp alone (pdq_comp on the masked ciphertexts), the whole Answer and
    the client's Decomp for each shape, on the paper's ring and modulus (one
    54-bit special prime, one prime per key-switching digit: our choice)."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2408_17063_gb300 import pdq

    base = W.CONFIGS["paper"]
    ctx = pdq.Context.from_config(base)
    stream = torch.cuda.current_stream()
    out = []
    for n, s_, paper_s in PAPER_SHAPES:
        import dataclasses
        cfg = dataclasses.replace(base, n=n, s=s_)
        q = W.draw_query(cfg, cfg.seed + rank)
        plan = ctx.plan(n, s_, 0)
        galois = ctx.plan_galois(plan)
        sk = ctx.secret_prepare(torch.from_numpy(q.sk))
        keys = ctx._u64(len(galois) * ctx.key_elems)
        kv = keys.view(len(galois), -1)
        kr = W.rotation_key_randomness(ctx.moduli, ctx.N, ctx.ndigits, galois, cfg.seed + rank)
        for i, k in enumerate(galois):
            a, e = kr[k]
            ctx.rotkey_gen(sk, k, torch.from_numpy(a.view(np.int64)).cuda(),
                           torch.from_numpy(e).cuda(), out=kv[i])
        db = ctx.db_encode(torch.from_numpy(q.db.astype(np.int32)).cuda())
        consts = ctx.plan_constants(plan)
        a, e = W.encryption_randomness(ctx.moduli[:ctx.L], ctx.N, plan.J, cfg.seed + rank)
        v = np.zeros(plan.J * ctx.N, dtype=np.int32)
        v[:n] = q.v
        v_cts = ctx.encrypt(sk, torch.from_numpy(v).cuda(), torch.from_numpy(a.view(np.int64)).cuda(),
                            torch.from_numpy(e).cuda())
        masked = ctx.mask(plan, v_cts, db)
        cws = ctx.comp_workspace(plan)
        aws = ctx.answer_workspace(plan)
        res = ctx._u64(plan.n_out * ctx.ct_elems)

        def timed(f, steps=5):
            for _ in range(2):
                f()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            for _ in range(steps):
                f()
            ev[1].record(stream)
            torch.cuda.synchronize()
            return ev[0].elapsed_time(ev[1]) / steps

        comp_ms = timed(lambda: ctx.comp(plan, masked, keys, galois, consts, ws=cws, out=res,
                                         stream=stream))
        ans_ms = timed(lambda: ctx.answer(plan, v_cts, db, keys, galois, consts, ws=aws, out=res,
                                          stream=stream))
        slots = ctx.decrypt(sk, res).cpu().numpy()
        t0 = time.perf_counter()
        got = ctx.decomp(plan, slots)
        dec_ms = (time.perf_counter() - t0) * 1e3
        out.append({"n": n, "s": s_, "B": plan.B, "giants": plan.giants, "groups": plan.G,
                    "comp_ms": comp_ms, "answer_ms": ans_ms, "decomp_host_ms": dec_ms,
                    "decompress_exactly": got == [(int(i), int(q.db[i])) for i in q.positions],
                    "paper_comp_s": paper_s})
        del keys, db, consts, v_cts, masked, cws, aws, res
        torch.cuda.empty_cache()
    return out


# Queries of one plan answered together: (configuration, records, matches,
# queries) -- the benchmark's large query, the plain N = 2^13 query and the
# paper's Table II/III ring at n = 16384, s = 16.
STACK_SHAPES = [("c3", 1 << 20, 256, 4), ("c2", 1 << 16, 64, 16), ("paper", 16384, 16, 32)]


def run_stacked(args, rank: int) -> list:
    """Clients of one database asking for the same numbers of records and
    matches (each with its own secret, keys and matches): one
    pdq_answer_stacked call for all of them against the same queries one
    pdq_answer at a time, device time (CUDA events); every stacked output is
    compared bit for bit with the query's answer alone and decompressed."""
    import dataclasses
    import numpy as np
    import torch
    import workloads as W
    from paper_2408_17063_gb300 import pdq

    stream = torch.cuda.current_stream()
    rows = []
    only = {x for x in args.stacked_configs.split(",") if x}
    for name, n, s_, Q in STACK_SHAPES:
        if only and name not in only:
            continue
        cfg = dataclasses.replace(W.CONFIGS[name], n=n, s=s_)
        ctx = pdq.Context.from_config(cfg)
        q0 = W.draw_query(cfg, cfg.seed + rank)
        db = ctx.db_encode(torch.from_numpy(q0.db.astype(np.int32)).cuda())
        plan = ctx.plan(n, s_, 0)
        galois = ctx.plan_galois(plan)
        consts = ctx.plan_constants(plan)
        v_all = ctx._u64(Q * plan.J * ctx.ct_elems).view(Q, -1)
        keys, sks, truths = [], [], []
        for i in range(Q):
            seed = cfg.seed + 7919 * (i + 1) + rank
            qi = W.draw_query(cfg, seed)          # own secret and matches; q0's database
            sk = ctx.secret_prepare(torch.from_numpy(qi.sk))
            ks = ctx._u64(len(galois) * ctx.key_elems)
            kv = ks.view(len(galois), -1)
            kr = W.rotation_key_randomness(ctx.moduli, ctx.N, ctx.ndigits, galois, seed)
            for j, k in enumerate(galois):
                a, e = kr[k]
                ctx.rotkey_gen(sk, k, torch.from_numpy(a.view(np.int64)).cuda(),
                               torch.from_numpy(e).cuda(), out=kv[j])
            a, e = W.encryption_randomness(ctx.moduli[:ctx.L], ctx.N, plan.J, seed)
            v = np.zeros(plan.J * ctx.N, dtype=np.int32)
            v[:n] = qi.v
            v_all[i].copy_(ctx.encrypt(sk, torch.from_numpy(v).cuda(),
                                       torch.from_numpy(a.view(np.int64)).cuda(),
                                       torch.from_numpy(e).cuda()).reshape(-1))
            keys.append(ks)
            sks.append(sk)
            truths.append([(int(p), int(q0.db[p])) for p in qi.positions])
        aws = ctx.answer_workspace(plan)
        sws = ctx.answer_stacked_workspace(plan, Q)
        alone = ctx._u64(Q * plan.n_out * ctx.ct_elems).view(Q, -1)
        stacked = ctx._u64(Q * plan.n_out * ctx.ct_elems)

        def plain():
            for i in range(Q):
                ctx.answer(plan, v_all[i], db, keys[i], galois, consts, ws=aws, out=alone[i],
                           stream=stream)

        def together():
            ctx.answer_stacked(plan, v_all, db, keys, galois, consts, ws=sws, out=stacked,
                               stream=stream)

        def timed(f, reps):
            for _ in range(2):
                f()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            for _ in range(reps):
                f()
            ev[1].record(stream)
            torch.cuda.synchronize()
            return ev[0].elapsed_time(ev[1]) / reps

        reps = 3 if name == "c3" else 10
        t_plain = timed(plain, reps)
        l0 = pdq.pdq_launch_count()
        # (NVTX ranges let a profiler select one stacked call and one alone)
        torch.cuda.nvtx.range_push(f"stacked_{name}")
        together()
        torch.cuda.nvtx.range_pop()
        launches = pdq.pdq_launch_count() - l0
        torch.cuda.nvtx.range_push(f"alone_{name}")
        ctx.answer(plan, v_all[0], db, keys[0], galois, consts, ws=aws, out=alone[0],
                   stream=stream)
        torch.cuda.nvtx.range_pop()
        t_stacked = timed(together, reps)
        torch.cuda.synchronize()
        out_q = stacked.view(Q, -1)
        same = all(torch.equal(out_q[i], alone[i]) for i in range(Q))
        ok = all(ctx.decomp(plan, ctx.decrypt(sks[i], out_q[i]).cpu().numpy()) == truths[i]
                 for i in range(Q))
        rows.append({"config": name, "N": ctx.N, "n": n, "s": s_, "queries": Q,
                     "B": plan.B, "giants": plan.giants, "groups": plan.G,
                     "plain_ms_per_query": t_plain / Q, "stacked_ms_per_query": t_stacked / Q,
                     "speedup": t_plain / t_stacked, "launches_per_stacked_call": int(launches),
                     "bit_identical_to_alone": bool(same), "all_decompress_exactly": bool(ok),
                     "stacked_workspace_gib": sws.numel() / 2**30})
        del keys, v_all, db, consts, aws, sws, alone, stacked, ctx
        torch.cuda.empty_cache()
    return rows


def run_gpu(args, cfg, rank: int, world: int):
    import numpy as np
    import torch
    import workloads as W
    from paper_2408_17063_gb300 import build, pdq

    build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    ctx = pdq.Context.from_config(cfg)
    q = W.draw_query(cfg, cfg.seed + rank)
    plan = ctx.plan(cfg.n, cfg.s, args.B)
    sched_tuning = None
    if args.tune_schedule:
        # the launch schedule of the context (transform phase split,
        # multiply-accumulate tiles): timed on a synthetic query of this shape,
        # the fastest kept; every schedule gives the same bits
        from paper_2408_17063_gb300 import tune
        t0 = time.perf_counter()
        hit = tune.ScheduleTuner(args.tune_cache or None, reps=2).best(ctx, cfg.n, cfg.s, args.B)
        sched_tuning = dict(hit, tuning_s=time.perf_counter() - t0)
        torch.cuda.empty_cache()
    galois = ctx.plan_galois(plan)
    sk = ctx.secret_prepare(torch.from_numpy(q.sk))
    N = ctx.N
    # rotation keys, database, diagonals: resident
    keys = ctx._u64(len(galois) * ctx.key_elems)
    kv = keys.view(len(galois), -1)
    kr = W.rotation_key_randomness(ctx.moduli, N, ctx.ndigits, galois, cfg.seed + rank)
    for i, k in enumerate(galois):
        a, e = kr[k]
        ctx.rotkey_gen(sk, k, torch.from_numpy(a.view(np.int64)).cuda(),
                       torch.from_numpy(e).cuda(), out=kv[i])
    db = ctx.db_encode(torch.from_numpy(q.db.astype(np.int32)).cuda())
    consts = ctx.plan_constants(plan)
    # the query: encrypted index vector
    a, e = W.encryption_randomness(ctx.moduli[:ctx.L], N, plan.J, cfg.seed + rank)
    v = np.zeros(plan.J * N, dtype=np.int32)
    v[:cfg.n] = q.v
    v_cts = ctx.encrypt(sk, torch.from_numpy(v).cuda(), torch.from_numpy(a.view(np.int64)).cuda(),
                        torch.from_numpy(e).cuda())
    ws = ctx.answer_workspace(plan)
    out = ctx._u64(plan.n_out * ctx.ct_elems)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()

    def step():
        ctx.answer(plan, v_cts, db, keys, galois, consts, ws=ws, out=out, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # correctness of what is timed: decrypt and decompress the answer
    slots = ctx.decrypt(sk, out).cpu().numpy()
    got = ctx.decomp(plan, slots)
    truth = [(int(i), int(q.db[i])) for i in q.positions]
    if got != truth:
        raise SystemExit("benchmark answer does not decompress to the query result")

    clocks = ClockSampler(local)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ctx.profile_enable(True)
    launches0 = pdq.pdq_launch_count()
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    ev[0].record(stream)
    for i in range(args.steps):
        step()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    launches = pdq.pdq_launch_count() - launches0
    clk = clocks.stop()
    stages = ctx.profile_read()
    ctx.profile_enable(False)
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = max_over_ranks(ev[0].elapsed_time(ev[-1]), dist)
    value = job_throughput(total_ms, args.steps, world)
    # latency distribution of the plain path over more steps (each step timed
    # by its own pair of events on the stream)
    lev = [torch.cuda.Event(enable_timing=True) for _ in range(args.latency_steps + 1)]
    lev[0].record(stream)
    for i in range(args.latency_steps):
        step()
        lev[i + 1].record(stream)
    torch.cuda.synchronize()
    lat = sorted(lev[i].elapsed_time(lev[i + 1]) for i in range(args.latency_steps))

    # the same Answer holding at most a budget of baby-step rotations (made and
    # consumed a chunk of primes at a time): its workspace and time
    budget_leg = None
    if args.rotation_budget_gib > 0:
        lib = pdq.load()
        full_ws = lib.pdq_answer_workspace_bytes(ctx.h, plan)
        ctx.set_rotation_budget(int(args.rotation_budget_gib * 2**30))
        bws = ctx.answer_workspace(plan)
        bout = ctx._u64(plan.n_out * ctx.ct_elems)

        def bstep():
            ctx.answer(plan, v_cts, db, keys, galois, consts, ws=bws, out=bout, stream=stream)

        bstep()
        torch.cuda.synchronize()
        same = torch.equal(bout, out)
        bev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        bev[0].record(stream)
        for _ in range(args.steps):
            bstep()
        bev[1].record(stream)
        torch.cuda.synchronize()
        ctx.set_rotation_budget(0)
        budget_leg = {"budget_gib": args.rotation_budget_gib,
                      "workspace_gib": bws.numel() / 2**30, "full_workspace_gib": full_ws / 2**30,
                      "ms_per_query": bev[0].elapsed_time(bev[1]) / args.steps,
                      "same_bits_as_unbudgeted": bool(same)}
        del bws, bout
        torch.cuda.empty_cache()

    # end to end through the host-buffer entry point (pinned host buffers,
    # coefficient form, copies inside the timed region)
    e2e = None
    if args.e2e_steps > 0:
        e2e = run_e2e(args, ctx, plan, v_cts, db, keys, galois, consts, ws, stream, dist, world)
    del ws

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # roofline of the diagonal multiply-accumulate kernel (one launch per query):
    # it is bound by the integer multiply-add pipe, so achieved and peak are
    # 60-bit modular multiply-accumulates per second
    mac_ms, mac_calls = stages["mac"]
    mac_ms_per = mac_ms / max(1, mac_calls)
    roofline = mac_roofline(ctx, plan, mac_ms_per)
    if ctx.schedule()["mac_tiles"] or ctx.schedule()["mac_bc"]:
        roofline["traffic"] = None        # captured under the default tiles
    ms_sorted = lat if lat else sorted(per)
    p50 = statistics.median(ms_sorted)
    p99 = ms_sorted[min(len(ms_sorted) - 1, int(round(0.99 * (len(ms_sorted) - 1))))]
    line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64 (exact modular integers)", "data": "synthetic",
            "config": config_dict(cfg, {"parallelism": f"replicas x{world}",
                                        "baby_steps_B": plan.B, "giant_steps": plan.giants,
                                        "l2": "inputs larger than L2 (per query: "
                                              f"{consts.numel() * 8 / 2**30:.2f} GiB of plan constants, "
                                              f"{keys.numel() * 8 / 2**20:.0f} MiB of rotation keys, "
                                              f"{v_cts.numel() * 8 / 2**20:.0f} MiB query, "
                                              f"{db.numel() * 8 / 2**20:.0f} MiB database read)"}),
            "latency_ms": {"p50": p50, "p99": p99, "min": ms_sorted[0], "max": ms_sorted[-1],
                           "steps": len(ms_sorted)},
            "stages_ms_per_query": {k: v[0] / max(1, args.steps) for k, v in stages.items()},
            "gpu_launches": int(launches), "gpu_launches_per_step": int(launches) / args.steps,
            "clocks": clk, "e2e": e2e, "roofline": roofline}
    line["config"]["schedule"] = ctx.schedule()
    if sched_tuning:
        line["schedule_tuning"] = sched_tuning
    if budget_leg:
        line["rotation_budget"] = budget_leg
    if args.paper_shapes:
        line["paper_shapes"] = {
            "what": ("the paper's Table II/III shapes (ring 2^13, t=65537, 2x54-bit primes + one "
                     "54-bit special prime, dnum 2): GPU Comp alone, Answer (Mask + Comp) and "
                     "host Decomp per query; paper_comp_s is the paper's single-thread Xeon time "
                     "(context, other hardware and scheme)"),
            "rows": run_paper_shapes(args, rank)}
    if args.plain_db:
        line["plain_db"] = run_plain_db(args, cfg, ctx, q, v_cts, sk, stream, rank)
    if args.stacked:
        line["stacked"] = {
            "what": ("queries of one plan (one database, the same numbers of records and "
                     "matches, own secret and keys each) answered by one pdq_answer_stacked "
                     "call, every step one launch over all of them, against pdq_answer one "
                     "query at a time; device time per query"),
            "rows": run_stacked(args, rank)}
    if args.switch_L and 0 < args.switch_L < cfg.L:
        line["switched"] = run_switched(args, cfg, ctx, plan, q, v_cts, stream, rank)
        if args.ring_log_n and args.ring_log_n < cfg.log_n:
            line["ring_switched"] = run_ring_switched(args, cfg, ctx, plan, q, v_cts, stream, rank)
    if args.mix > 0:
        del v_cts, keys, db, consts, out
        torch.cuda.empty_cache()
        mix = Mix(args.mix, args.lanes)
        line["batched"] = run_batched(args, mix)
        line["served"] = run_served(args, mix)
        if args.served_stack > 1:
            line["served_stacked"] = run_served(args, mix, stack=args.served_stack,
                                                rates=args.stack_rates)
        if args.clients > 0:
            del mix
            torch.cuda.empty_cache()
            mix = Mix(args.mix, args.lanes, clients=args.clients)
            line["batched_shared_keys"] = dict(run_batched(args, mix), clients=args.clients)
        if args.tune:
            from paper_2408_17063_gb300 import tune
            del mix
            torch.cuda.empty_cache()
            tuner = tune.PlanTuner(args.tune_cache or None, reps=2)
            t0 = time.perf_counter()
            mix = Mix(args.mix, args.lanes, tuner=tuner)
            tune_s = time.perf_counter() - t0
            res = run_batched(args, mix)
            changed = {k: {"B": v["B"], "default_B": v["default_B"], "ms": v["ms"]}
                       for k, v in tuner.cache.items() if v["B"] != v["default_B"]}
            line["batched_tuned"] = dict(res, tuning_s=tune_s, shapes_tuned=len(tuner.cache),
                                         shapes_changed=changed)
    if not args.no_cpu_baseline:
        from oracle import baseline
        line["cpu_baseline"] = baseline.baseline(cfg)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    import dataclasses
    import workloads as W
    cfg = W.CONFIGS[args.config]
    if args.n or args.s or args.L or args.K or args.dnum:
        cfg = dataclasses.replace(cfg, n=args.n or cfg.n, s=args.s or cfg.s, L=args.L or cfg.L,
                                  K=args.K or cfg.K, dnum=args.dnum or cfg.dnum)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, cfg, rank)
        return
    run_gpu(args, cfg, rank, world)


if __name__ == "__main__":
    main()
