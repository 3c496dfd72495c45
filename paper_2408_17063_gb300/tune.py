"""Autotuner of the Answer's baby-step/giant-step split.

The split B of the diagonal method (Sec. 5.2: k = gB + a, B - 1 hoisted baby
rotations per half-block, s'/B - 1 giant-step key switches per group) fixes
which kernels run and how large they are, and the best B depends on the
ring, the prime chain, the record count and the sparsity.  The library's
default (pdq_plan_make with B = 0) is a fixed cost model; this tuner times
every admissible B (powers of two, B <= min(s', 128), at most 32 giant steps)
on synthetic inputs of the query's shape through the C ABI (CUDA events on
the stream, after a warm-up) and keeps the fastest.  The timing does not
depend on the values, so a random secret, keys and index vector serve.

Choices persist in a JSON file keyed by the parameter set and the plan shape
(ring dimension, primes, digits, t, records, s', and the Answer kind), so a
server tunes each shape once.  Tuning allocates the keys, plan constants and
workspace of each candidate in turn (at N = 2^15, n = 2^20: about 17 GB).

ScheduleTuner does the same for the launch schedule of a context
(pdq_ctx_set_schedule: the phase split of the transforms and their
polynomials per launch, the position tiles per CTA and the baby steps per
copy step of the multiply-accumulate), by
coordinate descent over the knobs on one query shape (a knob moves only for a
gain above 1%); every schedule gives the same bits, so only the time decides.
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

from . import pdq

_LOCK = threading.Lock()


def shape_key(ctx: pdq.Context, n: int, s: int, kind: str = "answer") -> str:
    sp = 1 << math.ceil(math.log2(max(1, s)))
    return (f"{kind}:N{ctx.N}:L{ctx.L}:K{ctx.K}:d{ctx.ndigits}:t{ctx.t}:q{ctx.moduli[0]}:"
            f"n{n}:s{sp}")


def candidates(ctx: pdq.Context, n: int, s: int) -> list[int]:
    sp = 1 << math.ceil(math.log2(max(1, s)))
    out, b = [], 1
    while b <= min(sp, 128):
        if sp // b <= 32:
            out.append(b)
        b *= 2
    return out


class PlanTuner:
    """Times the admissible B of a shape once and remembers the fastest."""

    def __init__(self, path: str | None = None, reps: int = 3):
        self.path = path
        self.reps = reps
        self.cache: dict = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.cache = json.load(f)

    def save(self):
        if not self.path:
            return
        tmp = f"{self.path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self.cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def best(self, ctx: pdq.Context, n: int, s: int, stream=None) -> int:
        """The fastest B for an Answer of n records and sparsity s on ctx."""
        key = shape_key(ctx, n, s)
        with _LOCK:
            if key in self.cache:
                return int(self.cache[key]["B"])
        times = {b: self.time_answer(ctx, n, s, b, stream) for b in candidates(ctx, n, s)}
        best = min(times, key=lambda b: (times[b], b))
        with _LOCK:
            self.cache[key] = {"B": best, "ms": {str(b): t for b, t in times.items()},
                               "default_B": ctx.plan(n, s).B}
            self.save()
        return best

    def time_answer(self, ctx: pdq.Context, n: int, s: int, B: int, stream=None) -> float:
        """Milliseconds per Answer with plan B on synthetic inputs."""
        rig = AnswerRig(ctx, n, s, B, stream)
        ms = rig.time(self.reps)
        rig.close()
        return ms


class AnswerRig:
    """One synthetic Answer of a shape (random secret, keys, database and index
    vector: the timing does not depend on the values), ready to be timed."""

    def __init__(self, ctx: pdq.Context, n: int, s: int, B: int = 0, stream=None):
        stream = stream or torch.cuda.current_stream()
        self.ctx, self.stream = ctx, stream
        gen = torch.Generator(device="cpu").manual_seed(B * 1_000_003 + n)
        plan = ctx.plan(n, s, B)
        galois = ctx.plan_galois(plan)
        secret = torch.randint(-1, 2, (ctx.N,), generator=gen, dtype=torch.int8)
        sk = ctx.secret_prepare(secret, stream=stream)
        keys = ctx._u64(len(galois) * ctx.key_elems)
        kv = keys.view(len(galois), -1)
        for i, k in enumerate(galois):
            a = torch.stack([torch.randint(0, 1 << 62, (ctx.ndigits, ctx.N), generator=gen,
                                           dtype=torch.int64) % q for q in ctx.moduli], dim=1)
            e = torch.randint(-3, 4, (ctx.ndigits, ctx.N), generator=gen, dtype=torch.int32)
            ctx.rotkey_gen(sk, k, a.contiguous(), e, out=kv[i], stream=stream)
        values = torch.randint(0, ctx.t, (n,), generator=gen, dtype=torch.int32)
        db = ctx.db_encode(values, stream=stream)
        consts = ctx.plan_constants(plan, stream=stream)
        slots = torch.zeros(plan.J * ctx.N, dtype=torch.int32)
        slots[torch.randperm(n, generator=gen)[:s]] = 1
        a = torch.stack([torch.randint(0, 1 << 62, (plan.J, ctx.N), generator=gen,
                                       dtype=torch.int64) % q for q in ctx.moduli[:ctx.L]], dim=1)
        e = torch.randint(-3, 4, (plan.J, ctx.N), generator=gen, dtype=torch.int32)
        v_cts = ctx.encrypt(sk, slots, a.contiguous(), e, stream=stream)
        self.plan = plan
        self.bufs = dict(v_cts=v_cts, db=db, keys=keys, galois=galois, consts=consts,
                         ws=ctx.answer_workspace(plan), out=ctx._u64(plan.n_out * ctx.ct_elems))

    def run(self):
        b = self.bufs
        self.ctx.answer(self.plan, b["v_cts"], b["db"], b["keys"], b["galois"], b["consts"],
                        ws=b["ws"], out=b["out"], stream=self.stream)

    def time(self, reps: int = 3) -> float:
        """Milliseconds per Answer (CUDA events on the stream, after one warm-up)."""
        self.run()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(self.stream)
        for _ in range(reps):
            self.run()
        ev[1].record(self.stream)
        ev[1].synchronize()
        return ev[0].elapsed_time(ev[1]) / reps

    def close(self):
        self.bufs = {}
        torch.cuda.empty_cache()


# knob -> candidate values (0: the library's rule)
SCHEDULE_KNOBS = {"ntt_row_bits": [8, 9, 10], "mac_tiles": [2, 4, 8], "mac_bc": [8, 16],
                  "ntt_chunk": [256, 1024]}


def schedule_candidates(ctx: pdq.Context, knob: str) -> list[int]:
    vals = SCHEDULE_KNOBS[knob]
    if knob == "ntt_row_bits":       # two-phase transforms (N > 2^11), both phases <= 2^11
        vals = [r for r in vals if ctx.log_n > 11 and r < ctx.log_n and ctx.log_n - r <= 11]
    return [0] + vals


class ScheduleTuner:
    """Coordinate descent over the launch-schedule knobs of a context, timed on
    one Answer shape; persisted like PlanTuner's choices."""

    def __init__(self, path: str | None = None, reps: int = 3, min_gain: float = 0.01):
        self.path = path
        self.reps = reps
        # a knob leaves the library's rule only for a gain above this fraction
        # (smaller differences are run-to-run noise)
        self.min_gain = min_gain
        self.cache: dict = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.cache = json.load(f)

    save = PlanTuner.save

    def best(self, ctx: pdq.Context, n: int, s: int, B: int = 0, stream=None) -> dict:
        """The fastest schedule for Answers of n records and sparsity s (plan
        B) on ctx; the context is left on it."""
        key = "schedule:" + shape_key(ctx, n, s) + f":B{B}"
        with _LOCK:
            hit = self.cache.get(key)
        if hit is None:
            rig = AnswerRig(ctx, n, s, B, stream)
            cur = {k: 0 for k in SCHEDULE_KNOBS}
            ctx.set_schedule(**cur)
            default_ms = rig.time(self.reps)
            tried = {json.dumps(cur, sort_keys=True): default_ms}
            best_ms = default_ms
            for knob in SCHEDULE_KNOBS:
                for v in schedule_candidates(ctx, knob):
                    cand = dict(cur, **{knob: v})
                    tag = json.dumps(cand, sort_keys=True)
                    if tag not in tried:
                        ctx.set_schedule(**cand)
                        tried[tag] = rig.time(self.reps)
                    if tried[tag] < best_ms * (1 - self.min_gain):
                        best_ms, cur = tried[tag], cand
            rig.close()
            hit = {"schedule": cur, "ms": best_ms, "default_ms": default_ms,
                   "tried": {k: v for k, v in sorted(tried.items())}}
            with _LOCK:
                self.cache[key] = hit
                self.save()
        ctx.set_schedule(**hit["schedule"])
        return hit


def tune_plan(ctx: pdq.Context, n: int, s: int, tuner: PlanTuner | None = None, stream=None):
    """The plan of pdq_plan_make with the tuned B."""
    tuner = tuner or PlanTuner()
    return ctx.plan(n, s, tuner.best(ctx, n, s, stream))


__all__ = ["PlanTuner", "ScheduleTuner", "AnswerRig", "tune_plan", "candidates",
           "schedule_candidates", "shape_key"]
