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
        stream = stream or torch.cuda.current_stream()
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
        ws = ctx.answer_workspace(plan)
        out = ctx._u64(plan.n_out * ctx.ct_elems)

        def run():
            ctx.answer(plan, v_cts, db, keys, galois, consts, ws=ws, out=out, stream=stream)

        run()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        for _ in range(self.reps):
            run()
        ev[1].record(stream)
        ev[1].synchronize()
        ms = ev[0].elapsed_time(ev[1]) / self.reps
        del keys, consts, ws, out, v_cts, db, sk
        torch.cuda.empty_cache()
        return ms


def tune_plan(ctx: pdq.Context, n: int, s: int, tuner: PlanTuner | None = None, stream=None):
    """The plan of pdq_plan_make with the tuned B."""
    tuner = tuner or PlanTuner()
    return ctx.plan(n, s, tuner.best(ctx, n, s, stream))


__all__ = ["PlanTuner", "tune_plan", "candidates", "shape_key"]
