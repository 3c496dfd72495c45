"""Timing of the CPU oracle for the benchmark's CPU-baseline leg and its
reference arm.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): nothing here is tuned; it
times the oracle's functions as they stand.

A full-size Answer (N = 2^15, n = 2^20) takes the single-threaded oracle
hours, so it is modelled: one of each of the operations an Answer is made of
(a raise of c1, a rotation with its ModDown, an extended-basis rotation, a
ModDown of one polynomial, a Mask product, a diagonal product over Q u P) is
timed at full size and the times are weighted by the oracle's own operation
counts for the plan.  The operations of one Answer are independent across
half-blocks (baby steps, Mask), across (group, giant step) pairs (diagonal
products) and across groups (giant steps, rotate-and-sum), so on P cores the
oracle takes its single-core time over P, with each operation as slow as it
runs while P copies of it run at once: ``all_cores`` times the same sample in
P spawned processes that start each round together.  The model is checked by
whole Answers measured at the small configurations (c1, c2), and the
plaintext closed form of Eq. 1 is timed as the slot-domain reference point.
"""
from __future__ import annotations

import dataclasses
import multiprocessing as mp
import os
import platform
import subprocess
import time

import numpy as np


def _timed(f):
    t0 = time.perf_counter()
    r = f()
    return r, time.perf_counter() - t0


def op_counts(par, plan) -> dict:
    """How many of each sampled operation one Answer (oracle.pdq.answer) runs."""
    from . import pdq as opdq
    levels = opdq.rotsum_levels(par, plan)
    rot_giant = plan.G * (plan.giants - 1)
    return {
        "rotations": plan.J,                                    # Rot_col of each index ciphertext
        "raises": (plan.H if plan.B > 1 else 0) + rot_giant + plan.G * len(levels),
        "ext_rotations": plan.H * (plan.B - 1) + rot_giant + plan.G * sum(r - 1 for _, r in levels),
        "moddowns": rot_giant + plan.G * len(levels) + 2 * plan.G,
        "diag_products": plan.H * plan.B * plan.giants,
        "mask_products": 4 * plan.J,
    }


def _setup(cfg):
    import workloads as W
    from . import bfv, pdq as opdq
    par = bfv.Params.from_config(cfg)
    plan = opdq.make_plan(par, cfg.n, cfg.s)
    sk = W.draw_ternary(par.N, W.rng_for(cfg.seed, 3))
    a, e = W.encryption_randomness(par.q, par.N, 1, cfg.seed)
    ct = bfv.encrypt(par, sk, bfv.encode(par, np.arange(par.N) % par.t), a[0], e[0])
    k = par.galois_rot(1)
    kr = W.rotation_key_randomness(par.ext, par.N, len(par.digits), [k], cfg.seed)
    key = bfv.rotation_key(par, sk, k, *kr[k])
    return dict(par=par, plan=plan, ct=ct, ct_ext=bfv.ct_times_P(par, ct), k=k, key=key,
                pt=opdq.lifted_pt(par, np.arange(par.N) % par.t),
                pt_ext=bfv.lift(par, bfv.encode(par, np.arange(par.N) % par.t), par.ext))


def _sample(s) -> dict:
    """One round: each operation once at full size (two diagonal products)."""
    from . import bfv, pdq as opdq
    par, ct, ct_ext, k, key = s["par"], s["ct"], s["ct_ext"], s["k"], s["key"]
    raised, t_raise = _timed(lambda: bfv.mod_up_all(par, ct[1]))
    _, t_apply = _timed(lambda: bfv.rotate_hoisted(par, ct, raised, k, key))
    _, t_ext = _timed(lambda: bfv.rotate_ext_lazy(par, ct_ext, raised, k, key))
    _, t_down = _timed(lambda: bfv.mod_down(par, ct_ext[1]))
    _, t_ptmul = _timed(lambda: bfv.pt_mul(par, ct, s["pt"]))
    nmac = 2
    _, t = _timed(lambda: opdq.ring_dot_ext(par, [s["pt_ext"]] * nmac, [ct_ext] * nmac))
    times = {"raise": t_raise, "rotation": t_apply, "ext_rotation": t_ext, "moddown": t_down,
             "mask_product": t_ptmul, "diag_product": t / nmac}
    n = op_counts(par, s["plan"])
    per_query = (n["rotations"] * (t_raise + t_apply) + n["raises"] * t_raise
                 + n["ext_rotations"] * t_ext + n["moddowns"] * t_down
                 + n["diag_products"] * times["diag_product"] + n["mask_products"] * t_ptmul)
    return {"times_s": times, "seconds_per_query": per_query,
            "sampled_s": t_raise + t_apply + t_ext + t_down + t_ptmul + t}


def single_thread(cfg) -> dict:
    """The sample in this process, one thread."""
    return _sample(_setup(cfg))


def _worker(cfg_fields: dict, rounds: int, barrier, queue) -> None:
    import workloads as W
    cfg = W.Config(**cfg_fields)
    s = _setup(cfg)
    for _ in range(rounds):
        barrier.wait()
        queue.put(_sample(s))


def all_cores(cfg, procs: int | None = None, rounds: int = 1, timeout_s: float = 900.0):
    """The sample in `procs` spawned processes (default: every host core),
    `rounds` times, each round started together.  Returns, per round, the
    modelled seconds per query on `procs` cores (the mean per-process model
    over procs) and the round's wall time."""
    procs = procs or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs)
    queue = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(dataclasses.asdict(cfg), rounds, barrier, queue),
                      daemon=True) for _ in range(procs)]
    for p in ps:
        p.start()
    out = []
    try:
        for _ in range(rounds):
            t0 = time.perf_counter()
            res = [queue.get(timeout=timeout_s) for _ in range(procs)]
            wall = time.perf_counter() - t0
            spq = float(np.mean([r["seconds_per_query"] for r in res])) / procs
            out.append({"seconds_per_query": spq, "round_wall_s": wall,
                        "sampled_s_per_process": float(np.mean([r["sampled_s"] for r in res]))})
    finally:
        for p in ps:
            p.join(timeout=30)
            if p.is_alive():
                p.terminate()
    return procs, out


def answer_seconds(cfg) -> float:
    """One whole oracle Answer (Mask then Comp), single thread; keys and the
    encrypted query are made before the clock starts."""
    import workloads as W
    from . import bfv, pdq as opdq
    par = bfv.Params.from_config(cfg)
    plan = opdq.make_plan(par, cfg.n, cfg.s)
    q = W.draw_query(cfg)
    a, e = W.encryption_randomness(par.q, par.N, plan.J, cfg.seed)
    v = opdq.encrypt_index(par, q.sk, q.v, plan, a, e)
    gal = opdq.galois_elements(par, plan)
    kr = W.rotation_key_randomness(par.ext, par.N, len(par.digits), gal, cfg.seed)
    keys = {k: bfv.rotation_key(par, q.sk, k, *kr[k]) for k in gal}
    _, t = _timed(lambda: opdq.answer(par, v, q.db, keys, plan))
    return t


def closed_form_seconds(cfg) -> float:
    """The plaintext result C v, C d of Eq. 1 straight in Z_t (numpy)."""
    import workloads as W
    from . import bfv, pdq as opdq
    par = bfv.Params.from_config(cfg)
    plan = opdq.make_plan(par, cfg.n, cfg.s)
    q = W.draw_query(cfg)
    _, t = _timed(lambda: opdq.closed_form(par, plan, q.v, q.db))
    return t


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


def baseline(cfg, procs: int | None = None, checks=("c1", "c2")) -> dict:
    """The benchmark's cpu_baseline object for workload cfg: the oracle on all
    host cores (value), single-threaded, the model checked against whole
    Answers measured at the small configurations, and the closed form."""
    import workloads as W
    st = single_thread(cfg)
    procs, rounds = all_cores(cfg, procs)
    par_spq = rounds[0]["seconds_per_query"]
    checked = {}
    for name in checks:
        c = W.CONFIGS[name]
        checked[name] = {"measured_s": answer_seconds(c),
                         "model_s": single_thread(c)["seconds_per_query"]}
    closed = closed_form_seconds(cfg)
    t = st["times_s"]
    return {
        "value": 1.0 / par_spq, "unit": "queries/s", "cores": procs, "kind": "oracle",
        "cpu_model": cpu_model(), "nproc": os.cpu_count(),
        "seconds_per_query": par_spq,
        "single_thread": {"value": 1.0 / st["seconds_per_query"], "unit": "queries/s",
                          "seconds_per_query": st["seconds_per_query"], "op_times_s": t},
        "all_cores_round_wall_s": rounds[0]["round_wall_s"],
        "closed_form_s": closed,
        **{f"{k}_measured_s": v["measured_s"] for k, v in checked.items()},
        **{f"{k}_model_s": v["model_s"] for k, v in checked.items()},
        "sample": (f"oracle (plain C + Python, untuned) timed on one full-size raise, rotation "
                   f"with ModDown, extended-basis rotation, polynomial ModDown, Mask product and "
                   f"two diagonal products over Q u P ({st['sampled_s']:.1f} s single-thread), "
                   f"weighted by the oracle's operation counts per Answer "
                   f"({st['seconds_per_query']:.0f} s per query on one core); the same sample "
                   f"in {procs} processes at once gives {par_spq:.0f} s per query on {procs} "
                   f"cores (the Answer's operations are independent across half-blocks, "
                   f"giant steps and groups); model checked against whole Answers measured at "
                   + ", ".join(f"{k} ({v['measured_s']:.2f} s measured, {v['model_s']:.2f} s "
                               f"modelled)" for k, v in checked.items())
                   + f"; closed form of Eq. 1 in Z_t {closed:.2f} s"),
    }
