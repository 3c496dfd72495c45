"""The benchmark's reference arm (the CPU oracle on a bounded sample of the
c3 workload) runs without a GPU and prints one JSON line with the fields the
benchmark contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "queries/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["ms_per_step"] > 0
    assert d["config"]["N"] == 1 << 15 and d["config"]["n"] == 1 << 20 and d["config"]["s"] == 256
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == os.cpu_count() and cb["value"] == d["value"]
    assert isinstance(cb["sample"], str) and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_oracle_baseline_counts_and_model():
    """The operation counts of the CPU model are the oracle's own: at the c1
    plan (J = 1, H = 2, B = 8, 2 giant steps, one group, one rotate-and-sum
    level of 8) they are those of oracle.pdq.answer, and the model of a c1
    Answer is within a factor of two of a measured one."""
    import workloads as W
    from oracle import baseline, bfv, pdq as opdq
    cfg = W.CONFIGS["c1"]
    par = bfv.Params.from_config(cfg)
    plan = opdq.make_plan(par, cfg.n, cfg.s)
    assert (plan.J, plan.H, plan.B, plan.giants, plan.G) == (1, 2, 8, 2, 1)
    assert opdq.rotsum_levels(par, plan) == [(16, 8), (128, 4), (512, 4)]
    n = baseline.op_counts(par, plan)
    # Rot_col once; raises: 2 baby + 1 giant + 3 levels; extended rotations:
    # 2*7 baby + 1 giant + 7+3+3 rotate-and-sum; ModDowns: 1 + 3 + 2
    assert n == {"rotations": 1, "raises": 6, "ext_rotations": 28, "moddowns": 6,
                 "diag_products": 32, "mask_products": 4}
    model = baseline.single_thread(cfg)["seconds_per_query"]
    measured = baseline.answer_seconds(cfg)
    assert 0.5 < model / measured < 2.0
