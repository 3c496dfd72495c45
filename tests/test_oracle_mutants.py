"""The oracle's planted-mistake list stays applicable, and a sample of it is
killed by the pins here (the whole list: ``python -m oracle.mutants``)."""
import pytest

from oracle import mutants as M


def test_every_mutant_applies_to_the_current_oracle():
    names = [m.name for m in M.MUTANTS]
    assert len(names) == len(set(names)) and len(names) >= 70
    for m in M.MUTANTS:
        M.check(m)
    # every oracle source is covered
    assert {m.path for m in M.MUTANTS} == {"oracle/ref_ring.c", "oracle/ring.py", "oracle/bfv.py",
                                           "oracle/pdq.py"}


SAMPLE = ["automorphism_no_sign", "delta_off_by_one", "row_mask_short", "no_consistency_rows"]


def test_a_sample_of_mutants_is_killed():
    res = M.run(SAMPLE, jobs=len(SAMPLE))
    assert {name: verdict for name, (verdict, _) in res.items()} == {n: "killed" for n in SAMPLE}, res


@pytest.mark.parametrize("name", ["automorphism_no_sign"])
def test_a_mutant_is_applied_to_a_copy_only(name):
    """Running a mutant leaves the repository's own oracle untouched."""
    m = next(x for x in M.MUTANTS if x.name == name)
    before = open(f"{M.ROOT}/{m.path}").read()
    M.run_one(m)
    assert open(f"{M.ROOT}/{m.path}").read() == before
