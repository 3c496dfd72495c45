"""The library and the oracle stay independent: no source of the product
package (its Python modules and the CUDA/C++ of libpdq.so) imports, includes
or loads anything under oracle/, and no oracle source reaches into the
package.  The one module both sides use is workloads/ (random draws only),
which itself imports neither."""
import pathlib
import re

ROOT = pathlib.Path(__file__).resolve().parents[1]
PKG = ROOT / "paper_2408_17063_gb300"
ORACLE = ROOT / "oracle"
WORKLOADS = ROOT / "workloads"

_SOURCES = ("*.py", "*.cu", "*.cuh", "*.h", "*.cpp", "*.c")


def _files(base):
    for pat in _SOURCES:
        for f in base.rglob(pat):
            if "_build" not in f.parts and "__pycache__" not in f.parts:
                yield f


def _hits(files, pattern):
    rx = re.compile(pattern)
    return [f"{f.relative_to(ROOT)}:{i}: {line.strip()}"
            for f in files
            for i, line in enumerate(f.read_text(errors="replace").splitlines(), 1)
            if rx.search(line)]


def test_product_never_reaches_the_oracle():
    files = list(_files(PKG))
    assert files, "no product sources found"
    hits = _hits(files, r"(\bimport\s+oracle\b|\bfrom\s+oracle\b|#\s*include\s*[<\"][^>\"]*oracle"
                        r"|oracle/|ref_ring|importlib.*oracle)")
    assert not hits, "product sources reach the oracle:\n" + "\n".join(hits)


def test_oracle_never_reaches_the_product():
    files = list(_files(ORACLE))
    assert files, "no oracle sources found"
    hits = _hits(files, r"(\bimport\s+paper_2408_17063_gb300|\bfrom\s+paper_2408_17063_gb300"
                        r"|libpdq|csrc/|#\s*include\s*\"pdq)")
    assert not hits, "oracle sources reach the product:\n" + "\n".join(hits)


def test_shared_input_module_imports_neither_side():
    files = list(_files(WORKLOADS))
    assert files
    hits = _hits(files, r"(\bimport\s+oracle\b|\bfrom\s+oracle\b|paper_2408_17063_gb300)")
    assert not hits, "workloads/ imports a side:\n" + "\n".join(hits)
