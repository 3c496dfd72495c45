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


def _oracle_imports(path):
    """(enclosing function, imported module or name) for every import of the
    oracle in a Python file."""
    import ast
    tree = ast.parse(path.read_text())
    found = []

    def walk(node, fn):
        for ch in ast.iter_child_nodes(node):
            if isinstance(ch, (ast.FunctionDef, ast.AsyncFunctionDef)):
                walk(ch, ch.name)
                continue
            if isinstance(ch, ast.Import):
                found.extend((fn, a.name) for a in ch.names if a.name.split(".")[0] == "oracle")
            elif isinstance(ch, ast.ImportFrom) and (ch.module or "").split(".")[0] == "oracle":
                found.extend((fn, f"{ch.module}.{a.name}") for a in ch.names)
            walk(ch, fn)

    walk(tree, None)
    return found


def test_benchmark_reaches_the_oracle_only_for_the_cpu_baseline():
    """bench.py imports nothing of the oracle but its timing module, and only
    in the reference arm and the cpu_baseline leg; __graft_entry__ only in
    build() (compiling the oracle's C core) and smoke() (the check)."""
    bench = _oracle_imports(ROOT / "bench.py")
    assert bench and all(mod == "oracle.baseline" for _, mod in bench), bench
    assert {fn for fn, _ in bench} <= {"run_reference", "run_gpu"}, bench
    text = (ROOT / "bench.py").read_text()
    # inside run_gpu the import sits under the cpu_baseline leg alone
    i = text.index("def run_gpu(")
    body = text[i:text.index("\ndef ", i + 1)]
    j = body.index("from oracle import baseline")
    assert "no_cpu_baseline" in body[max(0, j - 120):j]
    assert 'line["cpu_baseline"] = baseline.baseline(' in body[j:j + 120]
    entry = _oracle_imports(ROOT / "__graft_entry__.py")
    assert entry and {fn for fn, _ in entry} <= {"build", "smoke"}, entry
