"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point declared in include/pdq.h, each citing its passage; a plain C99
client compiles and links against it (no compute calls)."""
import ctypes
import re

from paper_2408_17063_gb300 import build


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    from paper_2408_17063_gb300 import pdq
    declared = pdq.header_symbols()
    assert len(declared) >= 25
    missing = [s for s in declared if not hasattr(lib, s)]
    assert missing == []
    # the binding covers every declared entry point and nothing else
    assert sorted(pdq._SIGS) == declared


_DECL = re.compile(r"^\s*(?:const\s+)?(?:int|size_t|void|unsigned long long|uint\d+_t|const char\*)"
                   r"\s*\*?\s*(pdq_[a-z0-9_]+)\s*\(")
_CITES = re.compile(r"(Sec\.|Alg\.|Eq\.|Def\.|Table|[Rr]emark)")
_NO_COUNTERPART = re.compile(r"(no operation of the paper|not part of the paper|[Nn]ot part of the "
                             r"paper's method|no counterpart|library bookkeeping)")


def _declarations_with_comments():
    """(name, the comment block that precedes its declaration group) for every
    function declared in include/pdq.h."""
    lines = open(build.os.path.join(build.INCLUDE, "pdq.h")).read().splitlines()
    out, last, cur, in_comment = [], "", [], False
    for ln in lines:
        s = ln.strip()
        if in_comment:
            cur.append(s)
            if "*/" in s:
                in_comment, last = False, " ".join(cur)
            continue
        if s.startswith("/*"):
            cur = [s]
            if "*/" in s:
                last = s
            else:
                in_comment = True
            continue
        m = _DECL.match(ln)
        if m:
            out.append((m.group(1), last))
    return out


def test_header_cites_the_passage_of_every_entry_point():
    """Each entry point's comment names the passage of the paper it follows
    (section, algorithm, equation, definition, table or remark), or says that
    the paper has no counterpart (bookkeeping, workspaces, instrumentation)."""
    decls = _declarations_with_comments()
    from paper_2408_17063_gb300 import pdq
    assert sorted(n for n, _ in decls) == pdq.header_symbols()
    bare = [n for n, c in decls if not (_CITES.search(c) or _NO_COUNTERPART.search(c))]
    assert bare == [], f"entry points without a cited passage: {bare}"


_C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "pdq.h"

int main(void) {
    pdq_ctx* ctx = NULL;
    pdq_schedule sched;
    int rc;
    if (pdq_launch_count() != 0) return 10;
    if (pdq_rotate_noalloc_max_bytes() != (size_t)32 << 20) return 11;
    /* refusals come back as codes with a message, never as a crash */
    rc = pdq_ctx_create(NULL, &ctx);
    if (rc != PDQ_E_PARAM || ctx != NULL) return 12;
    if (strlen(pdq_last_error()) == 0) return 13;
    if (pdq_ctx_destroy(NULL) != PDQ_OK) return 14;
    memset(&sched, 0, sizeof sched);
    if (pdq_ctx_set_schedule(NULL, &sched) != PDQ_E_PARAM) return 15;
    printf("ok %s\n", pdq_last_error());
    return 0;
}
"""


def test_c_client_compiles_links_and_gets_error_codes(tmp_path):
    """The boundary is a C ABI: a C99 program (no C++ and no Python) compiles
    against include/pdq.h with -pedantic -Werror, links libpdq.so and gets
    error codes and messages back from refused calls (no GPU is touched)."""
    import shutil
    import subprocess
    import pytest
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    path = build.build()
    src = tmp_path / "client.c"
    src.write_text(_C_CLIENT)
    exe = tmp_path / "client"
    libdir = build.os.path.dirname(path)
    cmd = [cc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I", build.INCLUDE,
           str(src), "-o", str(exe), f"-L{libdir}", f"-l:{build.os.path.basename(path)}",
           f"-Wl,-rpath,{libdir}"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, (run.returncode, run.stdout, run.stderr)
    assert run.stdout.startswith("ok ")


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2408_17063_gb300 import pdq
    monkeypatch.setattr(pdq, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pdq, "_lib", None)
    import pytest
    with pytest.raises(ImportError):
        pdq.load()


def test_context_refuses_bad_parameters_before_any_device_work():
    """pdq_ctx_create checks the parameter set of Sec. 5.1 (ring, prime t =
    1 mod 2N, chain and digit counts) on the host and returns PDQ_E_PARAM with
    a message, leaving *out NULL, before it touches a device."""
    from paper_2408_17063_gb300 import pdq
    lib = pdq.load()
    good = dict(log_n=10, prime_bits=40, L=2, K=1, dnum=2, t=65537)
    bad = [dict(log_n=2), dict(log_n=17), dict(prime_bits=19), dict(prime_bits=61),
           dict(L=0), dict(L=31), dict(K=0), dict(K=9), dict(dnum=0), dict(dnum=3),
           dict(t=65539), dict(t=12289 * 2 + 1), dict(t=7681), dict(t=2),
           dict(log_n=16, t=65537),              # 65536 is not a multiple of 2^17
           dict(prime_bits=20, L=30, K=8)]       # too few primes = 1 mod 2N below 2^20
    for change in bad:
        p = pdq.Params(**{**good, **change})
        out = ctypes.c_void_p(1234)
        rc = lib.pdq_ctx_create(ctypes.byref(p), ctypes.byref(out))
        assert rc == pdq.PDQ_E_PARAM, (change, rc, lib.pdq_last_error())
        assert out.value is None
        assert lib.pdq_last_error()


def test_every_entry_point_refuses_null_arguments():
    """Called with every pointer NULL and every number 0, each entry point
    returns an error code with a message (an int call), or 0 (a size query),
    without touching memory or a device: NULL is never dereferenced across
    the ABI.  Destroying NULL is a no-op that succeeds."""
    from paper_2408_17063_gb300 import pdq
    lib = pdq.load()
    no_error = {"pdq_ctx_destroy", "pdq_server_destroy"}
    not_calls = {"pdq_last_error", "pdq_launch_count", "pdq_rotate_noalloc_max_bytes"}
    for name, (res, args) in sorted(pdq._SIGS.items()):
        if name in not_calls:
            continue
        vals = [None if (a is pdq._P or (isinstance(a, type) and issubclass(a, ctypes._Pointer)))
                else 0 for a in args]
        rc = getattr(lib, name)(*vals)
        if res is pdq._SZ:
            assert rc == 0, name
        elif name in no_error:
            assert rc == pdq.PDQ_OK, name
        else:
            assert rc == pdq.PDQ_E_PARAM, (name, rc)
            assert lib.pdq_last_error(), name
