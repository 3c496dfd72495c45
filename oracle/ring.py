"""Limb-wise ring arithmetic of the oracle (ctypes over ref_ring.c).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

A polynomial over an RNS basis is a uint64 array [limbs][N] of canonical
residues, limb i modulo moduli[i], in coefficient form.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

_lib = ctypes.CDLL(_build.build())
_u64p = ctypes.POINTER(ctypes.c_uint64)
_u64 = ctypes.c_uint64

for name, args, res in [
    ("ref_powmod", [_u64, _u64, _u64], _u64),
    ("ref_invmod", [_u64, _u64], _u64),
    ("ref_vec_mul", [_u64p, _u64p, _u64p, _u64, _u64], None),
    ("ref_vec_mac", [_u64p, _u64p, _u64p, _u64, _u64], None),
    ("ref_vec_add", [_u64p, _u64p, _u64p, _u64, _u64], None),
    ("ref_vec_sub", [_u64p, _u64p, _u64p, _u64, _u64], None),
    ("ref_vec_scale", [_u64p, _u64, _u64p, _u64, _u64], None),
    ("ref_negacyclic_schoolbook", [_u64p, _u64p, _u64p, _u64, _u64], None),
    ("ref_ntt_forward", [_u64p, ctypes.c_int, _u64, _u64], None),
    ("ref_ntt_inverse", [_u64p, ctypes.c_int, _u64, _u64], None),
    ("ref_negacyclic_mul", [_u64p, _u64p, _u64p, ctypes.c_int, _u64, _u64], None),
    ("ref_automorphism", [_u64p, _u64p, _u64, _u64, _u64], None),
    ("ref_basis_convert", [_u64p, _u64p, _u64p, _u64, _u64p, _u64, _u64p, _u64], None),
    ("ref_vec_reduce", [_u64p, _u64p, _u64, _u64], None),
]:
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res


def _p(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"], (a.dtype, a.flags)
    return a.ctypes.data_as(_u64p)


def _u(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint64)


def powmod(a: int, e: int, q: int) -> int:
    return int(_lib.ref_powmod(a % q, e, q))


def invmod(a: int, q: int) -> int:
    return int(_lib.ref_invmod(a % q, q))


def log2_exact(N: int) -> int:
    lg = N.bit_length() - 1
    assert 1 << lg == N
    return lg


# ---- single-limb operations --------------------------------------------------

def ntt_forward(a, q: int, psi: int) -> np.ndarray:
    """Values a(psi^{2j+1}), j = 0..N-1 (natural order)."""
    x = _u(a).copy()
    _lib.ref_ntt_forward(_p(x), log2_exact(x.shape[-1]), q, psi)
    return x


def ntt_inverse(a, q: int, psi: int) -> np.ndarray:
    x = _u(a).copy()
    _lib.ref_ntt_inverse(_p(x), log2_exact(x.shape[-1]), q, psi)
    return x


def schoolbook(a, b, q: int) -> np.ndarray:
    a, b = _u(a), _u(b)
    c = np.empty_like(a)
    _lib.ref_negacyclic_schoolbook(_p(a), _p(b), _p(c), a.shape[-1], q)
    return c


def negacyclic_mul(a, b, q: int, psi: int) -> np.ndarray:
    a, b = _u(a), _u(b)
    c = np.empty_like(a)
    _lib.ref_negacyclic_mul(_p(a), _p(b), _p(c), log2_exact(a.shape[-1]), q, psi)
    return c


def automorphism(a, k: int, q: int) -> np.ndarray:
    a = _u(a)
    out = np.empty_like(a)
    _lib.ref_automorphism(_p(a), _p(out), a.shape[-1], k % (2 * a.shape[-1]), q)
    return out


def vec_mul(a, b, q: int) -> np.ndarray:
    a, b = _u(a), _u(b)
    c = np.empty_like(a)
    _lib.ref_vec_mul(_p(a), _p(b), _p(c), a.size, q)
    return c


def vec_add(a, b, q: int) -> np.ndarray:
    a, b = _u(a), _u(b)
    c = np.empty_like(a)
    _lib.ref_vec_add(_p(a), _p(b), _p(c), a.size, q)
    return c


def vec_sub(a, b, q: int) -> np.ndarray:
    a, b = _u(a), _u(b)
    c = np.empty_like(a)
    _lib.ref_vec_sub(_p(a), _p(b), _p(c), a.size, q)
    return c


def vec_scale(a, w: int, q: int) -> np.ndarray:
    a = _u(a)
    c = np.empty_like(a)
    _lib.ref_vec_scale(_p(a), w % q, _p(c), a.size, q)
    return c


def vec_reduce(a, r: int) -> np.ndarray:
    a = _u(a)
    c = np.empty_like(a)
    _lib.ref_vec_reduce(_p(a), _p(c), a.size, r)
    return c


def basis_convert(x, src, r: int) -> np.ndarray:
    """Fast basis conversion of x ([len(src)][N], residues modulo the primes
    src) to the prime r:  sum_i [x_i * (S/s_i)^{-1}]_{s_i} * (S/s_i)  mod r,
    S = prod(src).  No overflow correction."""
    x = _u(x)
    src = [int(s) for s in src]
    S = 1
    for s in src:
        S *= s
    hat_inv = _u([invmod((S // s) % s, s) for s in src])
    hat_mod_r = _u([(S // s) % r for s in src])
    srcs = _u(src)
    y = np.empty(x.shape[-1], dtype=np.uint64)
    _lib.ref_basis_convert(_p(x), _p(srcs), _p(hat_inv), len(src), _p(hat_mod_r), r,
                           _p(y), x.shape[-1])
    return y
