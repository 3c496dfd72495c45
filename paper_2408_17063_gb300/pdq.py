"""Python binding of the PDQ C ABI (include/pdq.h).

Argument marshalling only: every function forwards to the entry point of the
same name in ``_lib/libpdq.so``; tensors are passed as device pointers and
sizes.  PyTorch supplies device memory and streams.  There is no fallback:
if the compiled library is missing, loading raises.

The ``Context`` class bundles a ``pdq_ctx`` with its parameters and offers
the same calls with workspace allocation from PyTorch's caching allocator.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libpdq.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pdq.h")

PDQ_OK, PDQ_E_PARAM, PDQ_E_NOMEM, PDQ_E_CUDA, PDQ_E_DECODE, PDQ_E_KEY = 0, 1, 2, 3, 4, 5
PDQ_E_TIMEOUT, PDQ_E_BUSY = 6, 7
PDQ_REQ_QUEUED, PDQ_REQ_RUNNING, PDQ_REQ_DONE = 0, 1, 2
MAX_MODULI = 40


class PdqError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pdq error {code}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_uint32), ("prime_bits", ctypes.c_uint32),
                ("L", ctypes.c_uint32), ("K", ctypes.c_uint32), ("dnum", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("t", ctypes.c_uint64)]


class Info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint32), ("L", ctypes.c_uint32), ("K", ctypes.c_uint32),
                ("ndigits", ctypes.c_uint32), ("t", ctypes.c_uint64), ("zeta", ctypes.c_uint64),
                ("moduli", ctypes.c_uint64 * MAX_MODULI), ("psi", ctypes.c_uint64 * MAX_MODULI)]


class Schedule(ctypes.Structure):
    _fields_ = [("ntt_row_bits", ctypes.c_uint32), ("mac_tiles", ctypes.c_uint32),
                ("mac_bc", ctypes.c_uint32), ("ntt_chunk", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {"ntt_row_bits": self.ntt_row_bits, "mac_tiles": self.mac_tiles,
                "mac_bc": self.mac_bc, "ntt_chunk": self.ntt_chunk}


class Plan(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64)] + [(f, ctypes.c_uint32) for f in (
        "s", "s_prime", "B", "giants", "J", "H", "G_sz", "hpg", "G", "hclass", "per_out",
        "n_out", "ring_ratio", "plain_db")]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class Query(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("v_cts", ctypes.c_void_p), ("db", ctypes.c_void_p),
                ("keys", ctypes.c_void_p), ("galois", ctypes.c_void_p),
                ("nkeys", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("consts", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class TicketInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32),
                ("t_submit_ns", ctypes.c_uint64), ("t_start_ns", ctypes.c_uint64),
                ("t_done_ns", ctypes.c_uint64), ("stacked", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


_P = ctypes.c_void_p
_U32 = ctypes.c_uint32
_U64 = ctypes.c_uint64
_SZ = ctypes.c_size_t
_I = ctypes.c_int

_SIGS = {
    "pdq_ctx_create": (_I, [ctypes.POINTER(Params), ctypes.POINTER(_P)]),
    "pdq_ctx_destroy": (_I, [_P]),
    "pdq_ctx_info": (_I, [_P, ctypes.POINTER(Info)]),
    "pdq_last_error": (ctypes.c_char_p, []),
    "pdq_ntt_forward": (_I, [_P, _P, _U32, _U32, _U32, _U64, _P]),
    "pdq_ntt_inverse": (_I, [_P, _P, _U32, _U32, _U32, _U64, _P]),
    "pdq_encode": (_I, [_P, _P, _U32, _U32, _P, _P]),
    "pdq_secret_prepare": (_I, [_P, _P, _P, _P]),
    "pdq_encrypt": (_I, [_P, _P, _P, _U32, _P, _P, _P, _P]),
    "pdq_rotkey_gen": (_I, [_P, _P, _U64, _P, _P, _P, _P]),
    "pdq_decrypt_workspace_bytes": (_SZ, [_P, _U32]),
    "pdq_decrypt": (_I, [_P, _P, _P, _U32, _P, _P, _SZ, _P]),
    "pdq_mod_switch_workspace_bytes": (_SZ, [_P, _U32]),
    "pdq_mod_switch": (_I, [_P, _P, _P, _U32, _P, _P, _SZ, _P]),
    "pdq_rotate_workspace_bytes": (_SZ, [_P, _U32]),
    "pdq_rotate": (_I, [_P, _P, _U32, _U64, _P, _P, _P, _SZ, _P]),
    "pdq_ctx_set_rotation_budget": (_I, [_P, _U64]),
    "pdq_ctx_set_schedule": (_I, [_P, ctypes.POINTER(Schedule)]),
    "pdq_ctx_get_schedule": (_I, [_P, ctypes.POINTER(Schedule)]),
    "pdq_plan_make": (_I, [_P, _U64, _U32, _U32, ctypes.POINTER(Plan)]),
    "pdq_plan_make_client": (_I, [_U64, _U32, _U64, _U32, _U32, ctypes.POINTER(Plan)]),
    "pdq_plan_galois_client": (_I, [_U64, _U32, ctypes.POINTER(Plan), _P, _U32,
                                    ctypes.POINTER(_U32)]),
    "pdq_plan_make_switched": (_I, [_P, _U32, _U64, _U32, _U32, ctypes.POINTER(Plan)]),
    "pdq_plan_make_plain_db": (_I, [_P, _U64, _U32, _U32, ctypes.POINTER(Plan)]),
    "pdq_db_diagonals_bytes": (_SZ, [_P, ctypes.POINTER(Plan)]),
    "pdq_db_diagonals_build": (_I, [_P, ctypes.POINTER(Plan), _P, _P, _P]),
    "pdq_answer_plain_db_workspace_bytes": (_SZ, [_P, ctypes.POINTER(Plan)]),
    "pdq_answer_plain_db": (_I, [_P, ctypes.POINTER(Plan), _P, _P, _P, _U32, _P, _P, _P, _SZ,
                                 _P]),
    "pdq_ctx_create_subring": (_I, [_P, _U32, ctypes.POINTER(_P)]),
    "pdq_ring_switch_key_gen": (_I, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "pdq_ring_switch_workspace_bytes": (_SZ, [_P, _U32]),
    "pdq_ring_switch": (_I, [_P, _P, _P, _U32, _U32, _P, _P, _P, _SZ, _P]),
    "pdq_plan_galois": (_I, [_P, ctypes.POINTER(Plan), _P, _U32, ctypes.POINTER(_U32)]),
    "pdq_plan_constants_bytes": (_SZ, [_P, ctypes.POINTER(Plan)]),
    "pdq_plan_constants_build": (_I, [_P, ctypes.POINTER(Plan), _P, _P]),
    "pdq_db_bytes": (_SZ, [_P, _U64]),
    "pdq_db_encode": (_I, [_P, _P, _U64, _P, _P]),
    "pdq_mask": (_I, [_P, ctypes.POINTER(Plan), _P, _P, _P, _P]),
    "pdq_db_plain_bytes": (_SZ, [_P, _U64]),
    "pdq_db_encode_plain": (_I, [_P, _P, _U64, _P, _P]),
    "pdq_mask_literal": (_I, [_P, ctypes.POINTER(Plan), _P, _P, _P, _P]),
    "pdq_comp_workspace_bytes": (_SZ, [_P, ctypes.POINTER(Plan)]),
    "pdq_comp": (_I, [_P, ctypes.POINTER(Plan), _P, _P, _P, _U32, _P, _P, _P, _SZ, _P]),
    "pdq_answer_workspace_bytes": (_SZ, [_P, ctypes.POINTER(Plan)]),
    "pdq_answer": (_I, [_P, ctypes.POINTER(Plan), _P, _P, _P, _P, _U32, _P, _P, _P, _SZ, _P]),
    "pdq_answer_stacked_workspace_bytes": (_SZ, [_P, ctypes.POINTER(Plan), _U32]),
    "pdq_answer_stacked": (_I, [_P, ctypes.POINTER(Plan), _U32, _P, _P, _P, _P, _U32, _P, _P, _P,
                                _SZ, _P]),
    "pdq_answer_host_workspace_bytes": (_SZ, [_P, ctypes.POINTER(Plan)]),
    "pdq_answer_host": (_I, [_P, ctypes.POINTER(Plan), _P, _P, _P, _P, _U32, _P, _P, _P, _SZ,
                             _P]),
    "pdq_decomp": (_I, [_P, ctypes.POINTER(Plan), _P, _P, _P, _U64, ctypes.POINTER(_U64)]),
    "pdq_decomp_client": (_I, [_U64, _U32, ctypes.POINTER(Plan), _P, _P, _P, _U64,
                               ctypes.POINTER(_U64)]),
    "pdq_launch_count": (ctypes.c_ulonglong, []),
    "pdq_answer_batch": (_I, [_P, ctypes.POINTER(Query), _U32, _P, _P, _U32, _P]),
    "pdq_server_create": (_I, [_P, _SZ, _U32, _U32, ctypes.POINTER(_P)]),
    "pdq_server_submit": (_I, [_P, _P, ctypes.POINTER(Query), ctypes.POINTER(_U64)]),
    "pdq_server_status": (_I, [_P, _U64, ctypes.POINTER(TicketInfo)]),
    "pdq_server_wait": (_I, [_P, _U64, _U32]),
    "pdq_server_drain": (_I, [_P, _U32]),
    "pdq_server_set_stacking": (_I, [_P, _U32]),
    "pdq_server_destroy": (_I, [_P]),
    "pdq_cts_serialized_bytes": (_SZ, [_P, _U32]),
    "pdq_cts_export": (_I, [_P, _P, _U32, _P, _SZ, _P, _P]),
    "pdq_cts_import": (_I, [_P, _P, _SZ, _P, _U32, ctypes.POINTER(_U32), _P]),
    "pdq_sk_serialized_bytes": (_SZ, [_P]),
    "pdq_sk_export": (_I, [_P, _P, _P, _SZ, _P, _P]),
    "pdq_sk_import": (_I, [_P, _P, _SZ, _P, _P]),
    "pdq_rotkeys_serialized_bytes": (_SZ, [_P, _U32]),
    "pdq_rotkeys_export": (_I, [_P, _P, _P, _U32, _P, _SZ, _P, _P]),
    "pdq_rotkeys_import": (_I, [_P, _P, _SZ, _P, _P, _U32, ctypes.POINTER(_U32), _P]),
    "pdq_rotate_noalloc_max_bytes": (_SZ, []),
    "pdq_rotate_noalloc": (_I, [_P, _P, _U32, _U64, _P, _P, _P]),
    "pdq_profile_enable": (_I, [_P, _I]),
    "pdq_profile_read": (_I, [_P, _P, _P, _U32]),
}

STAGES = ["mask", "pack", "baby", "mac", "giant", "rotsum", "combine", "acc_moddown"]


def pdq_launch_count() -> int:
    return int(load().pdq_launch_count())

_lib = None


def header_symbols() -> list[str]:
    """Every entry point declared in include/pdq.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(pdq_[a-z0-9_]+)\s*\(", text)))


def load() -> ctypes.CDLL:
    """Load libpdq.so (built by paper_2408_17063_gb300.build); raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2408_17063_gb300.build.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != PDQ_OK:
        raise PdqError(rc, load().pdq_last_error().decode())


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        assert t.is_contiguous(), "tensors passed to the C ABI must be contiguous"
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    return int(t)


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _decomp(call, plan: Plan, slots) -> list[tuple[int, int]]:
    """Marshals one Decomp call: call(plan, slots, idx, val, cap, count)."""
    s = np.ascontiguousarray(torch.as_tensor(slots).cpu().numpy().astype(np.uint32))
    cap = max(1, plan.G * plan.s_prime)
    idx = np.zeros(cap, dtype=np.uint64)
    val = np.zeros(cap, dtype=np.uint32)
    cnt = _U64()
    _check(call(ctypes.byref(plan), _ptr(s), _ptr(idx), _ptr(val), cap, ctypes.byref(cnt)))
    n = cnt.value
    return [(int(i), int(v)) for i, v in zip(idx[:n], val[:n])]


def plan_make_client(t: int, log_n: int, n: int, s: int, B: int = 0) -> Plan:
    """pdq_plan_make_client: the Answer's layout from t and the ring alone."""
    pl = Plan()
    _check(load().pdq_plan_make_client(t, log_n, n, s, B, ctypes.byref(pl)))
    return pl


def plan_galois_client(t: int, log_n: int, plan: Plan) -> list[int]:
    """pdq_plan_galois_client: the plan's Galois elements from t and the ring."""
    lib = load()
    cnt = _U32()
    _check(lib.pdq_plan_galois_client(t, log_n, ctypes.byref(plan), None, 0, ctypes.byref(cnt)))
    arr = (ctypes.c_uint64 * max(1, cnt.value))()
    _check(lib.pdq_plan_galois_client(t, log_n, ctypes.byref(plan), ctypes.cast(arr, _P),
                                      cnt.value, ctypes.byref(cnt)))
    return [int(x) for x in arr[:cnt.value]]


def decomp_client(t: int, log_n: int, plan: Plan, slots) -> list[tuple[int, int]]:
    """pdq_decomp_client: Decomp on the host with no context or GPU; slots
    [n_out][N] decrypted answer; returns sorted (record index, value) pairs."""
    lib = load()
    return _decomp(lambda *a: lib.pdq_decomp_client(t, log_n, *a), plan, slots)


class Context:
    """A parameter set on the current CUDA device (owns a pdq_ctx)."""

    def __init__(self, log_n: int, t: int, prime_bits: int, L: int, K: int, dnum: int,
                 _handle=None):
        lib = load()
        if _handle is None:
            p = Params(log_n, prime_bits, L, K, dnum, 0, t)
            h = _P()
            _check(lib.pdq_ctx_create(ctypes.byref(p), ctypes.byref(h)))
        else:
            h = _handle
        self.h = h
        info = Info()
        _check(lib.pdq_ctx_info(h, ctypes.byref(info)))
        self.N, self.L, self.K, self.ndigits = info.N, info.L, info.K, info.ndigits
        self.t, self.zeta = info.t, info.zeta
        self.m = self.N // 2
        self.E = self.L + self.K
        self.moduli = [int(info.moduli[i]) for i in range(self.E)]
        self.psi = [int(info.psi[i]) for i in range(self.E + 1)]
        self.log_n = log_n

    @classmethod
    def from_config(cls, cfg) -> "Context":
        return cls(cfg.log_n, cfg.t, cfg.prime_bits, cfg.L, cfg.K, cfg.dnum)

    def set_rotation_budget(self, nbytes: int):
        """pdq_ctx_set_rotation_budget: hold at most nbytes of baby-step
        rotations (0: all), made and consumed a chunk of primes at a time."""
        _check(load().pdq_ctx_set_rotation_budget(self.h, int(nbytes)))

    def set_schedule(self, ntt_row_bits: int = 0, mac_tiles: int = 0, mac_bc: int = 0,
                     ntt_chunk: int = 0):
        """pdq_ctx_set_schedule: launch-schedule knobs (0: the library's rule);
        results are the same bits under every schedule."""
        sc = Schedule(ntt_row_bits, mac_tiles, mac_bc, ntt_chunk)
        _check(load().pdq_ctx_set_schedule(self.h, ctypes.byref(sc)))

    def schedule(self) -> dict:
        sc = Schedule()
        _check(load().pdq_ctx_get_schedule(self.h, ctypes.byref(sc)))
        return sc.as_dict()

    def subring(self, log_n: int) -> "Context":
        """pdq_ctx_create_subring: the subring of dimension 2^log_n on this
        context's primes (ring switching)."""
        h = _P()
        _check(load().pdq_ctx_create_subring(self.h, log_n, ctypes.byref(h)))
        return Context(log_n, self.t, 0, self.L, self.K, 0, _handle=h)

    def plan_switched(self, big_log_n: int, n: int, s: int, B: int = 0) -> Plan:
        """pdq_plan_make_switched: Comp in this subring on a query switched
        from the ring of dimension 2^big_log_n."""
        pl = Plan()
        _check(load().pdq_plan_make_switched(self.h, big_log_n, n, s, B, ctypes.byref(pl)))
        return pl

    def plan_plain_db(self, n: int, s: int, B: int = 0) -> Plan:
        """pdq_plan_make_plain_db: the Answer on an unencrypted database."""
        pl = Plan()
        _check(load().pdq_plan_make_plain_db(self.h, n, s, B, ctypes.byref(pl)))
        return pl

    def db_diagonals(self, plan: Plan, values, stream=None) -> torch.Tensor:
        """pdq_db_diagonals_build: database-specific diagonals and group masks."""
        values = values.to(device="cuda", dtype=torch.int32).contiguous()
        lib = load()
        out = self._u64(lib.pdq_db_diagonals_bytes(self.h, ctypes.byref(plan)) // 8)
        _check(lib.pdq_db_diagonals_build(self.h, ctypes.byref(plan), _ptr(values), _ptr(out),
                                          _stream(stream)))
        return out

    def answer_plain_db_workspace(self, plan: Plan) -> torch.Tensor:
        return self._ws(load().pdq_answer_plain_db_workspace_bytes(self.h, ctypes.byref(plan)))

    def answer_plain_db(self, plan: Plan, v_cts, keys, galois, consts, ws=None, out=None,
                        stream=None) -> torch.Tensor:
        """pdq_answer_plain_db: the Answer without Mask, [C; C diag(DB)] v."""
        ws = self.answer_plain_db_workspace(plan) if ws is None else ws
        out = self._u64(plan.n_out * self.ct_elems) if out is None else out
        gal = (ctypes.c_uint64 * len(galois))(*galois)
        _check(load().pdq_answer_plain_db(self.h, ctypes.byref(plan), _ptr(v_cts), _ptr(keys),
                                          ctypes.cast(gal, _P), len(galois), _ptr(consts),
                                          _ptr(out), _ptr(ws), ws.numel(), _stream(stream)))
        return out.view(plan.n_out, 2, self.L, self.N)

    def ring_switch_key_gen(self, small: "Context", sk, s_small, a, e, stream=None) -> torch.Tensor:
        """pdq_ring_switch_key_gen: key from this ring's s to s_small(X^R)."""
        s_small = s_small.to(device="cuda", dtype=torch.int8).contiguous()
        a = a.to(device="cuda").contiguous()
        e = e.to(device="cuda", dtype=torch.int32).contiguous()
        out = self._u64(self.key_elems)
        _check(load().pdq_ring_switch_key_gen(self.h, small.h, _ptr(sk), _ptr(s_small), _ptr(a),
                                              _ptr(e), _ptr(out), _stream(stream)))
        return out.view(self.ndigits, 2, self.E, self.N)

    def ring_switch(self, small: "Context", cts, key, group: int = 1, out=None, ws=None,
                    stream=None) -> torch.Tensor:
        """pdq_ring_switch: count ciphertexts of this ring -> R count of the
        subring (part r of ciphertext i at (i/group) group R + r group + i%group)."""
        count = cts.numel() // self.ct_elems
        R = self.N // small.N
        lib = load()
        if ws is None:
            ws = self._ws(lib.pdq_ring_switch_workspace_bytes(self.h, count))
        if out is None:
            out = small._u64(count * R * small.ct_elems)
        _check(lib.pdq_ring_switch(self.h, small.h, _ptr(cts), count, group, _ptr(key), _ptr(out),
                                   _ptr(ws), ws.numel(), _stream(stream)))
        return out.view(count * R, 2, small.L, small.N)

    def close(self):
        if getattr(self, "h", None):
            load().pdq_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # sizes
    @property
    def ct_elems(self) -> int:
        return 2 * self.L * self.N

    @property
    def key_elems(self) -> int:
        return self.ndigits * 2 * self.E * self.N

    def _u64(self, n: int, device="cuda") -> torch.Tensor:
        # 64-bit residues travel as int64 tensors (same bits; torch has few uint64 ops)
        return torch.empty(int(n), dtype=torch.int64, device=device)

    def _ws(self, nbytes: int) -> torch.Tensor:
        return torch.empty(max(int(nbytes), 8), dtype=torch.uint8, device="cuda")

    # transforms
    def ntt_forward(self, data, count, nlimbs, limb0=0, stride=None, stream=None):
        stride = nlimbs * self.N if stride is None else stride
        _check(load().pdq_ntt_forward(self.h, _ptr(data), count, nlimbs, limb0, stride,
                                      _stream(stream)))

    def ntt_inverse(self, data, count, nlimbs, limb0=0, stride=None, stream=None):
        stride = nlimbs * self.N if stride is None else stride
        _check(load().pdq_ntt_inverse(self.h, _ptr(data), count, nlimbs, limb0, stride,
                                      _stream(stream)))

    # client-side helpers
    def encode(self, slots: torch.Tensor, nlimbs=None, stream=None) -> torch.Tensor:
        slots = slots.to(device="cuda", dtype=torch.int32).contiguous()
        count = slots.numel() // self.N
        nlimbs = self.L if nlimbs is None else nlimbs
        out = self._u64(count * nlimbs * self.N)
        _check(load().pdq_encode(self.h, _ptr(slots), count, nlimbs, _ptr(out), _stream(stream)))
        return out.view(count, nlimbs, self.N)

    def secret_prepare(self, s: torch.Tensor, stream=None) -> torch.Tensor:
        s = s.to(device="cuda", dtype=torch.int8).contiguous()
        out = self._u64(self.E * self.N)
        _check(load().pdq_secret_prepare(self.h, _ptr(s), _ptr(out), _stream(stream)))
        return out.view(self.E, self.N)

    def encrypt(self, sk, slots, a, e, stream=None) -> torch.Tensor:
        slots = slots.to(device="cuda", dtype=torch.int32).contiguous()
        count = slots.numel() // self.N
        a = a.to(device="cuda").contiguous()
        e = e.to(device="cuda", dtype=torch.int32).contiguous()
        out = self._u64(count * self.ct_elems)
        _check(load().pdq_encrypt(self.h, _ptr(sk), _ptr(slots), count, _ptr(a), _ptr(e),
                                  _ptr(out), _stream(stream)))
        return out.view(count, 2, self.L, self.N)

    def rotkey_gen(self, sk, galois: int, a, e, out=None, stream=None) -> torch.Tensor:
        a = a.to(device="cuda").contiguous()
        e = e.to(device="cuda", dtype=torch.int32).contiguous()
        out = self._u64(self.key_elems) if out is None else out
        _check(load().pdq_rotkey_gen(self.h, _ptr(sk), galois, _ptr(a), _ptr(e), _ptr(out),
                                     _stream(stream)))
        return out.view(self.ndigits, 2, self.E, self.N)

    def decrypt(self, sk, ct, stream=None) -> torch.Tensor:
        count = ct.numel() // self.ct_elems
        out = torch.empty(count * self.N, dtype=torch.int32, device="cuda")
        lib = load()
        ws = self._ws(lib.pdq_decrypt_workspace_bytes(self.h, count))
        _check(lib.pdq_decrypt(self.h, _ptr(sk), _ptr(ct), count, _ptr(out), _ptr(ws),
                               ws.numel(), _stream(stream)))
        return out.view(count, self.N)

    # exchange format (host bytes)
    def cts_export(self, ct, stream=None) -> bytes:
        count = ct.numel() // self.ct_elems
        lib = load()
        nbytes = lib.pdq_cts_serialized_bytes(self.h, count)
        buf = ctypes.create_string_buffer(nbytes)
        ws = self._u64(max(count * self.ct_elems, 1))
        _check(lib.pdq_cts_export(self.h, _ptr(ct), count, buf, nbytes, _ptr(ws), _stream(stream)))
        return buf.raw

    def cts_import(self, data: bytes, stream=None) -> torch.Tensor:
        lib = load()
        hdr_count = int.from_bytes(data[20:24], "little") if len(data) >= 24 else 0
        out = self._u64(max(hdr_count * self.ct_elems, 1))
        cnt = _U32()
        _check(lib.pdq_cts_import(self.h, data, len(data), _ptr(out), hdr_count,
                                  ctypes.byref(cnt), _stream(stream)))
        return out[:cnt.value * self.ct_elems].view(cnt.value, 2, self.L, self.N)

    def sk_export(self, sk, stream=None) -> bytes:
        lib = load()
        nbytes = lib.pdq_sk_serialized_bytes(self.h)
        buf = ctypes.create_string_buffer(nbytes)
        ws = self._u64(self.N)
        _check(lib.pdq_sk_export(self.h, _ptr(sk), buf, nbytes, _ptr(ws), _stream(stream)))
        return buf.raw

    def sk_import(self, data: bytes, stream=None) -> torch.Tensor:
        out = self._u64(self.E * self.N)
        _check(load().pdq_sk_import(self.h, data, len(data), _ptr(out), _stream(stream)))
        return out.view(self.E, self.N)

    def rotkeys_export(self, keys, galois, stream=None) -> bytes:
        """pdq_rotkeys_export: keys [count][ndigits][2][E][N] (NTT form) with
        their Galois elements -> bytes."""
        gal = np.ascontiguousarray(galois, dtype=np.uint64)
        count = len(gal)
        lib = load()
        nbytes = lib.pdq_rotkeys_serialized_bytes(self.h, count)
        buf = ctypes.create_string_buffer(nbytes)
        ws = self._u64(self.key_elems)
        _check(lib.pdq_rotkeys_export(self.h, _ptr(keys), _ptr(gal), count, buf, nbytes,
                                      _ptr(ws), _stream(stream)))
        return buf.raw

    def rotkeys_import(self, data: bytes, stream=None):
        """pdq_rotkeys_import: bytes -> (keys [count * key_elems] NTT form on
        the device, Galois elements as a list)."""
        lib = load()
        hdr_count = int.from_bytes(data[20:24], "little") if len(data) >= 24 else 0
        keys = self._u64(max(hdr_count * self.key_elems, 1))
        gal = np.zeros(max(hdr_count, 1), dtype=np.uint64)
        cnt = _U32()
        _check(lib.pdq_rotkeys_import(self.h, data, len(data), _ptr(keys), _ptr(gal), hdr_count,
                                      ctypes.byref(cnt), _stream(stream)))
        return keys[:cnt.value * self.key_elems], [int(g) for g in gal[:cnt.value]]

    def rotate(self, ct, galois: int, key, stream=None) -> torch.Tensor:
        count = ct.numel() // self.ct_elems
        lib = load()
        ws = self._ws(lib.pdq_rotate_workspace_bytes(self.h, count))
        out = torch.empty_like(ct)
        _check(lib.pdq_rotate(self.h, _ptr(ct), count, galois, _ptr(key), _ptr(out), _ptr(ws),
                              ws.numel(), _stream(stream)))
        return out

    def mod_switch(self, to: "Context", cts, out=None, ws=None, stream=None) -> torch.Tensor:
        """pdq_mod_switch: ciphertexts of this context to the first to.L primes."""
        count = cts.numel() // self.ct_elems
        lib = load()
        ws = self._ws(lib.pdq_mod_switch_workspace_bytes(self.h, count)) if ws is None else ws
        out = to._u64(count * to.ct_elems) if out is None else out
        _check(lib.pdq_mod_switch(self.h, to.h, _ptr(cts), count, _ptr(out), _ptr(ws), ws.numel(),
                                  _stream(stream)))
        return out.view(count, 2, to.L, to.N)

    def rotate_noalloc(self, ct, galois: int, key, out=None, stream=None) -> torch.Tensor:
        """pdq_rotate without a workspace: the library's fixed device scratch
        is used (no allocation inside the call; `out` may be preallocated)."""
        count = ct.numel() // self.ct_elems
        out = torch.empty_like(ct) if out is None else out
        _check(load().pdq_rotate_noalloc(self.h, _ptr(ct), count, galois, _ptr(key), _ptr(out),
                                         _stream(stream)))
        return out

    # plans
    def plan(self, n: int, s: int, B: int = 0) -> Plan:
        pl = Plan()
        _check(load().pdq_plan_make(self.h, n, s, B, ctypes.byref(pl)))
        return pl

    def plan_galois(self, plan: Plan) -> list[int]:
        lib = load()
        cnt = _U32()
        _check(lib.pdq_plan_galois(self.h, ctypes.byref(plan), None, 0, ctypes.byref(cnt)))
        arr = (ctypes.c_uint64 * cnt.value)()
        _check(lib.pdq_plan_galois(self.h, ctypes.byref(plan), ctypes.cast(arr, _P), cnt.value,
                                   ctypes.byref(cnt)))
        return [int(x) for x in arr]

    def plan_constants(self, plan: Plan, stream=None) -> torch.Tensor:
        lib = load()
        nbytes = lib.pdq_plan_constants_bytes(self.h, ctypes.byref(plan))
        out = self._u64(nbytes // 8)
        _check(lib.pdq_plan_constants_build(self.h, ctypes.byref(plan), _ptr(out),
                                            _stream(stream)))
        return out

    def db_encode(self, values, stream=None) -> torch.Tensor:
        values = values.to(device="cuda", dtype=torch.int32).contiguous()
        n = values.numel()
        lib = load()
        out = self._u64(lib.pdq_db_bytes(self.h, n) // 8)
        _check(lib.pdq_db_encode(self.h, _ptr(values), n, _ptr(out), _stream(stream)))
        return out

    def db_encode_plain(self, values, stream=None) -> torch.Tensor:
        """pdq_db_encode_plain: DB_j without row masks, [J][L][N]."""
        values = values.to(device="cuda", dtype=torch.int32).contiguous()
        n = values.numel()
        lib = load()
        out = self._u64(lib.pdq_db_plain_bytes(self.h, n) // 8)
        _check(lib.pdq_db_encode_plain(self.h, _ptr(values), n, _ptr(out), _stream(stream)))
        return out

    def mask_literal(self, plan: Plan, v_cts, db_plain, stream=None) -> torch.Tensor:
        """pdq_mask_literal: d = v.DB first, then the row masks."""
        out = self._u64(plan.J * 4 * self.ct_elems)
        _check(load().pdq_mask_literal(self.h, ctypes.byref(plan), _ptr(v_cts), _ptr(db_plain),
                                       _ptr(out), _stream(stream)))
        return out.view(plan.J * 4, 2, self.L, self.N)

    # hot path
    def mask(self, plan: Plan, v_cts, db, out=None, stream=None) -> torch.Tensor:
        out = self._u64(plan.J * 4 * self.ct_elems) if out is None else out
        _check(load().pdq_mask(self.h, ctypes.byref(plan), _ptr(v_cts), _ptr(db), _ptr(out),
                               _stream(stream)))
        return out.view(plan.J * 4, 2, self.L, self.N)

    def comp_workspace(self, plan: Plan) -> torch.Tensor:
        return self._ws(load().pdq_comp_workspace_bytes(self.h, ctypes.byref(plan)))

    def answer_workspace(self, plan: Plan) -> torch.Tensor:
        return self._ws(load().pdq_answer_workspace_bytes(self.h, ctypes.byref(plan)))

    def comp(self, plan: Plan, masked, keys, galois, consts, ws=None, out=None, stream=None):
        ws = self.comp_workspace(plan) if ws is None else ws
        out = self._u64(plan.n_out * self.ct_elems) if out is None else out
        gal = (ctypes.c_uint64 * len(galois))(*galois)
        _check(load().pdq_comp(self.h, ctypes.byref(plan), _ptr(masked), _ptr(keys),
                               ctypes.cast(gal, _P), len(galois), _ptr(consts), _ptr(out),
                               _ptr(ws), ws.numel(), _stream(stream)))
        return out.view(plan.n_out, 2, self.L, self.N)

    def answer(self, plan: Plan, v_cts, db, keys, galois, consts, ws=None, out=None,
               stream=None):
        ws = self.answer_workspace(plan) if ws is None else ws
        out = self._u64(plan.n_out * self.ct_elems) if out is None else out
        gal = (ctypes.c_uint64 * len(galois))(*galois)
        _check(load().pdq_answer(self.h, ctypes.byref(plan), _ptr(v_cts), _ptr(db), _ptr(keys),
                                 ctypes.cast(gal, _P), len(galois), _ptr(consts), _ptr(out),
                                 _ptr(ws), ws.numel(), _stream(stream)))
        return out.view(plan.n_out, 2, self.L, self.N)

    def answer_stacked_workspace(self, plan: Plan, Q: int) -> torch.Tensor:
        return self._ws(load().pdq_answer_stacked_workspace_bytes(self.h, ctypes.byref(plan), Q))

    def answer_stacked(self, plan: Plan, v_cts, db, key_sets, galois, consts, ws=None, out=None,
                       stream=None):
        """Q = len(key_sets) queries of one plan in one launch sequence: v_cts
        holds their index ciphertexts one query after the other, key_sets[q]
        is query q's key set; returns [Q][n_out][2][L][N]."""
        Q = len(key_sets)
        ws = self.answer_stacked_workspace(plan, Q) if ws is None else ws
        out = self._u64(Q * plan.n_out * self.ct_elems) if out is None else out
        gal = (ctypes.c_uint64 * len(galois))(*galois)
        ptrs = (ctypes.c_uint64 * Q)(*[_ptr(k) or 0 for k in key_sets])
        _check(load().pdq_answer_stacked(self.h, ctypes.byref(plan), Q, _ptr(v_cts), _ptr(db),
                                         ctypes.cast(ptrs, _P), ctypes.cast(gal, _P), len(galois),
                                         _ptr(consts), _ptr(out), _ptr(ws), ws.numel(),
                                         _stream(stream)))
        return out.view(Q, plan.n_out, 2, self.L, self.N)

    def answer_host_workspace(self, plan: Plan) -> torch.Tensor:
        return self._ws(load().pdq_answer_host_workspace_bytes(self.h, ctypes.byref(plan)))

    def answer_host(self, plan: Plan, v_host, db, keys, galois, consts, out_host, ws=None,
                    stream=None):
        """v_host / out_host: host tensors (pinned for full bandwidth), coefficient form."""
        ws = self.answer_host_workspace(plan) if ws is None else ws
        gal = (ctypes.c_uint64 * len(galois))(*galois)
        _check(load().pdq_answer_host(self.h, ctypes.byref(plan), _ptr(v_host), _ptr(db),
                                      _ptr(keys), ctypes.cast(gal, _P), len(galois), _ptr(consts),
                                      _ptr(out_host), _ptr(ws), ws.numel(), _stream(stream)))
        return out_host

    def query(self, plan: Plan, v_cts, db, keys, galois, consts, out) -> "QueryHandle":
        """Bundle one query's buffers for pdq_answer_batch / the server."""
        return QueryHandle(self, plan, v_cts, db, keys, galois, consts, out)

    def answer_batch(self, handles, lane_ws, stream=None):
        """pdq_answer_batch over QueryHandles; lane_ws: list of workspaces."""
        qs = (Query * len(handles))(*[h.struct for h in handles])
        ws = (ctypes.c_void_p * len(lane_ws))(*[_ptr(w) for w in lane_ws])
        nb = (ctypes.c_size_t * len(lane_ws))(*[w.numel() for w in lane_ws])
        _check(load().pdq_answer_batch(self.h, qs, len(handles), ctypes.cast(ws, _P),
                                       ctypes.cast(nb, _P), len(lane_ws), _stream(stream)))

    def profile_enable(self, on: bool = True):
        _check(load().pdq_profile_enable(self.h, 1 if on else 0))

    def profile_read(self) -> dict:
        """Summed milliseconds and call counts per stage since enabling."""
        ms = (ctypes.c_float * len(STAGES))()
        calls = (ctypes.c_uint32 * len(STAGES))()
        _check(load().pdq_profile_read(self.h, ctypes.cast(ms, _P), ctypes.cast(calls, _P),
                                       len(STAGES)))
        return {name: (float(ms[i]), int(calls[i])) for i, name in enumerate(STAGES)}

    def decomp(self, plan: Plan, slots) -> list[tuple[int, int]]:
        """slots: [n_out][N] decrypted answer (host or device); returns sorted
        (record index, value) pairs."""
        lib = load()
        return _decomp(lambda *a: lib.pdq_decomp(self.h, *a), plan, slots)


class QueryHandle:
    """Keeps a query's plan, Galois list and tensors alive with its pdq_query."""

    def __init__(self, ctx: Context, plan: Plan, v_cts, db, keys, galois, consts, out):
        self.ctx, self.plan = ctx, plan
        self.tensors = (v_cts, db, keys, consts, out)
        self.galois = (ctypes.c_uint64 * len(galois))(*galois)
        self.struct = Query(ctypes.cast(ctypes.pointer(plan), _P).value, _ptr(v_cts), _ptr(db),
                            _ptr(keys), ctypes.cast(self.galois, _P).value, len(galois), 0,
                            _ptr(consts), _ptr(out))
        self.out = out


class Server:
    """pdq_server: continuous batching over `lanes` worker streams with the
    workspaces carved out of `arena` (a device tensor = the HBM budget)."""

    def __init__(self, arena: torch.Tensor, lanes: int = 4, max_queue: int = 0):
        self.arena = arena
        # the workers' streams do not wait on the caller's: work queued there
        # (on memory the caching allocator may have just handed to the arena)
        # must finish before the server starts
        torch.cuda.current_stream().synchronize()
        h = _P()
        _check(load().pdq_server_create(_ptr(arena), arena.numel() * arena.element_size(), lanes,
                                        max_queue, ctypes.byref(h)))
        self.h = h
        self.pending = {}

    def submit(self, handle: QueryHandle) -> int:
        t = _U64()
        _check(load().pdq_server_submit(self.h, handle.ctx.h, ctypes.byref(handle.struct),
                                        ctypes.byref(t)))
        self.pending[t.value] = handle
        return t.value

    def status(self, ticket: int) -> TicketInfo:
        info = TicketInfo()
        _check(load().pdq_server_status(self.h, ticket, ctypes.byref(info)))
        return info

    def set_stacking(self, max_stack: int):
        """Answer up to max_stack queued requests of one shape together."""
        _check(load().pdq_server_set_stacking(self.h, max_stack))

    def wait(self, ticket: int, timeout_ms: int = 600000):
        _check(load().pdq_server_wait(self.h, ticket, timeout_ms))

    def drain(self, timeout_ms: int = 600000):
        _check(load().pdq_server_drain(self.h, timeout_ms))

    def close(self):
        if getattr(self, "h", None):
            load().pdq_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
