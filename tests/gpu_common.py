"""Shared setup of the GPU parity tests: the same seeded inputs go to the
oracle and to the CUDA library; results are compared in coefficient form."""
from __future__ import annotations

import functools

import numpy as np
import torch

import workloads as W
from oracle import bfv, pdq as opdq


def to_dev(a: np.ndarray) -> torch.Tensor:
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a.copy()).cuda()


def to_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().contiguous().numpy().view(np.uint64)


def coeff(ctx, t: torch.Tensor, nlimbs: int) -> np.ndarray:
    """Coefficient form of NTT-form polynomials [..][nlimbs][N] (copy)."""
    c = t.clone().contiguous()
    count = c.numel() // (nlimbs * ctx.N)
    ctx.ntt_inverse(c, count, nlimbs)
    torch.cuda.synchronize()
    return to_np(c).reshape(t.shape)


@functools.lru_cache(maxsize=None)
def library():
    from paper_2408_17063_gb300 import build, pdq
    build.build()
    return pdq


class Setup:
    """Oracle and GPU state for one configuration with identical randomness."""

    def __init__(self, cfg_name: str, seed: int | None = None, s: int | None = None,
                 n: int | None = None, B: int = 0, pattern: str | None = None, ctx=None,
                 L: int | None = None, dnum: int | None = None):
        pdq = library()
        cfg = W.CONFIGS[cfg_name]
        if any(x is not None for x in (s, n, pattern, L, dnum)):
            import dataclasses
            cfg = dataclasses.replace(cfg, s=s or cfg.s, n=n or cfg.n,
                                      pattern=pattern or cfg.pattern, L=L or cfg.L,
                                      dnum=dnum or cfg.dnum)
        self.cfg = cfg
        self.par = bfv.Params.from_config(cfg)
        self.ctx = pdq.Context.from_config(cfg) if ctx is None else ctx
        self.q = W.draw_query(cfg, seed)
        self.seed = cfg.seed if seed is None else seed
        self.oplan = opdq.make_plan(self.par, cfg.n, cfg.s, B or None)
        self.plan = self.ctx.plan(cfg.n, cfg.s, B)
        self.galois = self.ctx.plan_galois(self.plan)
        self.sk = self.ctx.secret_prepare(torch.from_numpy(self.q.sk))
        N = self.par.N
        # index-vector encryptions
        self.enc_a, self.enc_e = W.encryption_randomness(self.par.q, N, self.oplan.J, self.seed)
        slots = np.stack([opdq.record_slots(self.par, self.q.v, j)
                          for j in range(self.oplan.J)]).astype(np.int32)
        self.v_slots = slots
        self.v_cts = self.ctx.encrypt(self.sk, torch.from_numpy(slots).cuda(),
                                      to_dev(self.enc_a), torch.from_numpy(self.enc_e).cuda())
        # rotation keys
        self.key_rand = W.rotation_key_randomness(self.par.ext, N, len(self.par.digits),
                                                  self.galois, self.seed)
        keys = self.ctx._u64(len(self.galois) * self.ctx.key_elems)
        kv = keys.view(len(self.galois), -1)
        for i, k in enumerate(self.galois):
            a, e = self.key_rand[k]
            self.ctx.rotkey_gen(self.sk, k, to_dev(a), torch.from_numpy(e).cuda(), out=kv[i])
        self.keys = keys
        self.db = self.ctx.db_encode(torch.from_numpy(self.q.db.astype(np.int32)).cuda())
        self.consts = self.ctx.plan_constants(self.plan)
        torch.cuda.synchronize()

    # oracle side (computed on demand)
    @functools.cached_property
    def o_keys(self):
        return {k: bfv.rotation_key(self.par, self.q.sk, k, *self.key_rand[k])
                for k in self.galois}

    @functools.cached_property
    def o_v_cts(self):
        return opdq.encrypt_index(self.par, self.q.sk, self.q.v, self.oplan, self.enc_a,
                                  self.enc_e)

    def answer(self):
        return self.ctx.answer(self.plan, self.v_cts, self.db, self.keys, self.galois,
                               self.consts)

    def handle(self, out=None):
        """A pdq_query over this setup's buffers (new output buffer)."""
        out = self.ctx._u64(self.plan.n_out * self.ctx.ct_elems) if out is None else out
        return self.ctx.query(self.plan, self.v_cts, self.db, self.keys, self.galois,
                              self.consts, out)
