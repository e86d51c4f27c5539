"""Helpers of the GPU parity tests: the same seeded inputs go to the oracle
and, through the Python binding, to the CUDA library."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from oracle import brsgd as ob
from oracle import tr
from tests._util import make_problem, random_cores, to_lib_cores

cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")


def api():
    from paper_2303_16492_gb300 import api as A
    from paper_2303_16492_gb300 import build
    build.build()
    return A


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


class Case:
    """One problem: oracle state + device tensors holding identical values."""

    def __init__(self, dims, ranks, J, seed=0, prec=1, noise_rel=0.05, init_std=0.5, planted_std=None,
                 **cfg):
        A = api()
        self.A = A
        self.dims, self.ranks, self.J = list(dims), list(ranks), J
        self.dtype_np = np.float64 if prec == 0 else np.float32
        self.dtype_t = torch.float64 if prec == 0 else torch.float32
        N = len(dims)
        std = planted_std if planted_std is not None else [
            (ranks[n] * ranks[(n + 1) % N]) ** -0.25 for n in range(N)][0]
        planted, X_true, X = make_problem(dims, ranks, seed, noise_rel=noise_rel, std=std)
        start = random_cores(dims, ranks, seed + 7, std=init_std * std)
        # round every input to the device precision so that both sides see the same values
        self.X = X.astype(self.dtype_np).astype(np.float64)
        self.X_true = X_true.astype(self.dtype_np).astype(np.float64)
        start = [G.astype(self.dtype_np).astype(np.float64) for G in start]
        self.state = ob.State.new(start)
        ocfg = dict(cfg)
        self.ocfg = ob.Config(J=J, seed=cfg.get("seed_key", 3), **{k: v for k, v in ocfg.items()
                                                                  if k in ("dist", "variant", "rule", "alpha",
                                                                           "eta", "b", "eps", "damping", "J_H")})
        dev = "cuda"
        self.Xd = torch.from_numpy(np.ascontiguousarray(self.X.ravel(order="F")).astype(self.dtype_np)).to(dev)
        self.Xtd = torch.from_numpy(np.ascontiguousarray(self.X_true.ravel(order="F")).astype(self.dtype_np)).to(dev)
        self.cores_d = [torch.from_numpy(G.astype(self.dtype_np)).to(dev) for G in to_lib_cores(start)]
        pc = A.ProblemConfig(dims=self.dims, ranks=self.ranks, J=J, prec=prec, seed=self.ocfg.seed,
                             **{k: v for k, v in ocfg.items() if k in ("dist", "variant", "rule", "alpha", "eta",
                                                                       "b", "eps", "damping", "J_H", "fp32_units")})
        self.pc = pc
        self.solver = A.Solver([pc], [self.Xd], [self.cores_d])

    def Q(self, n):
        N = len(self.dims)
        return self.ranks[n] * self.ranks[(n + 1) % N]

    def device_cores(self):
        N = len(self.dims)
        return [tr.fold2(c.double().cpu().numpy(), self.ranks[n], self.ranks[(n + 1) % N])
                for n, c in enumerate(self.cores_d)]

    def debug(self, rec_n):
        A = self.A
        s = self.solver
        N, J = len(self.dims), self.J
        In, Q = self.dims[rec_n], self.Q(rec_n)
        dt = self.dtype_np
        out = dict(
            n=int(s.get_debug(A._abi.DBG_MODE, np.int32, 1)[0]),
            idx=s.get_debug(A._abi.DBG_IDX, np.int32, J * N).reshape(J, N),
            pF=s.get_debug(A._abi.DBG_PF, np.float64, J),
            Z=s.get_debug(A._abi.DBG_Z, dt, J * Q).reshape(J, Q),
            E=s.get_debug(A._abi.DBG_E, dt, J * In).reshape(J, In).T,
            g=s.get_debug(A._abi.DBG_G, dt, In * Q).reshape(In, Q),
            p=s.get_debug(A._abi.DBG_P, dt, In * Q).reshape(In, Q),
        )
        if self.pc.variant == 1:
            out["h"] = s.get_debug(A._abi.DBG_H, np.float64, Q * Q).reshape(Q, Q)
        return out
