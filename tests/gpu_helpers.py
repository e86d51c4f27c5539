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
    """Frobenius relative difference (reported in messages; every parity
    assertion is element by element, see assert_close)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def rms(x):
    x = np.asarray(x, dtype=np.float64)
    return float(np.sqrt(np.mean(x * x))) if x.size else 0.0


# Element-wise parity bound: |got - want| <= rtol * (|want| + K_RMS * rms(want)) + atol,
# element by element.  The rms term is the scale of the quantity: an element
# whose exact value is near zero after cancellation still carries rounding of
# the size of the typical element (sums of products of that size), so its
# error is bounded relative to the rms, not to itself.  K_RMS = 8 covers the
# largest of ~1e6 independent roundings of one rms-relative size (about 5
# standard deviations) with margin; one element off by a whole rms (a wrong
# row, a dropped term) exceeds it by four orders of magnitude at rtol = 2e-5.
K_RMS = 8.0


def assert_close(got, want, rtol, what="", atol=0.0, k=K_RMS):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert got.shape == want.shape, f"{what}: shape {got.shape} != {want.shape}"
    bound = rtol * (np.abs(want) + k * rms(want)) + atol
    err = np.abs(got - want)
    bad = ~(err <= bound)
    if bad.any():
        i = np.unravel_index(int(np.argmax(np.where(bad, err / np.maximum(bound, 1e-300), -1.0))), err.shape)
        raise AssertionError(
            f"{what}: {int(bad.sum())} of {bad.size} elements outside rtol={rtol:g} (x{k:g} rms); "
            f"worst at {tuple(int(v) for v in i)}: got {got[i]!r}, want {want[i]!r}, bound {bound[i]:.3e}; "
            f"Frobenius rel {rel(got, want):.3e}")


def store_eps(dtype_np):
    """Unit roundoff of the stored core dtype (its rounding of G + step)."""
    return 2.0 ** -53 if np.dtype(dtype_np) == np.float64 else 2.0 ** -24


def assert_update_close(dev_after, dev_before, ora_after, ora_before, rtol, eps, what="core", rtol_core=None):
    """Cores compared through the step they took: (G_after - G_before) on the
    device against (O_after - O_before) of the oracle, element by element,
    plus the rounding of the stored core (2 eps |O_after|).  A wrong update
    smaller than the core itself cannot hide behind the core's size.  The
    cores themselves are compared too (rtol_core, default rtol).  The update
    is alpha p (or the AdaGrad step of p), so its tolerance is that of the
    direction."""
    for k, (G, S, O, T) in enumerate(zip(dev_after, dev_before, ora_after, ora_before)):
        G, S, O, T = (np.asarray(v, dtype=np.float64) for v in (G, S, O, T))
        assert_close(G - S, O - T, rtol, f"{what} {k} update", atol=2.0 * eps * np.abs(O))
        assert_close(G, O, rtol if rtol_core is None else rtol_core, f"{what} {k}")


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

    def resync(self):
        """Oracle state := device cores (so both take the next step from the
        same iterate); remembered as the starting point of that step."""
        cores = self.device_cores()
        for k, G in enumerate(cores):
            self.state.cores[k] = G
        self.before = ([G.copy() for G in cores], [G.copy() for G in cores])
        return cores

    def snapshot(self):
        """Remember both sides' cores before a step taken without resync."""
        self.before = (self.device_cores(), [G.copy() for G in self.state.cores])

    def assert_cores(self, rtol, rtol_update=None):
        """Cores after a step: the update element by element against the
        oracle's (from the remembered starting points; rtol_update, default
        rtol), and the cores (rtol)."""
        dev = self.device_cores()
        before = getattr(self, "before", None)
        if before is None:
            for k, (G, O) in enumerate(zip(dev, self.state.cores)):
                assert_close(G, O, rtol, f"core {k}")
            return
        assert_update_close(dev, before[0], self.state.cores, before[1],
                            rtol if rtol_update is None else rtol_update, store_eps(self.dtype_np), rtol_core=rtol)
        self.before = None

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
