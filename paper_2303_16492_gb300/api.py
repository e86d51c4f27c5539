"""Python binding of the TR-BRSGD library: same names as the C-ABI, argument
marshalling only.  Every step of the method runs in the CUDA kernels of
libtrsgd.so; PyTorch supplies device memory and streams.  There is no CPU
fallback: a missing library raises."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _abi
from ._abi import check

_TORCH_TO_DT = {torch.float64: _abi.DTYPE_F64, torch.float32: _abi.DTYPE_F32, torch.bfloat16: _abi.DTYPE_BF16}


@dataclass
class ProblemConfig:
    """Arguments of one TR problem (Algorithm 3) plus the step rule."""
    dims: list
    ranks: list
    J: int
    dist: int = _abi.DIST_UNIFORM
    variant: int = _abi.PLAIN
    rule: int = _abi.STEP_FIXED
    prec: int = _abi.FP32
    alpha: float = 0.01
    eta: float = 0.0
    b: float = 0.0
    eps: float = 0.0
    damping: float = 0.0
    J_H: int = 0
    seed: int = 0
    x_dtype: int | None = None
    path: int = _abi.PATH_AUTO
    fp32_units: int = _abi.FP32_PIECES

    def to_c(self) -> _abi.Config:
        c = _abi.Config()
        c.N = len(self.dims)
        c.dist = self.dist
        for k, (d, r) in enumerate(zip(self.dims, self.ranks)):
            c.I[k] = int(d)
            c.R[k] = int(r)
        c.J = int(self.J)
        c.J_H = int(self.J_H)
        c.variant = self.variant
        c.rule = self.rule
        c.prec = self.prec
        c.x_dtype = (_abi.DTYPE_F64 if self.prec == _abi.FP64 else _abi.DTYPE_F32) if self.x_dtype is None \
            else self.x_dtype
        c.alpha = self.alpha
        c.eta = self.eta
        c.b = self.b
        c.eps = self.eps
        c.damping = self.damping
        c.seed = int(self.seed)
        c.path = int(self.path)
        c.fp32_units = int(self.fp32_units)
        return c


def _ptrs(tensors):
    arr = (ctypes.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = ctypes.c_void_p(t.data_ptr())
    return arr


def _stream_ptr(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Solver:
    """trsgd_init / trsgd_step / trsgd_run / trsgd_rel_error on one handle.

    ``X`` is a list of device tensors (one per problem, i_1 fastest, i.e. a
    Fortran-ordered flat buffer); ``cores`` a list (per problem) of lists of
    device tensors in the G_{n(2)} layout (I_n x R_n R_{n+1}, row-major),
    updated in place.
    """

    def __init__(self, configs, X, cores, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("the TR-BRSGD library needs a CUDA device")
        self.configs = list(configs)
        self.X = list(X)
        self.cores = [list(c) for c in cores]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        n = len(self.configs)
        carr = (_abi.Config * n)(*[c.to_c() for c in self.configs])
        flat = [t for cs in self.cores for t in cs]
        h = ctypes.c_void_p()
        check(_abi.lib().trsgd_init(carr, n, _ptrs(self.X), _ptrs(flat), _stream_ptr(self.stream),
                                    ctypes.byref(h)), "trsgd_init")
        self._h = h

    def step(self, t: int):
        check(_abi.lib().trsgd_step(self._h, int(t)), "trsgd_step")

    def step_counter(self, T: int):
        """T iterations from the device-resident counter, which then advances by
        T; recordable in a CUDA graph on ``self.stream``."""
        check(_abi.lib().trsgd_step_counter(self._h, int(T)), "trsgd_step_counter")

    def set_counter(self, t: int):
        check(_abi.lib().trsgd_set_counter(self._h, int(t)), "trsgd_set_counter")

    def run(self, t0: int, T: int, chunk: int = 0, tol: float = 0.0, max_seconds: float = 0.0, Xref=None):
        done = ctypes.c_int64()
        rse = ctypes.c_double()
        ref = ctypes.c_void_p(Xref.data_ptr()) if Xref is not None else None
        check(_abi.lib().trsgd_run(self._h, int(t0), int(T), int(chunk), float(tol), float(max_seconds), ref,
                                   ctypes.byref(done), ctypes.byref(rse)), "trsgd_run")
        return done.value, rse.value

    def rel_error(self, problem: int = 0, Xref=None) -> float:
        out = ctypes.c_double()
        ref = ctypes.c_void_p(Xref.data_ptr()) if Xref is not None else None
        check(_abi.lib().trsgd_rel_error(self._h, int(problem), ref, ctypes.byref(out)), "trsgd_rel_error")
        return out.value

    def set_debug(self, on: bool = True):
        check(_abi.lib().trsgd_set_debug(self._h, 1 if on else 0), "trsgd_set_debug")

    def get_debug(self, item: int, dtype, count: int) -> np.ndarray:
        out = np.empty(count, dtype=dtype)
        written = ctypes.c_size_t()
        check(_abi.lib().trsgd_get_debug(self._h, int(item), out.ctypes.data_as(ctypes.c_void_p), out.nbytes,
                                         ctypes.byref(written)), "trsgd_get_debug")
        return out

    def adagrad_state(self, problem: int, core: int, array: np.ndarray, store: bool = False):
        check(_abi.lib().trsgd_adagrad_state(self._h, int(problem), int(core),
                                             array.ctypes.data_as(ctypes.c_void_p), array.nbytes,
                                             1 if store else 0), "trsgd_adagrad_state")
        return array

    def launch_shape(self, cluster: int | None = None, threads: int | None = None):
        c = ctypes.c_int32(cluster or 0)
        t = ctypes.c_int32(threads or 0)
        setf = 0 if cluster is None and threads is None else 1
        check(_abi.lib().trsgd_launch_shape(self._h, setf, ctypes.byref(c), ctypes.byref(t)), "trsgd_launch_shape")
        return c.value, t.value

    def autotune(self, steps_per_trial: int = 20):
        check(_abi.lib().trsgd_autotune(self._h, int(steps_per_trial)), "trsgd_autotune")
        return self.launch_shape()

    def launch_count(self) -> int:
        return int(_abi.lib().trsgd_launch_count(self._h))

    def gd_step(self, scaled: bool = False, alpha: float = 1e-3, damping: float = 0.0):
        """One full-gradient iteration (TR-GD, or TR-ScaledGD when ``scaled``) of
        problem 0, every core from the same iterate."""
        check(_abi.lib().trsgd_gd_step(self._h, 1 if scaled else 0, float(alpha), float(damping)), "trsgd_gd_step")

    def set_wait_limit(self, polls: int):
        """trsgd_set_wait_limit (failure-path testing; 0 restores the default)."""
        check(_abi.lib().trsgd_set_wait_limit(self._h, int(polls)), "trsgd_set_wait_limit")

    def debug_index_bound(self, k: int, bound: int):
        """trsgd_debug_index_bound (debug build only; 0 restores I_k)."""
        check(_abi.lib().trsgd_debug_index_bound(self._h, int(k), int(bound)), "trsgd_debug_index_bound")

    def shard_plan(self, t: int, rank: int, world: int) -> _abi.Shard:
        """trsgd_shard_plan: this rank's sample ranges of iteration t."""
        sh = _abi.Shard()
        check(_abi.lib().trsgd_shard_plan(self._h, int(t), int(rank), int(world), ctypes.byref(sh)),
              "trsgd_shard_plan")
        return sh

    def step_partial(self, t: int, plan: _abi.Shard, gpart, hpart=None):
        """trsgd_step_partial into FP32 device buffers of gsplits_max (hsplits_max) partials."""
        hp = ctypes.c_void_p(hpart.data_ptr()) if hpart is not None else None
        check(_abi.lib().trsgd_step_partial(self._h, int(t), ctypes.byref(plan), ctypes.c_void_p(gpart.data_ptr()),
                                            hp), "trsgd_step_partial")

    def step_apply(self, t: int, gparts, gsplits: int, hparts=None, hsplits: int = 0):
        """trsgd_step_apply over the gathered partials (rank order)."""
        hp = ctypes.c_void_p(hparts.data_ptr()) if hparts is not None else None
        check(_abi.lib().trsgd_step_apply(self._h, int(t), ctypes.c_void_p(gparts.data_ptr()), int(gsplits), hp,
                                          int(hsplits)), "trsgd_step_apply")

    def tensor_pieces(self) -> int:
        """BF16 pieces per tensor-core operand of the two contractions (0: FMA units)."""
        return int(_abi.lib().trsgd_tensor_pieces(self._h))

    def close(self):
        if getattr(self, "_h", None):
            _abi.lib().trsgd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe_peak(unit: int, iters: int = 4096, stream=None) -> float:
    """trsgd_probe_peak: measured flop/s of the FP32 (unit 0) or FP64 (unit 1) FMA units."""
    out = ctypes.c_double()
    check(_abi.lib().trsgd_probe_peak(int(unit), int(iters), _stream_ptr(stream), ctypes.byref(out)),
          "trsgd_probe_peak")
    return out.value


def reconstruct(cores, dims, ranks, out=None, stream=None):
    """trsgd_reconstruct: X = TR({G_n}) as a flat device tensor (i_1 fastest)."""
    dt = cores[0].dtype
    numel = int(np.prod(dims))
    if out is None:
        out = torch.empty(numel, dtype=dt, device=cores[0].device)
    N = len(dims)
    I = (ctypes.c_int64 * N)(*[int(d) for d in dims])
    R = (ctypes.c_int64 * N)(*[int(r) for r in ranks])
    check(_abi.lib().trsgd_reconstruct(N, I, R, _TORCH_TO_DT[dt], _ptrs(cores), ctypes.c_void_p(out.data_ptr()),
                                       _stream_ptr(stream)), "trsgd_reconstruct")
    return out


def sampled_loss_grad(cores, dims, ranks, n, idx, XS, w, want_grads=True, stream=None):
    """trsgd_sampled_loss_grad: loss (float tensor [1]) and, optionally, the
    gradient of every core in the G_{k(2)} layout."""
    N = len(dims)
    I = (ctypes.c_int64 * N)(*[int(d) for d in dims])
    R = (ctypes.c_int64 * N)(*[int(r) for r in ranks])
    loss = torch.empty(1, dtype=torch.float32, device=cores[0].device)
    grads = [torch.empty_like(c) for c in cores] if want_grads else None
    check(_abi.lib().trsgd_sampled_loss_grad(
        N, I, R, int(n), int(idx.shape[0]), ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(XS.data_ptr()),
        ctypes.c_void_p(w.data_ptr()), _ptrs(cores), _ptrs(grads) if grads else None,
        ctypes.c_void_p(loss.data_ptr()), _stream_ptr(stream)), "trsgd_sampled_loss_grad")
    return loss, grads


class TRLoss(torch.autograd.Function):
    """Sampled TR reconstruction loss with the hand-written adjoint for all
    cores: forward and backward both call trsgd_sampled_loss_grad."""

    @staticmethod
    def forward(ctx, idx, XS, w, dims, ranks, n, *cores):
        cores = [c.contiguous() for c in cores]
        loss, grads = sampled_loss_grad(cores, dims, ranks, n, idx, XS, w, want_grads=True)
        ctx.save_for_backward(*grads)
        return loss[0]

    @staticmethod
    def backward(ctx, gout):
        grads = ctx.saved_tensors
        return (None, None, None, None, None, None) + tuple(g * gout for g in grads)
