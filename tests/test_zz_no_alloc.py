"""trsgd_rel_error_static: the relative error for callers that cannot
allocate device memory (their memory belongs to another allocator, or they
cannot accept the synchronisation an allocation may cause).  Checked through
the C-ABI against the handle-based trsgd_rel_error and against the oracle's
RSE of the same cores, on two calls in a row.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import tr
from tests._util import make_problem, random_cores, to_lib_cores, to_oracle_cores
from tests.gpu_helpers import api, cuda

pytestmark = [pytest.mark.gpu, cuda]


def _ptrs(ts):
    arr = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = ctypes.c_void_p(t.data_ptr())
    return arr


@pytest.mark.parametrize("prec", [0, 1])
def test_static_rel_error_matches_rel_error_twice(prec):
    A = api()
    lib = A._abi.lib()
    dims, ranks = [14, 13, 12, 11], [3, 2, 4, 3]
    planted, X_true, X = make_problem(dims, ranks, seed=31, noise_rel=0.05)
    start = random_cores(dims, ranks, seed=32, std=0.4)
    dt = torch.float64 if prec == 0 else torch.float32
    Xd = torch.from_numpy(np.ascontiguousarray(X.ravel(order="F"))).to("cuda", dt)
    cores = [torch.from_numpy(G).to("cuda", dt) for G in to_lib_cores(start)]
    s = A.Solver([A.ProblemConfig(dims=dims, ranks=ranks, J=40, prec=prec, alpha=0.02, seed=5)], [Xd], [cores])
    N = len(dims)
    I = (ctypes.c_int64 * N)(*dims)
    R = (ctypes.c_int64 * N)(*ranks)
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    tol = 1e-12 if prec == 0 else 1e-6
    for call in range(2):
        want = s.rel_error(0)
        st = lib.trsgd_rel_error_static(N, I, R, 0 if prec == 0 else 1, _ptrs(cores),
                                        ctypes.c_void_p(Xd.data_ptr()), ctypes.c_void_p(out.data_ptr()), stream)
        assert st == A._abi.OK
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - want) <= tol * want, (call, got, want)
        # the oracle's RSE of the cores the device holds now (FP64, Sec. 4)
        ora = tr.rse(to_oracle_cores([c.double().cpu().numpy() for c in cores], ranks), X.astype(
            np.float64 if prec == 0 else np.float32).astype(np.float64))
        assert abs(got - ora) <= tol * ora, (call, got, ora)
        s.step(call)          # move the cores so that the second call sees new values
        torch.cuda.synchronize()
    s.close()


def test_static_rel_error_rejects_oversize_and_bad_args():
    A = api()
    lib = A._abi.lib()
    cores = [torch.zeros(4, dtype=torch.float32, device="cuda") for _ in range(3)]
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    I = (ctypes.c_int64 * 3)(2, 4096, 2048)          # prod_{k>1} I_k = 8,388,608 > 4,194,304
    R = (ctypes.c_int64 * 3)(1, 1, 1)
    st = lib.trsgd_rel_error_static(3, I, R, 1, _ptrs(cores), ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), None)
    assert st == A._abi.EINVAL
    # four large dims: the running product of I_2..I_4 would pass 2^63; the
    # bound is checked before each multiplication
    cores4 = cores + [cores[0]]
    I4 = (ctypes.c_int64 * 4)(2, 1 << 30, 1 << 30, 1 << 30)
    R4 = (ctypes.c_int64 * 4)(1, 1, 1, 1)
    assert lib.trsgd_rel_error_static(4, I4, R4, 1, _ptrs(cores4), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()), None) == A._abi.EINVAL
    I2 = (ctypes.c_int64 * 3)(2, 2, 2)
    assert lib.trsgd_rel_error_static(3, I2, R, 1, _ptrs(cores), None, ctypes.c_void_p(out.data_ptr()),
                                      None) == A._abi.EINVAL
