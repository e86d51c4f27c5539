"""Parity at the headline size (N=4, 100^4 FP32, R=10, |F|=1000) in the
launch configuration the benchmark times.

Both sides build X from the same seeded inputs (planted cores and noise from
the synth module): the device by the library's reconstruction, the oracle
fiber by fiber from the per-mode identity of Sec. 2 (X_[n](:, col) =
G_{n(2)} G^{!=n}_{[2]}(col, :)^T) at the sampled positions only.  Every
intermediate of three full-size steps is compared element by element.
"""
import numpy as np
import pytest
import torch

from oracle import brsgd as ob
from oracle import tr
from tests._util import to_oracle_cores
from tests.gpu_helpers import api, cuda, rel

pytestmark = [pytest.mark.gpu, cuda]


class LazyTensor:
    """X = TR(planted) + sigma * noise, evaluated by the oracle one mode-n fiber
    at a time (the only access the oracle step makes).  `noise` is an array or
    a function from flat positions to noise values."""

    def __init__(self, planted, dims, noise, sigma):
        self.P, self.shape, self.ndim = planted, tuple(dims), len(dims)
        self.noise, self.sigma = noise, sigma
        self.strides = np.cumprod([1] + list(dims[:-1]))

    def __getitem__(self, key):
        n = [k for k, v in enumerate(key) if isinstance(v, slice)][0]
        idx = np.array([[-1 if k == n else int(v) for k, v in enumerate(key)]], dtype=np.int64)
        z = ob.sampled_subchain(self.P, n, idx)[0]
        fiber = tr.unfold2(self.P[n]) @ z
        base = sum(int(v) * int(self.strides[k]) for k, v in enumerate(key) if k != n)
        pos = base + np.arange(self.shape[n]) * int(self.strides[n])
        nz = self.noise(pos) if callable(self.noise) else self.noise[pos]
        return fiber + self.sigma * np.asarray(nz, dtype=np.float64)


def test_headline_size_three_steps():
    from paper_2303_16492_gb300 import synth
    A = api()
    w = synth.workload("c2")
    planted = synth.planted_cores(w)
    P = to_oracle_cores(planted, w.ranks)
    noise = synth.noise(w.dims, w.seed + 1, dtype=np.float32)
    # noise scale from the oracle: rms of X_true estimated on 4000 oracle entries
    rng = np.random.default_rng(0)
    ent = [tr.tr_entry(P, [int(rng.integers(0, d)) for d in w.dims]) for _ in range(4000)]
    sigma = w.noise_rel * float(np.sqrt(np.mean(np.square(ent))))
    Xo = LazyTensor(P, w.dims, noise, sigma)

    planted_d = [torch.from_numpy(G).to("cuda", torch.float32) for G in planted]
    Xd = A.reconstruct(planted_d, w.dims, w.ranks)
    Xd.add_(torch.from_numpy(noise).cuda(), alpha=sigma)
    init = synth.initial_cores(w, float(torch.linalg.vector_norm(Xd.double()) ** 2))
    init = [G.astype(np.float32) for G in init]
    cores_d = [torch.from_numpy(G).cuda() for G in init]
    pc = A.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=1, alpha=w.alpha, seed=w.seed + 3)
    s = A.Solver([pc], [Xd], [cores_d])
    s.set_debug(True)
    st = ob.State.new(to_oracle_cores([G.astype(np.float64) for G in init], w.ranks))
    cfg = ob.Config(J=w.J, alpha=w.alpha, seed=w.seed + 3)
    for t in range(3):
        for k in range(4):
            st.cores[k] = tr.fold2(cores_d[k].double().cpu().numpy(), w.ranks[k], w.ranks[(k + 1) % 4])
        rec = ob.step(st, Xo, cfg, t)
        s.step(t)
        n, J, In, Q = rec["n"], w.J, w.dims[rec["n"]], 100
        assert int(s.get_debug(A._abi.DBG_MODE, np.int32, 1)[0]) == n
        np.testing.assert_array_equal(s.get_debug(A._abi.DBG_IDX, np.int32, J * 4).reshape(J, 4), rec["idx"])
        np.testing.assert_array_equal(s.get_debug(A._abi.DBG_PF, np.float64, J), rec["pF"])
        assert rel(s.get_debug(A._abi.DBG_Z, np.float32, J * Q).reshape(J, Q), rec["Z"]) < 2e-5
        assert rel(s.get_debug(A._abi.DBG_E, np.float32, J * In).reshape(J, In).T, rec["E"]) < 2e-5
        assert rel(s.get_debug(A._abi.DBG_G, np.float32, In * Q).reshape(In, Q), rec["g"]) < 2e-5
        for k in range(4):
            assert rel(cores_d[k].double().cpu().numpy(), tr.unfold2(st.cores[k])) < 2e-5
    s.close()


@pytest.mark.parametrize("bf16", [False, True], ids=["fp32x3", "bf16"])
def test_large_size_grid_path_steps(bf16):
    """The large workload (N=3, 1000^3, R=20, |F|=4096, AdaGrad) on the
    whole-GPU path against the oracle: two full-size iterations, every
    intermediate compared.  The noise is drawn on the device by a seeded
    generator and read at the sampled positions only; X_true on the oracle side
    is evaluated fiber by fiber from the planted cores.  Tolerances as in the
    grid-path tests (FP32 pieces 2e-5; BF16 operands: E 1e-2, g 2e-2, cores 1e-3)."""
    from paper_2303_16492_gb300 import synth
    A = api()
    w = synth.workload("c5")
    planted = synth.planted_cores(w)
    P = to_oracle_cores(planted, w.ranks)
    rng = np.random.default_rng(0)
    ent = [tr.tr_entry(P, [int(rng.integers(0, d)) for d in w.dims]) for _ in range(2000)]
    sigma = w.noise_rel * float(np.sqrt(np.mean(np.square(ent))))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(w.seed + 1)
    numel = int(np.prod(w.dims))
    noise_d = torch.randn(numel, generator=gen, device="cuda", dtype=torch.float32)
    Xo = LazyTensor(P, w.dims, lambda pos: noise_d[torch.from_numpy(pos).cuda()].double().cpu().numpy(), sigma)
    planted_d = [torch.from_numpy(G).to("cuda", torch.float32) for G in planted]
    Xd = A.reconstruct(planted_d, w.dims, w.ranks)
    Xd.add_(noise_d, alpha=sigma)
    init = synth.initial_cores(w, float(torch.linalg.vector_norm(Xd.double()) ** 2))
    init = [G.astype(np.float32) for G in init]
    cores_d = [torch.from_numpy(G).cuda() for G in init]
    pc = A.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=A._abi.BF16_MIXED if bf16 else A._abi.FP32,
                         x_dtype=A._abi.DTYPE_F32, rule=w.rule, eta=w.eta, seed=w.seed + 3)
    s = A.Solver([pc], [Xd], [cores_d])
    assert s.launch_shape() == (0, 256)     # R = 20: the whole-GPU path
    s.set_debug(True)
    st = ob.State.new(to_oracle_cores([G.astype(np.float64) for G in init], w.ranks))
    cfg = ob.Config(J=w.J, seed=w.seed + 3, rule=w.rule, eta=w.eta)
    tol_e, tol_g, tol_c = (1e-2, 2e-2, 1e-3) if bf16 else (2e-5, 2e-5, 2e-5)
    N, J, Q = 3, w.J, w.ranks[0] * w.ranks[1]
    for t in range(2):
        for k in range(N):
            st.cores[k] = tr.fold2(cores_d[k].double().cpu().numpy(), w.ranks[k], w.ranks[(k + 1) % N])
            acc = np.empty(w.dims[k] * Q, dtype=np.float32)
            s.adagrad_state(0, k, acc)
            st.acc[k] = acc.reshape(w.dims[k], Q).astype(np.float64)
        rec = ob.step(st, Xo, cfg, t)
        s.step(t)
        n, In = rec["n"], w.dims[rec["n"]]
        assert int(s.get_debug(A._abi.DBG_MODE, np.int32, 1)[0]) == n
        np.testing.assert_array_equal(s.get_debug(A._abi.DBG_IDX, np.int32, J * N).reshape(J, N), rec["idx"])
        np.testing.assert_array_equal(s.get_debug(A._abi.DBG_PF, np.float64, J), rec["pF"])
        assert rel(s.get_debug(A._abi.DBG_Z, np.float32, J * Q).reshape(J, Q), rec["Z"]) < 2e-5
        assert rel(s.get_debug(A._abi.DBG_E, np.float32, J * In).reshape(J, In).T, rec["E"]) < tol_e
        g_dev = s.get_debug(A._abi.DBG_G, np.float32, In * Q).reshape(In, Q)
        assert rel(g_dev, rec["g"]) < tol_g
        # AdaGrad's first step on an entry is eta * p / |p| = +-eta: where |g| is below the
        # comparison's resolution (10 x the tolerance of g, relative to its rms) the sign, and so
        # the step, is decided by rounding; everywhere else the updated core must agree
        sure = np.abs(rec["g"]) > 10 * tol_g * np.sqrt(np.mean(rec["g"] ** 2))
        assert sure.mean() > 0.5
        for k in range(N):
            dev, ora = cores_d[k].double().cpu().numpy(), tr.unfold2(st.cores[k])
            if k == n:
                assert rel(dev[sure], ora[sure]) < tol_c
                assert np.all(np.abs(dev - ora) <= 2 * w.eta + 1e-6)   # any other entry: at most one sign flip
            else:
                assert rel(dev, ora) < tol_c
    s.close()
