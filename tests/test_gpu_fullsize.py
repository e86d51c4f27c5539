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
from tests.gpu_helpers import api, assert_close, assert_update_close, cuda

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


@pytest.mark.parametrize("units", ["pieces", "fma"])
def test_headline_size_three_steps(units):
    from paper_2303_16492_gb300 import synth
    A = api()
    fu = A._abi.FP32_PIECES if units == "pieces" else A._abi.FP32_FMA
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
    pc = A.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=1, alpha=w.alpha, seed=w.seed + 3, fp32_units=fu)
    s = A.Solver([pc], [Xd], [cores_d])
    assert s.launch_shape() == (16, 512)   # the launch shape the benchmark times
    assert s.tensor_pieces() == (3 if units == "pieces" else 0)
    s.set_debug(True)
    st = ob.State.new(to_oracle_cores([G.astype(np.float64) for G in init], w.ranks))
    cfg = ob.Config(J=w.J, alpha=w.alpha, seed=w.seed + 3)
    for t in range(3):
        for k in range(4):
            st.cores[k] = tr.fold2(cores_d[k].double().cpu().numpy(), w.ranks[k], w.ranks[(k + 1) % 4])
        before = [cores_d[k].double().cpu().numpy() for k in range(4)]
        rec = ob.step(st, Xo, cfg, t)
        s.step(t)
        n, J, In, Q = rec["n"], w.J, w.dims[rec["n"]], 100
        assert int(s.get_debug(A._abi.DBG_MODE, np.int32, 1)[0]) == n
        np.testing.assert_array_equal(s.get_debug(A._abi.DBG_IDX, np.int32, J * 4).reshape(J, 4), rec["idx"])
        np.testing.assert_array_equal(s.get_debug(A._abi.DBG_PF, np.float64, J), rec["pF"])
        assert_close(s.get_debug(A._abi.DBG_Z, np.float32, J * Q).reshape(J, Q), rec["Z"], 2e-5, "Z")
        assert_close(s.get_debug(A._abi.DBG_E, np.float32, J * In).reshape(J, In).T, rec["E"], 2e-5, "E")
        assert_close(s.get_debug(A._abi.DBG_G, np.float32, In * Q).reshape(In, Q), rec["g"], 2e-5, "g")
        assert_update_close([cores_d[k].double().cpu().numpy() for k in range(4)], before,
                            [tr.unfold2(st.cores[k]) for k in range(4)], before, 2e-5, 2.0 ** -24)
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
        before = [cores_d[k].double().cpu().numpy() for k in range(N)]
        rec = ob.step(st, Xo, cfg, t)
        s.step(t)
        n, In = rec["n"], w.dims[rec["n"]]
        assert int(s.get_debug(A._abi.DBG_MODE, np.int32, 1)[0]) == n
        np.testing.assert_array_equal(s.get_debug(A._abi.DBG_IDX, np.int32, J * N).reshape(J, N), rec["idx"])
        np.testing.assert_array_equal(s.get_debug(A._abi.DBG_PF, np.float64, J), rec["pF"])
        assert_close(s.get_debug(A._abi.DBG_Z, np.float32, J * Q).reshape(J, Q), rec["Z"], 2e-5, "Z")
        assert_close(s.get_debug(A._abi.DBG_E, np.float32, J * In).reshape(J, In).T, rec["E"], tol_e, "E")
        g_dev = s.get_debug(A._abi.DBG_G, np.float32, In * Q).reshape(In, Q)
        assert_close(g_dev, rec["g"], tol_g, "g")
        # AdaGrad's first step on an entry is eta * p / |p| = +-eta: where |g| is below the
        # comparison's resolution (10 x the tolerance of g, relative to its rms) the sign, and so
        # the step, is decided by rounding; everywhere else the updated core must agree
        sure = np.abs(rec["g"]) > 10 * tol_g * np.sqrt(np.mean(rec["g"] ** 2))
        assert sure.mean() > 0.5
        for k in range(N):
            dev, ora = cores_d[k].double().cpu().numpy(), tr.unfold2(st.cores[k])
            if k == n:
                assert_close((dev - before[k])[sure], (ora - before[k])[sure], tol_c, "core update (decided entries)")
                assert np.all(np.abs(dev - ora) <= 2 * w.eta + 1e-6)   # any other entry: at most one sign flip
            else:
                assert_close(dev - before[k], ora - before[k], tol_c, "unchanged core")
    s.close()


@pytest.mark.parametrize("bf16", [False, True], ids=["fp32x3", "bf16_x_stored_bf16"])
def test_large_size_scaled_steps(bf16):
    """The large workload as its recipe states it: the scaled variant (Sec.
    3.3, Q = R^2 = 400) with AdaGrad on the whole-GPU path, X stored in BF16
    (2 GB) for the BF16 run.  Two full-size iterations against the oracle:
    indices bit-exact; Z, E, g element by element; h from three BF16 pieces
    of Z (FP32 accuracy in both modes) within 2e-5; the direction against an
    FP64 Cholesky solve of the device's own h and g (1e-6: the double-float
    factorisation and solves), and against the oracle's direction within the
    direction's FP32/BF16 bound amplified by cond(h); the core update."""
    from paper_2303_16492_gb300 import synth
    A = api()
    w = synth.workload("c5")
    eta = w.extra.get("eta_scaled", w.eta)
    planted = synth.planted_cores(w)
    P = to_oracle_cores(planted, w.ranks)
    rng = np.random.default_rng(0)
    ent = [tr.tr_entry(P, [int(rng.integers(0, d)) for d in w.dims]) for _ in range(2000)]
    sigma = w.noise_rel * float(np.sqrt(np.mean(np.square(ent))))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(w.seed + 1)
    numel = int(np.prod(w.dims))
    noise_d = torch.randn(numel, generator=gen, device="cuda", dtype=torch.float32)
    lazy = LazyTensor(P, w.dims, lambda pos: noise_d[torch.from_numpy(pos).cuda()].double().cpu().numpy(), sigma)
    if bf16:   # the oracle's fibers rounded as the stored X is (FP32, then BF16)
        class _Rounded:
            shape, ndim = lazy.shape, lazy.ndim

            def __getitem__(self, key):
                f = torch.from_numpy(lazy[key].astype(np.float32))
                return f.to(torch.bfloat16).double().numpy()
        Xo = _Rounded()
    else:
        Xo = lazy
    planted_d = [torch.from_numpy(G).to("cuda", torch.float32) for G in planted]
    Xd = A.reconstruct(planted_d, w.dims, w.ranks)
    Xd.add_(noise_d, alpha=sigma)
    init = synth.initial_cores(w, float(torch.linalg.vector_norm(Xd.double()) ** 2))
    init = [G.astype(np.float32) for G in init]
    if bf16:
        Xd = Xd.to(torch.bfloat16)
    cores_d = [torch.from_numpy(G).cuda() for G in init]
    pc = A.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=A._abi.BF16_MIXED if bf16 else A._abi.FP32,
                         x_dtype=A._abi.DTYPE_BF16 if bf16 else A._abi.DTYPE_F32, rule=w.rule, eta=eta,
                         variant=1, seed=w.seed + 3)
    s = A.Solver([pc], [Xd], [cores_d])
    assert s.launch_shape() == (0, 256)
    s.set_debug(True)
    st = ob.State.new(to_oracle_cores([G.astype(np.float64) for G in init], w.ranks))
    cfg = ob.Config(J=w.J, seed=w.seed + 3, rule=w.rule, eta=eta, variant=1)
    tol_e, tol_g = (1e-2, 2e-2) if bf16 else (2e-5, 2e-5)
    N, J, Q = 3, w.J, w.ranks[0] * w.ranks[1]
    for t in range(2):
        for k in range(N):
            st.cores[k] = tr.fold2(cores_d[k].double().cpu().numpy(), w.ranks[k], w.ranks[(k + 1) % N])
            acc = np.empty(w.dims[k] * Q, dtype=np.float32)
            s.adagrad_state(0, k, acc)
            st.acc[k] = acc.reshape(w.dims[k], Q).astype(np.float64)
        before = [cores_d[k].double().cpu().numpy() for k in range(N)]
        rec = ob.step(st, Xo, cfg, t)
        s.step(t)
        n, In = rec["n"], w.dims[rec["n"]]
        assert int(s.get_debug(A._abi.DBG_MODE, np.int32, 1)[0]) == n
        np.testing.assert_array_equal(s.get_debug(A._abi.DBG_IDX, np.int32, J * N).reshape(J, N), rec["idx"])
        assert_close(s.get_debug(A._abi.DBG_Z, np.float32, J * Q).reshape(J, Q), rec["Z"], 2e-5, "Z")
        assert_close(s.get_debug(A._abi.DBG_E, np.float32, J * In).reshape(J, In).T, rec["E"], tol_e, "E")
        g_dev = s.get_debug(A._abi.DBG_G, np.float32, In * Q).reshape(In, Q).astype(np.float64)
        assert_close(g_dev, rec["g"], tol_g, "g")
        h_dev = s.get_debug(A._abi.DBG_H, np.float64, Q * Q).reshape(Q, Q)
        assert_close(h_dev, rec["h"], 2e-5, "h")
        p_dev = s.get_debug(A._abi.DBG_P, np.float32, In * Q).reshape(In, Q)
        L = np.linalg.cholesky(h_dev)
        assert_close(p_dev, -np.linalg.solve(L.T, np.linalg.solve(L, g_dev.T)).T, 1e-6, "p vs FP64 solve")
        kappa = np.linalg.cond(rec["h"])
        tol_p = tol_g + 2e-7 * kappa
        assert_close(p_dev, rec["p"], tol_p, f"p (cond {kappa:.1e})")
        # the update from the device's own direction (AdaGrad of Sec. 3.1's remark, FP32)
        dev = cores_d[n].double().cpu().numpy()
        acc = np.empty(In * Q, dtype=np.float32)
        s.adagrad_state(0, n, acc)
        A32 = acc.reshape(In, Q).astype(np.float64)
        want = before[n] + np.where(A32 > 0, eta / np.sqrt(np.maximum(A32, 1e-300)), 0.0) * p_dev
        assert_close(dev - before[n], want - before[n], 1e-5, "update from the device's p")
    s.close()


def _problem(A, name):
    """A named workload from the synth module: device X by the library's
    reconstruction plus seeded device noise (noise_rel of the rms of X_true,
    estimated on 2000 oracle entries); the oracle's X evaluated fiber by fiber
    from the planted cores and the same noise values."""
    from paper_2303_16492_gb300 import synth
    w = synth.workload(name)
    planted = synth.planted_cores(w)
    P = to_oracle_cores(planted, w.ranks)
    Xd = A.reconstruct([torch.from_numpy(G).to("cuda", torch.float32) for G in planted], w.dims, w.ranks)
    if w.noise_rel > 0:
        rng = np.random.default_rng(0)
        ent = [tr.tr_entry(P, [int(rng.integers(0, d)) for d in w.dims]) for _ in range(2000)]
        sigma = w.noise_rel * float(np.sqrt(np.mean(np.square(ent))))
        gen = torch.Generator(device="cuda")
        gen.manual_seed(w.seed + 1)
        noise_d = torch.randn(int(np.prod(w.dims)), generator=gen, device="cuda", dtype=torch.float32)
        Xo = LazyTensor(P, w.dims, lambda pos: noise_d[torch.from_numpy(pos).cuda()].double().cpu().numpy(), sigma)
        Xd.add_(noise_d, alpha=sigma)
    else:
        Xo = LazyTensor(P, w.dims, lambda pos: np.zeros(len(pos)), 0.0)
    init = [G.astype(np.float32) for G in synth.initial_cores(w, float(torch.linalg.vector_norm(Xd.double()) ** 2))]
    return w, P, Xo, Xd, init


def _c3_problem(A):
    """The c3 workload (N=5, 40^5, R=8, |F|=2048, Gaussian cores N(0, 1/8),
    noise 1e-3)."""
    return _problem(A, "c3")


@pytest.mark.parametrize("dist", [ob.DIST_UNIFORM, ob.DIST_LEVERAGE, ob.DIST_EUCLIDEAN],
                         ids=["uniform", "leverage", "euclidean"])
def test_c3_size_distributions(dist):
    """N=5, 40^5, R=8, |F|=2048 with three of the four distributions, two
    iterations each: indices bit-exact and p_F bit-exact for the uniform and
    Euclidean tables (built from the same cores on both sides); at I_k = 40 <
    R^2 = 64 leverage is exactly uniform, 1/I_k on the device and to 1e-15
    from the oracle's SVD; every intermediate within the FP32 tolerance.  The
    optimal distribution needs the full residual on the oracle side (10^8
    entries per iteration) and is checked at the smaller sizes of
    test_gpu_step."""
    A = api()
    w, P, Xo, Xd, init = _c3_problem(A)
    cores_d = [torch.from_numpy(G).cuda() for G in init]
    pc = A.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=1, alpha=w.alpha, dist=dist, seed=w.seed + 3)
    s = A.Solver([pc], [Xd], [cores_d])
    s.set_debug(True)
    N, J, Q = 5, w.J, 64
    st = ob.State.new(to_oracle_cores([G.astype(np.float64) for G in init], w.ranks))
    cfg = ob.Config(J=w.J, alpha=w.alpha, dist=dist, seed=w.seed + 3)
    for t in range(2):
        for k in range(N):
            st.cores[k] = tr.fold2(cores_d[k].double().cpu().numpy(), w.ranks[k], w.ranks[(k + 1) % N])
        before = [cores_d[k].double().cpu().numpy() for k in range(N)]
        rec = ob.step(st, Xo, cfg, t)
        s.step(t)
        n, In = rec["n"], w.dims[rec["n"]]
        np.testing.assert_array_equal(s.get_debug(A._abi.DBG_IDX, np.int32, J * N).reshape(J, N), rec["idx"])
        pf = s.get_debug(A._abi.DBG_PF, np.float64, J)
        if dist == ob.DIST_LEVERAGE:   # exactly 1/I_k on the device, 1/I_k to rounding from the oracle's SVD
            np.testing.assert_allclose(pf, rec["pF"], rtol=1e-12)
        else:
            np.testing.assert_array_equal(pf, rec["pF"])
        assert_close(s.get_debug(A._abi.DBG_Z, np.float32, J * Q).reshape(J, Q), rec["Z"], 2e-5, "Z")
        assert_close(s.get_debug(A._abi.DBG_E, np.float32, J * In).reshape(J, In).T, rec["E"], 2e-5, "E")
        assert_close(s.get_debug(A._abi.DBG_G, np.float32, In * Q).reshape(In, Q), rec["g"], 2e-5, "g")
        assert_update_close([cores_d[k].double().cpu().numpy() for k in range(N)], before,
                            [tr.unfold2(st.cores[k]) for k in range(N)], before, 2e-5, 2.0 ** -24)
    s.close()


def test_c3_size_adjoint():
    """The hand-written adjoint of the sampled loss for all five cores at the
    c3 size (|F| = 2048 samples of mode n, 40^5, R = 8) against the oracle's
    product-rule gradient (pinned by central differences at small sizes)."""
    A = api()
    from paper_2303_16492_gb300 import synth
    w = synth.workload("c3")
    cores = [G.astype(np.float32).astype(np.float64) for G in to_oracle_cores(synth.planted_cores(w), w.ranks)]
    n = 2
    idx = ob.draw_indices(11, 5, n, w.J, w.dims, None)
    XS = np.random.default_rng(3).standard_normal((w.dims[n], w.J)).astype(np.float32).astype(np.float64)
    wt = np.random.default_rng(4).uniform(0.5, 1.5, w.J).astype(np.float32).astype(np.float64)
    loss = ob.sampled_loss(cores, n, idx, XS, wt)
    grads = ob.sampled_loss_grads(cores, n, idx, XS, wt)
    cd = [torch.from_numpy(tr.unfold2(G)).to("cuda", torch.float32) for G in cores]
    idx_d = torch.from_numpy(np.where(idx < 0, 0, idx).astype(np.int32)).cuda()
    XS_d = torch.from_numpy(np.ascontiguousarray(XS.T).astype(np.float32)).cuda()
    w_d = torch.from_numpy(wt.astype(np.float32)).cuda()
    lg, gg = A.sampled_loss_grad(cd, w.dims, w.ranks, n, idx_d, XS_d, w_d)
    assert abs(float(lg.item()) - loss) < 1e-5 * abs(loss)
    for k in range(5):
        assert_close(gg[k].double().cpu().numpy(), tr.unfold2(grads[k]), 3e-5, "gg[k]")


@pytest.mark.parametrize("name", ["e1", "e1s", "e1s4", "hsi-salinas", "hsi-salinas-s", "hsi-indian",
                                  "hsi-indian-s", "hsi-pavia", "hsi-pavia-s"])
def test_paper_experiment_shapes(name):
    """The shapes of the paper's own experiments (Sec. 4): Experiment I (300^3,
    R = 10, |F| = 200; plain, and scaled with |H| = 200 and 400) and stand-ins
    for the three hyperspectral images (83x86x224 R=5, 145x145x220 R=10,
    610x340x103 R=10, |F| = 200; plain, and scaled with |H| = 1000), in the
    launch shape the library picks.  Two iterations from shared cores:
    indices and p_F bit-exact, every intermediate (and h for the scaled
    variant) within the FP32 tolerance."""
    A = api()
    w, P, Xo, Xd, init = _problem(A, name)
    N, J = 3, w.J
    cores_d = [torch.from_numpy(G).cuda() for G in init]
    pc = A.ProblemConfig(dims=w.dims, ranks=w.ranks, J=J, prec=1, alpha=w.alpha, variant=w.variant, J_H=w.JH,
                         damping=w.damping, seed=w.seed + 3)
    s = A.Solver([pc], [Xd], [cores_d])
    s.set_debug(True)
    st = ob.State.new(to_oracle_cores([G.astype(np.float64) for G in init], w.ranks))
    cfg = ob.Config(J=J, alpha=w.alpha, variant=w.variant, J_H=w.JH, damping=w.damping, seed=w.seed + 3)
    tol = 1e-4 if w.variant == 1 else 2e-5
    for t in range(2):
        for k in range(N):
            st.cores[k] = tr.fold2(cores_d[k].double().cpu().numpy(), w.ranks[k], w.ranks[(k + 1) % N])
        before = [cores_d[k].double().cpu().numpy() for k in range(N)]
        rec = ob.step(st, Xo, cfg, t)
        s.step(t)
        n, In, Q = rec["n"], w.dims[rec["n"]], w.ranks[rec["n"]] * w.ranks[(rec["n"] + 1) % N]
        assert int(s.get_debug(A._abi.DBG_MODE, np.int32, 1)[0]) == n
        np.testing.assert_array_equal(s.get_debug(A._abi.DBG_IDX, np.int32, J * N).reshape(J, N), rec["idx"])
        np.testing.assert_array_equal(s.get_debug(A._abi.DBG_PF, np.float64, J), rec["pF"])
        assert_close(s.get_debug(A._abi.DBG_Z, np.float32, J * Q).reshape(J, Q), rec["Z"], tol, "Z")
        assert_close(s.get_debug(A._abi.DBG_E, np.float32, J * In).reshape(J, In).T, rec["E"], tol, "E")
        assert_close(s.get_debug(A._abi.DBG_G, np.float32, In * Q).reshape(In, Q), rec["g"], tol, "g")
        if w.variant == 1:
            assert_close(s.get_debug(A._abi.DBG_H, np.float64, Q * Q).reshape(Q, Q), rec["h"], tol, "h")
        assert_close(s.get_debug(A._abi.DBG_P, np.float32, In * Q).reshape(In, Q), rec["p"], tol, "p")
        assert_update_close([cores_d[k].double().cpu().numpy() for k in range(N)], before,
                            [tr.unfold2(st.cores[k]) for k in range(N)], before, tol, 2.0 ** -24)
    s.close()


@pytest.mark.parametrize("name,dist", [("e2-k6", ob.DIST_LEVERAGE), ("e2-k6-s", ob.DIST_EUCLIDEAN),
                                       ("e2-k2-s", ob.DIST_UNIFORM)])
def test_experiment_2_shapes(name, dist):
    """Experiment II (Sec. 4) at 300^3: ill-conditioned U S V^T cores with
    condition number 1e6 or 1e2, R = 5, |F| = 200, plain and scaled with
    |H| = 1200, with non-uniform distributions built from the same cores on
    both sides.  Two iterations from shared cores; indices bit-exact; p_F
    bit-exact (Euclidean, uniform) or to 1e-5 (leverage of float cores: the
    device's Gram and Cholesky in the core precision against the oracle's
    SVD, about 1e-7 apart); intermediates within the FP32 bound."""
    A = api()
    w, P, Xo, Xd, init = _problem(A, name)
    N, J = 3, w.J
    cores_d = [torch.from_numpy(G).cuda() for G in init]
    pc = A.ProblemConfig(dims=w.dims, ranks=w.ranks, J=J, prec=1, alpha=w.alpha, variant=w.variant, J_H=w.JH,
                         dist=dist, seed=w.seed + 3)
    s = A.Solver([pc], [Xd], [cores_d])
    s.set_debug(True)
    st = ob.State.new(to_oracle_cores([G.astype(np.float64) for G in init], w.ranks))
    cfg = ob.Config(J=J, alpha=w.alpha, variant=w.variant, J_H=w.JH, dist=dist, seed=w.seed + 3)
    tol = 1e-4 if w.variant == 1 else 2e-5
    for t in range(2):
        for k in range(N):
            st.cores[k] = tr.fold2(cores_d[k].double().cpu().numpy(), w.ranks[k], w.ranks[(k + 1) % N])
        before = [cores_d[k].double().cpu().numpy() for k in range(N)]
        rec = ob.step(st, Xo, cfg, t)
        s.step(t)
        n, In, Q = rec["n"], w.dims[rec["n"]], w.ranks[rec["n"]] * w.ranks[(rec["n"] + 1) % N]
        np.testing.assert_array_equal(s.get_debug(A._abi.DBG_IDX, np.int32, J * N).reshape(J, N), rec["idx"])
        pf = s.get_debug(A._abi.DBG_PF, np.float64, J)
        if dist == ob.DIST_LEVERAGE:
            np.testing.assert_allclose(pf, rec["pF"], rtol=1e-5)
        else:
            np.testing.assert_array_equal(pf, rec["pF"])
        assert_close(s.get_debug(A._abi.DBG_Z, np.float32, J * Q).reshape(J, Q), rec["Z"], tol, "Z")
        assert_close(s.get_debug(A._abi.DBG_E, np.float32, J * In).reshape(J, In).T, rec["E"], tol, "E")
        # the weights 1 / (|F| J_n p_F) carry the leverage scores' ~1e-7 into g
        assert_close(s.get_debug(A._abi.DBG_G, np.float32, In * Q).reshape(In, Q), rec["g"], tol, "g")
        if w.variant == 1:
            assert_close(s.get_debug(A._abi.DBG_H, np.float64, Q * Q).reshape(Q, Q), rec["h"], tol, "h")
        assert_update_close([cores_d[k].double().cpu().numpy() for k in range(N)], before,
                            [tr.unfold2(st.cores[k]) for k in range(N)], before, tol, 2.0 ** -24)
    s.close()


@pytest.mark.parametrize("scaled", [False, True], ids=["gd", "scaled_gd"])
def test_experiment_1_full_gradient_iteration(scaled):
    """One TR-GD / TR-ScaledGD iteration at the Experiment I size (300^3, R =
    10, J_n = 90,000 columns per mode): the device forms Z, X_[n] Z and Z^T Z
    from the mode-major copies; the oracle from X = TR(planted) built on the
    host.  Every updated core within the FP32 bound (sums over 9e4 terms)."""
    A = api()
    from paper_2303_16492_gb300 import synth
    w = synth.workload("e1")
    planted = synth.planted_cores(w)
    P = to_oracle_cores(planted, w.ranks)
    X = tr.reconstruct(P)
    Xd = torch.from_numpy(np.ascontiguousarray(X.ravel(order="F")).astype(np.float32)).cuda()
    X = Xd.double().cpu().numpy().reshape(w.dims, order="F")
    init = [G.astype(np.float32) for G in synth.initial_cores(w, float(np.sum(X ** 2)))]
    cores_d = [torch.from_numpy(G).cuda() for G in init]
    pc = A.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=1, alpha=w.alpha, seed=w.seed + 3)
    s = A.Solver([pc], [Xd], [cores_d])
    start = to_oracle_cores([G.astype(np.float64) for G in init], w.ranks)
    if scaled:
        alpha = 1.0   # the ALS update of every core
    else:             # a step of ~5 % of the cores, so that the step itself is compared
        unit = ob.gd_step(start, X, 1.0)
        alpha = 0.05 * np.sqrt(sum(np.sum(g ** 2) for g in start)) / np.sqrt(
            sum(np.sum((u - g) ** 2) for u, g in zip(unit, start)))
    want = ob.gd_step(start, X, alpha, scaled=scaled)
    s.gd_step(scaled=scaled, alpha=alpha)
    torch.cuda.synchronize()
    for k in range(3):
        got = cores_d[k].double().cpu().numpy() - tr.unfold2(start[k])
        assert_close(got, tr.unfold2(want[k]) - tr.unfold2(start[k]), (1e-4 if scaled else 2e-5), "core update")
    s.close()


def test_batched_recipe_graph_replay_per_problem():
    """The batched recipe at its stated size: 64 independent N = 3 problems,
    each I_n ~ U{30..200} and R_n ~ U{4..16} drawn independently (rectangular
    slices, Q up to 256), Gaussian planted cores, noise 1e-3, |F| = 256, FP32
    on the tensor cores as three BF16 pieces, launch shape picked by the
    autotuner, every iteration replayed from one captured CUDA graph of the
    device-counter step.  After each replay every problem's cores are
    compared, update by update and element by element, with its own oracle
    step from the same starting cores (the oracle reads X fiber by fiber from
    the planted cores and the device's noise values)."""
    from paper_2303_16492_gb300 import synth
    A = api()
    ws = synth.batched_workloads(64)
    assert len({tuple(w.ranks) for w in ws}) > 32 and any(w.ranks[0] != w.ranks[1] for w in ws)
    Xs, cores_d, lazies, pcs, cfgs = [], [], [], [], []
    gen = torch.Generator(device="cuda")
    for w in ws:
        planted = synth.planted_cores(w)
        P = to_oracle_cores(planted, w.ranks)
        rng = np.random.default_rng(w.seed)
        ent = [tr.tr_entry(P, [int(rng.integers(0, d)) for d in w.dims]) for _ in range(500)]
        sigma = w.noise_rel * float(np.sqrt(np.mean(np.square(ent))))
        gen.manual_seed(w.seed + 1)
        noise_d = torch.randn(int(np.prod(w.dims)), generator=gen, device="cuda", dtype=torch.float32)
        Xd = A.reconstruct([torch.from_numpy(G).to("cuda", torch.float32) for G in planted], w.dims, w.ranks)
        Xd.add_(noise_d, alpha=sigma)
        lazies.append(LazyTensor(P, w.dims, lambda pos, nd=noise_d: nd[torch.from_numpy(pos).cuda()]
                                 .double().cpu().numpy(), sigma))
        init = [G.astype(np.float32) for G in synth.initial_cores(w, float(torch.linalg.vector_norm(Xd.double()) ** 2))]
        Xs.append(Xd)
        cores_d.append([torch.from_numpy(G).cuda() for G in init])
        pcs.append(A.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=A._abi.FP32, alpha=w.alpha,
                                   seed=w.seed + 3))
        cfgs.append(ob.Config(J=w.J, alpha=w.alpha, seed=w.seed + 3))
    side = torch.cuda.Stream()
    s = A.Solver(pcs, Xs, cores_d, stream=side)
    s.autotune(5)
    assert s.tensor_pieces() in (0, 3)   # FP32 on the tensor pieces or the FMA units: same bound
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        s.step_counter(1)
    for t in range(2):
        before = [[c.double().cpu().numpy() for c in cs] for cs in cores_d]
        g.replay()
        torch.cuda.synchronize()
        for p, w in enumerate(ws):
            st = ob.State.new(to_oracle_cores(before[p], w.ranks))
            ob.step(st, lazies[p], cfgs[p], t)
            assert_update_close([c.double().cpu().numpy() for c in cores_d[p]], before[p],
                                [tr.unfold2(G) for G in st.cores], before[p], 2e-5, 2.0 ** -24,
                                what=f"problem {p} core")
    s.close()
