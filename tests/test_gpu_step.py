"""GPU parity of the fused step kernel against the FP64 oracle.

Tolerances (derived from the arithmetic, stated per path):
  FP64 path: every recorded intermediate and the cores within 1e-12 relative
    for single steps from a shared state, 1e-10 after long trajectories.
  FP32 path: single steps within 2e-5 relative (sums of at most a few
    hundred FP32 products: sqrt(K) * 2^-24 ~ 1e-6 typical, K * 2^-24 ~ 1e-5
    worst case); indices and p_F bit-exact whenever both sides start from the
    same cores.  The same bound holds for the contractions on three BF16
    pieces per operand: each operand is split exactly up to 2^-24 of its
    value and the dropped piece products are below 2^-23 of each term.
"""
import numpy as np
import pytest
import torch

from oracle import brsgd as ob
from oracle import tr
from tests.gpu_helpers import Case, api, assert_close, cuda

pytestmark = [pytest.mark.gpu, cuda]


def _compare_step(case, rec, tol, check_p=True):
    d = case.debug(rec["n"])
    assert d["n"] == rec["n"]
    np.testing.assert_array_equal(d["idx"], rec["idx"])
    np.testing.assert_array_equal(d["pF"], rec["pF"])
    assert_close(d["Z"], rec["Z"], tol, "Z")
    assert_close(d["E"], rec["E"], tol, "E")
    assert_close(d["g"], rec["g"], tol, "g")
    if check_p:
        assert_close(d["p"], rec["p"], tol, "p")
    if "h" in d and rec["h"] is not None:
        assert_close(d["h"], rec["h"], tol, "h")
    case.assert_cores(tol)


SHAPES_FP32 = [
    dict(dims=[12, 9, 10, 11], ranks=[3, 4, 2, 3], J=100),
    dict(dims=[7, 6, 5, 6, 7], ranks=[2, 3, 2, 3, 2], J=64),
    dict(dims=[30, 40], ranks=[4, 3], J=50),
    dict(dims=[9, 8, 10], ranks=[1, 1, 1], J=33),
    dict(dims=[1, 7, 8], ranks=[2, 3, 2], J=20),
    dict(dims=[15, 14, 13], ranks=[4, 5, 3], J=1),
]


@pytest.mark.parametrize("units", ["pieces", "fma"])
@pytest.mark.parametrize("shape", SHAPES_FP32, ids=lambda s: "x".join(map(str, s["dims"])) + f"_J{s['J']}")
@pytest.mark.parametrize("cluster", [1, 4, 16])
def test_fp32_single_steps(shape, cluster, units):
    """FP32 on the FMA units and on the tensor cores as three BF16 pieces per
    operand (the six products of order <= 2): both within the FP32 bound."""
    A = api()
    fu = A._abi.FP32_PIECES if units == "pieces" else A._abi.FP32_FMA
    case = Case(prec=1, alpha=0.05, fp32_units=fu, **shape)
    case.solver.launch_shape(cluster=cluster, threads=256 if cluster == 4 else 512)
    # these shapes are small enough for the pieces at every cluster size
    assert case.solver.tensor_pieces() == (3 if units == "pieces" else 0)
    case.solver.set_debug(True)
    for t in range(4):
        # restart both sides from identical cores so each step is a single-step comparison
        case.resync()
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        _compare_step(case, rec, 2e-5)


@pytest.mark.parametrize("rank", [4, 8, 10, 16])
@pytest.mark.parametrize("cluster", [1, 16])
def test_fp32_uniform_rank_chain(rank, cluster):
    """Equal ranks take the register-blocked chain (two output columns per
    lane, one lane group per sample): N = 4 runs its first factor on the
    column-major staged slice and the second on a row-major intermediate;
    J = 77 leaves ragged lane groups at both cluster sizes."""
    case = Case(dims=[9, 11, 10, 12], ranks=[rank] * 4, J=77, prec=1, alpha=0.02)
    case.solver.launch_shape(cluster=cluster, threads=512)
    case.solver.set_debug(True)
    for t in range(4):
        case.resync()
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        _compare_step(case, rec, 2e-5)


@pytest.mark.parametrize("cluster", [1, 4])
def test_fp32_slices_staged_in_groups(cluster):
    """N = 5 with equal ranks 8 and J = 300: on one CTA the sampled slices of
    all 300 samples (1 KB each) do not fit shared memory at once, so they are
    staged and chained in groups of samples with a ragged last group."""
    case = Case(dims=[8, 7, 9, 6, 8], ranks=[8] * 5, J=300, prec=1, alpha=0.02)
    case.solver.launch_shape(cluster=cluster, threads=512)
    case.solver.set_debug(True)
    for t in range(4):
        case.resync()
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        _compare_step(case, rec, 2e-5)


def test_fp32_chunked_rows_ragged_tail():
    """I_n = 300 with Q = 256 does not fit one chunk: rows are processed in
    chunks with a ragged last chunk."""
    case = Case(dims=[300, 20, 25], ranks=[16, 16, 16], J=64, prec=1, alpha=0.01)
    case.solver.launch_shape(cluster=16, threads=512)
    case.solver.set_debug(True)
    for t in range(3):
        case.resync()
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        _compare_step(case, rec, 3e-5)


@pytest.mark.parametrize("cluster", [1, 8])
def test_fp64_single_steps(cluster):
    case = Case(dims=[20, 20, 20], ranks=[3, 3, 3], J=50, prec=0, alpha=0.01)
    case.solver.launch_shape(cluster=cluster, threads=512)
    case.solver.set_debug(True)
    for t in range(6):
        case.snapshot()
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        _compare_step(case, rec, 1e-12)


def test_fp64_trajectory_2000_steps():
    """Plain method, FP64 20^3, R=3, J=50, alpha 0.01, 2000 steps: cores and RSE
    within 1e-10 relative of the oracle trajectory."""
    from paper_2303_16492_gb300 import synth
    A = api()
    w = synth.workload("c1")
    planted = synth.planted_cores(w)
    from tests._util import to_oracle_cores
    pc_or = to_oracle_cores(planted, w.ranks)
    X_true = tr.reconstruct(pc_or)
    noise = synth.noise(w.dims, w.seed + 1).reshape(w.dims, order="F")
    X = X_true + noise * (w.noise_rel * np.linalg.norm(X_true) / np.linalg.norm(noise))
    init = synth.initial_cores(w, float(np.sum(X * X)))
    st = ob.State.new(to_oracle_cores(init, w.ranks))
    cfg = ob.Config(J=w.J, alpha=w.alpha, seed=w.seed + 3)
    ob.run(st, X, cfg, 2000)
    rse_oracle = tr.rse(st.cores, X_true)

    Xd = torch.from_numpy(np.ascontiguousarray(X.ravel(order="F"))).cuda()
    Xtd = torch.from_numpy(np.ascontiguousarray(X_true.ravel(order="F"))).cuda()
    cores = [torch.from_numpy(np.ascontiguousarray(G)).cuda() for G in init]
    s = A.Solver([A.ProblemConfig(dims=w.dims, ranks=w.ranks, J=w.J, prec=0, alpha=w.alpha, seed=w.seed + 3)],
                 [Xd], [cores])
    done, _ = s.run(0, 2000)
    assert done == 2000
    rse_gpu = s.rel_error(0, Xtd)
    for n, G in enumerate(cores):
        O = tr.unfold2(st.cores[n])
        assert_close(G.cpu().numpy(), O, 1e-10, "G")
    assert abs(rse_gpu - rse_oracle) <= 1e-10 * rse_oracle


@pytest.mark.parametrize("prec", [0, 1])
def test_euclidean_distribution_steps(prec):
    """Lemma euc_est sampling: from identical cores the integer CDF of both sides
    is bit-identical, so the indices and p_F are bit-exact."""
    case = Case(dims=[14, 11, 13], ranks=[3, 2, 4], J=80, prec=prec, alpha=0.05, dist=ob.DIST_EUCLIDEAN)
    case.solver.set_debug(True)
    tol = 1e-12 if prec == 0 else 2e-5
    for t in range(6):
        # restart the oracle from the device cores: its tables are then built from
        # the same values as the kernel's in-kernel table update, so p_F is bit-exact
        case.resync()
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        _compare_step(case, rec, tol)


@pytest.mark.parametrize("prec,damping", [(0, 0.0), (0, 0.5), (1, 0.0)])
def test_scaled_variant_steps(prec, damping):
    """Eq. scaledsg_direction with the damped preconditioner: h and p against
    the oracle's Cholesky solve."""
    case = Case(dims=[16, 15, 14], ranks=[3, 2, 3], J=90, prec=prec, alpha=0.3, variant=ob.VARIANT_SCALED,
                damping=damping)
    case.solver.set_debug(True)
    tol = 1e-11 if prec == 0 else 1e-4
    for t in range(5):
        if prec == 1:
            case.resync()
        else:
            case.snapshot()
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        _compare_step(case, rec, tol)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("ranks", [[3, 11, 3], [6, 8, 7]])
def test_scaled_variant_ragged_diagonal_blocks(prec, ranks):
    """Eq. scaledsg_direction through the blocked solves when Q is not a
    multiple of their 32-row diagonal blocks: Q = 33 (the last block one row)
    and 9 for ranks 3, 11, 3; Q = 48, 56, 42 (two blocks, the second ragged)
    for ranks 6, 8, 7; FP64 and double-float solves."""
    case = Case(dims=[12, 11, 10], ranks=ranks, J=120, prec=prec, alpha=0.3, variant=ob.VARIANT_SCALED,
                damping=0.05)
    case.solver.set_debug(True)
    tol = 1e-11 if prec == 0 else 1e-4
    for t in range(6):
        if prec == 1:
            case.resync()
        else:
            case.snapshot()
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        _compare_step(case, rec, tol)


@pytest.mark.parametrize("units", ["pieces", "fma"])
@pytest.mark.parametrize("J_H", [0, 70])
def test_scaled_variant_row_chunks(units, J_H):
    """Scaled variant with I_1 = 300 rows of Q = 100 columns: the rows of G_1
    are processed in chunks (128 rows on the tensor-core path), each CTA
    keeps its owned rows of every chunk for the solve against the damped
    Gram factor; with and without an independent Hessian batch H."""
    A = api()
    fu = A._abi.FP32_PIECES if units == "pieces" else A._abi.FP32_FMA
    case = Case(dims=[300, 9, 11], ranks=[10, 10, 10], J=60, prec=1, alpha=0.3, variant=ob.VARIANT_SCALED,
                damping=0.05, J_H=J_H, fp32_units=fu)
    # 8 CTAs: three chunks of 128 rows on the pieces; 4 CTAs on the FMA units: two chunks
    case.solver.launch_shape(cluster=8 if units == "pieces" else 4, threads=512)
    assert case.solver.tensor_pieces() == (3 if units == "pieces" else 0)
    case.solver.set_debug(True)
    for t in range(6):
        case.resync()
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        _compare_step(case, rec, 1e-4)


@pytest.mark.parametrize("prec,J_H", [(0, 0), (0, 70), (1, 70)])
def test_scaled_variant_leverage(prec, J_H):
    """Scaled variant with leverage-score sampling (Lemma lev_est) for F and
    the Hessian batch: tall cores (I_1 = 300 rows in three chunks of the
    tensor-core path, Q = 25), the weights 1 / (|H| J_n p_H) in h."""
    case = Case(dims=[300, 30, 28], ranks=[5, 5, 5], J=60, prec=prec, alpha=0.09, variant=ob.VARIANT_SCALED,
                J_H=J_H, dist=ob.DIST_LEVERAGE)
    case.solver.set_debug(True)
    tol = 1e-10 if prec == 0 else 1e-4
    for t in range(8):
        case.resync()
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        d = case.debug(rec["n"])
        np.testing.assert_array_equal(d["idx"], rec["idx"])
        np.testing.assert_allclose(d["pF"], rec["pF"], rtol=1e-12 if prec == 0 else 1e-5)
        assert_close(d["g"], rec["g"], tol, "g")
        assert_close(d["h"], rec["h"], tol, "h")
        assert_close(d["p"], rec["p"], tol, "p")
        case.assert_cores(tol)


def test_leverage_table_of_rank_deficient_core():
    """A tall float core whose columns are all equal (rank 1): its Gram cannot
    be factored, so the leverage table is rebuilt from ridge-shifted Grams and
    normalised.  The run goes on without a numerical error latched, every
    drawn index is in range with a positive, finite p_F, and the cores stay
    finite."""
    A = api()
    dims, ranks, J = [40, 9, 10], [4, 4, 4], 64
    rng = np.random.default_rng(3)
    X = torch.from_numpy(rng.standard_normal(int(np.prod(dims))).astype(np.float32)).cuda()
    cores = [torch.from_numpy((rng.standard_normal((dims[k], ranks[k] * ranks[(k + 1) % 3])) * 0.3)
                              .astype(np.float32)).cuda() for k in range(3)]
    cores[0][:] = cores[0][:, :1]          # every column equal: A^T A has rank 1
    pc = A.ProblemConfig(dims=dims, ranks=ranks, J=J, prec=1, alpha=1e-3, dist=ob.DIST_LEVERAGE, seed=5)
    s = A.Solver([pc], [X], [cores])
    s.set_debug(True)
    for t in range(12):
        s.step(t)
        torch.cuda.synchronize()
        n = int(s.get_debug(A._abi.DBG_MODE, np.int32, 1)[0])
        idx = s.get_debug(A._abi.DBG_IDX, np.int32, J * 3).reshape(J, 3)
        pf = s.get_debug(A._abi.DBG_PF, np.float64, J)
        assert np.all(pf > 0) and np.all(np.isfinite(pf))
        for k in range(3):
            if k != n:
                assert np.all((idx[:, k] >= 0) & (idx[:, k] < dims[k]))
    for c in cores:
        assert torch.isfinite(c).all()
    s.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("scaled", [False, True], ids=["gd", "scaled_gd"])
@pytest.mark.parametrize("shape", [dict(dims=[12, 9, 10], ranks=[3, 4, 2]),
                                   dict(dims=[7, 6, 5, 8], ranks=[2, 3, 2, 3])],
                         ids=["N3", "N4"])
def test_full_gradient_iterations(shape, scaled, prec):
    """TR-GD and TR-ScaledGD (Sec. 3, Eq. gradient and Eq. scaled_gd): every
    core updated from the same iterate, three iterations, each compared with
    the oracle from shared cores."""
    case = Case(prec=prec, J=16, alpha=0.05, **shape)
    damping = 1e-3 if scaled else 0.0
    tol = 1e-10 if prec == 0 else (1e-4 if scaled else 2e-5)
    for _ in range(3):
        start = case.device_cores()
        # the step is compared, so that a wrong gradient cannot hide behind the
        # cores' own size: alpha makes it ~5 % of the cores
        unit = ob.gd_step(start, case.X, 1.0, scaled=scaled, damping=damping)
        du = np.sqrt(sum(np.sum((u - g) ** 2) for u, g in zip(unit, start)))
        alpha = 0.05 * np.sqrt(sum(np.sum(g ** 2) for g in start)) / du
        want = ob.gd_step(start, case.X, alpha, scaled=scaled, damping=damping)
        case.solver.gd_step(scaled=scaled, alpha=alpha, damping=damping)
        torch.cuda.synchronize()
        for G, O, S in zip(case.device_cores(), want, start):
            assert_close(G - S, O - S, tol, "core update")


def test_full_gradient_rejects_unsupported():
    """Non-uniform handles (their sampling tables would go stale) and
    invalid arguments are refused on the host."""
    A = api()
    case = Case(dims=[8, 7, 9], ranks=[2, 2, 2], J=8, prec=1, dist=ob.DIST_EUCLIDEAN)
    with pytest.raises(A._abi.TrsgdError):
        case.solver.gd_step(alpha=0.1)
    case = Case(dims=[8, 7, 9], ranks=[2, 2, 2], J=8, prec=1)
    with pytest.raises(A._abi.TrsgdError):
        case.solver.gd_step(alpha=float("nan"))


def test_adagrad_steps_and_state():
    case = Case(dims=[12, 10, 11], ranks=[2, 3, 2], J=40, prec=0, rule=ob.RULE_ADAGRAD, eta=0.02)
    case.solver.set_debug(True)
    for t in range(8):
        case.snapshot()
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        _compare_step(case, rec, 1e-12)
    for k in range(3):
        acc = np.empty((case.dims[k], case.Q(k)), dtype=np.float64)
        case.solver.adagrad_state(0, k, acc)
        assert_close(acc, case.state.acc[k], 1e-12, f"AdaGrad sum of core {k}")


def test_scaled_adagrad_fp32():
    case = Case(dims=[10, 12, 9], ranks=[2, 2, 3], J=60, prec=1, variant=ob.VARIANT_SCALED,
                rule=ob.RULE_ADAGRAD, eta=0.05, damping=1e-3)
    case.solver.set_debug(True)
    for t in range(4):
        case.resync()
        acc = [np.empty((case.dims[k], case.Q(k)), dtype=np.float32) for k in range(3)]
        for k in range(3):
            case.solver.adagrad_state(0, k, acc[k])
            case.state.acc[k] = acc[k].astype(np.float64)
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        _compare_step(case, rec, 1e-4)


def test_non_finite_step_is_latched():
    """A divergent step size makes the cores non-finite: the device status
    word turns that into TRSGD_ENUMERIC at the next synchronising call."""
    A = api()
    case = Case(dims=[8, 9, 7], ranks=[2, 2, 2], J=16, prec=1, alpha=1e30)
    with pytest.raises(A._abi.TrsgdError) as ei:
        case.solver.run(0, 20)
    assert ei.value.status == A._abi.ENUMERIC


def test_run_stops_at_tolerance():
    """Sec. 4 stopping rule: trsgd_run stops once RSE <= tol (checked every chunk)."""
    case = Case(dims=[10, 10, 10], ranks=[2, 2, 2], J=40, prec=0, alpha=0.05, noise_rel=0.0, init_std=0.0)
    # start from the planted cores: RSE is already ~0
    done, r = case.solver.run(0, 1000, chunk=10, tol=1.0, Xref=case.Xtd)
    assert done == 10 and 0 <= r <= 1.0


def _bf16_round(a):
    t = torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64)
    return t.numpy()


@pytest.mark.parametrize("shape,cluster", [
    (dict(dims=[12, 9, 10, 11], ranks=[3, 4, 2, 3], J=100), 4),
    (dict(dims=[40, 30, 20], ranks=[4, 4, 4], J=90), 16),
    (dict(dims=[150, 20, 25], ranks=[8, 8, 8], J=64), 2),     # 2 row chunks of the 128-row tile
    (dict(dims=[30, 40], ranks=[4, 3], J=17), 1),
])
def test_bf16_mixed_tensor_core_steps(shape, cluster):
    """BF16_MIXED: fibers stored in bfloat16, residual on tensor cores with
    split-BF16 operands (hi*hi + hi*lo + lo*hi, about 2^-16 relative per
    product), gradient on tensor cores with the weighted residual in BF16
    (2^-9 relative per entry), FP32 accumulation.  The oracle gets the same
    BF16-rounded X.  Bounds: Z 2e-5, E 2e-4, g 1e-2, cores 1e-4 (one step)."""
    A = api()
    case = Case(prec=1, alpha=0.05, **shape)
    Xb = _bf16_round(case.X)
    case.X = Xb
    pc = A.ProblemConfig(dims=case.dims, ranks=case.ranks, J=case.J, prec=A._abi.BF16_MIXED,
                         x_dtype=A._abi.DTYPE_F32, alpha=0.05, seed=case.ocfg.seed)
    case.solver.close()
    case.solver = A.Solver([pc], [case.Xd], [case.cores_d])
    case.pc = pc
    case.solver.launch_shape(cluster=cluster, threads=512)
    case.solver.set_debug(True)
    for t in range(4):
        case.resync()
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        d = case.debug(rec["n"])
        np.testing.assert_array_equal(d["idx"], rec["idx"])
        assert_close(d["Z"], rec["Z"], 2e-5, "Z")
        assert_close(d["E"], rec["E"], 2e-4, "E")
        assert_close(d["g"], rec["g"], 1e-2, "g")
        case.assert_cores(1e-4, rtol_update=1e-2)   # the update is alpha p = -alpha g


@pytest.mark.parametrize("prec,dims,ranks", [
    (0, [20, 18, 22], [3, 3, 3]),        # tall cores (I > Q): l_i from the Cholesky factor of A^T A
    (0, [8, 30, 9], [3, 4, 3]),          # mixed: core 0 wide (8 <= 12), cores 1, 2 tall
    (1, [10, 12, 9], [4, 4, 4]),         # all wide (I <= Q): leverage is exactly uniform
])
def test_leverage_distribution_steps(prec, dims, ranks):
    """Lemma lev_est: p_k(i) = l_i(G_{k(2)}) / rank, rebuilt for the updated
    core after every step.  FP64 leverage scores agree with the oracle's SVD to
    ~1e-15, so the integer CDFs agree and indices and p_F match."""
    case = Case(dims=dims, ranks=ranks, J=60, prec=prec, alpha=0.05, dist=ob.DIST_LEVERAGE)
    case.solver.set_debug(True)
    tol = 1e-12 if prec == 0 else 2e-5
    for t in range(6):
        case.resync()
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        d = case.debug(rec["n"])
        np.testing.assert_array_equal(d["idx"], rec["idx"])
        assert_close(d["pF"], rec["pF"], 1e-12, "pF")
        assert_close(d["g"], rec["g"], tol, "g")
        case.assert_cores(tol)


@pytest.mark.parametrize("prec,dist", [(0, ob.DIST_UNIFORM), (0, ob.DIST_EUCLIDEAN), (1, ob.DIST_UNIFORM)])
def test_scaled_independent_hessian_batch(prec, dist):
    """Eq. S_hessian with H independent of F: |H| = 70 rows drawn on the H
    stream (same distributions), weights 1/(|H| J_n p_H)."""
    case = Case(dims=[16, 15, 14], ranks=[3, 2, 3], J=45, prec=prec, alpha=0.3, variant=ob.VARIANT_SCALED,
                damping=1e-3, J_H=70, dist=dist)
    case.solver.set_debug(True)
    tol = 1e-11 if prec == 0 else 1e-4
    for t in range(4):
        case.resync()
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        _compare_step(case, rec, tol)


def _encode_col(row, n, dims):
    col, stride = 0, 1
    N = len(dims)
    for s in range(1, N):
        k = (n + s) % N
        col += int(row[k]) * stride
        stride *= dims[k]
    return col


def test_optimal_distribution_fp64_steps():
    """Theorem variance / Eq. optimal_prob: the full residual of mode n is
    evaluated every step and |F| whole columns are drawn with the integer CDF;
    in FP64 the weights agree with the oracle to ~1e-15, so the draws match."""
    case = Case(dims=[9, 8, 10], ranks=[2, 3, 2], J=40, prec=0, alpha=0.05, dist=ob.DIST_OPTIMAL, noise_rel=0.2)
    case.solver.set_debug(True)
    for t in range(5):
        case.resync()
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        d = case.debug(rec["n"])
        np.testing.assert_array_equal(d["idx"], rec["idx"])
        assert_close(d["pF"], rec["pF"], 1e-12, "pF")
        assert_close(d["g"], rec["g"], 1e-11, "g")
        case.assert_cores(1e-11)


def test_optimal_distribution_fp32_draws_valid():
    """FP32 residuals move the integer CDF by up to ~1e-6 of its total, so a
    draw may land in a neighbouring column near a boundary: every device draw
    must lie within that tolerance of the oracle's CDF interval, and its p_F
    must equal the oracle's q of the drawn column to FP32 accuracy."""
    from oracle import philox as px
    case = Case(dims=[12, 10, 11], ranks=[3, 3, 3], J=64, prec=1, alpha=0.05, dist=ob.DIST_OPTIMAL, noise_rel=0.2)
    case.solver.set_debug(True)
    for t in range(3):
        case.resync()
        n = ob.draw_mode(case.ocfg.seed, t, 3)
        q = ob.optimal_dist(case.state.cores, case.X, n)
        _, cdf = px.integer_weights(q)
        W = int(cdf[-1])
        case.solver.step(t)
        d = case.debug(n)
        u = px.draw_u64(case.ocfg.seed, t, px.STREAM_OPT, 0, np.arange(case.J, dtype=np.uint64))
        for j in range(case.J):
            col = _encode_col(d["idx"][j], n, case.dims)
            target = (int(u[j]) * W) >> 64
            lo = int(cdf[col - 1]) if col > 0 else 0
            tol = int(1e-5 * W)
            assert lo - tol <= target < int(cdf[col]) + tol
            assert abs(d["pF"][j] - q[col]) <= 1e-4 * q[col]
        ob.step(case.state, case.X, case.ocfg, t)


@pytest.mark.parametrize("prec", [0, 1])
def test_scaled_damping_ladder_first_rung(prec):
    """A zero column in every slice of the core before n in the ring zeroes
    columns of Z, so h has exact zero rows: the undamped factorisation fails
    and the first rung of the ladder (damping 1e-12 tr(h)/Q) factors it, on
    both sides.  The recorded h carries that damping on its diagonal."""
    case = Case(dims=[12, 11, 10], ranks=[3, 2, 4], J=60, prec=prec, alpha=0.2, variant=ob.VARIANT_SCALED)
    case.solver.set_debug(True)
    t = 0
    n = ob.draw_mode(case.ocfg.seed, t, 3)
    k = (n + 2) % 3
    Rk = case.ranks[k]
    case.cores_d[k].view(case.dims[k], -1)[:, :Rk] = 0   # column 0 of every slice G_k(i)
    case.resync()
    rec = ob.step(case.state, case.X, case.ocfg, t)
    case.solver.step(t)
    d = case.debug(rec["n"])
    h_or = rec["h"]
    Q = h_or.shape[0]
    zero = [q for q in range(Q) if q % case.ranks[n] == 0]
    used = h_or[zero[0], zero[0]]
    assert used > 0 and np.allclose(np.diag(h_or)[zero], used)
    tr_h = np.trace(h_or) - Q * used
    assert used == pytest.approx(1e-12 * tr_h / Q, rel=1e-10)
    assert_close(np.diag(d["h"])[zero], np.diag(h_or)[zero], 1e-5, "damped zero pivots")
    assert_close(d["h"], h_or, 1e-11 if prec == 0 else 2e-5, "h")
    case.assert_cores(1e-10 if prec == 0 else 1e-4)


@pytest.mark.parametrize("prec", [0, 1])
def test_scaled_zero_subchain_is_a_numerical_error(prec):
    """Every core but G_n zero: Z = 0, h = 0, no rung of the ladder factors
    it (the oracle raises); the kernel latches TRSGD_ENUMERIC, reported at the
    next synchronising call, and the cores stay as they were."""
    A = api()
    case = Case(dims=[12, 11, 10], ranks=[3, 2, 4], J=60, prec=prec, alpha=0.2, variant=ob.VARIANT_SCALED)
    t = 0
    n = ob.draw_mode(case.ocfg.seed, t, 3)
    for k, c in enumerate(case.cores_d):
        if k != n:
            c.zero_()
    before = [c.clone() for c in case.cores_d]
    with pytest.raises(ob.NumericError):
        ob.step(ob.State.new(case.device_cores()), case.X, case.ocfg, t)
    case.solver.step(t)
    with pytest.raises(A._abi.TrsgdError) as ei:
        case.solver.rel_error(0)
    assert ei.value.status == A._abi.ENUMERIC
    for c, b in zip(case.cores_d, before):
        assert torch.equal(c, b)


def test_cores_changed_between_launches_are_used():
    """FP32 on the tensor pieces keeps every core as BF16 operand pieces that
    each launch rebuilds: cores overwritten by the caller between launches
    must be the ones the next steps use.  After a 3-step launch the device
    cores get fresh values in place; then a 2-step launch (the pieces of the
    updated rows rewritten inside it) and single steps are compared with the
    oracle from the new values.  I_1 = 150 rows: two row chunks of G_1."""
    A = api()
    case = Case(dims=[150, 20, 25], ranks=[8, 8, 8], J=64, prec=1, alpha=0.05)
    assert case.solver.tensor_pieces() == 3
    case.solver.run(0, 3)
    rng = np.random.default_rng(77)
    for G in case.cores_d:
        G.copy_(torch.from_numpy(rng.standard_normal(tuple(G.shape)).astype(np.float32) * 0.3).cuda())
    torch.cuda.synchronize()
    case.resync()
    for t in (3, 4):
        ob.step(case.state, case.X, case.ocfg, t)
    case.solver.run(3, 2)
    torch.cuda.synchronize()
    case.assert_cores(2e-5)
    for t in (5, 6):
        case.resync()
        ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        torch.cuda.synchronize()
        case.assert_cores(2e-5)
