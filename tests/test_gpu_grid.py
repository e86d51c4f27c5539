"""GPU parity of the whole-GPU path (TRSGD_PATH_GRID) against the FP64 oracle.

The grid path runs an iteration as five kernels over the whole GPU with the
residual and gradient contractions on the tensor cores.  Its draws use the
same Philox counters as the fused kernel and the oracle, so indices, fiber
columns and p_F are bit-exact.

Tolerances (from the arithmetic):
  BF16 operands (BF16_MIXED): G, Z and the weighted residual rounded to BF16
    (2^-9 relative each), products accumulated in FP32: E within 1e-2 and the
    gradient within 2e-2 relative; Z (formed in FP32) within 2e-5; the cores
    after one step within 1e-3.
  FP32 as three BF16 pieces (24 significant bits, six products of piece order
    <= 2): within 2e-5 relative like the FP32 SIMT path.
"""
import numpy as np
import pytest
import torch

from oracle import brsgd as ob
from tests.gpu_helpers import Case, api, assert_close, cuda

pytestmark = [pytest.mark.gpu, cuda]


def _bf16_round(x):
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    return t.to(torch.bfloat16).to(torch.float64).numpy()


SHAPES = [
    dict(dims=[150, 90, 130], ranks=[9, 10, 8], J=300),
    dict(dims=[40, 30, 50, 35], ranks=[5, 4, 6, 3], J=500),
    dict(dims=[30, 40], ranks=[6, 5], J=70),
    dict(dims=[130, 100, 90], ranks=[20, 20, 20], J=600),
]


def _util_oracle(cores2, ranks):
    from tests._util import to_oracle_cores
    return to_oracle_cores(cores2, ranks)


def _grid_case(shape, bf16, start=None, **cfg):
    """A Case on the whole-GPU path; `start` (library layout) replaces the
    initial cores on both sides."""
    A = api()
    case = Case(prec=1, alpha=0.05, **shape, **cfg)
    if start is not None:
        for k, G in enumerate(start):
            case.cores_d[k].copy_(torch.from_numpy(np.asarray(G, dtype=np.float32)))
        case.resync()
        case.before = None
    if bf16:
        case.X = _bf16_round(case.X)
    pc = A.ProblemConfig(dims=case.dims, ranks=case.ranks, J=case.J,
                         prec=A._abi.BF16_MIXED if bf16 else A._abi.FP32, x_dtype=A._abi.DTYPE_F32,
                         alpha=case.ocfg.alpha, seed=case.ocfg.seed, path=A._abi.PATH_GRID,
                         **{k: v for k, v in cfg.items() if k in ("rule", "eta", "b", "eps", "variant", "J_H",
                                                                  "damping")})
    case.solver.close()
    case.solver = A.Solver([pc], [case.Xd], [case.cores_d])
    case.pc = pc
    case.solver.set_debug(True)
    return case


def _check(case, rec, bf16):
    d = case.debug(rec["n"])
    assert d["n"] == rec["n"]
    np.testing.assert_array_equal(d["idx"], rec["idx"])
    np.testing.assert_array_equal(d["pF"], rec["pF"])
    assert_close(d["Z"], rec["Z"], 2e-5, "Z")
    tol_e, tol_g, tol_c = (1e-2, 2e-2, 1e-3) if bf16 else (2e-5, 2e-5, 2e-5)
    assert_close(d["E"], rec["E"], tol_e, "E")
    assert_close(d["g"], rec["g"], tol_g, "g")
    assert_close(d["p"], rec["p"], tol_g, "p")
    case.assert_cores(tol_c, rtol_update=tol_g)   # the update is alpha p (or AdaGrad's step of p)


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s["dims"])) + f"_R{s['ranks'][0]}")
@pytest.mark.parametrize("bf16", [True, False], ids=["bf16", "fp32x3"])
def test_grid_single_steps(shape, bf16):
    case = _grid_case(shape, bf16)
    assert case.solver.launch_shape() == (0, 256)
    for t in range(4):
        case.resync()
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        _check(case, rec, bf16)


def test_grid_adagrad_steps():
    """AdaGrad on the grid path: accumulators and steps against the oracle."""
    case = _grid_case(SHAPES[0], False, rule=ob.RULE_ADAGRAD, eta=0.05)
    for t in range(4):
        case.resync()
        acc = [np.empty((case.dims[k], case.Q(k)), dtype=np.float32) for k in range(3)]
        for k in range(3):
            case.solver.adagrad_state(0, k, acc[k])
            case.state.acc[k] = acc[k].astype(np.float64)
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        _check(case, rec, False)


def test_grid_is_chosen_for_large_ranks_and_follows_the_oracle():
    """R_1 = 20 exceeds the fused kernel, so the automatic choice is the grid
    path.  Uneven ranks give each mode its own padded Q, so the buffers are
    reused across modes of different sizes; 30 iterations without
    resynchronising stay within 1e-4 of the oracle's trajectory."""
    A = api()
    case = Case(dims=[60, 50, 40], ranks=[20, 12, 16], J=400, prec=1, alpha=0.05)
    assert case.solver.launch_shape() == (0, 256)
    with pytest.raises(A._abi.TrsgdError):
        case.solver.step_counter(1)
    for t in range(30):
        ob.step(case.state, case.X, case.ocfg, t)
    case.solver.run(0, 30)
    case.assert_cores(1e-4)
    assert abs(case.solver.rel_error(0, case.Xtd) - float(
        np.linalg.norm(ob.tr.reconstruct(case.state.cores) - case.X_true) / np.linalg.norm(case.X_true))) < 1e-4


# ---- scaled variant on the whole-GPU path (Sec. 3.3) ---------------------------

def _solve_fp64(g, h):
    """-g h^{-1} in FP64 (Cholesky), the reference for the device's solve."""
    L = np.linalg.cholesky(h)
    return -np.linalg.solve(L.T, np.linalg.solve(L, g.T)).T


SCALED_SHAPES = [
    dict(dims=[150, 90, 130], ranks=[9, 10, 8], J=300),      # Q = 90, 80, 72: ragged 32-blocks
    dict(dims=[130, 100, 90], ranks=[20, 20, 20], J=600),    # Q = 400, 13 blocks
    dict(dims=[40, 30, 50, 35], ranks=[5, 4, 6, 3], J=500),  # N = 4, uneven Q
]


@pytest.mark.parametrize("shape", SCALED_SHAPES, ids=lambda s: "x".join(map(str, s["dims"])) + f"_R{s['ranks'][0]}")
@pytest.mark.parametrize("bf16", [False, True], ids=["fp32x3", "bf16"])
@pytest.mark.parametrize("J_H", [0, 700])
def test_grid_scaled_steps(shape, bf16, J_H):
    """Eq. S_hessian and Eq. scaledsg_direction on the whole-GPU path: the
    Gram from three BF16 pieces of Z on the tensor cores (FP32 accuracy in
    both modes), the double-float factorisation and solves.  h element by
    element against the oracle's (2e-5), the direction against an FP64
    Cholesky solve of the device's own h and g (the solve's precision alone:
    1e-6 of the direction's rms, FP32 storage of p), and against the oracle's
    direction within the FP32 bound amplified by cond(h)."""
    A = api()
    case = _grid_case(shape, bf16, variant=ob.VARIANT_SCALED, J_H=J_H, damping=1e-3)
    assert case.solver.launch_shape() == (0, 256)
    for t in range(3):
        case.resync()
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        d = case.debug(rec["n"])
        assert d["n"] == rec["n"]
        np.testing.assert_array_equal(d["idx"], rec["idx"])
        assert_close(d["h"], rec["h"], 2e-5, "h")
        tol_g = 2e-2 if bf16 else 2e-5
        assert_close(d["g"], rec["g"], tol_g, "g")
        assert_close(d["p"], _solve_fp64(d["g"].astype(np.float64), d["h"]), 1e-6, "p vs FP64 solve of device h, g")
        kappa = np.linalg.cond(rec["h"])
        tol_p = tol_g + 2e-7 * kappa
        assert_close(d["p"], rec["p"], tol_p, f"p (cond {kappa:.1e})")
        case.assert_cores(1e-4 if not bf16 else 1e-3, rtol_update=tol_p)


@pytest.mark.parametrize("bf16", [False, True], ids=["fp32x3", "bf16"])
def test_grid_scaled_solve_matches_fp64_at_cond_1e6(bf16):
    """The double-float factorisation and solves against FP64 on a Gram
    matrix of condition number near 1e6: the columns r' of every slice
    G_k(i) are scaled by s_r' (geometric from 1 to 1e-3), so column
    r + r' R_n of Z = G^{!=n}_{[2]} carries s_r and cond(Z^T Z) ~ 1e6.  The
    device's p agrees with an FP64 Cholesky solve of its own h and g to 1e-6
    of the rms (an FP32 factor would be off by ~cond * 2^-24 ~ 6e-2)."""
    from tests._util import random_cores, to_lib_cores
    dims, R, J = [150, 130, 120], 10, 1024
    sc = np.geomspace(1.0, 1e-3, R)
    start = []
    for G in to_lib_cores(random_cores(dims, [R] * 3, seed=4, std=0.3)):
        start.append(G * np.tile(sc[:, None], (1, R)).T.ravel()[None, :])   # column r + r' R scaled by s_r'
    case = _grid_case(dict(dims=dims, ranks=[R] * 3, J=J), bf16, variant=ob.VARIANT_SCALED, start=start)
    seen = []
    for t in range(3):
        case.resync()
        rec = ob.step(case.state, case.X, case.ocfg, t)
        case.solver.step(t)
        d = case.debug(rec["n"])
        kappa = np.linalg.cond(d["h"])
        seen.append(kappa)
        assert_close(d["p"], _solve_fp64(d["g"].astype(np.float64), d["h"]), 1e-6, f"p (cond {kappa:.1e})")
    assert max(seen) > 1e5, seen


def test_grid_scaled_zero_subchain_is_a_numerical_error():
    """Every core but one zero: Z = 0 and h = 0, so no rung of the damping
    ladder factors h (the oracle raises NumericError); the grid path latches
    TRSGD_ENUMERIC and leaves G_n unchanged."""
    A = api()
    case = _grid_case(SCALED_SHAPES[1], False, variant=ob.VARIANT_SCALED)
    for c in case.cores_d:
        c.zero_()
    t = 0
    n = ob.draw_mode(case.ocfg.seed, t, 3)
    case.cores_d[n].normal_()
    before = [c.clone() for c in case.cores_d]
    with pytest.raises(ob.NumericError):
        ob.step(ob.State.new(case.device_cores()), case.X, case.ocfg, t)
    case.solver.step(t)
    with pytest.raises(A._abi.TrsgdError) as ei:
        case.solver.rel_error(0)
    assert ei.value.status == A._abi.ENUMERIC
    for c, b in zip(case.cores_d, before):
        assert torch.equal(c, b)
