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
from tests.gpu_helpers import Case, api, cuda, assert_close

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


def _grid_case(shape, bf16, **cfg):
    A = api()
    case = Case(prec=1, alpha=0.05, **shape, **cfg)
    if bf16:
        case.X = _bf16_round(case.X)
    pc = A.ProblemConfig(dims=case.dims, ranks=case.ranks, J=case.J,
                         prec=A._abi.BF16_MIXED if bf16 else A._abi.FP32, x_dtype=A._abi.DTYPE_F32,
                         alpha=case.ocfg.alpha, seed=case.ocfg.seed, path=A._abi.PATH_GRID,
                         **{k: v for k, v in cfg.items() if k in ("rule", "eta", "b", "eps")})
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
