"""Sample-sharded iterations (trsgd_shard_plan / trsgd_step_partial /
trsgd_step_apply) on one GPU: the ranks' partial sums, gathered in rank
order and summed by the library in a fixed order, give the single-device
iteration bit for bit (plain and scaled, H = F and an independent H, a rank
without samples).  Ranks are emulated one after the other on the same GPU;
no kernel waits on another."""
import numpy as np
import pytest
import torch

from oracle import brsgd as ob
from tests.gpu_helpers import Case, api, cuda

pytestmark = [pytest.mark.gpu, cuda]


def _pair(bf16, **cfg):
    """Two grid-path handles on identical copies of X and the cores."""
    A = api()
    case = Case(dims=[130, 100, 90], ranks=[20, 20, 20], J=1200, prec=1, alpha=0.05, **cfg)
    case.solver.close()
    pc = A.ProblemConfig(dims=case.dims, ranks=case.ranks, J=case.J,
                         prec=A._abi.BF16_MIXED if bf16 else A._abi.FP32, x_dtype=A._abi.DTYPE_F32,
                         alpha=0.05, seed=case.ocfg.seed, path=A._abi.PATH_GRID,
                         **{k: v for k, v in cfg.items() if k in ("variant", "J_H", "damping", "rule", "eta")})
    ca = [c.clone() for c in case.cores_d]
    cb = [c.clone() for c in case.cores_d]
    return A, A.Solver([pc], [case.Xd], [ca]), ca, A.Solver([pc], [case.Xd], [cb]), cb


def _sharded_step(sh, t, world):
    """One iteration as `world` ranks would run it, emulated one rank after
    the other: each rank's partials into its slot of the gathered buffer,
    then the apply over all of them."""
    plans = [sh.shard_plan(t, r, world) for r in range(world)]
    g = torch.empty(world * plans[0].gsplits_max * plans[0].gelems, device="cuda")
    h = torch.empty(world * plans[0].hsplits_max * plans[0].helems, device="cuda") if plans[0].helems else None
    for r, p in enumerate(plans):
        gs = g[r * p.gsplits_max * p.gelems:(r + 1) * p.gsplits_max * p.gelems]
        hs = h[r * p.hsplits_max * p.helems:(r + 1) * p.hsplits_max * p.helems] if h is not None else None
        sh.step_partial(t, p, gs, hs)
    sh.step_apply(t, g, world * plans[0].gsplits_max, h, world * plans[0].hsplits_max if h is not None else 0)
    return plans


@pytest.mark.parametrize("world", [2, 3, 8])
@pytest.mark.parametrize("cfg", [dict(), dict(variant=ob.VARIANT_SCALED, damping=1e-3),
                                 dict(variant=ob.VARIANT_SCALED, J_H=700, damping=1e-3),
                                 dict(rule=ob.RULE_ADAGRAD, eta=0.01)],
                         ids=["plain", "scaled", "scaled_H", "adagrad"])
@pytest.mark.parametrize("bf16", [False, True], ids=["fp32x3", "bf16"])
def test_sharded_steps_equal_single_device_steps(world, cfg, bf16):
    """Against trsgd_step where it runs the same kernels (FP32 pieces, the
    scaled variant), and against the one-rank plan where trsgd_step takes the
    fused BF16 kernel (plain direction), whose sums run in another order."""
    from paper_2303_16492_gb300.shard import unit_ranges
    A, ref, ref_cores, sh, sh_cores = _pair(bf16, **cfg)
    fused = bf16 and cfg.get("variant", 0) == 0
    for t in range(4):
        if fused:
            _sharded_step(ref, t, 1)
        else:
            ref.step(t)
        plans = [sh.shard_plan(t, r, world) for r in range(world)]
        # the plan follows the documented dealing rule and covers every sample once
        for r, p in enumerate(plans):
            j0, j1, cnt, mx = unit_ranges(1200, p.gunit, world, r)
            assert (p.j0, p.j1, p.gsplits, p.gsplits_max) == (j0, j1, cnt, mx)
        assert [p.j0 for p in plans][0] == 0 and plans[-1].j1 == 1200
        assert all(plans[r].j1 == plans[r + 1].j0 for r in range(world - 1))
        if world == 8:
            assert any(p.gsplits == 0 for p in plans)   # a rank without samples
        _sharded_step(sh, t, world)
        torch.cuda.synchronize()
        for a, b in zip(sh_cores, ref_cores):
            assert torch.equal(a, b), t
    ref.close()
    sh.close()


def test_shard_calls_reject_bad_ranges_and_other_paths():
    A, ref, _, sh, _ = _pair(False)
    p = sh.shard_plan(0, 0, 2)
    bad = A._abi.Shard.from_buffer_copy(p)
    bad.j0 = 1           # not on a unit boundary
    g = torch.empty(4 * p.gsplits_max * p.gelems, device="cuda")
    with pytest.raises(A._abi.TrsgdError):
        sh.step_partial(0, bad, g)
    bad = A._abi.Shard.from_buffer_copy(p)
    bad.mode = (p.mode + 1) % 3   # not iteration 0's mode
    with pytest.raises(A._abi.TrsgdError):
        sh.step_partial(0, bad, g)
    with pytest.raises(A._abi.TrsgdError):
        sh.shard_plan(0, 2, 2)
    ref.close()
    sh.close()
    c = Case(dims=[12, 9, 10], ranks=[3, 4, 2], J=40, prec=1)   # cluster path
    with pytest.raises(A._abi.TrsgdError) as ei:
        c.solver.shard_plan(0, 0, 2)
    assert ei.value.status == A._abi.EUNSUPPORTED
