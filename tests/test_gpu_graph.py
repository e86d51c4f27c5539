"""Device-resident iteration counter, CUDA-graph replay and checkpoint/resume.

The sampler is a pure function of (seed, t, stream, slot, j) (Philox
counters), so an iteration depends only on t and the current state: a run
split into pieces — by the device counter, by graph replays, or by a
checkpoint written to the host and loaded into a new handle — must give
bit-identical cores.
"""
import numpy as np
import pytest
import torch

from tests.gpu_helpers import Case, cuda
from tests.gpu_helpers import api as api_mod

pytestmark = [pytest.mark.gpu, cuda]


def _fresh(case, stream=None, cores=None):
    A = case.A
    cs = [c.clone() for c in (cores if cores is not None else case.start_cores)]
    return A.Solver([case.pc], [case.Xd], [cs], stream=stream), cs


def _case(**kw):
    c = Case([12, 9, 10, 7], [3, 4, 2, 3], 40, seed=5, prec=1, alpha=0.05, **kw)
    c.start_cores = [t.clone() for t in c.cores_d]
    c.solver.close()
    return c


def _same(a, b):
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("dist", [0, 2])
def test_counter_pieces_equal_one_run(dist):
    case = _case(dist=dist)
    ref, ref_cores = _fresh(case)
    ref.run(0, 30)
    s, cores = _fresh(case)
    for _ in range(3):
        s.step_counter(10)
    torch.cuda.synchronize()
    _same(cores, ref_cores)
    # the counter can be moved: iterations 30..39 from both
    ref.run(30, 10)
    s.set_counter(30)
    s.step_counter(10)
    torch.cuda.synchronize()
    _same(cores, ref_cores)
    ref.close()
    s.close()


def test_graph_replays_continue_the_sequence():
    case = _case()
    ref, ref_cores = _fresh(case)
    ref.run(0, 4 * 25)
    side = torch.cuda.Stream()
    s, cores = _fresh(case, stream=side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        s.step_counter(25)
    # capture records the launches without running them: the counter is still 0
    for _ in range(4):
        g.replay()
    torch.cuda.synchronize()
    _same(cores, ref_cores)
    assert s.launch_count() >= 1
    ref.close()
    s.close()


@pytest.mark.parametrize("rule,dist", [(1, 0), (1, 2), (0, 1)])
def test_checkpoint_resume_is_bit_exact(rule, dist):
    """Cores and AdaGrad accumulators saved to the host after T iterations
    and loaded into a new handle continue exactly like one 2T run; the
    distribution tables are rebuilt from the saved cores at init."""
    case = _case(rule=rule, dist=dist, eta=0.05)
    T = 20
    ref, ref_cores = _fresh(case)
    ref.run(0, 2 * T)
    torch.cuda.synchronize()

    a, cores_a = _fresh(case)
    a.run(0, T)
    torch.cuda.synchronize()
    saved = [c.cpu().clone() for c in cores_a]
    acc = []
    if rule == 1:
        for k, c in enumerate(saved):
            acc.append(a.adagrad_state(0, k, np.empty(c.numel(), dtype=np.float32)).copy())
    a.close()

    b, cores_b = _fresh(case, cores=[c.cuda() for c in saved])
    for k, arr in enumerate(acc):
        b.adagrad_state(0, k, arr, store=True)
    b.run(T, T)
    torch.cuda.synchronize()
    _same(cores_b, ref_cores)
    ref.close()
    b.close()


@pytest.mark.parametrize("threads", [128, 256, 512])
@pytest.mark.parametrize("prec", [0, 1])
def test_pipelined_launch_equals_single_steps(threads, prec):
    """Within one launch of many uniform iterations, the draws and fiber copies
    of iteration t+1 are issued by half of each CTA while the other half
    reduces iteration t.  The draws depend on t only, so one launch of 40
    iterations must give the same cores, bit for bit, as 40 launches of one
    iteration (no pipelining), for every block size."""
    c = Case([12, 9, 10, 7], [3, 4, 2, 3], 40, seed=5, prec=prec, alpha=0.05)
    start = [t.clone() for t in c.cores_d]
    c.solver.close()
    a, ca = _fresh(c, cores=start)
    b, cb = _fresh(c, cores=start)
    for s in (a, b):
        s.launch_shape(cluster=4, threads=threads)
    a.run(0, 40)                 # one launch (no stopping checks)
    for t in range(40):
        b.step(t)
    torch.cuda.synchronize()
    _same(ca, cb)
    a.close()
    b.close()


@pytest.mark.parametrize("prec,dims", [(1, [12, 9, 10, 7]), (1, [300, 20, 25]), (0, [300, 20, 25])],
                         ids=["fp32_pieces", "fp32_bulk_fibers", "fp64_bulk_fibers"])
def test_forced_wait_timeout_is_reported_and_drained(prec, dims):
    """Bounded waits on the failure path: with trsgd_set_wait_limit(-1) the
    first try of every mbarrier wait (tensor-core completion; bulk copies of
    fibers of 1 KB or more, mode 1 of the 300-row shapes) times out at once,
    latches TRSGD_ETIMEOUT, and a second wait of the default length drains
    the operation, so the launch still completes: the next synchronising
    call reports the timeout, the cores are finite and equal to those of a
    run without the forced timeouts, and limit 0 restores normal operation."""
    A = api_mod()
    ranks = [3, 4, 2, 3][:len(dims)]
    c = Case(dims, ranks, 40, seed=5, prec=prec, alpha=0.05)
    start = [t.clone() for t in c.cores_d]
    c.solver.close()
    ref, ref_cores = _fresh(c, cores=start)
    s, cores = _fresh(c, cores=start)
    ref.run(0, 12)
    s.set_wait_limit(-1)
    for t in range(12):
        s.step(t)
    with pytest.raises(A._abi.TrsgdError) as ei:
        s.rel_error(0)
    assert ei.value.status == A._abi.ETIMEOUT
    torch.cuda.synchronize()
    for x, y in zip(cores, ref_cores):
        assert torch.isfinite(x).all()
    _same(cores, ref_cores)
    s.set_wait_limit(0)
    ref.run(12, 4)
    s.run(12, 4)   # synchronising: no status latched any more
    _same(cores, ref_cores)
    ref.close()
    s.close()
