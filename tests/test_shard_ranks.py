"""Host logic of the sample-sharded iteration on CPU (gloo, world sizes 2
and 3): the units of a batch dealt to the ranks cover every sample once;
each rank's partial sums of Eq. S_gradient and Eq. S_hessian (computed by
the oracle on its samples only, the estimator's normalisation by the whole
batch), gathered in rank order by the same all-gather the sharded solver uses
and summed in that order, equal the whole-batch estimators; every rank holds
the same bytes and takes the same scaled step.  The kernels are not involved
(the library's own sums are checked bit for bit on the GPU)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DIMS, RANKS, J, UNIT = [9, 8, 7], [3, 2, 4], 37, 8


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    from tests._util import make_problem, random_cores
    _, _, X = make_problem(DIMS, RANKS, seed=61, noise_rel=0.1)
    return random_cores(DIMS, RANKS, seed=62, std=0.5), X


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from oracle import brsgd as ob
    from paper_2303_16492_gb300.shard import gather_in_rank_order, unit_ranges
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cores, X = _problem()
    t, seed = 3, 17
    n = ob.draw_mode(seed, t, 3)
    idx = ob.draw_indices(seed, t, n, J, DIMS, None)            # every rank: the same counters
    pF = ob.sample_probability(idx, n, [ob.uniform_dist(G) for G in cores])
    j0, j1, cnt, mx = unit_ranges(J, UNIT, world, rank)
    Q = RANKS[n] * RANKS[(n + 1) % 3]
    gl = torch.zeros(mx, DIMS[n] * Q, dtype=torch.float64)
    hl = torch.zeros(mx, Q * Q, dtype=torch.float64)
    for u in range(cnt):   # one partial per unit of this rank's range, scaled by its share of the batch
        a, b = j0 + u * UNIT, min(j0 + (u + 1) * UNIT, j1)
        Z, _, _, g, Jn = ob.estimate_gradient(cores, X, n, idx[a:b], pF[a:b])
        gl[u] = torch.from_numpy((g * (b - a) / J).ravel())
        hl[u] = torch.from_numpy((ob.preconditioner(Z, pF[a:b], Jn) * (b - a) / J).ravel())
    G = gather_in_rank_order(gl.ravel(), world)
    H = gather_in_rank_order(hl.ravel(), world)
    gs = torch.zeros(DIMS[n] * Q, dtype=torch.float64)
    hs = torch.zeros(Q * Q, dtype=torch.float64)
    for z in range(world * mx):   # the fixed order of the library's update
        gs += G[z * DIMS[n] * Q:(z + 1) * DIMS[n] * Q]
        hs += H[z * Q * Q:(z + 1) * Q * Q]
    g = gs.numpy().reshape(DIMS[n], Q)
    h = hs.numpy().reshape(Q, Q)
    p, _ = ob.scaled_direction(g, h, 1e-3)
    q.put((rank, (j0, j1, cnt, mx), g.tobytes(), p.tobytes()))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_partials_gloo(world):
    sys.path.insert(0, ROOT)
    from oracle import brsgd as ob
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ranges = [o[1] for o in out]
    assert ranges[0][0] == 0 and ranges[-1][1] == J
    assert all(ranges[r][1] == ranges[r + 1][0] for r in range(world - 1))
    assert sum(r[2] for r in ranges) == (J + UNIT - 1) // UNIT
    # every rank: the same bytes
    assert len({o[2] for o in out}) == 1 and len({o[3] for o in out}) == 1
    # equal to the whole-batch estimators (up to the order of the sums)
    cores, X = _problem()
    t, seed = 3, 17
    n = ob.draw_mode(seed, t, 3)
    idx = ob.draw_indices(seed, t, n, J, DIMS, None)
    pF = ob.sample_probability(idx, n, [ob.uniform_dist(G) for G in cores])
    Z, _, _, g, Jn = ob.estimate_gradient(cores, X, n, idx, pF)
    p, _ = ob.scaled_direction(g, ob.preconditioner(Z, pF, Jn), 1e-3)
    Q = RANKS[n] * RANKS[(n + 1) % 3]
    got_g = np.frombuffer(out[0][2]).reshape(DIMS[n], Q)
    got_p = np.frombuffer(out[0][3]).reshape(DIMS[n], Q)
    assert np.allclose(got_g, g, rtol=1e-12, atol=1e-15 * np.abs(g).max())
    assert np.allclose(got_p, p, rtol=1e-10, atol=1e-13 * np.abs(p).max())


def test_unit_ranges_rule():
    sys.path.insert(0, ROOT)
    from paper_2303_16492_gb300.shard import unit_ranges
    for total, unit in [(1200, 256), (37, 8), (4096, 1024), (100, 256)]:
        for world in range(1, 10):
            rs = [unit_ranges(total, unit, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == total
            assert all(rs[r][1] == rs[r + 1][0] for r in range(world - 1))
            assert all(r[0] % unit == 0 for r in rs)
            assert max(r[2] for r in rs) == rs[0][3]
            assert sum(r[2] for r in rs) == (total + unit - 1) // unit
