"""GPU parity of reconstruction, relative error, the adjoint (autograd) and
batched stepping against the oracle."""
import numpy as np
import pytest
import torch

from oracle import brsgd as ob
from oracle import tr
from tests._util import random_cores, to_lib_cores
from tests.gpu_helpers import Case, api, cuda, assert_close, assert_update_close

pytestmark = [pytest.mark.gpu, cuda]


@pytest.mark.parametrize("dims,ranks", [([20, 21, 22], [3, 4, 2]), ([9, 8, 7, 6], [2, 3, 4, 2]),
                                        ([70, 3, 5], [5, 2, 3]), ([5, 6], [3, 2]), ([4, 3, 5, 3, 4], [2, 2, 1, 3, 2])])
@pytest.mark.parametrize("prec", [0, 1])
def test_reconstruct_matches_element_formula(dims, ranks, prec):
    A = api()
    cores = random_cores(dims, ranks, seed=3, std=0.7)
    want = tr.reconstruct(cores)
    dt = torch.float64 if prec == 0 else torch.float32
    cd = [torch.from_numpy(G).to("cuda", dt) for G in to_lib_cores(cores)]
    got = A.reconstruct(cd, dims, ranks).double().cpu().numpy().reshape(dims, order="F")
    assert_close(got, want, (1e-13 if prec == 0 else 2e-6), "got")


def test_rel_error_matches_oracle():
    case = Case(dims=[18, 17, 16], ranks=[3, 3, 3], J=30, prec=0, alpha=0.05, noise_rel=0.1)
    r_true = case.solver.rel_error(0, case.Xtd)
    r_x = case.solver.rel_error(0)
    assert abs(r_true - tr.rse(case.state.cores, case.X_true)) < 1e-13 * max(1, r_true)
    assert abs(r_x - tr.rse(case.state.cores, case.X)) < 1e-13 * max(1, r_x)


@pytest.mark.parametrize("dims,ranks,n", [([12, 11, 10], [3, 4, 2], 1), ([7, 6, 5, 6, 7], [2, 3, 2, 3, 2], 3),
                                          ([20, 20, 20, 20, 20], [8, 8, 8, 8, 8], 0), ([9, 10], [3, 4], 1)])
def test_adjoint_all_cores_matches_oracle(dims, ranks, n):
    """trsgd_sampled_loss_grad against the oracle's product-rule gradient of
    the sampled loss (itself pinned by finite differences)."""
    A = api()
    cores = random_cores(dims, ranks, seed=5, std=(ranks[0] * ranks[1]) ** -0.25)
    X = np.random.default_rng(6).standard_normal(dims).astype(np.float32).astype(np.float64)
    cores = [c.astype(np.float32).astype(np.float64) for c in cores]
    J = 64
    idx = ob.draw_indices(9, 4, n, J, dims, None)
    XS = ob.sampled_fibers(X, n, idx)
    w = np.random.default_rng(7).uniform(0.5, 1.5, J).astype(np.float32).astype(np.float64)
    loss = ob.sampled_loss(cores, n, idx, XS, w)
    grads = ob.sampled_loss_grads(cores, n, idx, XS, w)
    cd = [torch.from_numpy(G).to("cuda", torch.float32) for G in to_lib_cores(cores)]
    idx_d = torch.from_numpy(np.where(idx < 0, 0, idx).astype(np.int32)).cuda()
    XS_d = torch.from_numpy(np.ascontiguousarray(XS.T).astype(np.float32)).cuda()
    w_d = torch.from_numpy(w.astype(np.float32)).cuda()
    lg, gg = A.sampled_loss_grad(cd, dims, ranks, n, idx_d, XS_d, w_d)
    assert abs(float(lg.item()) - loss) < 1e-5 * abs(loss)
    for k in range(len(dims)):
        assert_close(gg[k].double().cpu().numpy(), tr.unfold2(grads[k]), 3e-5, "gg[k]")


def test_autograd_function_backward():
    """TRLoss.apply: torch autograd routes the hand-written adjoint to every core."""
    A = api()
    dims, ranks, n = [10, 9, 8], [2, 3, 2], 2
    cores = random_cores(dims, ranks, seed=8, std=0.6)
    X = np.random.default_rng(9).standard_normal(dims)
    idx = ob.draw_indices(1, 2, n, 32, dims, None)
    XS = ob.sampled_fibers(X, n, idx)
    w = np.ones(32)
    grads = ob.sampled_loss_grads(cores, n, idx, XS, w)
    cd = [torch.from_numpy(G).to("cuda", torch.float32).requires_grad_(True) for G in to_lib_cores(cores)]
    idx_d = torch.from_numpy(np.where(idx < 0, 0, idx).astype(np.int32)).cuda()
    XS_d = torch.from_numpy(np.ascontiguousarray(XS.T).astype(np.float32)).cuda()
    w_d = torch.ones(32, device="cuda")
    L = A.TRLoss.apply(idx_d, XS_d, w_d, dims, ranks, n, *cd)
    (2.0 * L).backward()
    for k in range(3):
        assert_close(cd[k].grad.double().cpu().numpy(), 2.0 * tr.unfold2(grads[k]), 3e-5, "cd[k]")


def test_batched_problems_match_independent_oracle_runs():
    """Several problems of uneven dims and ranks stepped together in one
    persistent launch: each equals its own oracle trajectory."""
    A = api()
    rng = np.random.default_rng(12)
    specs = []
    for p in range(6):
        dims = [int(v) for v in rng.integers(8, 30, size=3)]
        ranks = [int(v) for v in rng.integers(2, 6, size=3)]
        specs.append((dims, ranks))
    Xs, cores_d, states, cfgs, pcs = [], [], [], [], []
    for p, (dims, ranks) in enumerate(specs):
        cores = random_cores(dims, ranks, seed=100 + p, std=(ranks[0] * ranks[1]) ** -0.25)
        X = tr.reconstruct(random_cores(dims, ranks, seed=200 + p, std=(ranks[0] * ranks[1]) ** -0.25))
        Xs.append(torch.from_numpy(np.ascontiguousarray(X.ravel(order="F"))).cuda())
        cores_d.append([torch.from_numpy(G).cuda() for G in to_lib_cores(cores)])
        states.append((ob.State.new(cores), X))
        cfgs.append(ob.Config(J=24 + p, alpha=0.02, seed=50 + p))
        pcs.append(A.ProblemConfig(dims=dims, ranks=ranks, J=24 + p, prec=0, alpha=0.02, seed=50 + p))
    s = A.Solver(pcs, Xs, cores_d)
    s.run(0, 40)
    for p in range(6):
        st, X = states[p]
        ob.run(st, X, cfgs[p], 40)
        for k in range(3):
            assert_close(cores_d[p][k].cpu().numpy(), tr.unfold2(st.cores[k]), 1e-11, "cores_d[p][k]")


def test_mixed_variant_batch_on_tensor_pieces():
    """Plain and scaled problems stepped together in one launch, FP32 on the
    tensor cores as three BF16 pieces, clusters of several CTAs.  With a
    scaled problem in the launch, CTA 0 of every cluster takes no samples (it
    factorises the Gram matrix of a scaled problem meanwhile), so CTA 0 of a
    plain problem updates its rows of G_n from a zero partial gradient.  Every
    problem's cores are compared, update by update and element by element,
    with its own oracle step from the same starting cores."""
    from tests._util import make_problem
    A = api()
    rng = np.random.default_rng(31)
    variants = [ob.VARIANT_PLAIN, ob.VARIANT_SCALED, ob.VARIANT_PLAIN, ob.VARIANT_SCALED]
    Xs, Xd, cores_d, pcs, cfgs, ranks_l = [], [], [], [], [], []
    for p, var in enumerate(variants):
        dims = [int(v) for v in rng.integers(20, 45, size=3)]
        ranks = [int(v) for v in rng.integers(3, 6, size=3)]
        std = (ranks[0] * ranks[1]) ** -0.25
        _, _, X = make_problem(dims, ranks, 300 + p, noise_rel=0.05, std=std)
        X = X.astype(np.float32).astype(np.float64)
        start = [G.astype(np.float32).astype(np.float64) for G in random_cores(dims, ranks, 400 + p, std=0.5 * std)]
        alpha = 0.3 if var == ob.VARIANT_SCALED else 0.05
        Xs.append(X)
        Xd.append(torch.from_numpy(np.ascontiguousarray(X.ravel(order="F")).astype(np.float32)).cuda())
        cores_d.append([torch.from_numpy(G.astype(np.float32)).cuda() for G in to_lib_cores(start)])
        pcs.append(A.ProblemConfig(dims=dims, ranks=ranks, J=150, prec=A._abi.FP32, alpha=alpha, variant=var,
                                   seed=60 + p))
        cfgs.append(ob.Config(J=150, alpha=alpha, variant=var, seed=60 + p))
        ranks_l.append(ranks)
    s = A.Solver(pcs, Xd, cores_d)
    assert s.tensor_pieces() == 3
    for t in range(3):
        before = [[c.double().cpu().numpy() for c in cs] for cs in cores_d]
        s.run(t, 1)
        torch.cuda.synchronize()
        for p, var in enumerate(variants):
            N = 3
            st = ob.State.new([tr.fold2(before[p][k], ranks_l[p][k], ranks_l[p][(k + 1) % N]) for k in range(N)])
            ob.step(st, Xs[p], cfgs[p], t)
            assert_update_close([c.double().cpu().numpy() for c in cores_d[p]], before[p],
                                [tr.unfold2(G) for G in st.cores], before[p],
                                1e-4 if var == ob.VARIANT_SCALED else 2e-5, 2.0 ** -24,
                                what=f"problem {p} core")
    s.close()


def test_adjoint_is_bit_reproducible():
    """The sampled-loss adjoint adds its per-sample terms in a fixed order (no
    atomics): two calls on the same inputs give identical bits, here with
    many samples hitting the same slices (J = 2048 over I_k = 12)."""
    A = api()
    dims, ranks, n = [12, 10, 11, 9], [3, 4, 2, 3], 1
    cores = random_cores(dims, ranks, seed=41, std=0.6)
    X = np.random.default_rng(42).standard_normal(dims)
    J = 2048
    idx = ob.draw_indices(3, 7, n, J, dims, None)
    XS = ob.sampled_fibers(X, n, idx)
    w = np.random.default_rng(43).uniform(0.5, 1.5, J)
    cd = [torch.from_numpy(G).to("cuda", torch.float32) for G in to_lib_cores(cores)]
    idx_d = torch.from_numpy(np.where(idx < 0, 0, idx).astype(np.int32)).cuda()
    XS_d = torch.from_numpy(np.ascontiguousarray(XS.T).astype(np.float32)).cuda()
    w_d = torch.from_numpy(w.astype(np.float32)).cuda()
    l1, g1 = A.sampled_loss_grad(cd, dims, ranks, n, idx_d, XS_d, w_d)
    l2, g2 = A.sampled_loss_grad(cd, dims, ranks, n, idx_d, XS_d, w_d)
    assert torch.equal(l1, l2)
    for a, b in zip(g1, g2):
        assert torch.equal(a, b)
    grads = ob.sampled_loss_grads(cores, n, idx, XS, w)
    for k in range(len(dims)):
        assert_close(g1[k].double().cpu().numpy(), tr.unfold2(grads[k]), 3e-5, f"g[{k}]")
