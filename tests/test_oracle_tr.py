"""Pins of the TR definitions of Sec. 2 (oracle, CPU only).

Brute force, invariances and textbook special cases: a dropped term, a wrong
index order or a transposed slice in the oracle fails at least one of these.
"""
import itertools

import numpy as np
import pytest

from oracle import tr
from tests._util import random_cores

SHAPES = [
    ([3, 4, 5], [2, 3, 1]),
    ([2, 3, 2, 4], [1, 2, 3, 2]),
    ([3, 2, 2, 3, 2], [2, 1, 3, 2, 2]),
    ([4, 3, 5], [3, 3, 3]),
]


@pytest.mark.parametrize("dims,ranks", SHAPES)
def test_per_mode_identity_matches_element_formula(dims, ranks):
    """X_[n] = G_{n(2)} (G^{!=n}_{[2]})^T for every n (Sec. 2) against the
    element formula Trace(prod_n G_n(i_n)) evaluated entry by entry."""
    cores = random_cores(dims, ranks, seed=1)
    X = tr.tr_full_bruteforce(cores)
    for n in range(len(dims)):
        Xn = tr.unfold2(cores[n]) @ tr.subchain_unfold(cores, n).T
        assert np.allclose(Xn, tr.unfold_mode(X, n), rtol=1e-12, atol=1e-12)
    assert np.allclose(tr.reconstruct(cores), X, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dims,ranks", SHAPES[:3])
def test_unfoldings_by_explicit_index_maps(dims, ranks):
    """Mode-n and classical unfoldings against their index definitions,
    written as explicit loops over all multi-indices."""
    rng = np.random.default_rng(0)
    X = rng.standard_normal(dims)
    N = len(dims)
    for n in range(N):
        Xn = tr.unfold_mode(X, n)
        Xc = tr.unfold_classical(X, n)
        for idx in itertools.product(*[range(d) for d in dims]):
            # mode-n: i_{n+1} fastest, then ..., i_N, i_1, ..., i_{n-1}
            col, stride = 0, 1
            for k in list(range(n + 1, N)) + list(range(0, n)):
                col += idx[k] * stride
                stride *= dims[k]
            assert Xn[idx[n], col] == X[idx]
            # classical: i_1 fastest, skipping n
            col, stride = 0, 1
            for k in range(N):
                if k == n:
                    continue
                col += idx[k] * stride
                stride *= dims[k]
            assert Xc[idx[n], col] == X[idx]
        assert np.array_equal(tr.fold_mode(Xn, n, dims), X)


def test_multi_index_is_column_major_flat_order():
    dims = [3, 4, 2, 5]
    X = np.arange(np.prod(dims)).reshape(dims, order="F")
    for idx in itertools.product(*[range(d) for d in dims]):
        assert X[idx] == tr.multi_index(idx, dims)


def test_core_unfolding_layout():
    """G_{n(2)}(i, r + r' R_n) = G_n(r, i, r') and fold2 inverts it."""
    G = np.random.default_rng(3).standard_normal((2, 5, 3))
    G2 = tr.unfold2(G)
    for r, i, rp in itertools.product(range(2), range(5), range(3)):
        assert G2[i, r + rp * 2] == G[r, i, rp]
    assert np.array_equal(tr.fold2(G2, 2, 3), G)


def test_subchain_product_and_hadamard_definitions():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((2, 3, 4))
    B = rng.standard_normal((4, 5, 3))
    C = tr.subchain_product(A, B)
    for j1, j2 in itertools.product(range(3), range(5)):
        assert np.allclose(C[:, j1 + j2 * 3, :], A[:, j1, :] @ B[:, j2, :])
    B2 = rng.standard_normal((4, 3, 2))
    H = tr.slices_hadamard(A, B2)
    for j in range(3):
        assert np.allclose(H[:, j, :], A[:, j, :] @ B2[:, j, :])


def test_trace_cyclicity_rotation():
    """Rotating the cores and the index order leaves every entry unchanged."""
    dims, ranks = [3, 4, 2, 3], [2, 3, 2, 1]
    cores = random_cores(dims, ranks, seed=5)
    X = tr.reconstruct(cores)
    for s in range(1, 4):
        rot = cores[s:] + cores[:s]
        Xr = tr.reconstruct(rot)
        assert np.allclose(np.moveaxis(Xr, list(range(4)), [(k + s) % 4 for k in range(4)]), X)


def test_gauge_invariance():
    """G_n(i) -> A_n^{-1} G_n(i) A_{n+1} leaves TR(G) unchanged."""
    dims, ranks = [3, 4, 3], [2, 3, 2]
    cores = random_cores(dims, ranks, seed=6)
    rng = np.random.default_rng(7)
    As = [rng.standard_normal((r, r)) + 3 * np.eye(r) for r in ranks]
    new = []
    for n, G in enumerate(cores):
        A_in = np.linalg.inv(As[n])
        A_out = As[(n + 1) % 3]
        new.append(np.einsum("ab,bic,cd->aid", A_in, G, A_out))
    assert np.allclose(tr.reconstruct(new), tr.reconstruct(cores), rtol=1e-10, atol=1e-10)


def test_rank_one_is_outer_product():
    dims = [3, 4, 5]
    cores = random_cores(dims, [1, 1, 1], seed=8)
    vecs = [G[0, :, 0] for G in cores]
    assert np.allclose(tr.reconstruct(cores), np.einsum("i,j,k->ijk", *vecs))


def test_order_two_is_matrix_product():
    """N = 2: X(i, j) = Trace(G_1(i) G_2(j)) = (A B^T)(i, j) with A = G_{1(2)}
    and B the (I_2 x R_1 R_2) matrix B(j, r + r' R_1) = G_2(r', j, r)."""
    G1 = np.random.default_rng(9).standard_normal((2, 4, 3))
    G2 = np.random.default_rng(10).standard_normal((3, 5, 2))
    A = tr.unfold2(G1)
    B = np.empty((5, 6))
    for j, r, rp in itertools.product(range(5), range(2), range(3)):
        B[j, r + rp * 2] = G2[rp, j, r]
    assert np.allclose(tr.reconstruct([G1, G2]), A @ B.T)


def test_rse_and_loss_definitions():
    dims, ranks = [3, 3, 4], [2, 2, 2]
    cores = random_cores(dims, ranks, seed=11)
    X = tr.reconstruct(cores)
    assert tr.rse(cores, X) == 0.0
    Y = X + 0.5
    assert np.isclose(tr.loss(cores, Y), 0.5 * 0.25 * X.size)
    assert np.isclose(tr.rse(cores, Y), 0.5 * np.sqrt(X.size) / np.linalg.norm(Y))
