"""Pins of the sampler: Philox4x32-10 known answers, the integer index maps and
the four distributions of Sec. 3.2 (oracle, CPU only)."""
import os

import numpy as np
import pytest

from oracle import brsgd as ob
from oracle import philox as px
from oracle import tr
from tests._util import random_cores

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    """Known-answer vectors of the Philox4x32-10 reference implementation
    (Salmon et al., SC'11)."""
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        w = [int(x, 16) for x in row]
        out = px.philox4x32_10(*w[:6])
        assert [int(o) for o in out] == w[6:]


def test_mulhi64_exact():
    rng = np.random.default_rng(0)
    for _ in range(200):
        u = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
        m = int(rng.integers(1, 2**53))
        assert int(px.mulhi64(np.array([u], dtype=object), m)[0]) == (u * m) >> 64


def test_counter_layout_distinct_streams():
    """Different (t, stream, slot, j) give different draws; the same counter
    gives the same draw (the sampler is a pure function of its counter)."""
    a = px.draw_u64(5, 7, px.STREAM_F, 2, np.arange(4, dtype=np.uint64))
    b = px.draw_u64(5, 7, px.STREAM_F, 2, np.arange(4, dtype=np.uint64))
    c = px.draw_u64(5, 7, px.STREAM_H, 2, np.arange(4, dtype=np.uint64))
    d = px.draw_u64(5, 8, px.STREAM_F, 2, np.arange(4, dtype=np.uint64))
    e = px.draw_u64(6, 7, px.STREAM_F, 2, np.arange(4, dtype=np.uint64))
    assert list(a) == list(b)
    assert len(set(a) | set(c) | set(d) | set(e)) == 16


def _chi2_ok(counts, probs, n):
    exp = probs * n
    keep = exp > 5
    stat = np.sum((counts[keep] - exp[keep]) ** 2 / exp[keep])
    dof = keep.sum() - 1
    return stat < dof + 6 * np.sqrt(2 * dof)


def test_uniform_index_histogram():
    I, J = 37, 40000
    idx = ob.draw_indices(11, 3, 0, J, [5, I, 4], None)
    assert idx[:, 0].min() == -1 and idx[:, 0].max() == -1
    counts = np.bincount(idx[:, 1], minlength=I)
    assert _chi2_ok(counts, np.full(I, 1 / I), J)
    assert idx[:, 2].min() >= 0 and idx[:, 2].max() < 4


def test_mode_draw_uniform():
    modes = np.array([ob.draw_mode(3, t, 5) for t in range(5000)])
    assert _chi2_ok(np.bincount(modes, minlength=5), np.full(5, 0.2), 5000)


def test_integer_cdf_histogram_and_zero_weight():
    p = np.array([0.5, 0.0, 0.25, 0.125, 0.125])
    w, cdf = px.integer_weights(p)
    assert int(cdf[-1]) == 2**52 and w[1] == 0
    u = px.draw_u64(1, 0, px.STREAM_F, 0, np.arange(20000, dtype=np.uint64))
    idx = px.cdf_index(u, cdf)
    counts = np.bincount(idx, minlength=5)
    assert counts[1] == 0
    assert _chi2_ok(counts, p, 20000)


def test_cdf_index_boundaries():
    """The smallest i with target < C[i]: targets exactly at a boundary go right."""
    cdf = np.array([3, 3, 7, 10], dtype=np.uint64)
    # u chosen so that mulhi64(u, 10) equals a given target: u = target * 2^64 / 10 rounded up
    for target, want in [(0, 0), (2, 0), (3, 2), (6, 2), (7, 3), (9, 3)]:
        u = -(-(target << 64) // 10)
        assert (u * 10) >> 64 == target
        assert int(px.cdf_index(np.array([u], dtype=object), cdf)[0]) == want


@pytest.mark.parametrize("seed", [0, 1])
def test_distributions_sum_to_one_and_beta_bounds(seed):
    """Lemma euc_est and Lemma lev_est: the product distribution q over all
    J_n rows satisfies q(i) >= beta_n p^{!=n}(i), checked by brute force."""
    dims, ranks = [6, 7, 5], [2, 3, 2]
    cores = random_cores(dims, ranks, seed)
    N = 3
    for n in range(N):
        Z = tr.subchain_unfold(cores, n)
        order = tr.ring_order(n, N)
        # Euclidean
        pe = [ob.euclidean_dist(G) for G in cores]
        for p in pe:
            assert np.isclose(p.sum(), 1.0) and np.all(p >= 0)
        qe_cols = np.ones(Z.shape[0])
        for col in range(Z.shape[0]):
            row = ob.decode_column(col, n, dims)
            qe_cols[col] = np.prod([pe[k][row[k]] for k in order])
        pz = np.sum(Z ** 2, axis=1) / np.sum(Z ** 2)
        beta_e = 1.0 / np.prod([np.sum(cores[k] ** 2) for k in order])
        # the proof's bound q(i) >= beta_n ||G^{!=n}(:, i, :)||^2 (submultiplicativity);
        # the Lemma's q(i) >= beta_n p^{!=n}(i) follows when ||G^{!=n}||^2 >= 1
        assert np.all(qe_cols >= beta_e * np.sum(Z ** 2, axis=1) - 1e-15)
        assert np.sum(Z ** 2) >= 1.0
        assert np.all(qe_cols >= beta_e * pz - 1e-15)
        assert np.isclose(qe_cols.sum(), 1.0)
        # leverage
        pl = [ob.leverage_dist(G) for G in cores]
        for p in pl:
            assert np.isclose(p.sum(), 1.0) and np.all(p >= 0)
        ql = np.array([np.prod([pl[k][ob.decode_column(c, n, dims)[k]] for k in order])
                       for c in range(Z.shape[0])])
        Qz, _ = np.linalg.qr(Z)
        rank_z = np.linalg.matrix_rank(Z)
        pz_lev = np.sum(Qz[:, :rank_z] ** 2, axis=1) / rank_z
        Rn, Rn1 = ranks[n], ranks[(n + 1) % N]
        beta_l = 1.0 / (Rn * Rn1 * np.prod([ranks[k] ** 2 for k in range(N) if k not in (n, (n + 1) % N)]))
        assert np.all(ql >= beta_l * pz_lev - 1e-12)
        assert np.isclose(ql.sum(), 1.0)


def test_leverage_against_projection_diagonal():
    """l_i = (A (A^T A)^{-1} A^T)_{ii} for full column rank A (textbook),
    independent of the SVD route of the oracle."""
    G = random_cores([9, 12, 9], [2, 2, 2], seed=3)[1]       # G_{(2)} is 12 x 4
    A = tr.unfold2(G)
    P = A @ np.linalg.solve(A.T @ A, A.T)
    assert np.allclose(ob.leverage_dist(G), np.diag(P) / 4, rtol=1e-10, atol=1e-14)


def test_leverage_is_uniform_when_rows_do_not_exceed_columns():
    """I_k <= R_k R_{k+1} with full row rank: every leverage score is 1, so
    the leverage distribution is exactly uniform."""
    G = random_cores([4, 6, 4], [3, 3, 3], seed=4)[1]        # 6 x 9
    assert np.allclose(ob.leverage_dist(G), np.full(6, 1 / 6), rtol=1e-12)


def test_euclidean_is_proportional_to_slice_norms():
    G = random_cores([3, 8, 3], [2, 3, 2], seed=5)[1]
    p = ob.euclidean_dist(G)
    s = np.array([np.sum(G[:, i, :] ** 2) for i in range(8)])
    assert np.allclose(p, s / s.sum(), rtol=1e-14)


def test_optimal_distribution_definition():
    """Eq. optimal_prob by brute force over all J_n fibers."""
    dims, ranks = [4, 5, 3], [2, 2, 3]
    cores = random_cores(dims, ranks, seed=6)
    X = np.random.default_rng(7).standard_normal(dims)
    for n in range(3):
        q = ob.optimal_dist(cores, X, n)
        Z = tr.subchain_unfold(cores, n)
        a = []
        for col in range(Z.shape[0]):
            row = ob.decode_column(col, n, dims)
            fib = X[ob.fiber_index_tuple(row, n)]
            est = np.array([tr.tr_entry(cores, [i if k == n else row[k] for k in range(3)])
                            for i in range(dims[n])])
            a.append(np.linalg.norm(est - fib) * np.linalg.norm(Z[col]))
        a = np.array(a)
        assert np.allclose(q, a / a.sum(), rtol=1e-10)


def test_decode_column_inverts_mode_unfolding():
    dims = [3, 4, 2, 5]
    X = np.random.default_rng(8).standard_normal(dims)
    for n in range(4):
        Xn = tr.unfold_mode(X, n)
        for col in range(Xn.shape[1]):
            row = ob.decode_column(col, n, dims)
            assert np.array_equal(Xn[:, col], X[ob.fiber_index_tuple(row, n)])
