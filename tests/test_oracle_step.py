"""Pins of one TR-BRSGD / TR-ScaledBRSGD iteration (oracle, CPU only).

Closed forms (planted exact fit, full enumeration, weighted least squares,
damping limit, AdaGrad first step), finite differences, the exact variance of
Theorem variance by enumeration, Monte-Carlo unbiasedness and descent, and
recovery of planted cores.
"""
import numpy as np
import pytest

from oracle import brsgd as ob
from oracle import tr
from tests._util import make_problem, random_cores

DIMS, RANKS = [5, 6, 4], [2, 3, 2]


def _all_columns(dims, n):
    N = len(dims)
    Jn = int(np.prod([dims[k] for k in range(N) if k != n]))
    return np.array([ob.decode_column(c, n, dims) for c in range(Jn)], dtype=np.int64)


def _uniform_pF(idx, n, cores):
    return ob.sample_probability(idx, n, [ob.uniform_dist(G) for G in cores])


def test_planted_exact_fit_gives_zero_step():
    """Noise-free planted data: E = 0, g = 0 and the step leaves the cores
    unchanged (Eq. S_gradient on an exact fit)."""
    planted, _, X = make_problem(DIMS, RANKS, seed=1)
    st = ob.State.new(planted)
    cfg = ob.Config(J=16, alpha=0.5, seed=3)
    for t in range(6):
        rec = ob.step(st, X, cfg, t)
        assert np.max(np.abs(rec["E"])) < 1e-12
        assert np.max(np.abs(rec["g"])) < 1e-12
    for G, P in zip(st.cores, planted):
        assert np.allclose(G, P, atol=1e-12)


def test_sampled_rows_and_fibers_match_full_unfoldings():
    """Algorithm 2: Z(j, :) = G^{!=n}_{[2]}(col_j, :) and X_S(:, j) = X_[n](:, col_j)."""
    cores = random_cores(DIMS, RANKS, seed=2)
    X = np.random.default_rng(3).standard_normal(DIMS)
    for n in range(3):
        idx = ob.draw_indices(5, 9, n, 12, DIMS, None)
        Zfull = tr.subchain_unfold(cores, n)
        Xn = tr.unfold_mode(X, n)
        Z = ob.sampled_subchain(cores, n, idx)
        XS = ob.sampled_fibers(X, n, idx)
        for j in range(12):
            col = 0
            stride = 1
            for k in tr.ring_order(n, 3):
                col += idx[j, k] * stride
                stride *= DIMS[k]
            assert np.allclose(Z[j], Zfull[col], rtol=1e-13, atol=1e-14)
            assert np.array_equal(XS[:, j], Xn[:, col])


@pytest.mark.parametrize("n", [0, 1, 2])
def test_full_enumeration_gives_gradient_over_Jn(n):
    """F = every row once with uniform p: g = grad f / J_n exactly
    (Eq. S_gradient against Eq. gradient)."""
    cores = random_cores(DIMS, RANKS, seed=4)
    X = np.random.default_rng(5).standard_normal(DIMS)
    idx = _all_columns(DIMS, n)
    pF = _uniform_pF(idx, n, cores)
    _, _, _, g, Jn = ob.estimate_gradient(cores, X, n, idx, pF)
    assert np.allclose(g * Jn, tr.full_gradient(cores, X, n), rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("n", [0, 1, 2])
def test_full_gradient_central_differences(n):
    """Eq. gradient against central finite differences of f, every coordinate."""
    cores = random_cores([3, 4, 3], [2, 2, 2], seed=6)
    X = np.random.default_rng(7).standard_normal([3, 4, 3])
    grad = tr.full_gradient(cores, X, n)
    h = 1e-5
    G2 = tr.unfold2(cores[n])
    fd = np.zeros_like(G2)
    for i in range(G2.shape[0]):
        for q in range(G2.shape[1]):
            for s in (+1, -1):
                Gp = G2.copy()
                Gp[i, q] += s * h
                c2 = list(cores)
                c2[n] = tr.fold2(Gp, cores[n].shape[0], cores[n].shape[2])
                fd[i, q] += s * tr.loss(c2, X) / (2 * h)
    assert np.allclose(fd, grad, rtol=1e-6, atol=1e-7)


def _exact_single_sample_variance(cores, X, n, q):
    """E||g - E g||^2 for |F| = 1 by enumerating every row c with prob q_c."""
    idx = _all_columns(DIMS, n)
    gs = []
    for c in range(idx.shape[0]):
        _, _, _, g, Jn = ob.estimate_gradient(cores, X, n, idx[c:c + 1], np.array([q[c]]))
        gs.append(g)
    gs = np.array(gs)
    mean = np.einsum("c,cij->ij", q, gs)
    var = np.einsum("c,c->", q, np.sum((gs - mean) ** 2, axis=(1, 2)))
    return mean, var, Jn


@pytest.mark.parametrize("dist", ["uniform", "euclidean", "optimal"])
def test_exact_variance_matches_theorem(dist):
    """Theorem variance (Eq. var) for |F| = 1, enumerated exactly: the mean is
    grad f / J_n and the variance is Eq. var divided by J_n^2 (the estimator of
    Eq. S_gradient is the paper's f_i-based one divided by J_n).  For the
    optimal q of Eq. optimal_prob it equals Eq. optimal_var / J_n^2 and is the
    smallest of the three."""
    cores = random_cores(DIMS, RANKS, seed=8)
    _, _, X = make_problem(DIMS, RANKS, seed=9, noise_rel=0.3)
    n = 1
    Z = tr.subchain_unfold(cores, n)
    R = tr.unfold2(cores[n]) @ Z.T - tr.unfold_mode(X, n)
    grad = tr.full_gradient(cores, X, n)
    idx = _all_columns(DIMS, n)
    if dist == "uniform":
        q = np.full(Z.shape[0], 1.0 / Z.shape[0])
    elif dist == "euclidean":
        q = ob.sample_probability(idx, n, [ob.euclidean_dist(G) for G in cores])
    else:
        q = ob.optimal_dist(cores, X, n)
    mean, var, Jn = _exact_single_sample_variance(cores, X, n, q)
    assert np.allclose(mean * Jn, grad, rtol=1e-10, atol=1e-10)
    rn = np.linalg.norm(R, axis=0) ** 2
    zn = np.linalg.norm(Z, axis=1) ** 2
    eq_var = np.sum(rn * zn / q) - np.sum(grad ** 2)
    assert np.isclose(var * Jn ** 2, eq_var, rtol=1e-9)
    if dist == "optimal":
        eq_opt = np.sum(np.sqrt(rn * zn)) ** 2 - np.sum(grad ** 2)
        assert np.isclose(var * Jn ** 2, eq_opt, rtol=1e-9)
        q_u = np.full(Z.shape[0], 1.0 / Z.shape[0])
        _, var_u, _ = _exact_single_sample_variance(cores, X, n, q_u)
        assert var <= var_u


def test_monte_carlo_unbiased_minibatch():
    """Lemma unbias_gradient (up to the 1/J_n factor) with |F| = 8 under the
    Euclidean distribution: the mean over M draws of the full step machinery
    is within a chi-square bound of grad f / J_n, with the per-entry variance
    taken from the exact single-sample enumeration."""
    cores = random_cores(DIMS, RANKS, seed=10)
    _, _, X = make_problem(DIMS, RANKS, seed=11, noise_rel=0.5)
    n, J, M = 2, 8, 600
    cfg = ob.Config(J=J, dist=ob.DIST_EUCLIDEAN, seed=21)
    dists = [ob.euclidean_dist(G) for G in cores]
    gs = []
    for t in range(M):
        idx = ob.draw_indices(cfg.seed, t, n, J, DIMS, dists)
        pF = ob.sample_probability(idx, n, dists)
        gs.append(ob.estimate_gradient(cores, X, n, idx, pF)[3])
    gs = np.array(gs)
    idx_all = _all_columns(DIMS, n)
    q = ob.sample_probability(idx_all, n, dists)
    singles = np.array([ob.estimate_gradient(cores, X, n, idx_all[c:c + 1], q[c:c + 1])[3]
                        for c in range(idx_all.shape[0])])
    Jn = idx_all.shape[0]
    mean1 = np.einsum("c,cij->ij", q, singles)
    var1 = np.einsum("c,cij->ij", q, (singles - mean1) ** 2)
    target = tr.full_gradient(cores, X, n) / Jn
    assert np.allclose(mean1, target, rtol=1e-10, atol=1e-12)
    z2 = (gs.mean(axis=0) - target) ** 2 / (var1 / (J * M))
    dof = z2.size
    assert z2.sum() < dof + 6 * np.sqrt(2 * dof)


def test_scaled_step_is_weighted_least_squares():
    """H = F, eta = 0, alpha = 1: G+ = argmin_G ||D^{1/2}(Z G^T - X_S^T)||
    (Eq. scaledsg_direction with Eq. S_hessian), against numpy lstsq."""
    cores = random_cores(DIMS, RANKS, seed=12)
    X = np.random.default_rng(13).standard_normal(DIMS)
    for dist in (ob.DIST_UNIFORM, ob.DIST_EUCLIDEAN):
        st = ob.State.new(cores)
        cfg = ob.Config(J=40, dist=dist, variant=ob.VARIANT_SCALED, alpha=1.0, seed=14)
        rec = ob.step(st, X, cfg, 0, force_mode=0)
        w = np.sqrt(1.0 / rec["pF"])[:, None]
        sol = np.linalg.lstsq(w * rec["Z"], w * rec["XS"].T, rcond=None)[0].T
        assert np.allclose(tr.unfold2(st.cores[0]), sol, rtol=1e-9, atol=1e-10)


def test_full_batch_scaled_step_is_als():
    """Full enumeration, uniform, alpha = 1: the scaled step is the TR-ALS
    update of Algorithm 1 (ScaledGD with alpha = 1, Eq. scaled_gd)."""
    cores = random_cores(DIMS, RANKS, seed=15)
    X = np.random.default_rng(16).standard_normal(DIMS)
    n = 1
    idx = _all_columns(DIMS, n)
    pF = _uniform_pF(idx, n, cores)
    Z, XS, E, g, Jn = ob.estimate_gradient(cores, X, n, idx, pF)
    h = ob.preconditioner(Z, pF, Jn)
    p, _ = ob.scaled_direction(g, h, 0.0)
    new = tr.unfold2(cores[n]) + p
    assert np.allclose(new, ob.als_update(cores, X, n), rtol=1e-9, atol=1e-10)


def test_scaled_gd_alpha_one_is_jacobi_als():
    """TR-ScaledGD with alpha = 1 and no damping replaces every core by its
    TR-ALS update (Algorithm 1) computed from the same iterate: checked
    against numpy's least-squares solver, core by core."""
    cores = random_cores(DIMS, RANKS, seed=21)
    X = np.random.default_rng(22).standard_normal(DIMS)
    new = ob.gd_step(cores, X, 1.0, scaled=True)
    for n in range(len(DIMS)):
        assert np.allclose(tr.unfold2(new[n]), ob.als_update(cores, X, n), rtol=1e-8, atol=1e-10)


def test_gd_first_order_decrease():
    """TR-GD moves every core along -grad_n at once, so the loss decreases by
    alpha * sum_n ||grad_n||^2 to first order: (f(Y) - f(Y_alpha)) / alpha
    tends to that sum as alpha -> 0 (error O(alpha))."""
    cores = random_cores(DIMS, RANKS, seed=23)
    X = np.random.default_rng(24).standard_normal(DIMS)
    f0 = tr.loss(cores, X)
    want = sum(float(np.sum(tr.full_gradient(cores, X, n) ** 2)) for n in range(len(DIMS)))
    errs = []
    for alpha in (1e-7, 1e-8):
        got = (f0 - tr.loss(ob.gd_step(cores, X, alpha), X)) / alpha
        errs.append(abs(got - want) / want)
    assert errs[1] < 2e-5 and errs[1] < errs[0] / 5


def test_damping_limit_recovers_plain_step():
    """Damped preconditioner: with eta^t -> infinity and step alpha * eta^t the
    scaled step tends to the plain BRSGD step, error O(||h|| / eta^t)."""
    cores = random_cores(DIMS, RANKS, seed=17)
    X = np.random.default_rng(18).standard_normal(DIMS)
    plain = ob.step(ob.State.new(cores), X, ob.Config(J=10, alpha=0.01, seed=2), 0)["delta"]
    errs = []
    for eta in (1e3, 1e5):
        rec = ob.step(ob.State.new(cores), X,
                      ob.Config(J=10, variant=ob.VARIANT_SCALED, alpha=0.01 * eta, damping=eta, seed=2), 0)
        errs.append(np.linalg.norm(rec["delta"] - plain) / np.linalg.norm(plain))
    assert errs[1] < 2e-2 * errs[0] + 1e-12 and errs[1] < 1e-3


def test_only_the_chosen_core_changes():
    cores = random_cores(DIMS, RANKS, seed=19)
    X = np.random.default_rng(20).standard_normal(DIMS)
    st = ob.State.new(cores)
    rec = ob.step(st, X, ob.Config(J=10, alpha=0.05, seed=4), 3)
    for k in range(3):
        if k != rec["n"]:
            assert np.array_equal(st.cores[k], cores[k])
    assert not np.array_equal(st.cores[rec["n"]], cores[rec["n"]])


def test_adagrad_first_steps_closed_form():
    """Remark after Algorithm 3 with b = eps = 0: the first step on a core is
    eta * sign(p); the second is eta * p2 / sqrt(p1^2 + p2^2)."""
    cores = random_cores(DIMS, RANKS, seed=21)
    X = np.random.default_rng(22).standard_normal(DIMS)
    st = ob.State.new(cores)
    cfg = ob.Config(J=10, rule=ob.RULE_ADAGRAD, eta=0.03, seed=5)
    r1 = ob.step(st, X, cfg, 0, force_mode=1)
    assert np.allclose(r1["delta"], 0.03 * np.sign(r1["p"]), rtol=1e-14, atol=0)
    r2 = ob.step(st, X, cfg, 1, force_mode=1)
    assert np.allclose(r2["delta"], 0.03 * r2["p"] / np.sqrt(r1["p"] ** 2 + r2["p"] ** 2), rtol=1e-12)
    # a core never chosen keeps a zero accumulator
    assert np.all(st.acc[0] == 0) and np.all(st.acc[2] == 0)


def test_expected_descent_small_step():
    """Proof of Theorem conv_brsgd: for a small step the expected loss after
    one iteration is below the current loss (Monte Carlo over mode and batch)."""
    cores = random_cores(DIMS, RANKS, seed=23, std=0.8)
    _, _, X = make_problem(DIMS, RANKS, seed=24, noise_rel=0.1)
    f0 = tr.loss(cores, X)
    M = 300
    diffs = []
    for t in range(M):
        st = ob.State.new(cores)
        ob.step(st, X, ob.Config(J=6, alpha=1e-3, seed=31), t)
        diffs.append(tr.loss(st.cores, X) - f0)
    diffs = np.array(diffs)
    assert diffs.mean() + 4 * diffs.std() / np.sqrt(M) < 0


def test_recovery_of_planted_cores():
    """Noise-free planted data, start at planted + 1e-2 perturbation:
    fixed-step BRSGD drives the RSE below 1e-8 (interpolation regime)."""
    planted, X_true, X = make_problem([6, 7, 5], [2, 2, 2], seed=25)
    rng = np.random.default_rng(26)
    start = [G + 1e-2 * rng.standard_normal(G.shape) for G in planted]
    st = ob.State.new(start)
    cfg = ob.Config(J=24, alpha=0.05, seed=7)
    r0 = tr.rse(st.cores, X_true)
    ob.run(st, X, cfg, T=4000)
    r1 = tr.rse(st.cores, X_true)
    assert r0 > 1e-3 and r1 < 1e-8


@pytest.mark.parametrize("n", [0, 1, 2])
def test_adjoint_all_cores_central_differences(n):
    """Gradient of the sampled loss w.r.t. every core against central finite
    differences (h = 1e-5), and the core-n block equals Eq. S_gradient's g
    when w_j = 1/(|F| J_n p_F(j))."""
    dims, ranks = [3, 4, 3], [2, 3, 2]
    cores = random_cores(dims, ranks, seed=27)
    X = np.random.default_rng(28).standard_normal(dims)
    idx = ob.draw_indices(3, 1, n, 5, dims, None)
    pF = _uniform_pF(idx, n, cores)
    XS = ob.sampled_fibers(X, n, idx)
    Jn = int(np.prod([dims[k] for k in range(3) if k != n]))
    w = 1.0 / (5 * Jn * pF)
    grads = ob.sampled_loss_grads(cores, n, idx, XS, w)
    h = 1e-5
    for k in range(3):
        fd = np.zeros_like(cores[k])
        for pos in np.ndindex(cores[k].shape):
            for s in (+1, -1):
                c2 = [G.copy() for G in cores]
                c2[k][pos] += s * h
                fd[pos] += s * ob.sampled_loss(c2, n, idx, XS, w) / (2 * h)
        assert np.allclose(fd, grads[k], rtol=1e-6, atol=1e-8)
    g = ob.estimate_gradient(cores, X, n, idx, pF)[3]
    assert np.allclose(tr.unfold2(grads[n]), g, rtol=1e-12, atol=1e-14)


def test_hessian_mean_with_independent_H_by_enumeration():
    """Sec. 3.3, the unbiased-Hessian lemma: with |H| i.i.d. draws from a
    non-uniform p, E[h] = Z^T Z / J_n, Z = G^{!=n}_{[2]} in full.  Exact
    expectation by enumerating every ordered pair of columns (|H| = 2, weight
    p(c1) p(c2)): a normalisation by any count other than |H| (for instance
    the 1/(|F| J_n) printed in Eq. S_hessian, with |F| != |H|) moves the
    mean by the ratio of the two counts."""
    cores = random_cores(DIMS, RANKS, seed=41)
    for n in range(3):
        dists = [ob.euclidean_dist(G) for G in cores]
        idx_all = _all_columns(DIMS, n)
        q = ob.sample_probability(idx_all, n, dists)
        Zf = tr.subchain_unfold(cores, n)
        Jn = Zf.shape[0]
        assert abs(q.sum() - 1.0) < 1e-12 and np.ptp(q) > 0
        mean = np.zeros((Zf.shape[1], Zf.shape[1]))
        for c1 in range(Jn):
            for c2 in range(Jn):
                rows = [c1, c2]
                mean += q[c1] * q[c2] * ob.preconditioner(Zf[rows], q[rows], Jn)
        assert np.allclose(mean, Zf.T @ Zf / Jn, rtol=1e-12, atol=1e-14)


def test_step_hessian_mean_uses_the_H_batch():
    """The step's own h with an independent H (|H| = 7, |F| = 3, Euclidean
    p_H): alpha = 0 keeps the cores fixed, so over M iterations the mean of
    the recorded h minus the damping is a Monte-Carlo estimate of
    Z^T Z / J_n (unbiased-Hessian lemma, Sec. 3.3).  Each entry lies within
    5 standard errors (its variance from the exact single-draw enumeration);
    a 1/(|F| J_n) normalisation would put the mean at 7/3 of the target."""
    cores = random_cores(DIMS, RANKS, seed=42)
    X = np.random.default_rng(43).standard_normal(DIMS)
    n, JH, M, damping = 1, 7, 1500, 1e-3
    cfg = ob.Config(J=3, J_H=JH, dist=ob.DIST_EUCLIDEAN, variant=ob.VARIANT_SCALED, alpha=0.0,
                    damping=damping, seed=44)
    st = ob.State.new(cores)
    hs = np.array([ob.step(st, X, cfg, t, force_mode=n)["h"] for t in range(M)])
    Q = hs.shape[1]
    hs -= damping * np.eye(Q)[None]
    dists = [ob.euclidean_dist(G) for G in cores]
    idx_all = _all_columns(DIMS, n)
    q = ob.sample_probability(idx_all, n, dists)
    Zf = tr.subchain_unfold(cores, n)
    Jn = Zf.shape[0]
    target = Zf.T @ Zf / Jn
    singles = np.einsum("ca,cb->cab", Zf, Zf) / (q[:, None, None] * Jn)
    var1 = np.einsum("c,cab->ab", q, (singles - target[None]) ** 2)
    se = np.sqrt(var1 / (JH * M)) + 1e-15
    assert np.all(np.abs(hs.mean(axis=0) - target) < 5 * se)
    wrong = target * JH / 3
    assert np.mean(np.abs(hs.mean(axis=0) - wrong) > 5 * se) > 0.5


def test_damping_ladder_sequence_and_failure():
    """Reading of the damped preconditioner (Sec. 3.3): when the Cholesky
    factorisation of h + eta I fails, the damping becomes
    eta + 1e-12 tr(h)/Q * 10^m for m = 0, 1, ..., 6, and the step fails after
    that.  h = diag(1, 1, 1, -c) fails while the added damping is below c:
    c = 1e-9 first factors at m = 4 (7.5e-9 > 1e-9 > 7.5e-10); c = 1 never
    does; a zero h (no trace to scale) fails at once."""
    c = 1e-9
    h = np.diag([1.0, 1.0, 1.0, -c])
    L, used = ob.cholesky_damped(h, 0.0)
    tr_h = 3.0 - c
    assert used == pytest.approx(1e-12 * tr_h / 4 * 1e4, rel=1e-14)
    assert np.allclose(L @ L.T, h + used * np.eye(4), rtol=1e-14, atol=1e-18)
    for m in range(4):   # every earlier rung leaves a negative pivot
        assert -c + 1e-12 * tr_h / 4 * 10.0 ** m < 0
    # an explicit damping that already suffices is used unchanged
    L, used = ob.cholesky_damped(np.diag([1.0, 1.0, 0.0]), 0.5)
    assert used == 0.5 and np.allclose(np.diag(L), np.sqrt([1.5, 1.5, 0.5]))
    # exact zero pivot: the first rung (m = 0) already factors
    L, used = ob.cholesky_damped(np.diag([2.0, 0.0, 2.0, 0.0]), 0.0)
    assert used == pytest.approx(1e-12 * 4.0 / 4, rel=1e-14)
    with pytest.raises(ob.NumericError):
        ob.cholesky_damped(np.diag([1.0, 1.0, 1.0, -1.0]), 0.0)
    with pytest.raises(ob.NumericError):
        ob.cholesky_damped(np.zeros((3, 3)), 0.0)


def test_scaled_step_with_zero_subchain_fails_and_damped_one_does_not():
    """Degenerate case of the scaled variant: with every core but G_n zero,
    Z = 0, so h = 0 and no rung of the ladder can factor it (the step raises);
    with a damping eta > 0, h = eta I and the direction -g / eta is zero
    because g = 0 too."""
    cores = random_cores(DIMS, RANKS, seed=45)
    X = np.random.default_rng(46).standard_normal(DIMS)
    n = 0
    zc = [G if k == n else np.zeros_like(G) for k, G in enumerate(cores)]
    with pytest.raises(ob.NumericError):
        ob.step(ob.State.new(zc), X, ob.Config(J=5, variant=ob.VARIANT_SCALED, seed=1), 0, force_mode=n)
    rec = ob.step(ob.State.new(zc), X, ob.Config(J=5, variant=ob.VARIANT_SCALED, damping=0.25, seed=1), 0,
                  force_mode=n)
    assert np.array_equal(rec["h"], 0.25 * np.eye(rec["h"].shape[0]))
    assert not np.any(rec["p"])
