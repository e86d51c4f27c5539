"""One TR-BRSGD / TR-ScaledBRSGD iteration, step by step (oracle side).

Test infrastructure only (see ``oracle/__init__``).

The iteration follows Algorithm 3 (TR-BRSGD) of Sec. 3.1 with the sampled
subchain and data of Algorithm 2 (SSDTP):

  1. draw the mode n uniformly from {1..N}                  (Algorithm 3)
  2. for k = n+1..N, 1..n-1 draw |F| slice indices of core k with
     replacement from p_k, and p_F = prod_k p_k(idx_k)      (Algorithm 2)
  3. G^{!=n}(:, F, :) = I  *  G_{n+1}(:, idx, :) * ... * G_{n-1}(:, idx, :)
     (slices-Hadamard products), i.e. rows Z = G^{!=n}_{[2]}(F, :)
  4. X_S = X_[n](:, F): one mode-n fiber per sample
  5. g = (G_{n(2)} Z^T D Z - X_S D Z) / (|F| J_n), D = diag(1/p_F)
                                                            (Eq. S_gradient)
  6. direction p = -g (Algorithm 3) or p = -g h^{-1} with
     h = Z_H^T D_H Z_H / (|H| J_n) + eta^t I             (Eq. S_hessian,
     Eq. scaledsg_direction and the damped preconditioner, Sec. 3.3)
  7. G_{n(2)} += alpha p (Eq. update_brsgd) or the AdaGrad step of the Remark
     after Algorithm 3.

Readings of points the paper leaves open:
  * Eq. S_gradient is implemented literally; its expectation is the full
    gradient divided by J_n (the factor J_n in f_i of Sec. 3.1 is not
    carried into the estimator).
  * Eq. S_hessian is normalised by |H| J_n (it prints |F| J_n; the two agree
    when H = F, the default).
  * With-replacement duplicates stay separate samples.
  * AdaGrad squares the search direction p (the scaled one under
    TR-ScaledBRSGD); its sum runs over the steps at which core n was chosen,
    including the current one; the AdaGrad step replaces alpha; an entry with
    b + sum = 0 gets a zero step.
  * The damping is constant; when the Cholesky factorisation fails the damping
    grows to 1e-12 tr(h)/Q * 10^m for m = 0..6, then the step fails.
  * Euclidean slice norms and the core norm are left-to-right sums (the core
    norm is the sum of the slice norms in increasing i) so that both sides can
    form bit-identical integer sampling weights.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import philox as px
from . import tr

DIST_UNIFORM, DIST_LEVERAGE, DIST_EUCLIDEAN, DIST_OPTIMAL = 0, 1, 2, 3
VARIANT_PLAIN, VARIANT_SCALED = 0, 1
RULE_FIXED, RULE_ADAGRAD = 0, 1


class NumericError(RuntimeError):
    pass


@dataclass
class Config:
    J: int
    dist: int = DIST_UNIFORM
    variant: int = VARIANT_PLAIN
    rule: int = RULE_FIXED
    alpha: float = 0.01
    eta: float = 0.01          # AdaGrad eta (Remark after Algorithm 3)
    b: float = 0.0
    eps: float = 0.0
    damping: float = 0.0       # eta^t of the damped preconditioner (Sec. 3.3)
    J_H: int = 0               # |H|; 0 means H = F
    seed: int = 0


@dataclass
class State:
    cores: list                               # (R_n, I_n, R_{n+1}) float64
    acc: list = field(default_factory=list)   # AdaGrad sums, G_{n(2)} layout

    @staticmethod
    def new(cores):
        cores = [np.array(G, dtype=np.float64, copy=True) for G in cores]
        acc = [np.zeros((G.shape[1], G.shape[0] * G.shape[2])) for G in cores]
        return State(cores, acc)


def dims_of(cores):
    return [G.shape[1] for G in cores]


# --------------------------------------------------------------------------
# Sampling distributions (Sec. 3.2)
# --------------------------------------------------------------------------

def uniform_dist(G):
    """p(i) = 1/I  (uniform distribution, Sec. 3.2)."""
    I = G.shape[1]
    return np.full(I, 1.0 / I)


def euclidean_dist(G):
    """p(i) = ||G(:, i, :)||_F^2 / ||G||_F^2  (Lemma euc_est).

    The slice norm sums the squares in the G_{n(2)} column order
    (r + r' R_n increasing) from left to right; ||G||_F^2 is the left-to-right
    sum of the slice norms in increasing i.
    """
    G2 = tr.unfold2(G)
    s = np.array([np.cumsum(row * row)[-1] for row in G2])   # left-to-right
    total = np.cumsum(s)[-1]
    if not total > 0:
        raise NumericError("Euclidean distribution of a zero core")
    return s / total


def leverage_dist(G):
    """p(i) = l_i(G_{n(2)}) / rank(G_{n(2)})  (Lemma lev_est, Definition of
    leverage scores): l_i = ||Q(i, :)||^2 for an orthonormal basis Q of the
    column space, taken from a thin SVD; the numerical rank counts singular
    values above max(m, n) * eps * s_max."""
    A = tr.unfold2(G)
    U, s, _ = np.linalg.svd(A, full_matrices=False)
    if s.size == 0 or s[0] == 0:
        raise NumericError("leverage distribution of a zero core")
    tol = max(A.shape) * np.finfo(np.float64).eps * s[0]
    rank = int(np.sum(s > tol))
    lev = np.sum(U[:, :rank] ** 2, axis=1)
    return lev / rank


def core_dists(cores, dist: int):
    if dist == DIST_UNIFORM:
        return [uniform_dist(G) for G in cores]
    if dist == DIST_EUCLIDEAN:
        return [euclidean_dist(G) for G in cores]
    if dist == DIST_LEVERAGE:
        return [leverage_dist(G) for G in cores]
    raise ValueError("per-core distributions exist for uniform, Euclidean and leverage")


def optimal_dist(cores, X, n: int):
    """q(i) proportional to ||R_[n](:, i)||_2 ||G^{!=n}_{[2]}(i, :)||_2 over all
    J_n fibers, R_[n] = G_{n(2)} (G^{!=n}_{[2]})^T - X_[n]  (Eq. optimal_prob).
    An exact fit (all residuals zero) falls back to the uniform distribution."""
    Z = tr.subchain_unfold(cores, n)
    R = tr.unfold2(cores[n]) @ Z.T - tr.unfold_mode(X, n)
    a = np.linalg.norm(R, axis=0) * np.linalg.norm(Z, axis=1)
    total = np.sum(a)
    if not total > 0:
        return np.full(Z.shape[0], 1.0 / Z.shape[0])
    return a / total


# --------------------------------------------------------------------------
# Algorithm 2 (SSDTP) and the mode draw of Algorithm 3
# --------------------------------------------------------------------------

def draw_mode(seed: int, t: int, N: int) -> int:
    """n ~ Uniform{0..N-1} (Algorithm 3): mulhi64 of the mode-stream draw."""
    u = px.draw_u64(seed, t, px.STREAM_MODE, 0, 0)
    return int(px.mulhi64(u, N))


def draw_indices(seed, t, n, J, dims, dists, stream=px.STREAM_F):
    """idx[j, k] for k != n drawn with replacement from p_k (Algorithm 2);
    slot n holds -1.  ``dists[k]`` is None for the uniform distribution
    (integer draw mulhi64(u, I_k)) or a probability vector (integer CDF)."""
    N = len(dims)
    idx = np.full((J, N), -1, dtype=np.int64)
    js = np.arange(J, dtype=np.uint64)
    for k in tr.ring_order(n, N):
        u = px.draw_u64(seed, t, stream, k, js)
        if dists is None or dists[k] is None:
            idx[:, k] = px.mulhi64(u, dims[k])
        else:
            _, cdf = px.integer_weights(dists[k])
            idx[:, k] = px.cdf_index(u, cdf)
    return idx


def sample_probability(idx, n, probs):
    """p_F(j) = prod_k p_k(idx[j, k]) over k = n+1..N, 1..n-1 in that order
    (Algorithm 2), one rounded product per factor."""
    J, N = idx.shape
    pF = np.ones(J)
    for k in tr.ring_order(n, N):
        pF = pF * probs[k][idx[:, k]]
    return pF


def sampled_subchain(cores, n, idx):
    """Z = G^{!=n}_{[2]}(F, :) (J x R_n R_{n+1}) built as in Algorithm 2: the
    identity-sliced tensor is multiplied (slices-Hadamard) by
    G_k(:, idx(:, k), :) for k = n+1..N, 1..n-1."""
    N = len(cores)
    J = idx.shape[0]
    Rn1 = cores[(n + 1) % N].shape[0]
    S = np.repeat(np.eye(Rn1)[:, None, :], J, axis=1)      # R_{n+1} x J x R_{n+1}
    for k in tr.ring_order(n, N):
        S = tr.slices_hadamard(S, cores[k][:, idx[:, k], :])
    return tr.unfold_mode(S, 1)                            # S: R_{n+1} x J x R_n


def fiber_index_tuple(idx_row, n):
    return tuple(slice(None) if k == n else int(i) for k, i in enumerate(idx_row))


def sampled_fibers(X, n, idx):
    """X_S = X_[n](:, F): column j is the mode-n fiber of X through the
    sampled indices of row j (per-sample fibers)."""
    J = idx.shape[0]
    XS = np.empty((X.shape[n], J))
    for j in range(J):
        XS[:, j] = X[fiber_index_tuple(idx[j], n)]
    return XS


def decode_column(col, n, dims):
    """Column index of X_[n] -> (i_{n+1}, ..., i_N, i_1, ..., i_{n-1}) by the
    mode-n unfolding (i_{n+1} fastest); returns an idx row with -1 at n."""
    N = len(dims)
    row = [-1] * N
    rem = int(col)
    for k in tr.ring_order(n, N):
        row[k] = rem % dims[k]
        rem //= dims[k]
    return row


# --------------------------------------------------------------------------
# One iteration
# --------------------------------------------------------------------------

def _draw_batch(cores, X, cfg, t, n, J, stream):
    """Indices and p_F of one batch under cfg.dist."""
    dims = dims_of(cores)
    N = len(dims)
    if cfg.dist == DIST_OPTIMAL:
        q = optimal_dist(cores, X, n)
        _, cdf = px.integer_weights(q)
        u = px.draw_u64(cfg.seed, t, px.STREAM_OPT if stream == px.STREAM_F else stream,
                        0, np.arange(J, dtype=np.uint64))
        cols = px.cdf_index(u, cdf)
        idx = np.array([decode_column(c, n, dims) for c in cols], dtype=np.int64).reshape(J, N)
        pF = q[cols]
        return idx, pF
    if cfg.dist == DIST_UNIFORM:
        idx = draw_indices(cfg.seed, t, n, J, dims, None, stream)
        probs = [uniform_dist(G) for G in cores]
    else:
        probs = core_dists(cores, cfg.dist)
        idx = draw_indices(cfg.seed, t, n, J, dims, probs, stream)
    return idx, sample_probability(idx, n, probs)


def cholesky_damped(h, damping):
    """Cholesky of h + damping I; on failure the damping grows to
    1e-12 tr(h)/Q * 10^m, m = 0..6 (reading of the damped preconditioner)."""
    Q = h.shape[0]
    tries = [damping] + [damping + 1e-12 * np.trace(h) / Q * 10.0 ** m for m in range(7)]
    for d in tries:
        try:
            return np.linalg.cholesky(h + d * np.eye(Q)), d
        except np.linalg.LinAlgError:
            continue
    raise NumericError("preconditioner is not positive definite")


def estimate_gradient(cores, X, n, idx, pF):
    """Sampled quantities of one batch: Z = G^{!=n}_{[2]}(F, :), X_S, the
    residual E = G_{n(2)} Z^T - X_S and g of Eq. S_gradient,
    g = (G_{n(2)} Z^T D Z - X_S D Z) / (|F| J_n), D = diag(1/p_F)."""
    dims = dims_of(cores)
    N = len(dims)
    Jn = int(np.prod([dims[k] for k in range(N) if k != n], dtype=np.int64))
    J = idx.shape[0]
    Z = sampled_subchain(cores, n, idx)
    XS = sampled_fibers(X, n, idx)
    G2 = tr.unfold2(cores[n])
    D = np.diag(1.0 / pF)
    E = G2 @ Z.T - XS
    g = (G2 @ Z.T @ D @ Z - XS @ D @ Z) / (J * Jn)
    return Z, XS, E, g, Jn


def preconditioner(ZH, pH, Jn):
    """h = Z_H^T D_H Z_H / (|H| J_n)  (Eq. S_hessian, normalised by |H|)."""
    return ZH.T @ np.diag(1.0 / pH) @ ZH / (ZH.shape[0] * Jn)


def scaled_direction(g, h, damping):
    """p = -g (h + eta^t I)^{-1} through a Cholesky factorisation
    (Eq. scaledsg_direction with the damped preconditioner of Sec. 3.3).
    Returns p and the damping actually used."""
    L, used = cholesky_damped(h, damping)
    return -np.linalg.solve(L.T, np.linalg.solve(L, g.T)).T, used


def step(state: State, X, cfg: Config, t: int, force_mode: int | None = None):
    """Apply iteration t in place to ``state``; return a record of every
    intermediate (n, idx, pF, Z, XS, E, g, h, p, delta)."""
    cores = state.cores
    N = len(cores)
    n = draw_mode(cfg.seed, t, N) if force_mode is None else int(force_mode)

    idx, pF = _draw_batch(cores, X, cfg, t, n, cfg.J, px.STREAM_F)   # Algorithm 2
    Z, XS, E, g, Jn = estimate_gradient(cores, X, n, idx, pF)       # Eq. S_gradient

    h = None
    if cfg.variant == VARIANT_PLAIN:
        p = -g                                                       # Algorithm 3
    else:
        if cfg.J_H > 0:
            idxH, pH = _draw_batch(cores, X, cfg, t, n, cfg.J_H, px.STREAM_H)
            ZH = sampled_subchain(cores, n, idxH)
        else:
            pH, ZH = pF, Z
        h = preconditioner(ZH, pH, Jn)                               # Eq. S_hessian
        p, used = scaled_direction(g, h, cfg.damping)                # Eq. scaledsg_direction
        h = h + used * np.eye(h.shape[0])

    G2 = tr.unfold2(cores[n])
    if cfg.rule == RULE_FIXED:
        delta = cfg.alpha * p                                        # Eq. update_brsgd
    else:
        A = state.acc[n]
        A += p * p
        base = cfg.b + A
        scale = np.zeros_like(base)
        pos = base > 0
        scale[pos] = cfg.eta / base[pos] ** (0.5 + cfg.eps)
        delta = scale * p                                            # AdaGrad Remark

    Rn, Rn1 = cores[n].shape[0], cores[n].shape[2]
    cores[n] = tr.fold2(G2 + delta, Rn, Rn1)
    return dict(n=n, idx=idx, pF=pF, Z=Z, XS=XS, E=E, g=g, h=h, p=p, delta=delta, Jn=Jn)


def run(state: State, X, cfg: Config, T: int, t0: int = 0, X_ref=None, eval_every: int = 0):
    """T iterations from t0; optional RSE history against X_ref (Sec. 4)."""
    hist = []
    for t in range(t0, t0 + T):
        step(state, X, cfg, t)
        if eval_every and X_ref is not None and (t - t0 + 1) % eval_every == 0:
            hist.append((t + 1, tr.rse(state.cores, X_ref)))
    return hist


# --------------------------------------------------------------------------
# Full-batch baselines used only as pins (Sec. 3.1 and 3.3)
# --------------------------------------------------------------------------

def gd_step(cores, X, alpha, scaled=False, damping=0.0):
    """One iteration of the full-gradient methods of Sec. 3, every core from
    the same iterate: TR-GD, G_{n(2)} <- G_{n(2)} - alpha grad_n (the update
    after Eq. gradient), or TR-ScaledGD (Eq. scaled_gd), grad_n multiplied by
    (Z^T Z + damping I)^{-1}, Z = G^{!=n}_{[2]}.  Returns the new cores."""
    new = []
    for n in range(len(cores)):
        grad = tr.full_gradient(cores, X, n)
        if scaled:
            Z = tr.subchain_unfold(cores, n)
            L, _ = cholesky_damped(Z.T @ Z, damping)
            grad = np.linalg.solve(L.T, np.linalg.solve(L, grad.T)).T
        G2 = tr.unfold2(cores[n]) - alpha * grad
        new.append(tr.fold2(G2, cores[n].shape[0], cores[n].shape[2]))
    return new


def als_update(cores, X, n):
    """TR-ALS core update (Algorithm 1): G_{n(2)} = X_[n] Z (Z^T Z)^{-1}."""
    Z = tr.subchain_unfold(cores, n)
    return np.linalg.lstsq(Z, tr.unfold_mode(X, n).T, rcond=None)[0].T


def sampled_loss(cores, n, idx, XS, w):
    """1/2 sum_j w_j ||X_S(:, j) - G_{n(2)} Z(j, :)^T||^2 over a sampled batch."""
    Z = sampled_subchain(cores, n, idx)
    E = tr.unfold2(cores[n]) @ Z.T - XS
    return 0.5 * float(np.sum(w[None, :] * E * E))


def sampled_loss_grads(cores, n, idx, XS, w):
    """Gradient of ``sampled_loss`` w.r.t. every core, in the (R_k, I_k, R_{k+1})
    layout, by the product rule on Trace(G_n(i) G_{n+1}(i_{n+1}) ... ): the
    factor of core k sees the product of the slices before it (A) and after it
    (B) in the cyclic order starting at n; d/dG_k(i_k) = (B M A)^T with
    M = sum_i e(i, j) G_n(i)."""
    N = len(cores)
    J = idx.shape[0]
    Z = sampled_subchain(cores, n, idx)
    G2 = tr.unfold2(cores[n])
    E = G2 @ Z.T - XS
    grads = [np.zeros_like(G) for G in cores]
    grads_n2 = (E * w[None, :]) @ Z
    grads[n] = tr.fold2(grads_n2, cores[n].shape[0], cores[n].shape[2])
    order = tr.ring_order(n, N)
    for j in range(J):
        M = np.einsum("i,aib->ab", E[:, j] * w[j], cores[n])   # R_n x R_{n+1}
        slices = [cores[k][:, idx[j, k], :] for k in order]
        for pos, k in enumerate(order):
            A = np.eye(cores[(n + 1) % N].shape[0])
            for S in slices[:pos]:
                A = A @ S
            B = np.eye(cores[k].shape[2])
            for S in slices[pos + 1:]:
                B = B @ S
            grads[k][:, idx[j, k], :] += (B @ M @ A).T
    return grads
