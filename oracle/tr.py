"""TR model definitions of Sec. 2, written out plainly (oracle side).

Test infrastructure only (see ``oracle/__init__``).

Conventions
-----------
* A core is a float64 array ``G`` of shape (R_n, I_n, R_{n+1}); its lateral
  slice G_n(i) = G[:, i, :] (Introduction, element-wise TR formula).
* A tensor is a numpy array indexed X[i_1, ..., i_N] (0-based here; the paper
  is 1-based).  Its flat storage in the library has i_1 fastest (Definition
  of the multi-index), i.e. ``X.ravel(order="F")``.
* ``unfold2(G)`` is the classical mode-2 unfolding G_{n(2)} (I_n x R_n R_{n+1},
  column index r + r' R_n), which is also the library's core layout.
"""
from __future__ import annotations

import itertools

import numpy as np


def ring_order(n: int, N: int):
    """Core order n+1, ..., N, 1, ..., n-1 (0-based) used by the subchain
    tensor (Definition of the subchain tensor) and by Algorithm 2."""
    return [(n + s) % N for s in range(1, N)]


def tr_entry(cores, idx):
    """X(i_1..i_N) = Trace(G_1(i_1) G_2(i_2) ... G_N(i_N))  (Introduction)."""
    P = np.eye(cores[0].shape[0])
    for G, i in zip(cores, idx):
        P = P @ G[:, i, :]
    return float(np.trace(P))


def tr_full_bruteforce(cores):
    """Full tensor by the element formula, one entry at a time (tiny sizes)."""
    dims = [G.shape[1] for G in cores]
    X = np.empty(dims)
    for idx in itertools.product(*[range(d) for d in dims]):
        X[idx] = tr_entry(cores, idx)
    return X


def multi_index(idx, dims):
    """overline{i_1 ... i_N} = i_1 + i_2 I_1 + i_3 I_1 I_2 + ... (0-based form
    of the Definition of the multi-index)."""
    off, stride = 0, 1
    for i, d in zip(idx, dims):
        off += i * stride
        stride *= d
    return off


def unfold_mode(X, n: int):
    """Mode-n unfolding X_[n] (I_n x prod_{k!=n} I_k): column index is the
    multi-index of (i_{n+1}, ..., i_N, i_1, ..., i_{n-1}), i_{n+1} fastest."""
    N = X.ndim
    perm = [n] + ring_order(n, N)
    return np.transpose(X, perm).reshape(X.shape[n], -1, order="F")


def fold_mode(Xn, n: int, dims):
    """Inverse of ``unfold_mode``."""
    N = len(dims)
    perm = [n] + ring_order(n, N)
    Y = Xn.reshape([dims[p] for p in perm], order="F")
    return np.transpose(Y, np.argsort(perm))


def unfold_classical(X, n: int):
    """Classical mode-n unfolding X_(n): column multi-index of
    (i_1, ..., i_{n-1}, i_{n+1}, ..., i_N), i_1 fastest."""
    N = X.ndim
    perm = [n] + [k for k in range(N) if k != n]
    return np.transpose(X, perm).reshape(X.shape[n], -1, order="F")


def unfold2(G):
    """G_{n(2)} (I_n x R_n R_{n+1}); entry (i, r + r' R_n) = G[r, i, r']."""
    return unfold_classical(G, 1)


def fold2(G2, Rn: int, Rn1: int):
    """Inverse of ``unfold2``: (I_n x R_n R_{n+1}) -> (R_n, I_n, R_{n+1})."""
    I = G2.shape[0]
    return np.transpose(G2.reshape(I, Rn, Rn1, order="F"), (1, 0, 2))


def subchain_product(A, B):
    """Mode-2 subchain product (Definition): A (I1 x J1 x K), B (K x J2 x I2)
    -> C (I1 x J1 J2 x I2) with C(:, j1 + j2 J1, :) = A(j1) B(j2)."""
    I1, J1, K = A.shape
    K2, J2, I2 = B.shape
    assert K == K2
    C4 = np.einsum("ajk,kmc->amjc", A, B)          # [a, j2, j1, c]
    return C4.reshape(I1, J2 * J1, I2)              # column j1 + j2 J1


def slices_hadamard(A, B):
    """Mode-2 slices-Hadamard product (Definition): (A * B)(j) = A(j) B(j)."""
    assert A.shape[2] == B.shape[0] and A.shape[1] == B.shape[1]
    return np.einsum("ajk,kjc->ajc", A, B)


def subchain_tensor(cores, n: int):
    """G^{!=n} = G_{n+1} x G_{n+2} x ... x G_N x G_1 x ... x G_{n-1}
    (Definition of the subchain tensor), shape (R_{n+1}, J_n, R_n)."""
    order = ring_order(n, len(cores))
    S = cores[order[0]]
    for k in order[1:]:
        S = subchain_product(S, cores[k])
    return S


def subchain_unfold(cores, n: int):
    """G^{!=n}_{[2]} (J_n x R_n R_{n+1}): mode-2 unfolding of the subchain
    tensor; entry (j, r + r' R_n) = G^{!=n}(r', j, r)."""
    return unfold_mode(subchain_tensor(cores, n), 1)


def reconstruct(cores):
    """TR({G_n}) via the per-mode identity X_[1] = G_{1(2)} (G^{!=1}_{[2]})^T
    (Sec. 2, after Eq. tr_als_opt), folded back to a tensor."""
    dims = [G.shape[1] for G in cores]
    X1 = unfold2(cores[0]) @ subchain_unfold(cores, 0).T
    return fold_mode(X1, 0, dims)


def loss(cores, X):
    """f(Y) = 1/2 || TR({G_n}) - X ||_F^2   (Eq. trmin_opt)."""
    return 0.5 * float(np.sum((reconstruct(cores) - X) ** 2))


def full_gradient(cores, X, n: int):
    """grad_{G_{n(2)}} f = G_{n(2)} Z^T Z - X_[n] Z, Z = G^{!=n}_{[2]}
    (Eq. gradient); returned in the G_{n(2)} layout."""
    Z = subchain_unfold(cores, n)
    G2 = unfold2(cores[n])
    return G2 @ Z.T @ Z - unfold_mode(X, n) @ Z


def rse(cores, X_true):
    """RSE = ||TR(G) - X_true||_F / ||X_true||_F   (Sec. 4)."""
    Xh = reconstruct(cores)
    return float(np.linalg.norm((Xh - X_true).ravel()) / np.linalg.norm(X_true.ravel()))
