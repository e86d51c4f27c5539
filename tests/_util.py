"""Small helpers shared by the tests (no method arithmetic of their own)."""
from __future__ import annotations

import numpy as np

from oracle import tr


def to_oracle_cores(cores2, ranks):
    """Library-layout cores G_{n(2)} (I_n x R_n R_{n+1}) -> oracle (R_n, I_n, R_{n+1})."""
    N = len(cores2)
    return [tr.fold2(np.asarray(G, dtype=np.float64), ranks[n], ranks[(n + 1) % N])
            for n, G in enumerate(cores2)]


def to_lib_cores(cores):
    return [np.ascontiguousarray(tr.unfold2(G)) for G in cores]


def random_cores(dims, ranks, seed, std=1.0):
    rng = np.random.default_rng(seed)
    N = len(dims)
    return [rng.standard_normal((ranks[n], dims[n], ranks[(n + 1) % N])) * std for n in range(N)]


def make_problem(dims, ranks, seed, noise_rel=0.0, std=1.0):
    """Planted cores, X_true = TR(planted) by the oracle, X = X_true + noise."""
    planted = random_cores(dims, ranks, seed, std)
    X_true = tr.reconstruct(planted)
    X = X_true.copy()
    if noise_rel > 0:
        rng = np.random.default_rng(seed + 1)
        E = rng.standard_normal(X.shape)
        X = X + E * (noise_rel * np.linalg.norm(X_true) / np.linalg.norm(E))
    return planted, X_true, X
