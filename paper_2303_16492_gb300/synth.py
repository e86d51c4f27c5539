"""Seeded synthetic inputs for the TR-BRSGD workloads.

This module only draws random numbers: planted cores (Gaussian, or the
ill-conditioned U S V^T cores of Sec. 4, Experiment II), initial cores, and
noise tensors.  It holds none of the method's arithmetic: the tensor
X_true = TR(planted cores) is formed by the caller (the library's
``reconstruct`` on the GPU, or the oracle in tests), and the noise is scaled
by the caller to its relative norm.

Cores are returned in the library layout G_{n(2)}: a C-contiguous array of
shape (I_n, R_n * R_{n+1}) whose column r + r' R_n holds G_n(r, i, r')
(classical mode-2 unfolding, Sec. 2).  Core n has ranks
(R[n], R[(n + 1) % N]).

Seeds: a workload seed s gives the planted cores (s), the noise (s + 1), the
initial cores (s + 2) and the sampler key (s + 3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian_cores(dims, ranks, std, seed: int, dtype=np.float64):
    """i.i.d. N(0, std^2) cores; ``std`` is a scalar or one value per core."""
    rng = _rng(seed)
    N = len(dims)
    stds = std if np.ndim(std) else [std] * N
    out = []
    for n in range(N):
        Q = ranks[n] * ranks[(n + 1) % N]
        out.append((rng.standard_normal((dims[n], Q)) * stds[n]).astype(dtype))
    return out


def haar_orthonormal(rows: int, cols: int, rng) -> np.ndarray:
    """rows x cols matrix with orthonormal columns, Haar distributed (QR of a
    Gaussian matrix with the signs of R's diagonal moved into Q)."""
    A = rng.standard_normal((rows, cols))
    Qm, Rm = np.linalg.qr(A)
    return Qm * np.sign(np.diag(Rm))[None, :]


def illcond_cores(dims, rank: int, smin: float, seed: int, dtype=np.float64):
    """G_{n(2)} = U_n S V^T (Sec. 4, Experiment II): U_n (I_n x R^2) with
    orthonormal columns, S diagonal geometric from 1 down to ``smin``, V a
    R^2 x R^2 orthogonal matrix shared by all cores.  Needs I_n >= R^2."""
    rng = _rng(seed)
    Q = rank * rank
    V = haar_orthonormal(Q, Q, rng)
    S = np.array([smin ** (i / (Q - 1)) for i in range(Q)]) if Q > 1 else np.ones(1)
    out = []
    for I in dims:
        if I < Q:
            raise ValueError("ill-conditioned cores need I_n >= R^2")
        U = haar_orthonormal(I, Q, rng)
        out.append(((U * S[None, :]) @ V.T).astype(dtype))
    return out


def noise(shape, seed: int, dtype=np.float64):
    """Standard normal noise, flat, i_1 fastest (shape is the tensor dims)."""
    rng = _rng(seed)
    return rng.standard_normal(int(np.prod(shape))).astype(dtype)


def init_std(dims, ranks, x_sq_norm: float, frac: float = 0.01) -> float:
    """Common std s of i.i.d. Gaussian initial cores with
    E||TR(G0)||^2 = frac ||X||^2.  For i.i.d. N(0, s^2) cores every entry has
    E[x^2] = prod_n R_n * s^(2N), so s = (frac ||X||^2 / (prod I prod R))^(1/2N)."""
    N = len(dims)
    target = frac * x_sq_norm / (math.prod(dims) * math.prod(ranks))
    return target ** (1.0 / (2 * N))


@dataclass
class Workload:
    """One synthetic TR workload (dims, ranks, batch, step rule, precision)."""
    name: str
    dims: list
    ranks: list
    J: int
    planted: str = "gaussian"        # "gaussian" | "illcond"
    planted_std: float = 1.0
    smin: float = 1e-3               # ill-conditioned cores: last singular value
    noise_rel: float = 1e-3
    init: str = "scaled"             # "scaled" (init_std) | float std
    alpha: float = 0.01
    variant: int = 0                 # 0 plain, 1 scaled
    rule: int = 0                    # 0 fixed, 1 AdaGrad
    eta: float = 0.0
    damping: float = 0.0
    JH: int = 0                      # |H| of the scaled variant (0: H = F)
    dist: int = 0
    prec: int = 1                    # 0 FP64, 1 FP32, 2 BF16 storage / mixed
    seed: int = 0
    extra: dict = field(default_factory=dict)


def workload(name: str) -> Workload:
    """The workload recipes (sizes of the synthetic test problems)."""
    if name == "c1":   # plain method, FP64 20^3, R=3
        return Workload("c1", [20, 20, 20], [3, 3, 3], 50, "gaussian", 1 / math.sqrt(3),
                        noise_rel=1e-3, init=0.1, alpha=0.01, prec=0)
    if name == "c2":   # 100^4 FP32, R=10, ill-conditioned cores
        return Workload("c2", [100] * 4, [10] * 4, 1000, "illcond", smin=1e-3,
                        noise_rel=1e-4, alpha=5e6, prec=1)
    if name == "c3":   # 40^5 FP32, R=8, Gaussian cores N(0, 1/8)
        return Workload("c3", [40] * 5, [8] * 5, 2048, "gaussian", 1 / math.sqrt(8),
                        noise_rel=1e-3, alpha=2.5, prec=1)
    if name == "c5":   # 1000^3 BF16 storage, R=20, scaled variant with AdaGrad (whole-GPU path);
        # eta for the scaled direction from a sweep (0.003, 0.01 stall near RSE 0.78 in 2000
        # iterations; 0.03 reaches 2.3e-3 in 400), 0.01 for the plain direction
        return Workload("c5", [1000] * 3, [20] * 3, 4096, "illcond", smin=1e-2,
                        noise_rel=1e-3, variant=1, rule=1, eta=1e-2, prec=2, extra={"eta_scaled": 3e-2})
    if name in ("c5p", "c5ps"):  # profiling size of the large workload: its mode-1 contractions
        # (I_1 = 1000, R = 20, J = 4096) on a 1000 x 400 x 400 tensor that a full counter capture
        # can hold; c5p the plain direction, c5ps the scaled one
        return Workload(name, [1000, 400, 400], [20] * 3, 4096, "illcond", smin=1e-2,
                        noise_rel=1e-3, variant=1 if name == "c5ps" else 0, rule=1, eta=1e-2, prec=2,
                        extra={"eta_scaled": 3e-2})
    # Experiment I (Sec. 4): 300^3, Gaussian N(0, 1) cores 10 x 300 x 10, |F| = 200,
    # noiseless; the paper's step sizes (plain 6e-2; scaled 1e-1 with |H| = 200 or 400)
    if name == "e1":
        return Workload("e1", [300] * 3, [10] * 3, 200, "gaussian", 1.0, noise_rel=0.0, alpha=6e-2, prec=1)
    if name in ("e1s", "e1s4"):
        return Workload(name, [300] * 3, [10] * 3, 200, "gaussian", 1.0, noise_rel=0.0, alpha=1e-1, prec=1,
                        variant=1, JH=200 if name == "e1s" else 400)
    # Stand-ins shaped like the hyperspectral images of Sec. 4 (the images are not
    # available): planted ill-conditioned rank-R TR (singular values 1 .. 1e-2) plus
    # 5 % noise, |F| = 200; plain step 0.5 / lambda_max of the planted sampled-gradient
    # curvature (rounded), scaled variant with the paper's alpha and |H| = 1000
    hsi = {"hsi-salinas": ([83, 86, 224], 5, 8e3, 2e-2),
           "hsi-indian": ([145, 145, 220], 10, 3.5e4, 4e-3),
           "hsi-pavia": ([610, 340, 103], 10, 6e4, 4e-2)}
    base = name[:-2] if name.endswith("-s") else name
    if base in hsi:
        dims, R, a_plain, a_scaled = hsi[base]
        if name.endswith("-s"):
            return Workload(name, dims, [R] * 3, 200, "illcond", smin=1e-2, noise_rel=0.05, alpha=a_scaled,
                            prec=1, variant=1, JH=1000)
        return Workload(name, dims, [R] * 3, 200, "illcond", smin=1e-2, noise_rel=0.05, alpha=a_plain, prec=1)
    # Experiment II (Sec. 4): G_{n(2)} = U_n S V^T with condition number kappa in
    # {1e2, 1e4, 1e6}, R = 5, |F| = 200, noiseless; the dims are not stated (300^3
    # here); plain alpha 5e-4; scaled (-s) alpha 9e-2 with |H| = 1200
    kap = {"e2-k2": 1e2, "e2-k4": 1e4, "e2-k6": 1e6}
    if base in kap:
        if name.endswith("-s"):
            return Workload(name, [300] * 3, [5] * 3, 200, "illcond", smin=1.0 / kap[base], noise_rel=0.0,
                            alpha=9e-2, prec=1, variant=1, JH=1200)
        return Workload(name, [300] * 3, [5] * 3, 200, "illcond", smin=1.0 / kap[base], noise_rel=0.0,
                        alpha=5e-4, prec=1)
    raise KeyError(name)


EXP2_WORKLOADS = ["e2-k2", "e2-k4", "e2-k6"]

NEXT_WORKLOADS = ["e1", "e1s", "e1s4", "hsi-salinas", "hsi-salinas-s", "hsi-indian", "hsi-indian-s",
                  "hsi-pavia", "hsi-pavia-s"]


def batched_workloads(count: int = 64, seed: int = 0, J: int = 256):
    """Batched recipe: independent N=3 problems, each I_n ~ U{30..200} and
    each R_n ~ U{4..16} drawn independently (problem p uses seed + p)."""
    out = []
    for p in range(count):
        rng = _rng(seed + 1000 + p)
        dims = [int(v) for v in rng.integers(30, 201, size=3)]
        ranks = [int(v) for v in rng.integers(4, 17, size=3)]
        out.append(Workload(f"c4[{p}]", dims, ranks, J, "gaussian", 0.0,
                            noise_rel=1e-3, alpha=1.5, prec=1, seed=seed + p))
    return out


def planted_cores(w: Workload, dtype=np.float64):
    if w.planted == "illcond":
        return illcond_cores(w.dims, w.ranks[0], w.smin, w.seed, dtype)
    std = w.planted_std
    if std == 0.0:       # batched recipe: std_n^2 = 1 / sqrt(R_n R_{n+1})
        N = len(w.dims)
        std = [(w.ranks[n] * w.ranks[(n + 1) % N]) ** -0.25 for n in range(N)]
    return gaussian_cores(w.dims, w.ranks, std, w.seed, dtype)


def initial_cores(w: Workload, x_sq_norm: float, dtype=np.float64):
    std = init_std(w.dims, w.ranks, x_sq_norm) if w.init == "scaled" else float(w.init)
    return gaussian_cores(w.dims, w.ranks, std, w.seed + 2, dtype)
