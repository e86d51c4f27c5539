"""Philox4x32-10 and the integer index draws of the sampler (oracle side).

Test infrastructure only (see ``oracle/__init__``).

Philox4x32-10 follows its published definition (J. K. Salmon, M. A. Moraes,
R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11):
a 4-word counter and a 2-word key, ten rounds; each round multiplies counter
words 0 and 2 by two fixed odd constants, splits the 64-bit products into
high/low halves and mixes them with words 1, 3 and the key; the key is bumped
by the two Weyl constants between rounds.

Counter layout used by the method (shared convention, implemented twice):

  word 0 = sample index j             (32 bits)
  word 1 = (stream << 24) | slot      (stream: 0 mode, 1 fibers F, 2 Hessian
                                       batch H, 3 optimal distribution;
                                       slot: core index k, 0 otherwise)
  word 2 = t mod 2^32                 (iteration)
  word 3 = t div 2^32
  key    = (seed mod 2^32, seed div 2^32)

One draw uses output words 0 and 1 as u = x1 * 2^32 + x0 (a uniform 64-bit
integer).  A uniform index in [0, m) is mulhi64(u, m) = floor(u * m / 2^64);
its bias is at most m / 2^64.  A draw from a probability vector p uses integer
weights w_i = round_half_even(p_i * 2^52) and their inclusive prefix sums C;
with W = C[-1], the index is the smallest i with mulhi64(u, W) < C[i].
"""
from __future__ import annotations

import numpy as np

MASK32 = 0xFFFFFFFF
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85

STREAM_MODE = 0
STREAM_F = 1
STREAM_H = 2
STREAM_OPT = 3

WEIGHT_SCALE_LOG2 = 52


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on (broadcastable) arrays of 32-bit words.

    Returns the four output words as uint64 arrays holding 32-bit values.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    k0 = np.asarray(k0, dtype=np.uint64) & MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & MASK32
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(PHILOX_W0)) & MASK32
            k1 = (k1 + np.uint64(PHILOX_W1)) & MASK32
        p0 = m0 * c0          # < 2^64: exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def draw_u64(seed: int, t: int, stream: int, slot, j):
    """Uniform 64-bit integers (as Python ints in an object array) for counters
    (j, stream/slot, t) under key ``seed``; ``slot`` and ``j`` broadcast."""
    slot = np.asarray(slot, dtype=np.uint64)
    j = np.asarray(j, dtype=np.uint64)
    w1 = (np.uint64(stream) << np.uint64(24)) | slot
    x0, x1, _, _ = philox4x32_10(j, w1, t & MASK32, (t >> 32) & MASK32,
                                 seed & MASK32, (seed >> 32) & MASK32)
    x0, x1 = np.broadcast_arrays(x0, x1)
    out = np.empty(x0.shape, dtype=object)
    for pos in np.ndindex(x0.shape):
        out[pos] = (int(x1[pos]) << 32) | int(x0[pos])
    return out


def mulhi64(u, m: int):
    """floor(u * m / 2^64) elementwise, in exact integer arithmetic."""
    u = np.asarray(u, dtype=object)
    out = np.empty(u.shape, dtype=np.int64)
    for pos in np.ndindex(u.shape):
        out[pos] = (int(u[pos]) * int(m)) >> 64
    return out


def integer_weights(p):
    """w_i = round_half_even(p_i * 2^52) as uint64 and their inclusive prefix
    sums (exact integer arithmetic)."""
    p = np.asarray(p, dtype=np.float64)
    if np.any(p < 0) or not np.all(np.isfinite(p)):
        raise ValueError("probabilities must be finite and nonnegative")
    w = np.rint(np.ldexp(p, WEIGHT_SCALE_LOG2)).astype(np.uint64)
    c = np.cumsum(w, dtype=np.uint64)
    return w, c


def cdf_index(u, cdf):
    """Smallest i with mulhi64(u, W) < cdf[i], W = cdf[-1]."""
    total = int(cdf[-1])
    if total == 0:
        raise ValueError("all weights are zero")
    target = np.asarray([(int(x) * total) >> 64 for x in np.ravel(u)], dtype=object)
    cdf_py = [int(c) for c in cdf]
    out = np.empty(target.shape, dtype=np.int64)
    for pos, tv in enumerate(target):
        lo, hi = 0, len(cdf_py) - 1          # first index with cdf > tv
        while lo < hi:
            mid = (lo + hi) // 2
            if cdf_py[mid] > tv:
                hi = mid
            else:
                lo = mid + 1
        out[pos] = lo
    return out.reshape(np.shape(u))


def cdf_margin(u, cdf):
    """Distance (integer units) from each draw's target to the nearest CDF
    boundary; used to judge draws whose index could flip under a change of
    the last bits of the weights."""
    total = int(cdf[-1])
    cdf_py = np.asarray([0] + [int(c) for c in cdf], dtype=object)
    out = []
    for x in np.ravel(u):
        tv = (int(x) * total) >> 64
        out.append(min(abs(int(b) - tv) for b in cdf_py))
    return np.asarray(out, dtype=object).reshape(np.shape(u))
