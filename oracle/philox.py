"""Philox4x32-10 counter-based generator and the sampler's random numbers.

TEST INFRASTRUCTURE ONLY (see ``oracle/qmc_oracle.py``).

Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw, "Parallel
random numbers: as easy as 1, 2, 3" (SC'11): a 4 x 32-bit counter and a
2 x 32-bit key; each of the 10 rounds multiplies counter words 0 and 2 by
0xD2511F53 and 0xCD9E8D57 into 64-bit products and permutes/xors the halves
with the other words and the key; the key is advanced by the Weyl constants
0x9E3779B9 and 0xBB67AE85 between rounds.

Random-number layout used by the Metropolis step (both sides implement it):
key = (seed mod 2^32, seed div 2^32); counter = (block j, walker index,
step mod 2^32, step div 2^32).  Block j yields Gaussians 4j..4j+3 by
Box-Muller on the word pairs (x0, x1) and (x2, x3):
  u(x) = (x + 0.5) 2^-32,  rad = sqrt(-2 ln u(x0)),  th = 2 pi u(x1),
  z = (rad cos th, rad sin th, ...).
Block ceil(3N / 4) word x0 gives the acceptance uniform u(x0).
"""
from __future__ import annotations

import numpy as np

MASK = np.uint64(0xFFFFFFFF)
M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
TWO_PI = 6.283185307179586


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 on uint64 arrays holding 32-bit words."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & MASK
    k1 = np.asarray(k1, dtype=np.uint64) & MASK
    for rnd in range(10):
        if rnd:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        c0, c1, c2, c3 = ((p1 >> np.uint64(32)) ^ c1 ^ k0, p1 & MASK,
                          (p0 >> np.uint64(32)) ^ c3 ^ k1, p0 & MASK)
    return c0, c1, c2, c3


def u01(x):
    """32-bit word -> uniform in (0, 1): (x + 0.5) 2^-32 (exact in FP64)."""
    return (x.astype(np.float64) + 0.5) * 2.0 ** -32


def walker_normals_and_uniform(seed: int, walker_idx, step: int, n: int):
    """Gaussians [W, n] and the acceptance uniform [W] for one step."""
    walker_idx = np.asarray(walker_idx, dtype=np.uint64)
    W = walker_idx.shape[0]
    k0 = np.uint64(seed & 0xFFFFFFFF)
    k1 = np.uint64((seed >> 32) & 0xFFFFFFFF)
    s_lo = np.uint64(step & 0xFFFFFFFF)
    s_hi = np.uint64((step >> 32) & 0xFFFFFFFF)
    n_blk = (n + 3) // 4
    z = np.empty((W, 4 * n_blk), dtype=np.float64)
    for j in range(n_blk):
        x0, x1, x2, x3 = philox4x32_10(np.full(W, j, dtype=np.uint64), walker_idx, s_lo, s_hi, k0, k1)
        r1 = np.sqrt(-2.0 * np.log(u01(x0)))
        t1 = TWO_PI * u01(x1)
        r2 = np.sqrt(-2.0 * np.log(u01(x2)))
        t2 = TWO_PI * u01(x3)
        z[:, 4 * j + 0] = r1 * np.cos(t1)
        z[:, 4 * j + 1] = r1 * np.sin(t1)
        z[:, 4 * j + 2] = r2 * np.cos(t2)
        z[:, 4 * j + 3] = r2 * np.sin(t2)
    x0, _, _, _ = philox4x32_10(np.full(W, n_blk, dtype=np.uint64), walker_idx, s_lo, s_hi, k0, k1)
    return z[:, :n], u01(x0)
