"""Philox4x32-10 counter-based generator and Box-Muller normals (oracle side).

Test infrastructure only.  Written from the published definition: J. K.
Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random numbers: as
easy as 1, 2, 3", SC'11.  One round maps the counter (c0, c1, c2, c3) with key
(k0, k1) to (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
with the 32x32->64 products of multipliers M0 = 0xD2511F53, M1 = 0xCD9E8D57;
between rounds the key is bumped by the Weyl constants (0x9E3779B9,
0xBB67AE85).  Ten rounds.

Normal draws used by the CMA-ES sampler (the CUDA path implements the same
generator independently): element n of a generation's lam x d block of
standard normals comes from counter block b = n // 4,
counter = (b, generation, stream, 0), key = (seed mod 2^32, seed >> 32); the
four words r0..r3 give 24-bit uniforms u = ((r >> 8) + 0.5) / 2^24 and
Box-Muller pairs (evaluated here in FP64)
  z0 = sqrt(-2 ln u0) cos(2 pi u1), z1 = sqrt(-2 ln u0) sin(2 pi u1),
  z2 = sqrt(-2 ln u2) cos(2 pi u3), z3 = sqrt(-2 ln u2) sin(2 pi u3);
element n takes z_(n mod 4).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """ctr: uint array [..., 4]; key: uint array [..., 2].  Returns uint32 [..., 4]."""
    c = np.asarray(ctr, np.uint64) & MASK32
    k = np.asarray(key, np.uint64) & MASK32
    c0, c1, c2, c3 = (c[..., i].copy() for i in range(4))
    k0, k1 = k[..., 0].copy(), k[..., 1].copy()
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def normals(seed: int, stream: int, generation: int, count: int) -> np.ndarray:
    """The first `count` standard normals of (seed, stream, generation), FP64."""
    nb = (count + 3) // 4
    b = np.arange(nb, dtype=np.uint64)
    ctr = np.stack([b, np.full(nb, generation, np.uint64), np.full(nb, stream, np.uint64),
                    np.zeros(nb, np.uint64)], axis=-1)
    key = np.broadcast_to(np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], np.uint64), (nb, 2))
    r = philox4x32_10(ctr, key)
    u = ((r >> np.uint32(8)).astype(np.float64) + 0.5) / 16777216.0
    rad0 = np.sqrt(-2.0 * np.log(u[:, 0]))
    rad1 = np.sqrt(-2.0 * np.log(u[:, 2]))
    z = np.stack([rad0 * np.cos(2 * np.pi * u[:, 1]), rad0 * np.sin(2 * np.pi * u[:, 1]),
                  rad1 * np.cos(2 * np.pi * u[:, 3]), rad1 * np.sin(2 * np.pi * u[:, 3])], axis=-1)
    return z.reshape(-1)[:count]
