"""Philox4x32-10 counter-based generator and Box-Muller normals (oracle side).

Test infrastructure only: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.

The spontaneous-emission noise of the gain model (Sec. "Sample and numerical
approach", where it enters the field evolution as a random term) needs one Gaussian
number per gain cell, per polarization component and per time step.  Those are
too many to pass in as inputs, so both sides implement the same published
generator: Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11), written here from its definition:

  round:  (hi0, lo0) = 0xD2511F53 * x0,  (hi1, lo1) = 0xCD9E8D57 * x2   (32x32 -> 64)
          x' = (hi1 ^ x1 ^ k0,  lo1,  hi0 ^ x3 ^ k1,  lo0)
  key schedule between rounds: k0 += 0x9E3779B9, k1 += 0xBB67AE85 (mod 2^32)

Counter / key layout used by the gain noise (shared reading of both sides):
  key = (seed & 0xffffffff, seed >> 32)
  ctr = (cell & 0xffffffff, cell >> 32, step & 0xffffffff, step >> 32)
with cell = (k*ny + j)*nx + i and `step` the index n of the update n -> n+1.
Uniforms: u = ((x >> 9) + 0.5) * 2^-23 in (0, 1): 24 significant bits, so the
value is exact in binary32 as well as in binary64.
Normals (Box-Muller): rho = sqrt(-2 ln u0); xi_x = rho cos(2 pi u1),
xi_y = rho sin(2 pi u1); xi_z = sqrt(-2 ln u2) cos(2 pi u3).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)
S32 = np.uint64(32)


def philox4x32_10(ctr, key):
    """ctr: 4 arrays (or ints) of uint32 values; key: 2 of them. Returns 4 uint64 arrays < 2^32."""
    x0, x1, x2, x3 = (np.asarray(c, dtype=np.uint64) & MASK for c in ctr)
    k0, k1 = (np.asarray(k, dtype=np.uint64) & MASK for k in key)
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * x0          # < 2^64: exact in uint64
        p1 = M1 * x2
        hi0, lo0 = p0 >> S32, p0 & MASK
        hi1, lo1 = p1 >> S32, p1 & MASK
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return x0, x1, x2, x3


def uniforms24(x):
    """((x >> 9) + 0.5) * 2^-23 in float64 (exact, and exact in binary32)."""
    return ((np.asarray(x, dtype=np.uint64) >> np.uint64(9)).astype(np.float64) + 0.5) * (2.0 ** -23)


def gain_noise(seed: int, step: int, cells):
    """Three N(0,1) deviates per cell index for update `step`: float64[3, len(cells)]."""
    cells = np.asarray(cells, dtype=np.uint64)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    step = int(step) & 0xFFFFFFFFFFFFFFFF
    key = (seed & 0xFFFFFFFF, seed >> 32)
    ctr = (cells & MASK, cells >> S32, np.full_like(cells, step & 0xFFFFFFFF), np.full_like(cells, step >> 32))
    x0, x1, x2, x3 = philox4x32_10(ctr, key)
    u0, u1, u2, u3 = (uniforms24(x) for x in (x0, x1, x2, x3))
    rho01 = np.sqrt(-2.0 * np.log(u0))
    rho23 = np.sqrt(-2.0 * np.log(u2))
    return np.stack([rho01 * np.cos(2.0 * np.pi * u1), rho01 * np.sin(2.0 * np.pi * u1),
                     rho23 * np.cos(2.0 * np.pi * u3)])
