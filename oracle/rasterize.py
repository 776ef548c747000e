"""Rasterization of the sphere list into per-cell material bytes (oracle side).

Test infrastructure only: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.

The inverted opal (Sec. "Sample and numerical approach") is a set of spheres
with permittivity eps_sphere in a background eps_bg, inside a finite structure
box; outside the box the medium is eps_outside.  Each Yee E component samples
the permittivity at its own node:

  Ex at (i+1/2, j, k),  Ey at (i, j+1/2, k),  Ez at (i, j, k+1/2)   (grid units)

and the gain medium (when enabled) occupies the cells whose centre
(i+1/2, j+1/2, k+1/2) lies in a sphere.

Byte layout per cell: bits 2c..2c+1 = class of E_c (0 outside the box,
1 background, 2 sphere), bit 6 = cell centre inside a sphere and the box.

Inside test: strict  (dx*dx + dy*dy) + dz*dz < r*r  in FP64, each operation
rounded on its own, in exactly that order (a tie on the surface has measure
zero; the order makes the result reproducible bit for bit).
Box test: box_lo[d] <= p[d] < box_hi[d] for each axis.
"""
from __future__ import annotations

import math

import numpy as np

OFFSETS = ((0.5, 0.0, 0.0), (0.0, 0.5, 0.0), (0.0, 0.0, 0.5), (0.5, 0.5, 0.5))


def inside_masks(shape, spheres):
    """bool[4, nx, ny, nz]: sample point s (Ex, Ey, Ez, centre) inside any sphere."""
    nx, ny, nz = shape
    inside = np.zeros((4, nx, ny, nz), dtype=bool)
    for cx, cy, cz, r in np.asarray(spheres, dtype=np.float64).reshape(-1, 4):
        rr = r * r
        for s, (ox, oy, oz) in enumerate(OFFSETS):
            i0 = max(0, math.floor(cx - r - ox)); i1 = min(nx, math.ceil(cx + r - ox) + 1)
            j0 = max(0, math.floor(cy - r - oy)); j1 = min(ny, math.ceil(cy + r - oy) + 1)
            k0 = max(0, math.floor(cz - r - oz)); k1 = min(nz, math.ceil(cz + r - oz) + 1)
            if i0 >= i1 or j0 >= j1 or k0 >= k1:
                continue
            dx = (np.arange(i0, i1, dtype=np.float64) + ox) - cx
            dy = (np.arange(j0, j1, dtype=np.float64) + oy) - cy
            dz = (np.arange(k0, k1, dtype=np.float64) + oz) - cz
            d2 = ((dx * dx)[:, None, None] + (dy * dy)[None, :, None]) + (dz * dz)[None, None, :]
            inside[s, i0:i1, j0:j1, k0:k1] |= d2 < rr
    return inside


def in_box_masks(shape, box_lo, box_hi):
    nx, ny, nz = shape
    out = np.zeros((4, nx, ny, nz), dtype=bool)
    for s, off in enumerate(OFFSETS):
        ok = []
        for d, n in enumerate((nx, ny, nz)):
            p = np.arange(n, dtype=np.float64) + off[d]
            ok.append((p >= box_lo[d]) & (p < box_hi[d]))
        out[s] = ok[0][:, None, None] & ok[1][None, :, None] & ok[2][None, None, :]
    return out


def rasterize(shape, spheres, box_lo, box_hi) -> np.ndarray:
    """Material bytes in memory order uint8[nz, ny, nx] (x fastest)."""
    inside = inside_masks(shape, spheres)
    box = in_box_masks(shape, box_lo, box_hi)
    mat = np.zeros(tuple(shape), dtype=np.uint8)
    for c in range(3):
        cls = np.where(box[c], np.where(inside[c], 2, 1), 0).astype(np.uint8)
        mat |= (cls << (2 * c)).astype(np.uint8)
    mat |= ((inside[3] & box[3]).astype(np.uint8) << 6)
    return np.ascontiguousarray(mat.transpose(2, 1, 0))
