"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module draws the random numbers and builds the geometry inputs of a run;
it holds none of the stepping arithmetic.  Both the CUDA library and the CPU
oracle consume what it returns (a sphere list, probe cells, request streams),
so neither side depends on the other.

Geometry follows the paper's sample description (Sec. "Sample and numerical
approach"): an fcc inverted opal of air spheres of radius r0 = a/(2*sqrt(2))
(touching neighbours) in a high-index background, made disordered by random
radii.  Two disorder laws are offered:

* ``"paper"``    -- xi drawn uniformly from [-1/2, 1/2], r = r0 (1 + gamma xi),
                    radii only (the paper's law);
* ``"gaussian"`` -- independent Gaussian deviates delta ~ N(0, sigma) for the
                    radius and for each centre coordinate: r = r0 (1 + delta_r)
                    (clamped at 0), centre += a * delta_xyz.

Sphere lists are ``float64[n, 4]`` rows (cx, cy, cz, r) in grid units (one unit
= one cell edge), with the cell (i, j, k) occupying [i, i+1) x [j, j+1) x [k, k+1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# conventional-cube basis of the fcc lattice, in units of the lattice constant a
FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])

R0_OVER_A = 1.0 / (2.0 * math.sqrt(2.0))   # touching spheres (Sec. "Sample and numerical approach")


def rotation_111_to_z() -> np.ndarray:
    """Orthogonal matrix that maps the crystal [111] direction onto +z.

    Used for the plane wave launched along [111]: the grid stays axis-aligned and
    the lattice is rotated instead.
    """
    n = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
    z = np.array([0.0, 0.0, 1.0])
    v = np.cross(n, z)
    s = np.linalg.norm(v)
    c = float(n @ z)
    vx = np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])
    return np.eye(3) + vx + vx @ vx * ((1 - c) / (s * s))


def fcc_opal_spheres(box_lo, box_hi, res: float, *, rotation: str | np.ndarray = "identity",
                     disorder: str = "gaussian", sigma: float = 0.0, gamma: float = 0.0,
                     seed: int = 0) -> np.ndarray:
    """Sphere list of an fcc inverted opal filling the structure box.

    box_lo, box_hi : structure box corners in grid units (cells); the lattice
                     origin sits at box_lo (identity rotation) or the lattice is
                     rotated about the box centre.
    res            : cells per lattice constant a.
    Every lattice site whose (disordered) sphere intersects the box is kept;
    spheres are clipped by the box later, at rasterization.
    Draws use numpy's PCG64 generator seeded with ``seed``.
    """
    lo = np.asarray(box_lo, dtype=np.float64)
    hi = np.asarray(box_hi, dtype=np.float64)
    if isinstance(rotation, str):
        R = np.eye(3) if rotation == "identity" else rotation_111_to_z()
    else:
        R = np.asarray(rotation, dtype=np.float64)
    centre = 0.5 * (lo + hi)
    origin = lo if isinstance(rotation, str) and rotation == "identity" else centre
    # lattice-frame bounding region: inverse-rotate the box corners about `origin`
    corners = np.array([[x, y, z] for x in (lo[0], hi[0]) for y in (lo[1], hi[1]) for z in (lo[2], hi[2])])
    loc = (corners - origin) @ R  # row vectors: R^T applied
    rmax = R0_OVER_A * res * (1.0 + 6.0 * max(sigma, gamma))
    cmin = np.floor((loc.min(axis=0) - rmax) / res) - 1
    cmax = np.ceil((loc.max(axis=0) + rmax) / res) + 1
    ii = np.arange(int(cmin[0]), int(cmax[0]) + 1)
    jj = np.arange(int(cmin[1]), int(cmax[1]) + 1)
    kk = np.arange(int(cmin[2]), int(cmax[2]) + 1)
    cells = np.stack(np.meshgrid(ii, jj, kk, indexing="ij"), axis=-1).reshape(-1, 3).astype(np.float64)
    sites = (cells[:, None, :] + FCC_BASIS[None, :, :]).reshape(-1, 3) * res  # lattice frame, grid units
    sites = sites @ R.T + origin
    # deterministic site order (lexicographic in the rotated frame) before drawing
    order = np.lexsort((sites[:, 0], sites[:, 1], sites[:, 2]))
    sites = sites[order]
    n = sites.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    r0 = R0_OVER_A * res
    if disorder == "gaussian":
        d = rng.normal(0.0, 1.0, size=(n, 4)) * sigma
        radius = np.maximum(r0 * (1.0 + d[:, 0]), 0.0)
        sites = sites + res * d[:, 1:4]
    elif disorder == "paper":
        xi = rng.uniform(-0.5, 0.5, size=n)
        radius = np.maximum(r0 * (1.0 + gamma * xi), 0.0)
    else:
        raise ValueError(f"unknown disorder law {disorder!r}")
    # keep spheres whose ball meets the box (distance from centre to the box < r)
    q = np.clip(sites, lo, hi)
    dist2 = ((sites - q) ** 2).sum(axis=1)
    keep = (dist2 < radius * radius) & (radius > 0)
    out = np.concatenate([sites[keep], radius[keep, None]], axis=1)
    return np.ascontiguousarray(out, dtype=np.float64)


def probe_cells(shape, npml, count: int, seed: int) -> np.ndarray:
    """`count` probe cells drawn uniformly from the non-absorbing interior.

    shape = (nx, ny, nz); npml = (xlo, xhi, ylo, yhi, zlo, zhi).  Draws use
    PCG64(seed).  Returns int32[count, 3] rows (i, j, k).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    cols = []
    for d in range(3):
        lo_d = npml[2 * d]
        hi_d = shape[d] - npml[2 * d + 1]
        cols.append(rng.integers(lo_d, hi_d, size=count))
    return np.stack(cols, axis=1).astype(np.int32)


def random_fields(shape, seed: int, scale: float = 1.0, dtype=np.float64) -> np.ndarray:
    """Seeded N(0, scale^2) values for the six Yee arrays, float[6, nz, ny, nx]."""
    nx, ny, nz = shape
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.normal(0.0, scale, size=(6, nz, ny, nx))).astype(dtype)


def random_material(shape, seed: int, gain_fraction: float = 0.0, classes=(1, 2)) -> np.ndarray:
    """Seeded material bytes, uint8[nz, ny, nx]: random class per E component
    (bits 0-1 Ex, 2-3 Ey, 4-5 Ez) drawn from `classes`, gain bit 6 set with
    probability `gain_fraction`."""
    nx, ny, nz = shape
    rng = np.random.Generator(np.random.PCG64(seed))
    cl = np.asarray(classes, dtype=np.uint8)
    m = np.zeros((nz, ny, nx), dtype=np.uint8)
    for c in range(3):
        m |= (cl[rng.integers(0, len(cl), size=(nz, ny, nx))] << (2 * c)).astype(np.uint8)
    if gain_fraction > 0:
        m |= ((rng.random((nz, ny, nx)) < gain_fraction).astype(np.uint8) << 6)
    return m


# ----------------------------------------------------------------------------
# Workload descriptions (plain parameter records; no derived coefficients)
# ----------------------------------------------------------------------------

@dataclass
class SourceSpec:
    kind: str = "point"          # "point" or "sheet"
    comp: int = 2                # E component driven: 0=x, 1=y, 2=z
    pos: tuple = (0, 0, 0)       # point source cell (i, j, k)
    axis: int = 2                # sheet normal axis
    index: int = 0               # sheet plane index along `axis`
    waist: float = 0.0           # Gaussian transverse waist in cells (0 = uniform)
    f0_hat: float = 0.80         # centre frequency, normalized a/lambda
    rel_bw: float = 0.10         # FWHM of the power spectrum / f0
    t0_steps: float = 0.0        # pulse centre in time steps (0 = 5 tau)
    amplitude: float = 1.0       # V/m per step (see the source term of the E update)


@dataclass
class GainSpec:
    n_total: float = 1e24        # m^-3
    fa_hat: float = 0.80         # transition frequency, normalized a/lambda
    dw_rel: float = 0.02         # linewidth Delta omega / omega_a
    tau32: float = 100e-15
    tau21: float = 1e-9
    tau10: float = 100e-15
    pump: float = 1e9            # s^-1, rate 0 -> 3
    kappa: float = 0.0           # coupling; 0 = 6 pi eps0 c^3 / (omega_a^2 tau21)
    noise_amp: float = 0.0       # V/m (std of the normalized polarization kick per step)
    init: str = "steady"         # "steady" (N = N_eq) or "ground" (all in level 0)
    coupling: str = "cell"       # "cell": P on the cell's own E nodes; "centred": P at the cell centre


@dataclass
class FluxSpec:
    axis: int = 2
    index: int = 0
    sign: float = 1.0
    u: tuple = (0, 0)            # face range along the first transverse axis (cyclic order)
    v: tuple = (0, 0)            # face range along the second transverse axis


@dataclass
class RunSpec:
    """One realization: grid, geometry, sources, observers, gain."""
    shape: tuple
    res: float
    a: float = 480e-9
    courant: float = 0.5
    npml: tuple = (0, 0, 0, 0, 0, 0)
    periodic: tuple = (False, False, False)
    eps: tuple = (11.9, 11.9, 1.0)          # (outside, background, sphere)
    cpml_m: float = 3.0
    cpml_sigma_factor: float = 0.8
    cpml_kappa_max: float = 1.0
    cpml_alpha_max: float = 0.05
    cpml_f_hat: float = 0.80
    absorber: str = "cpml"                  # "cpml" or "upml" (same grading, no alpha)
    precision: str = "f32"
    spheres: np.ndarray | None = None
    box_lo: tuple = (0, 0, 0)
    box_hi: tuple = (0, 0, 0)
    sources: list = field(default_factory=list)
    probes: np.ndarray | None = None
    fluxes: list = field(default_factory=list)
    gain: GainSpec | None = None
    seed: int = 0
    steps: int = 0

    @property
    def cells(self) -> int:
        return int(self.shape[0]) * int(self.shape[1]) * int(self.shape[2])


def interior(spec: RunSpec):
    """Non-absorbing interior [lo, hi) per axis."""
    lo = tuple(spec.npml[2 * d] for d in range(3))
    hi = tuple(spec.shape[d] - spec.npml[2 * d + 1] for d in range(3))
    return lo, hi


def transverse_axes(axis: int):
    """Cyclic transverse axes (d1, d2) of a plane normal to `axis`."""
    return (axis + 1) % 3, (axis + 2) % 3


def flux_box(spec: RunSpec, inset: int = 2):
    """Six outward flux planes enclosing the interior, `inset` cells inside the CPML."""
    lo, hi = interior(spec)
    b0 = [lo[d] + inset for d in range(3)]
    b1 = [hi[d] - inset for d in range(3)]
    out = []
    for d in range(3):
        d1, d2 = transverse_axes(d)
        for idx, sg in ((b0[d], -1.0), (b1[d], 1.0)):
            out.append(FluxSpec(axis=d, index=idx, sign=sg, u=(b0[d1], b1[d1]), v=(b0[d2], b1[d2])))
    return out


def plane_flux(spec: RunSpec, axis: int, index: int, sign: float = 1.0) -> FluxSpec:
    """Flux plane normal to `axis` covering the interior faces."""
    lo, hi = interior(spec)
    d1, d2 = transverse_axes(axis)
    return FluxSpec(axis=axis, index=index, sign=sign, u=(lo[d1], hi[d1] - 1), v=(lo[d2], hi[d2] - 1))


# ----------------------------------------------------------------------------
# The workloads (parameter records only)
# ----------------------------------------------------------------------------

def opal_dipole_f64(steps: int = 2000) -> RunSpec:
    """40^3 FP64 dipole run: 2x2x2 unit cells at 12 cells/a + 8-cell CPML,
    air spheres in eps 11.9, Ez Gaussian pulse at the centre, 8 seeded probes."""
    res, ncell, npml = 12, 2, 8
    n = ncell * res + 2 * npml
    spec = RunSpec(shape=(n, n, n), res=res, npml=(npml,) * 6, eps=(11.9, 11.9, 1.0),
                   precision="f64", box_lo=(npml,) * 3, box_hi=(n - npml,) * 3, steps=steps)
    spec.spheres = fcc_opal_spheres(spec.box_lo, spec.box_hi, res, sigma=0.0, seed=0)
    c = n // 2
    spec.sources = [SourceSpec(kind="point", comp=2, pos=(c, c, c), f0_hat=0.80, rel_bw=0.10)]
    spec.probes = probe_cells(spec.shape, spec.npml, 8, seed=1)
    return spec


def opal_planewave_f32(ncell: int = 8, res: int = 20, npml: int = 12, sigma: float = 0.0,
                       realization: int = 0, steps: int = 20000, precision: str = "f32") -> RunSpec:
    """Passive disordered opal: ncell^3 unit cells at `res` cells/a + CPML, lattice
    rotated so [111] is along z, x-polarized plane-wave sheet at z = npml+2,
    transmitted-flux plane at z = nz-npml-3."""
    n = ncell * res + 2 * npml
    spec = RunSpec(shape=(n, n, n), res=res, npml=(npml,) * 6, eps=(11.9, 11.9, 1.0),
                   precision=precision, box_lo=(npml,) * 3, box_hi=(n - npml,) * 3, steps=steps,
                   seed=1000 + realization)
    spec.spheres = fcc_opal_spheres(spec.box_lo, spec.box_hi, res, rotation="111", sigma=sigma,
                                    seed=1000 + realization)
    spec.sources = [SourceSpec(kind="sheet", comp=0, axis=2, index=npml + 2, f0_hat=0.80, rel_bw=0.10)]
    spec.fluxes = [plane_flux(spec, 2, n - npml - 3)]
    spec.probes = probe_cells(spec.shape, spec.npml, 8, seed=1000 + realization + 1)
    return spec


def opal_lasing_f32(ncell: int = 6, res: int = 20, npml: int = 10, sigma: float = 0.0,
                    pump: float = 1e10, realization: int = 0, steps: int = 100000,
                    precision: str = "f32") -> RunSpec:
    """Maxwell-Bloch lasing: spheres filled with a four-level gain medium
    (eps_host 2.25, 1e24 m^-3, f_a = 0.80 a/lambda, linewidth 0.02 omega_a,
    tau32 = tau10 = 100 fs, tau21 = 1 ns), Gaussian polarization noise 1e-6."""
    n = ncell * res + 2 * npml
    spec = RunSpec(shape=(n, n, n), res=res, npml=(npml,) * 6, eps=(11.9, 11.9, 2.25),
                   precision=precision, box_lo=(npml,) * 3, box_hi=(n - npml,) * 3, steps=steps,
                   seed=2000 + realization)
    spec.spheres = fcc_opal_spheres(spec.box_lo, spec.box_hi, res, rotation="identity", sigma=sigma,
                                    seed=2000 + realization)
    spec.gain = GainSpec(n_total=1e24, fa_hat=0.80, dw_rel=0.02, tau32=100e-15, tau21=1e-9,
                         tau10=100e-15, pump=pump, noise_amp=1e-6, init="steady")
    spec.fluxes = flux_box(spec)
    spec.probes = probe_cells(spec.shape, spec.npml, 8, seed=2000 + realization + 1)
    return spec


def mixed_batch(count: int = 64, seed: int = 4000, steps: int = 20000, npml: int = 12,
                precision: str = "f32", ncell: int | None = None):
    """Mixed-size batch: n in 4..8 unit cells, 16..20 cells/a, sigma ~ U(0, 10%);
    even members passive plane-wave runs, odd members lasing runs.  `ncell`
    given: every member keeps its draws (resolution, sigma, seeds) but spans
    `ncell`^3 unit cells (the reduced members of the error checks)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    fixed = ncell
    for r in range(count):
        ncell = int(rng.integers(4, 9))
        res = int(rng.integers(16, 21))
        sigma = float(rng.uniform(0.0, 0.10))
        if fixed is not None:
            ncell = int(fixed)
        if r % 2 == 0:
            s = opal_planewave_f32(ncell=ncell, res=res, npml=npml, sigma=sigma, realization=r,
                                   steps=steps, precision=precision)
        else:
            s = opal_lasing_f32(ncell=ncell, res=res, npml=npml, sigma=sigma, realization=r,
                                steps=steps, precision=precision)
        s.seed = seed + r
        out.append(s)
    return out


def request_stream(count: int, rate_hz: float = 4.0, seed: int = 5000, n_range=(64, 200),
                   steps_range=(5000, 50000), npml: int = 12):
    """Poisson arrival stream of passive and lasing runs with grid edge in
    `n_range` (including CPML) and step counts in `steps_range`.
    Returns a list of (arrival_time_s, RunSpec)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for r in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        n_target = int(rng.integers(n_range[0], n_range[1] + 1))
        res = int(rng.integers(16, 21))
        ncell = max(2, int(round((n_target - 2 * npml) / res)))
        sigma = float(rng.uniform(0.0, 0.10))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        if rng.random() < 0.5:
            s = opal_planewave_f32(ncell=ncell, res=res, npml=npml, sigma=sigma, realization=r, steps=steps)
        else:
            s = opal_lasing_f32(ncell=ncell, res=res, npml=npml, sigma=sigma, realization=r, steps=steps)
        s.seed = seed + r
        out.append((t, s))
    return out
