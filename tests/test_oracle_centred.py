"""Pins of the oracle's centred Bloch coupling (no GPU).

The paper solves the Bloch variables in the middle of the Yee cell (Sec.
"Sample and numerical approach").  In the "centred" coupling the polarization
and the populations of cell (i, j, k) sit at its centre; the oscillator is
driven by the centre average A E of the four edges of each E component, and
the polarization current reaches each edge as A^T dP, the average over the
four cells sharing the edge.  Pinned by:

* linear fields: A reproduces a linear E field at the cell centres and A^T a
  linear cell field at the edges exactly (two-point averages along two axes
  are exact for linear functions);
* uniform fields: with a homogeneous gain medium in a periodic box and
  uniform fields the centred coupling equals the cell coupling bit for bit
  (the latter is pinned against an adaptive ODE solve of the zero-dimensional
  Maxwell-Bloch system);
* a field whose cell averages vanish (E_x alternating in sign along y) never
  drives the centred oscillators: the run equals the passive run bit for bit,
  while the cell coupling does couple;
* field-medium energy exchange: in a closed lossless box the field energy
  plus hbar omega_a N2 is conserved to rounding, which needs A^T to be the
  exact adjoint of A;
* the discrete Gauss law for eps E + A^T P and for H~ with random
  permittivity, gain cells, pump and noise.
"""
import math

import numpy as np
import pytest

import oracle.gain as G
from oracle import C0, EPS0, HBAR, Oracle
from paper_0802_3775_gb300 import inputs

# edge offsets of Ex, Ey, Ez in cells
NODE = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5)]
GAIN = dict(n_total=1e24, fa_hat=0.8, dw_rel=0.02, tau32=100e-15, tau21=1e-9, tau10=100e-15)


def _coords(shape, off):
    nx, ny, nz = shape
    return np.meshgrid(np.arange(nx) + off[0], np.arange(ny) + off[1], np.arange(nz) + off[2], indexing="ij")


def test_linear_fields_interpolate_exactly():
    shape = (7, 6, 8)
    o = Oracle(shape, 10)
    a = np.array([[0.3, -1.1, 2.0, 0.7], [1.5, 0.2, -0.4, 1.1], [-0.6, 0.9, 0.35, -2.0]])  # per component: c0 + g.r
    E = np.empty((3,) + shape)
    for c in range(3):
        X, Y, Z = _coords(shape, NODE[c])
        E[c] = a[c, 0] + a[c, 1] * X + a[c, 2] * Y + a[c, 3] * Z
    Ebar = o.to_cells(E)
    Xc, Yc, Zc = _coords(shape, (0.5, 0.5, 0.5))
    inner = (slice(0, -1), slice(0, -1), slice(0, -1))  # cells whose four edges are all on the grid
    for c in range(3):
        ref = a[c, 0] + a[c, 1] * Xc + a[c, 2] * Yc + a[c, 3] * Zc
        np.testing.assert_allclose(Ebar[c][inner], ref[inner], rtol=0, atol=1e-12)
    P = np.empty((3,) + shape)
    for c in range(3):
        P[c] = a[c, 0] + a[c, 1] * Xc + a[c, 2] * Yc + a[c, 3] * Zc
    Pe = o.to_edges(P)
    inner = (slice(1, None), slice(1, None), slice(1, None))  # edges whose four cells are all on the grid
    for c in range(3):
        X, Y, Z = _coords(shape, NODE[c])
        ref = a[c, 0] + a[c, 1] * X + a[c, 2] * Y + a[c, 3] * Z
        np.testing.assert_allclose(Pe[c][inner], ref[inner], rtol=0, atol=1e-12)


def _gain_box(shape, coupling, periodic=(True, True, True), **kw):
    o = Oracle(shape, 12, courant=0.5, periodic=periodic, eps=(2.25, 2.25, 2.25), seed=3)
    o.set_material(np.full(shape[::-1], 0b1010101, dtype=np.uint8))  # class 1 everywhere, all gain cells
    o.set_gain(**GAIN, pump=kw.get("pump", 1e12), noise_amp=0.0, coupling=coupling)
    return o


def test_uniform_fields_make_the_centred_coupling_equal_the_cell_coupling():
    shape = (5, 6, 4)
    runs = []
    for coupling in ("cell", "centred"):
        o = _gain_box(shape, coupling)
        E0 = np.array([3e5, -1e5, 2e5])
        o.E[:] = E0[:, None, None, None]
        o.P[:] = (0.1 * E0)[:, None, None, None]
        o.dN[1] += 1e21
        o.dN[2] -= 1e21
        o.step(400)
        runs.append((o.E.copy(), o.H.copy(), o.P.copy(), o.dN.copy()))
    for a, b in zip(*runs):
        assert np.array_equal(a, b)
    # the medium did act on the field
    assert np.max(np.abs(runs[0][2])) > 0.1 * 3e5 * 0.1


def test_a_field_with_vanishing_cell_averages_does_not_couple():
    shape = (4, 6, 5)
    Y = np.arange(shape[1])
    pattern = (-1.0) ** Y  # alternating along y (ny even: consistent across the periodic wrap)
    out = {}
    for coupling in ("cell", "centred", None):
        if coupling is None:
            o = Oracle(shape, 12, courant=0.5, periodic=(True, True, True), eps=(2.25, 2.25, 2.25))
            o.set_material(np.full(shape[::-1], 0b0010101, dtype=np.uint8))
        else:
            o = _gain_box(shape, coupling)
        o.E[0] = 1e6 * pattern[None, :, None]
        o.step(300)
        out[coupling] = o
    # the centred oscillators saw a zero drive: P stays zero and the run is the passive one
    assert np.array_equal(out["centred"].P, np.zeros_like(out["centred"].P))
    assert np.array_equal(out["centred"].E, out[None].E)
    assert np.array_equal(out["centred"].H, out[None].H)
    # the cell coupling is driven by the same field
    assert np.max(np.abs(out["cell"].P)) > 1e-4 * 1e6
    assert not np.array_equal(out["cell"].E, out[None].E)


def test_centred_energy_exchange_is_balanced():
    """Closed PEC box, every cell a gain cell, relaxation and pump off, an
    inverted start: field energy plus hbar w_a sum N2 is conserved to
    rounding, because sum_edges E_half . A^T dP = sum_cells (A E_half) . dP."""
    shape = (7, 8, 6)
    o = Oracle(shape, 12, courant=0.5, eps=(1.0, 2.5, 2.25))
    mat = inputs.random_material(shape, seed=21, classes=(1, 2)) | np.uint8(64)
    o.set_material(mat)
    n_total, fa = 1e24, 0.8
    omega_a = 2.0 * math.pi * fa * C0 / o.a
    o.set_gain(n_total=n_total, fa_hat=fa, dw_rel=0.02, tau32=1e6, tau21=1e6, tau10=1e6, pump=0.0,
               kappa=G.default_kappa(omega_a, 1e-9), noise_amp=0.0, init="ground", coupling="centred")
    o.dN[0] -= 0.4 * n_total
    o.dN[2] += 0.4 * n_total
    rng = np.random.Generator(np.random.PCG64(22))
    o.E[:] = 1e7 * rng.normal(size=o.E.shape)
    o._pec(o.E)
    dv = o.dx ** 3
    C, Wf = [], []
    for n in range(1500):
        E_n, H_before = o.E.copy(), o.H.copy()
        N2 = float(np.sum(o.populations()[2]))
        o.step(1)
        W = 0.5 * EPS0 * dv * (float(np.sum(o.eps_E * E_n * E_n)) + float(np.sum(o.H * H_before)))
        Wf.append(W)
        C.append(W + HBAR * o.gain["omega_a"] * dv * N2)
    C, Wf = np.asarray(C), np.asarray(Wf)
    moved = np.max(np.abs(Wf - Wf[0]))
    assert moved > 1e-5 * abs(C[0])
    assert np.max(np.abs(C - C[0])) <= 1e-14 * abs(C[0])
    assert np.max(np.abs(C - C[0])) <= 1e-9 * moved


def _div_nodes(F, periodic):
    out = np.zeros(F.shape[1:])
    for d in range(3):
        lo = np.roll(F[d], 1, axis=d)
        if not periodic[d]:
            idx = [slice(None)] * 3
            idx[d] = 0
            lo[tuple(idx)] = 0.0
        out += F[d] - lo
    return out


def _div_cells(F, periodic):
    out = np.zeros(F.shape[1:])
    for d in range(3):
        hi = np.roll(F[d], -1, axis=d)
        if not periodic[d]:
            idx = [slice(None)] * 3
            idx[d] = -1
            hi[tuple(idx)] = 0.0
        out += hi - F[d]
    return out


def test_centred_gauss_laws_with_gain_pump_and_noise():
    shape = (9, 8, 7)
    periodic = (False, True, False)
    o = Oracle(shape, 12, courant=0.5, periodic=periodic, eps=(1.0, 2.5, 11.9), seed=5)
    o.set_material(inputs.random_material(shape, seed=31, gain_fraction=0.5, classes=(0, 1, 2)))
    o.set_gain(**GAIN, pump=1e10, noise_amp=1e5, coupling="centred")
    o.set_fields_memory_order(inputs.random_fields(shape, seed=32, scale=1e7))
    o._pec(o.E)
    D0 = _div_nodes(o.eps_E * o.E + o.to_edges(o.P), periodic)
    B0 = _div_cells(o.H, periodic)
    o.step(200)
    assert np.max(np.abs(o.P)) > 0.1 * np.max(np.abs(o.E))
    inner = (slice(1, None), slice(None), slice(1, None))
    D1 = _div_nodes(o.eps_E * o.E + o.to_edges(o.P), periodic)
    assert np.max(np.abs(D1 - D0)[inner]) <= 1e-13 * np.max(np.abs(D0))
    assert np.max(np.abs(_div_cells(o.H, periodic) - B0)) <= 1e-13 * np.max(np.abs(B0))
    # the polarization counted on its own cells instead breaks the law
    assert np.max(np.abs(_div_nodes(o.eps_E * o.E + o.P, periodic) - D0)[inner]) > 1e-3 * np.max(np.abs(D0))
