"""Pins of the oracle's Yee update against closed forms (no GPU).

* periodic box: a discrete plane-wave eigenmode keeps the form
  cos(k.r - omega n dt) with sin^2(omega dt / 2) = (S^2/eps_r) sum_d sin^2(k_d/2)
  (Yee numerical dispersion; the Yee scheme is the paper's FDTD method,
  Sec. "Sample and numerical approach");
* PEC box: a discrete cavity eigenmode oscillates as cos(omega n dt) with the
  same dispersion and k_d = pi m_d / n_d;
* lossless closed box with random inhomogeneous eps: the discrete energy
  1/2 sum H~^{n+1/2}.H~^{n+1/2} + 1/2 sum eps E^{n+1}.E^n is invariant;
* a randomly excited PEC cavity rings at the discrete resonances, which
  approach the continuum ones c pi sqrt(sum (m_d/L_d)^2) as O(dx^2);
* discrete Gauss laws: with random eps, gain cells, pump and noise kicks, the
  node divergence of D~ = eps E + P~ and the cell divergence of H~ stay at
  their initial values (the divergence of a Yee curl vanishes identically),
  so a wrong index, sign or coefficient in a curl or in the polarization
  coupling breaks them.
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_0802_3775_gb300 import inputs

# node offsets of Ex, Ey, Ez, Hx, Hy, Hz in cells
NODE = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5), (0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]


def _coords(shape, off):
    nx, ny, nz = shape
    return np.meshgrid(np.arange(nx) + off[0], np.arange(ny) + off[1], np.arange(nz) + off[2], indexing="ij")


@pytest.mark.parametrize("eps_r,m,courant", [(1.0, (1, 2, -1), 0.5), (2.5, (2, -1, 3), 0.9), (11.9, (0, 1, 2), 0.3)])
def test_periodic_plane_wave_dispersion(eps_r, m, courant):
    shape = (12, 10, 14)
    o = Oracle(shape, 12, courant=courant, periodic=(True, True, True), eps=(eps_r, eps_r, eps_r))
    S = o.S
    k = np.array([2 * math.pi * m[d] / shape[d] for d in range(3)])
    K = 2.0 * np.sin(k / 2.0)
    E_hat = np.cross(K, [0.3, -0.7, 1.1])
    E_hat /= np.linalg.norm(E_hat)
    Om = S * np.linalg.norm(K) / math.sqrt(eps_r)
    w = 2.0 * math.asin(Om / 2.0)
    H_hat = (S / Om) * np.cross(K, E_hat)

    def field(c, n_time):
        X, Y, Z = _coords(shape, NODE[c])
        amp = E_hat[c] if c < 3 else H_hat[c - 3]
        return amp * np.cos(k[0] * X + k[1] * Y + k[2] * Z - w * n_time)

    for c in range(3):
        o.E[c] = field(c, 0.0)
        o.H[c] = field(c + 3, -0.5)
    o.add_probe(3, 4, 5)
    N = 300
    o.step(N)
    for c in range(3):
        np.testing.assert_allclose(o.E[c], field(c, N), rtol=0, atol=1e-11)
        np.testing.assert_allclose(o.H[c], field(c + 3, N - 0.5), rtol=0, atol=1e-11)
    # probes hold E^{n+1} after update n
    pr = o.probe_series()
    for n in (0, 17, N - 1):
        for c in range(3):
            X = 3 + NODE[c][0]; Y = 4 + NODE[c][1]; Z = 5 + NODE[c][2]
            ref = E_hat[c] * math.cos(k[0] * X + k[1] * Y + k[2] * Z - w * (n + 1))
            assert abs(pr[n, 0, c] - ref) < 1e-12


@pytest.mark.parametrize("m,eps_r", [((1, 2, 1), 1.0), ((2, 1, 3), 4.0)])
def test_pec_cavity_eigenmode(m, eps_r):
    shape = (10, 12, 9)
    o = Oracle(shape, 10, courant=0.5, eps=(eps_r, eps_r, eps_r))
    S = o.S
    k = np.array([math.pi * m[d] / shape[d] for d in range(3)])
    K = 2.0 * np.sin(k / 2.0)
    A = np.cross(K, [1.0, 0.4, -0.3])
    Om = S * np.linalg.norm(K) / math.sqrt(eps_r)
    w = 2.0 * math.asin(Om / 2.0)
    X, Y, Z = {}, {}, {}
    for c in range(6):
        X[c], Y[c], Z[c] = _coords(shape, NODE[c])
    sx, sy, sz = np.sin, np.sin, np.sin
    cx, cy, cz = np.cos, np.cos, np.cos
    E0 = [A[0] * cx(k[0] * X[0]) * sy(k[1] * Y[0]) * sz(k[2] * Z[0]),
          A[1] * sx(k[0] * X[1]) * cy(k[1] * Y[1]) * sz(k[2] * Z[1]),
          A[2] * sx(k[0] * X[2]) * sy(k[1] * Y[2]) * cz(k[2] * Z[2])]
    KA = np.cross(K, A)
    C = [KA[0] * sx(k[0] * X[3]) * cy(k[1] * Y[3]) * cz(k[2] * Z[3]),
         KA[1] * cx(k[0] * X[4]) * sy(k[1] * Y[4]) * cz(k[2] * Z[4]),
         KA[2] * cx(k[0] * X[5]) * cy(k[1] * Y[5]) * sz(k[2] * Z[5])]
    for c in range(3):
        o.E[c] = E0[c]
        o.H[c] = 0.5 * S * C[c]
    N = 400
    o.step(N)
    for c in range(3):
        np.testing.assert_allclose(o.E[c], E0[c] * math.cos(w * N), rtol=0, atol=1e-11)
        np.testing.assert_allclose(o.H[c], -(S / Om) * C[c] * math.sin(w * (N - 0.5)), rtol=0, atol=1e-11)


def test_discrete_energy_invariant_inhomogeneous():
    shape = (9, 10, 11)
    o = Oracle(shape, 10, courant=0.5, eps=(1.0, 2.5, 11.9))
    o.set_material(inputs.random_material(shape, seed=7, classes=(0, 1, 2)))
    F = inputs.random_fields(shape, seed=8)
    o.set_fields_memory_order(F)
    # tangential E on the index-0 planes is held at zero
    o.E[1][0] = o.E[2][0] = 0.0
    o.E[0][:, 0] = o.E[2][:, 0] = 0.0
    o.E[0][:, :, 0] = o.E[1][:, :, 0] = 0.0
    W = []
    for n in range(3000):
        Eprev = o.E.copy()
        o.step(1)
        W.append(0.5 * np.sum(o.H * o.H) + 0.5 * np.sum(o.eps_E * o.E * Eprev))
    W = np.asarray(W)
    assert np.max(np.abs(W - W[0])) / abs(W[0]) < 1e-12
    # a wrong eps weighting breaks the invariant
    Wbad = 0.5 * np.sum(o.H * o.H) + 0.5 * np.sum(o.E * Eprev)
    assert abs(Wbad - W[-1]) / abs(W[0]) > 1e-3


def test_pec_cavity_resonances_from_ringing():
    shape = (8, 7, 6)
    res = 10
    o = Oracle(shape, res, courant=0.5)
    rng = np.random.Generator(np.random.PCG64(3))
    o.E[:] = rng.normal(size=o.E.shape)
    o.E[1][0] = o.E[2][0] = 0.0
    o.E[0][:, 0] = o.E[2][:, 0] = 0.0
    o.E[0][:, :, 0] = o.E[1][:, :, 0] = 0.0
    o.add_probe(3, 2, 2)
    N = 8192
    o.step(N)
    sig = o.probe_series()[:, 0, :].sum(axis=1)
    spec = np.abs(np.fft.rfft(sig * np.hanning(N)))
    freqs = np.fft.rfftfreq(N)  # cycles per step
    # discrete resonances: sin^2(w/2) = S^2 sum sin^2(pi m_d / (2 n_d))
    res_f = []
    for mx in range(shape[0] + 1):
        for my in range(shape[1] + 1):
            for mz in range(shape[2] + 1):
                if (mx > 0) + (my > 0) + (mz > 0) < 2:
                    continue
                s2 = sum(math.sin(math.pi * mm / (2 * nn)) ** 2 for mm, nn in zip((mx, my, mz), shape))
                res_f.append(2 * math.asin(o.S * math.sqrt(s2)) / (2 * math.pi))
    res_f = np.array(res_f)
    peaks = [i for i in range(2, len(spec) - 1) if spec[i] > spec[i - 1] and spec[i] > spec[i + 1]]
    top = sorted(peaks, key=lambda i: -spec[i])[:8]
    bin_w = 1.0 / N
    for i in top:
        # parabolic peak interpolation
        a, b, c = np.log(spec[i - 1]), np.log(spec[i]), np.log(spec[i + 1])
        f = (i + 0.5 * (a - c) / (a - 2 * b + c)) * bin_w
        assert np.min(np.abs(res_f - f)) < 1.5 * bin_w
    # continuum limit of the (1,1,0) mode: omega = c pi sqrt(sum (m/L)^2), O(dx^2) away
    f_disc = 2 * math.asin(o.S * math.sqrt(math.sin(math.pi / 16) ** 2 + math.sin(math.pi / 14) ** 2)) / (2 * math.pi)
    f_cont = o.S * 0.5 * math.sqrt((1 / 8) ** 2 + (1 / 7) ** 2)
    assert abs(f_disc - f_cont) / f_cont < 0.01


def _div_nodes(F, periodic):
    """Backward-difference divergence of an E-staggered field at the nodes."""
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
    """Forward-difference divergence of an H-staggered field at the cell centres."""
    out = np.zeros(F.shape[1:])
    for d in range(3):
        hi = np.roll(F[d], -1, axis=d)
        if not periodic[d]:
            idx = [slice(None)] * 3
            idx[d] = -1
            hi[tuple(idx)] = 0.0
        out += hi - F[d]
    return out


def test_discrete_gauss_laws_with_gain_and_noise():
    shape = (9, 8, 7)
    periodic = (False, True, False)
    o = Oracle(shape, 12, courant=0.5, periodic=periodic, eps=(1.0, 2.5, 11.9), seed=5)
    o.set_material(inputs.random_material(shape, seed=31, gain_fraction=0.5, classes=(0, 1, 2)))
    o.set_gain(n_total=1e24, fa_hat=0.8, dw_rel=0.02, tau32=100e-15, tau21=1e-9, tau10=100e-15,
               pump=1e10, noise_amp=1e5)
    o.set_fields_memory_order(inputs.random_fields(shape, seed=32, scale=1e7))
    o._pec(o.E)
    D0 = _div_nodes(o.eps_E * o.E + o.P, periodic)
    B0 = _div_cells(o.H, periodic)
    o.step(200)
    # the polarization took part: it is of the field's size
    assert np.max(np.abs(o.P)) > 0.1 * np.max(np.abs(o.E))
    # nodes off the closed index-0 planes (tangential E held at zero there)
    inner = (slice(1, None), slice(None), slice(1, None))
    D1 = _div_nodes(o.eps_E * o.E + o.P, periodic)
    assert np.max(np.abs(D1 - D0)[inner]) <= 1e-13 * np.max(np.abs(D0))
    assert np.max(np.abs(_div_cells(o.H, periodic) - B0)) <= 1e-13 * np.max(np.abs(B0))
    # leaving out the polarization, or the permittivity, breaks the law
    assert np.max(np.abs(_div_nodes(o.eps_E * o.E, periodic) - D0)[inner]) > 1e-3 * np.max(np.abs(D0))
    assert np.max(np.abs(_div_nodes(o.E + o.P, periodic) - D0)[inner]) > 1e-3 * np.max(np.abs(D0))


# SI constants for the energy pins (CODATA 2018 mu0, exact c), written here so
# that the expected energies do not reuse the oracle's normalization
_MU0 = 1.25663706212e-6
_C = 299792458.0
_EPS0 = 1.0 / (_MU0 * _C * _C)


@pytest.mark.parametrize("eps_r,m,res", [(1.0, (1, 2, -1), 12), (11.9, (2, 0, 3), 20), (2.25, (0, -1, 1), 16)])
def test_energy_of_a_travelling_plane_wave(eps_r, m, res):
    """Oracle.energy() of a discrete travelling plane wave in a periodic box
    equals the continuum energy of a plane wave, (1/2) eps0 eps_r E0^2 V,
    at every step: its electric and magnetic parts are each half of it (the
    discrete H~ amplitude is sqrt(eps_r) E0 by the dispersion relation), and
    cos^2 summed over whole periods of the box is half the node count.  A
    dx^2 in place of dx^3, eps_r left out of the electric part or a missing
    1/2 each fail by a factor."""
    shape = (12, 10, 14)
    a = 480e-9
    o = Oracle(shape, res, a=a, courant=0.5, periodic=(True, True, True), eps=(eps_r, eps_r, eps_r))
    S = o.S
    k = np.array([2 * math.pi * m[d] / shape[d] for d in range(3)])
    K = 2.0 * np.sin(k / 2.0)
    E_hat = np.cross(K, [0.3, -0.7, 1.1])
    E0 = 37.0  # V/m
    E_hat *= E0 / np.linalg.norm(E_hat)
    Om = S * np.linalg.norm(K) / math.sqrt(eps_r)
    w = 2.0 * math.asin(Om / 2.0)
    H_hat = (S / Om) * np.cross(K, E_hat)
    for c in range(3):
        X, Y, Z = _coords(shape, NODE[c])
        o.E[c] = E_hat[c] * np.cos(k[0] * X + k[1] * Y + k[2] * Z)
        X, Y, Z = _coords(shape, NODE[c + 3])
        o.H[c] = H_hat[c] * np.cos(k[0] * X + k[1] * Y + k[2] * Z + 0.5 * w)
    dx = a / res
    V = shape[0] * shape[1] * shape[2] * dx ** 3
    U = 0.5 * _EPS0 * eps_r * E0 ** 2 * V
    assert abs(o.energy() / U - 1.0) < 1e-12
    for _ in range(3):
        o.step(37)
        assert abs(o.energy() / U - 1.0) < 1e-12


def test_energy_of_uniform_static_fields_in_a_layered_box():
    """A uniform E0 and H0 in a periodic box are static (every Yee difference
    of a uniform field is zero), so Oracle.energy() must equal the field energy
    of electrostatics and magnetostatics: (1/2) eps0 E0^2 (eps_1 V_1 + eps_2 V_2)
    + (1/2) mu0 H0^2 V for two layers of permittivity eps_1, eps_2 filling
    half the box each, with H0 = H~0 / eta0 the SI magnetic field."""
    shape = (6, 8, 10)
    res, a = 16, 480e-9
    eps1, eps2 = 1.0, 11.9
    o = Oracle(shape, res, a=a, periodic=(True, True, True), eps=(eps1, eps2, eps2))
    mat = np.zeros(shape[::-1], dtype=np.uint8)  # class 0 (eps1) for z < nz/2
    mat[shape[2] // 2:] = 0b010101                # class 1 (eps2) above
    o.set_material(mat)
    E0 = np.array([3.0, -4.0, 12.0])      # V/m
    Ht0 = np.array([-2.0, 5.0, 1.5])      # H~ = eta0 H, V/m
    for c in range(3):
        o.E[c] = E0[c]
        o.H[c] = Ht0[c]
    dx = a / res
    V = shape[0] * shape[1] * shape[2] * dx ** 3
    eta0 = _MU0 * _C
    H0 = Ht0 / eta0
    U = 0.5 * _EPS0 * (E0 @ E0) * (eps1 * V / 2 + eps2 * V / 2) + 0.5 * _MU0 * (H0 @ H0) * V
    assert abs(o.energy() / U - 1.0) < 1e-13
    o.step(5)
    assert abs(o.energy() / U - 1.0) < 1e-13
