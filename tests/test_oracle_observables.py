"""Pins of the oracle's flux, source, absorbing layer and rasterizer (no GPU).

* Poynting flux T^n of a discrete travelling eigenmode through a plane has the
  closed form  dx^2 N_faces E0^2 sqrt(eps_r) cos(k/2) cos(omega dt/2)
  cos^2(k p - omega n) / eta0  (the transmitted power T(t) of Sec. "Dynamical
  diffusion and localization" is this flux through the crystal's exit side);
* the source waveform has the stated centre frequency and power-spectrum FWHM
  (single-cycle / 100 fs pulses of Secs. "Wide-band excitation" and
  "Dynamical diffusion");
* a soft source in a one-cell periodic box drives E = -(A/eps_r) sum_n g(n);
* CPML reflection (the paper's absorbing layer, Sec. "Sample and numerical
  approach"): a probe near the layer agrees with a run in a much larger box
  to better than -40 dB until the outer box's echo returns, for a plain
  (kappa_max 1) and a stretched (kappa_max 3) layer;
* CPML memory: at slab nodes of each kind the memory series equals the
  recursive convolution of the raw differences (scipy's lfilter), and the
  update uses D / kappa + psi;
* rasterizer: brute force with scalar Python arithmetic on tiny grids equals the
  oracle bit for bit; touching fcc spheres fill pi/(3 sqrt 2) = 0.7405 of space;
* sheet source: in a transversely periodic box a uniform sheet radiates the
  field of a continuum current sheet, E = -eta K / 2 on each side, with a
  mismatch second order in k dx (it scales as eps_r f0^2); with a waist the
  sheet's profile is centred on the interior and isotropic on every axis;
* Poynting theorem: the flux a dipole pulse sends through the six faces of a
  closed cube, summed over time, equals the energy that ends up outside it,
  with a mismatch that falls as the square of the frequency (the faces' E and
  H are averaged to the face centres, a second-order approximation).
"""
import math

import numpy as np
import pytest

from oracle import EPS0, ETA0, Oracle, waveform
from oracle.rasterize import rasterize
from paper_0802_3775_gb300 import inputs


@pytest.mark.parametrize("axis,pol,eps_r", [(2, 0, 1.0), (2, 1, 2.0), (0, 1, 1.0), (0, 2, 3.0), (1, 2, 1.0), (1, 0, 1.5)])
def test_flux_of_travelling_eigenmode(axis, pol, eps_r):
    shape = [5, 6, 7]
    shape[axis] = 24
    shape = tuple(shape)
    o = Oracle(shape, 12, courant=0.5, periodic=(True, True, True), eps=(eps_r,) * 3)
    S = o.S
    kk = 2 * math.pi * 2 / shape[axis]
    k = np.zeros(3); k[axis] = kk
    K = 2 * np.sin(k / 2)
    E_hat = np.zeros(3); E_hat[pol] = 1.7
    Om = S * np.linalg.norm(K) / math.sqrt(eps_r)
    w = 2 * math.asin(Om / 2)
    H_hat = (S / Om) * np.cross(K, E_hat)
    NODE = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5), (0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]
    for c in range(6):
        X = np.meshgrid(*[np.arange(shape[d]) + NODE[c][d] for d in range(3)], indexing="ij")
        ph = k[0] * X[0] + k[1] * X[1] + k[2] * X[2]
        if c < 3:
            o.E[c] = E_hat[c] * np.cos(ph)
        else:
            o.H[c - 3] = H_hat[c - 3] * np.cos(ph + 0.5 * w)
    d1, d2 = (axis + 1) % 3, (axis + 2) % 3
    p = 9
    u = (1, shape[d1] - 2)
    v = (0, shape[d2] - 1)
    o.add_flux(axis, p, 1.0, u, v)
    N = 120
    o.step(N)
    T = o.flux_series()[0]
    nfaces = (u[1] - u[0]) * (v[1] - v[0])
    n = np.arange(N)
    ref = o.dx ** 2 * nfaces * 1.7 ** 2 * math.sqrt(eps_r) * math.cos(kk / 2) * math.cos(w / 2) * np.cos(kk * p - w * n) ** 2 / ETA0
    np.testing.assert_allclose(T, ref, rtol=0, atol=1e-10 * np.max(np.abs(ref)))


def test_waveform_centre_and_bandwidth():
    S, res, f0_hat, bw = 0.5 / math.sqrt(3), 20, 0.8, 0.1
    N = 1 << 16
    g = waveform(np.arange(N), f0_hat, bw, S, res)
    P = np.abs(np.fft.rfft(g)) ** 2
    f = np.fft.rfftfreq(N)
    f0 = f0_hat * S / res
    i = int(np.argmax(P))
    assert abs(f[i] - f0) / f0 < 0.01
    half = P >= 0.5 * P[i]
    lo = f[np.argmax(half)]
    hi = f[len(half) - 1 - np.argmax(half[::-1])]
    assert abs((hi - lo) / f0 - bw) / bw < 0.02
    # pulse centred at t0 = 5 tau: the envelope is below 1e-5 at n = 0
    tau = math.sqrt(math.log(2)) / (math.pi * bw * f0)
    assert abs(g[0]) < math.exp(-12.4)
    assert abs(np.argmax(np.abs(g)) + 0.5 - 5 * tau) < 1 / f0


def test_soft_source_in_one_cell_box():
    o = Oracle((1, 1, 1), 12, periodic=(True, True, True), eps=(1.0, 2.5, 1.0))
    o.add_source(kind="point", comp=1, pos=(0, 0, 0), amplitude=3.0, f0_hat=0.8, rel_bw=0.5)
    N = 700
    o.step(N)
    g = waveform(np.arange(N), 0.8, 0.5, o.S, 12)
    assert abs(o.E[1, 0, 0, 0] - (-(3.0 / 2.5) * g.sum())) < 1e-12
    assert o.E[0, 0, 0, 0] == 0.0 and o.E[2, 0, 0, 0] == 0.0


@pytest.mark.slow
@pytest.mark.parametrize("kappa_max", [1.0, 3.0])
def test_cpml_reflection_below_minus_40db(kappa_max):
    res, npml, interior, pad = 10, 8, 20, 16

    def run(n_extra):
        n = interior + 2 * npml + 2 * n_extra
        o = Oracle((n, n, n), res, npml=(npml,) * 6, eps=(1.0, 1.0, 1.0), cpml_f_hat=0.6,
                   cpml_kappa_max=kappa_max)
        c = n // 2
        o.add_source(kind="point", comp=2, pos=(c, c, c), f0_hat=0.6, rel_bw=1.0)
        # probe two cells inside the small box's absorbing layer boundary
        o.add_probe(c, c, n_extra + npml + 2)
        o.add_probe(n_extra + npml + 2, c + 3, c)
        o.step(150)
        return o.probe_series()

    small = run(0)
    big = run(pad)
    err = np.max(np.abs(small - big))
    ref = np.max(np.abs(big))
    # the bar is -40 dB; this layer reaches about -80 dB, so a broken
    # coefficient (which lands near the -20 dB of a bare PEC wall) cannot pass
    assert 20 * math.log10(err / ref) < -60.0


@pytest.mark.slow
@pytest.mark.parametrize("kappa_max", [1.0, 3.0])
def test_upml_reflection_below_minus_40db(kappa_max):
    """The uniaxial PML (the paper's absorber) on the same grading as the
    CPML: a dipole pulse near the layer seen from a small box and from a box
    larger by 16 cells on every side agree to better than -60 dB until the
    echo of the large box returns (the layer reaches about -80 dB; a node
    graded at the wrong half-integer offset lands near -22 dB, a sign slip in
    the D-to-E step near -39 dB)."""
    res, npml, interior, pad = 10, 8, 20, 16

    def run(n_extra):
        n = interior + 2 * npml + 2 * n_extra
        o = Oracle((n, n, n), res, npml=(npml,) * 6, eps=(1.0, 1.0, 1.0), cpml_f_hat=0.6,
                   cpml_kappa_max=kappa_max, absorber="upml")
        c = n // 2
        o.add_source(kind="point", comp=2, pos=(c, c, c), f0_hat=0.6, rel_bw=1.0)
        o.add_probe(c, c, n_extra + npml + 2)
        o.add_probe(n_extra + npml + 2, c + 3, c)
        o.step(150)
        return o.probe_series()

    small = run(0)
    big = run(pad)
    err = np.max(np.abs(small - big))
    ref = np.max(np.abs(big))
    assert 20 * math.log10(err / ref) < -60.0


def test_upml_without_conductivity_is_the_yee_update():
    """With zero conductivity and kappa 1 the layer's nodes, stepped through
    the auxiliary D~ and B~, give the plain Yee leapfrog of a grid without
    absorbing slabs to rounding (random fields, random permittivity, a PEC
    box)."""
    shape = (12, 11, 13)
    runs = []
    for npml, absorber in (((0,) * 6, "cpml"), ((4, 3, 4, 5, 3, 4), "upml")):
        o = Oracle(shape, 10, npml=npml, eps=(1.0, 2.5, 11.9), cpml_sigma_factor=0.0, absorber=absorber)
        o.set_material(inputs.random_material(shape, seed=41, classes=(0, 1, 2)))
        o.set_fields_memory_order(inputs.random_fields(shape, seed=42))
        o._pec(o.E)
        o.step(60)
        runs.append(o.fields_memory_order())
    assert np.max(np.abs(runs[0] - runs[1])) <= 1e-12 * np.max(np.abs(runs[0]))


def _brute_force_material(shape, spheres, lo, hi):
    nx, ny, nz = shape
    offs = ((0.5, 0.0, 0.0), (0.0, 0.5, 0.0), (0.0, 0.0, 0.5), (0.5, 0.5, 0.5))
    out = np.zeros((nz, ny, nx), dtype=np.uint8)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                byte = 0
                for s, (ox, oy, oz) in enumerate(offs):
                    p = (i + ox, j + oy, k + oz)
                    in_box = all(lo[d] <= p[d] < hi[d] for d in range(3))
                    ins = False
                    for (cx, cy, cz, r) in spheres:
                        dx = p[0] - cx; dy = p[1] - cy; dz = p[2] - cz
                        if (dx * dx + dy * dy) + dz * dz < r * r:
                            ins = True
                    if s < 3:
                        byte |= ((2 if ins else 1) if in_box else 0) << (2 * s)
                    elif ins and in_box:
                        byte |= 64
                out[k, j, i] = byte
    return out


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_rasterizer_brute_force(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (7, 5, 6)
    spheres = [(float(rng.uniform(-1, 8)), float(rng.uniform(-1, 6)), float(rng.uniform(-1, 7)), float(rng.uniform(0.5, 3)))
               for _ in range(4)]
    # a sphere whose surface passes exactly through sample points
    spheres.append((2.0, 2.0, 2.0, 1.5))
    lo, hi = (1, 0.5, 1), (6, 5, 5.5)
    ref = _brute_force_material(shape, spheres, lo, hi)
    got = rasterize(shape, np.array(spheres), lo, hi)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("res", [48, 64])
def test_touching_fcc_fill_fraction(res):
    n = res  # one conventional cube
    spheres = inputs.fcc_opal_spheres((0, 0, 0), (n, n, n), res, sigma=0.0)
    mat = rasterize((n, n, n), spheres, (0, 0, 0), (n, n, n))
    target = math.pi / (3 * math.sqrt(2))
    assert abs(float(np.mean((mat >> 6) & 1)) - target) < 0.005
    for c in range(3):
        cls = (mat >> (2 * c)) & 3
        assert set(np.unique(cls)) <= {1, 2}
        assert abs(float(np.mean(cls == 2)) - target) < 0.005


@pytest.mark.parametrize("kind,comp,d,where", [("H", 0, 2, "z+"), ("E", 1, 0, "x-"), ("E", 2, 1, "y+"), ("H", 2, 0, "x+")])
def test_cpml_memory_is_the_recursive_convolution(kind, comp, d, where):
    """Inside an absorbing slab the memory psi^n = b psi^{n-1} + c D^n is the
    recursive convolution of the raw difference D with c b^k: scipy's lfilter
    with numerator [c] and denominator [1, -b] reproduces the oracle's psi
    series at a slab node from the recorded D series, and the difference the
    update uses is D / kappa + psi (kappa_max = 3 here, so 1/kappa != 1)."""
    import dataclasses
    from scipy.signal import lfilter

    from helpers import small_opal

    class Recording(Oracle):
        def _term(self, D, dd, cc, kk):
            out = super()._term(D, dd, cc, kk)
            if (kk, cc, dd) == (kind, comp, d):
                self.rec.append((D[node], self.psi[kk][(cc, dd)][node], out[node]))
            return out

    spec = dataclasses.replace(small_opal(n_cells=2, res=8, npml=5, precision="f64", source="dipole"),
                               cpml_kappa_max=3.0)
    o = Recording.from_spec(spec)
    n3 = o.shape
    mid = [s // 2 for s in n3]
    depth = 2  # nodes into the slab
    axis = "xyz".index(where[0])
    mid[axis] = depth if where[1] == "-" else n3[axis] - 1 - depth
    node = tuple(mid)
    o.rec = []
    o.step(300)
    D, psi, used = map(np.array, zip(*o.rec))
    ik, b, c = (float(np.ravel(v)[node[d]]) for v in o.prof[kind][d])
    assert 0.0 < b < 1.0 and c < 0.0 and 0.0 < ik < 1.0
    assert np.max(np.abs(psi)) > 0.0
    ref = lfilter([c], [1.0, -b], D)
    assert np.max(np.abs(psi - ref)) <= 1e-13 * np.max(np.abs(psi))
    assert np.max(np.abs(used - (ik * D + psi))) <= 1e-15 * np.max(np.abs(used))


def _radiated_through_cube(f0_hat, n=48, half=6, steps=145):
    """z dipole at the centre of a closed lossless box; flux planes on the six
    faces of the cube [c - half, c + half]^3, outward signs.  Returns the
    time-summed outward flux of each face, the energy outside the cube and
    the energy inside it after `steps` (the pulse has left the cube, its
    echo from the walls has not come back)."""
    o = Oracle((n, n, n), 6, courant=0.5)
    c = n // 2
    o.add_source(kind="point", comp=2, pos=(c, c, c), f0_hat=f0_hat, rel_bw=1.0)
    lo, hi = c - half, c + half
    for d in range(3):
        o.add_flux(d, lo, -1.0, (lo, hi), (lo, hi))
        o.add_flux(d, hi, 1.0, (lo, hi), (lo, hi))
    for _ in range(steps - 1):
        o.step(1)
    E_prev = o.E.copy()
    o.step(1)
    # the discrete invariant 1/2 eps0 dx^3 (sum eps_r E^{n+1}.E^n + sum H~^{n+1/2}.H~^{n+1/2})
    dens = np.concatenate([o.eps_E * o.E * E_prev, o.H * o.H])
    inside = np.zeros((n, n, n), dtype=bool)
    inside[lo:hi + 1, lo:hi + 1, lo:hi + 1] = True
    w = 0.5 * EPS0 * o.dx ** 3
    u_in = w * float(np.sum(dens[:, inside]))
    u_out = w * float(np.sum(dens[:, ~inside]))
    faces = o.flux_series().sum(axis=1) * o.dt
    return faces, u_out, u_in


def test_poynting_theorem_over_a_closed_cube():
    m = {}
    for f0 in (0.5, 0.35):
        faces, u_out, u_in = _radiated_through_cube(f0)
        assert u_in < 2e-3 * u_out
        # the four side faces see the same flux, the two end faces of the dipole axis another
        np.testing.assert_allclose(faces[:4], faces[0], rtol=1e-12)
        m[f0] = (u_out - faces.sum()) / u_out
        assert 0 < m[f0] < 0.025
        # one face counted with the wrong orientation breaks the balance
        bad = faces.sum() - 2 * faces[1]
        assert abs(u_out - bad) / u_out > 0.2
    # second order: the mismatch scales as f0^2
    assert abs(m[0.5] / m[0.35] / (0.5 / 0.35) ** 2 - 1) < 0.03


def _sheet_mismatch(eps_r, f0_hat, amplitude=2.0, steps=1400):
    """Uniform x-polarized sheet at z = 200 of a 1 x 1 x 1200 box, periodic in
    x and y (a 1D problem), probe 100 cells downstream.  The soft term
    -(A/eps_r) g per step is a surface current K = eps0 A g c / S, whose
    continuum field is E = -(eta0 / sqrt(eps_r)) K / 2 = -A g / (2 S sqrt(eps_r)),
    delayed by the travel time.  Returns the relative mismatch of the
    time-summed E^2, the best correlation with the delayed continuum pulse and
    the delay of that best match beyond the continuum travel time."""
    o = Oracle((1, 1, 1200), 12, courant=0.5, periodic=(True, True, False), eps=(eps_r,) * 3)
    o.add_source(kind="sheet", comp=0, axis=2, index=200, f0_hat=f0_hat, rel_bw=0.5, amplitude=amplitude)
    o.add_probe(0, 0, 300)
    o.step(steps)
    e = o.probe_series()[:, 0, 0]
    ref = amplitude * waveform(np.arange(steps), f0_hat, 0.5, o.S, 12) / (2 * o.S * math.sqrt(eps_r))
    # best match over delays from the continuum travel time to a few steps
    # more (the grid's group velocity is a little lower)
    lag0 = 100 * math.sqrt(eps_r) / o.S
    corr = {lag: np.dot(e[lag:], ref[:-lag]) / math.sqrt(np.dot(e, e) * np.dot(ref, ref))
            for lag in range(int(lag0) - 1, int(lag0) + 8)}
    best = min(corr, key=corr.get)
    return float(np.sum(e * e) / np.sum(ref * ref) - 1.0), float(corr[best]), best - lag0


def test_sheet_source_radiates_the_current_sheet_field():
    m = {}
    for eps_r in (1.0, 2.5):
        for f0 in (0.25, 0.5):
            m[eps_r, f0], corr, delay = _sheet_mismatch(eps_r, f0)
            assert 0 < m[eps_r, f0] < 0.06
            assert corr < -0.99          # E = -eta K / 2: opposite to the current
            assert -1.0 < delay < 6.0
    for eps_r in (1.0, 2.5):
        assert abs(m[eps_r, 0.5] / m[eps_r, 0.25] / 4.0 - 1) < 0.1
    for f0 in (0.25, 0.5):
        assert abs(m[2.5, f0] / m[1.0, f0] / 2.5 - 1) < 0.1


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_sheet_waist_profile_is_centred_and_isotropic(axis):
    shape = (20, 26, 32)
    npml = (2, 4, 3, 5, 6, 2)
    o = Oracle(shape, 10, npml=npml)
    o.add_source(kind="sheet", comp=(axis + 1) % 3, axis=axis, index=9, waist=3.0)
    w = o.sources[-1]["w"]
    plane = np.take(w, 9, axis=axis)
    assert np.count_nonzero(w) == np.count_nonzero(plane)      # only the sheet plane is driven
    d1, d2 = (axis + 1) % 3, (axis + 2) % 3
    # the plane's array axes are the remaining axes in increasing order
    a1, a2 = sorted((d1, d2))
    lo = {d: npml[2 * d] for d in range(3)}
    hi = {d: shape[d] - npml[2 * d + 1] for d in range(3)}
    # zero outside the non-absorbing interior of the plane
    inside = np.zeros_like(plane, dtype=bool)
    inside[lo[a1]:hi[a1], lo[a2]:hi[a2]] = True
    assert np.all(plane[~inside] == 0) and np.all(plane[inside] > 0)
    # centred: the profile is mirror-symmetric about the interior centre on both axes
    sub = plane[lo[a1]:hi[a1], lo[a2]:hi[a2]]
    np.testing.assert_allclose(sub, sub[::-1, :], rtol=1e-13)
    np.testing.assert_allclose(sub, sub[:, ::-1], rtol=1e-13)
    # isotropic: one cell off the centre row weighs the same along either axis
    c1, c2 = 0.5 * (lo[a1] + hi[a1] - 1), 0.5 * (lo[a2] + hi[a2] - 1)
    i1, i2 = int(math.floor(c1)), int(math.floor(c2))
    f = lambda x1, x2: math.exp(-((x1 - c1) ** 2 + (x2 - c2) ** 2) / 9.0)
    assert math.isclose(plane[i1, i2] / plane[i1 + 1, i2], f(i1, i2) / f(i1 + 1, i2), rel_tol=1e-12)
    assert math.isclose(plane[i1, i2] / plane[i1, i2 + 1], f(i1, i2) / f(i1, i2 + 1), rel_tol=1e-12)


def test_rasterizer_degenerate_inputs():
    shape = (5, 4, 3)
    # no spheres: background inside the box, class 0 outside, no gain
    lo, hi = (1, 0, 1), (4, 4, 3)
    got = rasterize(shape, np.zeros((0, 4)), lo, hi)
    assert np.array_equal(got, _brute_force_material(shape, [], lo, hi))
    assert not np.any(got & 64)
    # an empty box: every node outside, whatever the spheres
    got = rasterize(shape, np.array([[2.0, 2.0, 1.0, 3.0]]), (2, 2, 2), (2, 2, 2))
    assert not np.any(got)
    # a zero-radius sphere on a sample point covers nothing (strict test)
    got = rasterize(shape, np.array([[1.5, 1.0, 1.0, 0.0]]), (0, 0, 0), shape)
    assert np.array_equal(got, np.full(shape[::-1], 0b010101, dtype=np.uint8))
