"""Pins of the oracle's four-level Maxwell-Bloch gain model and noise (no GPU).

The lasing model (paper, Secs. "Sample and numerical approach" and "3+1D
simulation of lasing": four-level system, three degenerate levels coupled to
the three field components, external pump, spontaneous-emission noise) is
checked against:

* the rate matrix conserving sum N and the closed-form steady state;
* zero field: the population relaxation against exp(t A) N(0) (scipy) and the
  Bateman cascade solution, with second-order convergence of Crank-Nicolson;
* a one-cell periodic box (no curl): the coupled E / P / N system against an
  independent high-accuracy ODE integration of the continuum equations, with
  second-order convergence, and exact conservation of D = eps_r E + P~;
* Philox4x32-10 published known-answer vectors and Gaussian statistics;
* a slab of inverted (or absorbing) medium in a 1D waveguide amplifies (or
  attenuates) a pulse by the plane-wave factor of a Lorentz medium,
  exp(-2 Im k L) with k = (w/c) sqrt(eps_r + chi(w)) and
  chi = (kappa/eps0)(N1 - N2)/(w_a^2 - w^2 - i w dw), averaged over the
  pulse spectrum, the exponent converging at second order in dx.
"""
import math
import os

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg
import scipy.stats

from oracle import C0, EPS0, HBAR, Oracle
from oracle import gain as G
from oracle.philox import gain_noise, philox4x32_10
from paper_0802_3775_gb300 import inputs

GAIN_BYTE = np.uint8(0b1101010)  # all three E components class 2, gain bit set


def one_cell(courant, eps_sphere=2.25, **gain):
    o = Oracle((1, 1, 1), 20, courant=courant, periodic=(True, True, True), eps=(1.0, 1.0, eps_sphere))
    o.set_material(np.full((1, 1, 1), GAIN_BYTE))
    o.set_gain(**gain)
    return o


def test_rate_matrix_and_equilibrium():
    W, t32, t21, t10 = 3e10, 100e-15, 1e-9, 100e-15
    A = G.rate_matrix(W, t32, t21, t10)
    assert np.allclose(A.sum(axis=0), 0.0, atol=0)
    Neq = G.equilibrium(1e24, W, t32, t21, t10)
    assert abs(Neq.sum() - 1e24) < 1e24 * 1e-15
    assert np.max(np.abs(A @ Neq)) < 1e24 * 1e-15 / t10
    # flux balance around the cycle 0 -> 3 -> 2 -> 1 -> 0
    assert math.isclose(W * Neq[0], Neq[3] / t32, rel_tol=1e-14)
    assert math.isclose(Neq[3] / t32, Neq[2] / t21, rel_tol=1e-14)
    assert math.isclose(Neq[2] / t21, Neq[1] / t10, rel_tol=1e-14)
    # Crank-Nicolson keeps sum N: 1^T (M - I) = 0 and 1^T w = 0
    MmI, w = G.crank_nicolson(A, 1e-17)
    assert np.max(np.abs(MmI.sum(axis=0))) < 1e-18
    assert abs(w.sum()) < 1e-15


def _relax(courant, steps_time, W, taus):
    o = one_cell(courant, n_total=1e24, fa_hat=0.8, dw_rel=0.02, tau32=taus[0], tau21=taus[1],
                 tau10=taus[2], pump=W, init="ground")
    nsteps = int(round(steps_time / o.dt))
    o.step(nsteps)
    return o.populations()[:, 0, 0, 0], nsteps * o.dt, o


@pytest.mark.parametrize("W", [0.0, 2e12])
def test_relaxation_matches_matrix_exponential(W):
    taus = (100e-15, 300e-15, 50e-15)
    t_end = 0.4e-12
    N, t, o = _relax(0.5, t_end, W, taus)
    A = G.rate_matrix(W, *taus)
    ref = scipy.linalg.expm(t * A) @ np.array([1e24, 0, 0, 0])
    err = np.max(np.abs(N - ref)) / 1e24
    assert err < 1e-7
    assert abs(N.sum() - 1e24) / 1e24 < 1e-13
    # second-order convergence in dt
    N2, t2, _ = _relax(0.25, t_end, W, taus)
    ref2 = scipy.linalg.expm(t2 * A) @ np.array([1e24, 0, 0, 0])
    err2 = np.max(np.abs(N2 - ref2)) / 1e24
    if err > 1e-12:
        assert 3.3 < err / err2 < 4.7


def test_relaxation_bateman_cascade():
    # all population in level 3, no pump: 3 -> 2 -> 1 -> 0 cascade in closed form
    taus = (100e-15, 300e-15, 50e-15)
    o = one_cell(0.5, n_total=1e24, fa_hat=0.8, dw_rel=0.02, tau32=taus[0], tau21=taus[1],
                 tau10=taus[2], pump=0.0, init="steady")
    # steady state without pump is the ground state; move everything to level 3
    o.dN[:, 0, 0, 0] = np.array([-1e24, 0.0, 0.0, 1e24])
    n = 9000
    o.step(n)
    t = n * o.dt
    a, b, c = 1 / taus[0], 1 / taus[1], 1 / taus[2]
    N3 = math.exp(-a * t)
    N2 = a / (b - a) * (math.exp(-a * t) - math.exp(-b * t))
    N1 = a * b * (math.exp(-a * t) / ((b - a) * (c - a)) + math.exp(-b * t) / ((a - b) * (c - b))
                  + math.exp(-c * t) / ((a - c) * (b - c)))
    ref = 1e24 * np.array([1 - N1 - N2 - N3, N1, N2, N3])
    assert np.max(np.abs(o.populations()[:, 0, 0, 0] - ref)) / 1e24 < 1e-7


def _zero_d_reference(t_end, eps_r, pars, drive):
    """Continuum E/P/N equations of a uniform field (no curl), integrated by DOP853.

    drive(t) is the source current term, in V/m per second, entering
    eps_r dE/dt = -dP~/dt - drive(t).
    """
    omega_a = 2 * math.pi * pars["fa_hat"] * C0 / 480e-9
    dw = pars["dw_rel"] * omega_a
    kappa = G.default_kappa(omega_a, pars["tau21"])
    A = G.rate_matrix(pars["pump"], pars["tau32"], pars["tau21"], pars["tau10"])
    Neq = G.equilibrium(pars["n_total"], pars["pump"], pars["tau32"], pars["tau21"], pars["tau10"])

    def rhs(t, y):
        E, P, Q, N = y[0:3], y[3:6], y[6:9], y[9:13]   # P = P~ = P/eps0, Q = dP~/dt
        dQ = -dw * Q - omega_a ** 2 * P + (kappa / EPS0) * (N[1] - N[2]) * E
        dE = -(Q + drive(t)) / eps_r
        R = EPS0 * float(E @ Q) / (HBAR * omega_a)
        dN = A @ N + R * np.array([0.0, -1.0, 1.0, 0.0])
        return np.concatenate([dE, Q, dQ, dN])

    y0 = np.concatenate([np.zeros(9), Neq])
    return scipy.integrate.solve_ivp(rhs, (0, t_end), y0, method="DOP853", rtol=1e-11, atol=1e-30,
                                     dense_output=True, max_step=t_end / 400)


@pytest.mark.parametrize("pump", [3e12, 1e8])
def test_zero_dimensional_maxwell_bloch_against_ode(pump):
    """Field driven from rest by a smooth pulse in a one-cell box with gain."""
    pars = dict(n_total=1e24, fa_hat=0.8, dw_rel=0.02, tau32=100e-15, tau21=1e-9, tau10=100e-15, pump=pump)
    rate = np.array([2e21, -3e21, 1e21])        # V/m/s: amplitude of the current term
    f0_hat, bw = 0.8, 0.5
    f0 = f0_hat * C0 / 480e-9
    tau = math.sqrt(math.log(2)) / (math.pi * bw * f0)

    def drive(t):
        x = t - 5 * tau
        return rate * math.exp(-x * x / (2 * tau * tau)) * math.sin(2 * math.pi * f0 * x)

    t_end = 25e-15
    errs, nerrs = [], []
    for courant in (0.5, 0.25):
        o = one_cell(courant, **pars, init="steady")
        for c in range(3):
            # amplitude is the per-step kick: rate * dt; pulse centred at 5 tau in steps
            o.add_source(kind="point", comp=c, pos=(0, 0, 0), amplitude=rate[c] * o.dt, f0_hat=f0_hat, rel_bw=bw)
        o.add_probe(0, 0, 0)
        n = int(round(t_end / o.dt))
        o.step(n)
        sol = _zero_d_reference(n * o.dt, 2.25, pars, drive)
        times = (np.arange(n) + 1) * o.dt
        Eref = sol.sol(times)[0:3].T
        Egot = o.probe_series()[:, 0, :]
        errs.append(np.max(np.abs(Egot - Eref)) / np.max(np.abs(Eref)))
        # D = eps_r E + P~ changes only through the source
        g = np.array([o.sources[c]["w"][0, 0, 0] for c in range(3)])
        from oracle import waveform
        gsum = waveform(np.arange(n), f0_hat, bw, o.S, o.res).sum()
        D = 2.25 * o.E[:, 0, 0, 0] + o.P[:, 0, 0, 0]
        assert np.max(np.abs(D + g * gsum)) < 1e-9 * np.max(np.abs(g * gsum))
        Nref = sol.y[9:13, -1]
        dN_ref = Nref - G.equilibrium(1e24, pump, 100e-15, 1e-9, 100e-15)
        nerrs.append(np.max(np.abs(o.dN[:, 0, 0, 0] - dN_ref)) / np.max(np.abs(dN_ref)))
    assert errs[1] < 2e-3 and nerrs[1] < 2e-3
    assert 3.3 < errs[0] / errs[1] < 4.7
    # the stimulated-exchange rate is centred in time: populations converge at second order too
    assert 3.3 < nerrs[0] / nerrs[1] < 4.7


def test_philox_known_answers(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = philox4x32_10(r[0:4], r[4:6])
        assert [int(x) for x in out] == r[6:10]


def test_noise_is_standard_normal():
    xi = gain_noise(seed=12345, step=7, cells=np.arange(200000))
    assert xi.shape == (3, 200000)
    for c in range(3):
        assert abs(xi[c].mean()) < 5 / math.sqrt(2e5)
        assert abs(xi[c].var() - 1) < 5 * math.sqrt(2 / 2e5)
        assert scipy.stats.kstest(xi[c], "norm").pvalue > 1e-4
    # different steps and seeds give independent draws
    xi2 = gain_noise(seed=12345, step=8, cells=np.arange(200000))
    xi3 = gain_noise(seed=12346, step=7, cells=np.arange(200000))
    assert abs(np.corrcoef(xi[0], xi2[0])[0, 1]) < 0.02
    assert abs(np.corrcoef(xi[0], xi3[0])[0, 1]) < 0.02


def test_noise_kick_statistics_in_gain_cells():
    # with the field held at zero by a huge permittivity the kicks accumulate in P
    o = Oracle((6, 5, 4), 20, periodic=(True, True, True), eps=(1.0, 1.0, 1e30))
    o.set_material(np.full((4, 5, 6), GAIN_BYTE))
    o.set_gain(n_total=1e24, fa_hat=0.8, dw_rel=0.02, tau32=100e-15, tau21=1e-9, tau10=100e-15,
               pump=0.0, noise_amp=1e-6)
    o.seed = 99
    o.step(1)
    xi = gain_noise(99, 0, np.arange(120))
    got = o.P.transpose(0, 3, 2, 1).reshape(3, -1)
    np.testing.assert_allclose(got, 1e-6 * xi, rtol=1e-15, atol=0)


def test_energy_bookkeeping_field_plus_upper_population_is_conserved():
    """Closed PEC box, every cell a gain cell, relaxation and pump off (rates
    ~1e-6 /s), an inverted initial population: the discrete field energy
    W^n = 1/2 eps0 dx^3 (sum eps_r E^n.E^n + sum H~^{n+1/2}.H~^{n-1/2}) plus
    hbar w_a dx^3 sum N2^n is conserved to rounding, because the field's work
    on the polarization, -(E^{n+1}+E^n)/2 . (P~^{n+1}-P~^n), is exactly the
    energy the rate equations hand to level 2 (paper, Sec. "Sample and
    numerical approach": energy exchange between field and medium)."""
    shape = (7, 8, 6)
    o = Oracle(shape, 12, courant=0.5, eps=(1.0, 2.5, 2.25))
    mat = inputs.random_material(shape, seed=21, classes=(1, 2)) | np.uint8(64)
    o.set_material(mat)
    n_total, fa = 1e24, 0.8
    omega_a = 2.0 * math.pi * fa * C0 / o.a
    o.set_gain(n_total=n_total, fa_hat=fa, dw_rel=0.02, tau32=1e6, tau21=1e6, tau10=1e6, pump=0.0,
               kappa=G.default_kappa(omega_a, 1e-9), noise_amp=0.0, init="ground")
    o.dN[0] -= 0.4 * n_total   # 40 % of the atoms moved from level 0 to level 2: inverted
    o.dN[2] += 0.4 * n_total
    rng = np.random.Generator(np.random.PCG64(22))
    o.E[:] = 1e7 * rng.normal(size=o.E.shape)   # strong enough that the exchange shows in N2 at FP64
    o.E[1][0] = o.E[2][0] = 0.0
    o.E[0][:, 0] = o.E[2][:, 0] = 0.0
    o.E[0][:, :, 0] = o.E[1][:, :, 0] = 0.0
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
    assert moved > 1e-5 * abs(C[0])                       # the field gained energy from level 2
    assert np.max(np.abs(C - C[0])) <= 1e-14 * abs(C[0])  # ... exactly what level 2 lost
    assert np.max(np.abs(C - C[0])) <= 1e-9 * moved


@pytest.mark.parametrize("steps_per_period", [20, 40, 80])
def test_polarization_recurrence_against_the_damped_oscillator(steps_per_period):
    """The P~ recurrence with constant drive: its characteristic roots give the
    damped oscillator's decay rate dw/2 and frequency sqrt(w_a^2 - dw^2/4) to
    second order in dt, and its fixed point is the static response
    kappa (N1-N2) E / (eps0 w_a^2) exactly (paper, Sec. "Sample and numerical
    approach": Lorentz polarization driven by the population difference)."""
    omega_a, domega, kappa = 2 * math.pi * 5e14, 0.2 * 2 * math.pi * 5e14, 3.0e-5
    dt = 2 * math.pi / omega_a / steps_per_period
    a1, a2, a3 = G.polarization_coefficients(omega_a, domega, kappa, dt)
    lam = np.roots([1.0, -a1, a2])
    decay = -math.log(abs(lam[0])) / dt
    freq = abs(np.angle(lam[0])) / dt
    w_d = math.sqrt(omega_a ** 2 - domega ** 2 / 4)
    h = omega_a * dt
    assert abs(decay / (domega / 2) - 1) < 0.5 * h * h
    assert abs(freq / w_d - 1) < 0.5 * h * h
    # fixed point of the driven recurrence
    dn, E = 2.5e23, 7.0
    P_star = a3 * dn * E / (1.0 - a1 + a2)
    assert abs(P_star / (kappa * dn * E / (EPS0 * omega_a ** 2)) - 1) < 1e-12
    # the recurrence itself converges to it
    p_prev = p = 0.0
    for _ in range(200 * steps_per_period):
        p, p_prev = a1 * p - a2 * p_prev + a3 * dn * E, p
    assert abs(p / P_star - 1) < 1e-9


def _slab_transmission(inversion, res, kappa=4.2e-7, f0=0.4, dw_rel=0.2, rel_bw=0.1):
    """x-polarized pulse from a uniform sheet through a 100-cell slab (at
    res = 12; lengths scale with res) of gain cells in a 1 x 1 x n box that
    is periodic across and absorbing at both z ends.  inversion: fraction of
    the atoms moved from level 0 to level 2 (> 0) or to level 1 (< 0), with
    relaxation and pump off.  Returns (sum of E^2 at a probe behind the slab,
    the oracle, the probe series)."""
    sc = res // 12
    n = 260 * sc
    o = Oracle((1, 1, n), res, courant=0.5, periodic=(True, True, False), npml=(0, 0, 0, 0, 20 * sc, 20 * sc))
    mat = np.full((n, 1, 1), 0b010101, dtype=np.uint8)
    mat[60 * sc:160 * sc] |= 64
    o.set_material(mat)
    o.set_gain(n_total=1e24, fa_hat=f0, dw_rel=dw_rel, tau32=1e6, tau21=1e6, tau10=1e6, pump=0.0,
               kappa=kappa, noise_amp=0.0, init="ground")
    m = o.gain["mask"]
    o.dN[0][m] -= abs(inversion) * 1e24
    o.dN[2 if inversion > 0 else 1][m] += abs(inversion) * 1e24
    o.add_source(kind="sheet", comp=0, axis=2, index=30 * sc, f0_hat=f0, rel_bw=rel_bw, amplitude=1.0)
    o.add_probe(0, 0, 200 * sc)
    o.step(4000 * sc)             # the whole pulse passes the probe
    e = o.probe_series()[:, 0, 0]
    return float(np.sum(e * e)), o, e


def _lorentz_factor(o, inversion, kappa, weights, length):
    """Spectrum-averaged plane-wave power factor of the continuum Lorentz medium."""
    m = 8 * len(weights)
    spec = np.abs(np.fft.rfft(weights, m)) ** 2
    w = 2 * np.pi * np.fft.rfftfreq(m, d=o.dt)
    wa, dwa = o.gain["omega_a"], o.gain["domega"]
    chi = (kappa / EPS0) * (-inversion * 1e24) / (wa ** 2 - w ** 2 - 1j * w * dwa)
    k = (w / C0) * np.sqrt(1.0 + chi + 0j)
    return float(np.sum(spec * np.exp(-2.0 * np.imag(k) * length)) / np.sum(spec))


def test_slab_gain_and_loss_match_the_lorentz_medium():
    kappa = 4.2e-7
    err = {}
    for res in (12, 24):
        ref, _, e0 = _slab_transmission(0.0, res, kappa)
        for inv in (0.5, -0.5):
            u, o, _ = _slab_transmission(inv, res, kappa)
            expect = _lorentz_factor(o, inv, kappa, e0, 100 * (res // 12) * o.dx)
            assert (expect > 2.0) if inv > 0 else (expect < 0.5)    # a strong effect
            err[res, inv] = math.log(u / ref) / math.log(expect) - 1.0
            # linear regime: the populations have not moved
            N = o.populations()[:, o.gain["mask"]]
            assert np.max(np.abs(N[2] - (0.5e24 if inv > 0 else 0.0))) < 1e-9 * 1e24
    for inv in (0.5, -0.5):
        assert abs(err[12, inv]) < 0.012
        assert abs(err[24, inv]) < 0.4 * abs(err[12, inv])        # second order in dx


def test_gain_model_without_gain_cells_leaves_the_passive_run_unchanged():
    """Degenerate case: a gain medium switched on in a grid whose cells are
    all outside the spheres changes nothing, noise included, bit for bit."""
    shape = (8, 7, 6)
    mat = inputs.random_material(shape, seed=41, classes=(1, 2))     # gain bit clear everywhere
    runs = []
    for with_gain in (False, True):
        o = Oracle(shape, 10, npml=(2, 2, 0, 0, 1, 3), eps=(1.0, 2.5, 11.9), seed=7)
        o.set_material(mat)
        if with_gain:
            o.set_gain(n_total=1e24, fa_hat=0.8, dw_rel=0.02, tau32=100e-15, tau21=1e-9, tau10=100e-15,
                       pump=1e12, noise_amp=1e3)
        o.add_source(kind="point", comp=1, pos=(4, 3, 3), f0_hat=0.8, rel_bw=0.5)
        o.step(120)
        runs.append(o)
    assert np.any(runs[0].E != 0)
    assert np.array_equal(runs[0].E, runs[1].E) and np.array_equal(runs[0].H, runs[1].H)
    assert not np.any(runs[1].P) and not np.any(runs[1].dN)
