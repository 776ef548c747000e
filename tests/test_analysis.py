"""Post-processing of the observation series, pinned by signals with known
answers (no GPU): a sinusoid's frequency, an exponential's time constant and
the diffusion constant of the closed form, and the weights of a known sum of
exponentials."""
import math

import numpy as np
import pytest

from paper_0802_3775_gb300 import analysis as A


def test_peak_frequency_of_a_sinusoid():
    dt = 1.0e-17
    f = 4.9e14                       # not on a bin of the transform
    n = np.arange(60000)
    rng = np.random.Generator(np.random.PCG64(1))
    phase = rng.uniform(0, 2 * np.pi, 3)
    series = np.stack([np.cos(2 * np.pi * f * n * dt + p) for p in phase], axis=1)
    series *= np.exp(1e-6 * n)[:, None]           # a slowly growing line, as past threshold
    bin_hz = 1.0 / (len(n) // 2 * dt)
    assert abs(A.peak_frequency(series, dt) - f) < 0.02 * bin_hz


def test_tail_fit_recovers_the_time_constant_and_diffusion_constant():
    dt = 2.0e-17
    tau_true = 3.3e-13
    t = np.arange(150000) * dt
    rise = 1 - np.exp(-t / 2e-14)
    T = rise * np.exp(-t / tau_true) + 0.5 * np.exp(-t / 2e-14)  # fast component dies before the edge
    tau = A.tail_time_constant(T, dt)
    assert abs(tau / tau_true - 1) < 1e-6
    L = 4.0e-6
    assert A.diffusion_constant(tau, L) == pytest.approx(L * L / (math.pi ** 2 * tau), rel=1e-15)
    # paper scale: a 4 um opal with tau0 ~ 1e-13 s gives D of order 10 m^2/s
    assert 5 < A.diffusion_constant(1.2e-13, 4.0e-6) < 20


def test_decay_time_distribution_recovers_two_components():
    dt = 1.0e-16
    taus = np.geomspace(1e-14, 1e-11, 61)
    w = np.zeros_like(taus)
    w[15], w[45] = 1.0, 0.3            # two components on the grid, one short-lived, one long-lived
    t = np.arange(6000) * dt
    T = np.exp(-t / taus[15]) * w[15] + np.exp(-t / taus[45]) * w[45]
    g = A.decay_time_distribution(T, dt, taus, window=(0, len(T)), alpha=1e-9)
    assert np.all(g >= 0)
    assert abs(g[15] - 1.0) < 1e-3 and abs(g[45] - 0.3) < 1e-3
    others = np.delete(g, [15, 45])
    assert np.max(others) < 1e-3
    # a single exponential gives a single peak at its time constant
    g1 = A.decay_time_distribution(np.exp(-t / taus[30]), dt, taus, window=(0, len(T)), alpha=1e-9)
    assert int(np.argmax(g1)) == 30


def test_trailing_edge_window():
    T = np.concatenate([np.linspace(0, 1, 50), np.exp(-np.arange(400) / 20.0)])
    i0, i1 = A.trailing_edge(T, start_fraction=0.1, end_fraction=1e-6)
    assert T[i0] < 0.1 <= T[i0 - 1]
    assert i1 == len(T) or T[i1] < 1e-6
