"""Host post-processing of the FP64 observation series (probe fields, flux
T^n): the quantities the paper extracts from its runs.

* `peak_frequency`: lasing line of a probe series (Sec. "3+1D simulation of
  lasing": emission spectra): Hann-windowed power spectrum of the last half
  of the series, peak refined by a parabola through the log power of the
  three bins around the maximum.
* `tail_time_constant` and `diffusion_constant`: the decaying tail of the
  transmitted power T(t) fitted by exp(-t/tau0) and D = L^2 / (pi^2 tau0) (Sec.
  "Dynamical diffusion and localization", diffusion constant and decay
  times).
* `decay_time_distribution`: the weights g(tau) >= 0 of a sum of
  exponentials exp(-t/tau) that best matches the trailing edge (same
  section), by non-negative least squares with a Tikhonov term.

Readings where the paper is silent: the trailing edge starts where T has
fallen below `start_fraction` of its maximum after the maximum and ends where
it falls below `end_fraction` of it (or at the end of the series); the
exponential fit is a least-squares line through log T over that window; the
regularization weight of g(tau) is alpha (relative to the largest singular
value of the kernel).  These run on the host on FP64 series read back from
the device; they are not part of the time stepping.
"""
from __future__ import annotations

import math

import numpy as np


def peak_frequency(series, dt: float) -> float:
    """Frequency (Hz) of the strongest line of a probe series [steps, 3] (or
    [steps]) sampled every dt seconds."""
    x = np.asarray(series, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    x = x[len(x) // 2:]
    x = x - x.mean(axis=0)
    w = np.hanning(len(x))[:, None]
    p = (np.abs(np.fft.rfft(x * w, axis=0)) ** 2).sum(axis=1)
    i = int(np.argmax(p[1:-1])) + 1
    a, b, c = np.log(p[i - 1]), np.log(p[i]), np.log(p[i + 1])
    shift = 0.5 * (a - c) / (a - 2.0 * b + c)
    return (i + shift) / (len(x) * dt)


def trailing_edge(T, start_fraction: float = 0.1, end_fraction: float = 1e-6):
    """Index range [i0, i1) of the trailing edge of a transmission series."""
    T = np.asarray(T, dtype=np.float64)
    k = int(np.argmax(T))
    peak = T[k]
    if not peak > 0:
        raise ValueError("the transmission has no positive maximum")
    after = np.nonzero(T[k:] < start_fraction * peak)[0]
    if len(after) == 0:
        raise ValueError("the transmission never falls below start_fraction of its maximum")
    i0 = k + int(after[0])
    below = np.nonzero(T[i0:] < end_fraction * peak)[0]
    i1 = i0 + int(below[0]) if len(below) else len(T)
    if i1 - i0 < 3:
        raise ValueError("trailing edge shorter than 3 samples")
    return i0, i1


def tail_time_constant(T, dt: float, window=None) -> float:
    """Leading time constant tau0 (s) of exp(-t/tau0) fitted to the trailing
    edge (least-squares line through log T)."""
    T = np.asarray(T, dtype=np.float64)
    i0, i1 = trailing_edge(T) if window is None else window
    t = np.arange(i0, i1) * dt
    y = T[i0:i1]
    keep = y > 0
    slope, _ = np.polyfit(t[keep], np.log(y[keep]), 1)
    if not slope < 0:
        raise ValueError("the trailing edge does not decay")
    return -1.0 / slope


def diffusion_constant(tau0: float, thickness: float) -> float:
    """D = L^2 / (pi^2 tau0) (m^2/s) for a slab of thickness L (m)."""
    return thickness * thickness / (math.pi * math.pi * tau0)


def decay_time_distribution(T, dt: float, taus, window=None, alpha: float = 1e-6):
    """g(tau_j) >= 0 minimizing ||sum_j g_j exp(-t/tau_j) - T(t)||^2 +
    (alpha s_max)^2 ||g||^2 over the trailing edge, t measured from the start
    of the window; s_max is the largest singular value of the kernel."""
    from scipy.optimize import nnls

    T = np.asarray(T, dtype=np.float64)
    taus = np.asarray(taus, dtype=np.float64)
    i0, i1 = trailing_edge(T) if window is None else window
    t = np.arange(0, i1 - i0) * dt
    K = np.exp(-t[:, None] / taus[None, :])
    s_max = np.linalg.norm(K, 2)
    A = np.vstack([K, alpha * s_max * np.eye(len(taus))])
    b = np.concatenate([T[i0:i1], np.zeros(len(taus))])
    g, _ = nnls(A, b, maxiter=50 * len(taus))
    return g
