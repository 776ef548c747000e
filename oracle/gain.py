"""Four-level gain model coefficients (oracle side, FP64).

Test infrastructure only: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.

The gain medium of the paper has four levels, three of them degenerate and
each tied to one field component (Sec. "Sample and
numerical approach"), pumped externally for the lasing runs (Sec. "3+1D
simulation of lasing").  Its su(4) density-matrix form lives in a cited work
that is not available here, so the model follows the rate-equation form of
the 1D/2D models the paper contrasts itself with:

  levels 0..3, pump W: 0 -> 3, decays 3 -> 2 (tau32), 2 -> 1 (tau21, lasing),
  1 -> 0 (tau10);
  dN/dt = A N + R b,  b = (0, -1, +1, 0),  R = E . dP/dt / (hbar omega_a);
  d2P/dt2 + dw dP/dt + omega_a^2 P = kappa (N1 - N2) E.

Time integration of the populations is Crank-Nicolson:
  N^{n+1} = M N^n + v R^{n+1/2},  M = (I - dt A/2)^-1 (I + dt A/2),
  v = dt (I - dt A/2)^-1 b,
with M - I = dt (I - dt A/2)^-1 A formed directly (no cancellation).
"""
from __future__ import annotations

import math

import numpy as np

C0 = 299792458.0
MU0 = 1.25663706212e-6
EPS0 = 1.0 / (MU0 * C0 * C0)
HBAR = 1.054571817e-34

B_STIM = np.array([0.0, -1.0, 1.0, 0.0])


def rate_matrix(pump: float, tau32: float, tau21: float, tau10: float) -> np.ndarray:
    """A with dN/dt = A N for N = (N0, N1, N2, N3) and no field."""
    return np.array([
        [-pump, 1.0 / tau10, 0.0, 0.0],
        [0.0, -1.0 / tau10, 1.0 / tau21, 0.0],
        [0.0, 0.0, -1.0 / tau21, 1.0 / tau32],
        [pump, 0.0, 0.0, -1.0 / tau32],
    ])


def equilibrium(n_total: float, pump: float, tau32: float, tau21: float, tau10: float) -> np.ndarray:
    """Steady state of A: N3 = W tau32 N0, N2 = W tau21 N0, N1 = W tau10 N0."""
    n0 = n_total / (1.0 + pump * (tau32 + tau21 + tau10))
    return np.array([n0, pump * tau10 * n0, pump * tau21 * n0, pump * tau32 * n0])


def crank_nicolson(A: np.ndarray, dt: float):
    """(M - I, w) with N^{n+1} = N^n + (M - I) N^n + w (R dt)."""
    L = np.eye(4) - 0.5 * dt * A
    m_minus_i = dt * np.linalg.solve(L, A)
    w = np.linalg.solve(L, B_STIM)
    return m_minus_i, w


def default_kappa(omega_a: float, tau21: float) -> float:
    """Classical-oscillator coupling 6 pi eps0 c^3 / (omega_a^2 tau21) (C/(kg m^3) ... per m^-3)."""
    return 6.0 * math.pi * EPS0 * C0 ** 3 / (omega_a ** 2 * tau21)


def polarization_coefficients(omega_a: float, domega: float, kappa: float, dt: float):
    """(a1, a2, a3) of P~^{n+1} = a1 P~^n - a2 P~^{n-1} + a3 (N1 - N2) E^n with P~ = P / eps0.

    Central differences of d2P/dt2 + dw dP/dt + omega_a^2 P = kappa (N1 - N2) E.
    """
    g = 0.5 * domega * dt
    a1 = (2.0 - (omega_a * dt) ** 2) / (1.0 + g)
    a2 = (1.0 - g) / (1.0 + g)
    a3 = kappa * dt * dt / (EPS0 * (1.0 + g))
    return a1, a2, a3
