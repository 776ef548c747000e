"""Plain, slow, FP64 CPU oracle of the Maxwell-Bloch FDTD hot path.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.
The CUDA library and its Python binding never import it, and it imports
nothing from them; the two share only the seeded input generators.

Modules:
  fdtd       -- the Yee / CPML / gain / noise / source / probe / flux stepper
  rasterize  -- sphere list -> per-cell material bytes
  gain       -- four-level rate matrix, equilibrium, Crank-Nicolson and
                polarization-oscillator coefficients
  philox     -- Philox4x32-10 and Box-Muller, written from their definitions
"""
from .fdtd import Oracle, waveform, C0, MU0, EPS0, ETA0, HBAR  # noqa: F401
