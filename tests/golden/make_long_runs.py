"""Writes the stored oracle results of the long-run parity tests.

Calls only the FP64 oracle (`oracle/`) and the seeded input generators; no
value here comes from the CUDA library.  Each run is a reduced copy of a
workload recipe, stepped for as long as the workload runs:

* ``long_opal64_f32.npz`` -- the passive [111] disordered-opal recipe at
  2x2x2 unit cells, 20 cells/a, 12-cell CPML (64^3 grid), sigma 6 %,
  20000 steps (the passive workload's run length), solved twice: with the
  binary32-rounded coefficient tables an FP32 run uses (``coef32``) and with
  exact coefficients.  Stored: the FP64 flux series T^n, the probe series at
  every 4th step (binary32: the bar is 1e-5), and the six fields at two full
  z-planes plus 2048 seeded cells (binary32) after SNAP_STEPS steps (while the
  pulse is inside the opal, on its trailing edge) and after the run.

Run from the repository root:  python tests/golden/make_long_runs.py [name ...]
(the two oracle runs of the 64^3 opal go to two processes, ~17 minutes).
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import Oracle  # noqa: E402
from paper_0802_3775_gb300 import inputs  # noqa: E402

OPAL64_STEPS = 20000
SNAP_STEPS = (2000, 5000)
OPAL64_PLANES = (20, 44)
OPAL64_NCELLS = 2048
PROBE_EVERY = 4


def opal64_spec():
    """The reduced passive workload run (also built by the test)."""
    return inputs.opal_planewave_f32(ncell=2, res=20, npml=12, sigma=0.06, realization=1, steps=OPAL64_STEPS)


def opal64_sample_cells(shape):
    """Seeded flat cell indices (x fastest) of the sampled final fields."""
    nx, ny, nz = shape
    rng = np.random.Generator(np.random.PCG64(64064))
    return np.sort(rng.choice(nx * ny * nz, size=OPAL64_NCELLS, replace=False)).astype(np.int64)


def sample_fields(F, shape):
    """F: float[6, nz, ny, nx] -> (planes float32[6, len(PLANES), ny, nx], cells float32[6, NCELLS])."""
    planes = np.stack([F[:, k] for k in OPAL64_PLANES], axis=1).astype(np.float32)
    cells = F.reshape(6, -1)[:, opal64_sample_cells(shape)].astype(np.float32)
    return planes, cells


def run_opal64(coef32):
    spec = opal64_spec()
    o = Oracle.from_spec(spec, coef32=coef32)
    t0 = time.perf_counter()
    out = {}
    for q, n in enumerate(SNAP_STEPS):
        o.step(n - o.n)
        planes, cells = sample_fields(o.fields_memory_order(), spec.shape)
        out[f"snap{q}_planes"], out[f"snap{q}_cells"] = planes, cells
    o.step(spec.steps - o.n)
    print(f"opal64 coef32={coef32}: {spec.steps} steps in {time.perf_counter() - t0:.0f} s", flush=True)
    planes, cells = sample_fields(o.fields_memory_order(), spec.shape)
    out.update(flux=o.flux_series()[0], probes=o.probe_series()[PROBE_EVERY - 1::PROBE_EVERY].astype(np.float32),
               planes=planes, cells=cells, energy=np.array([o.energy()]))
    return out


def make_opal64():
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(2) as pool:
        r32, rex = pool.map(run_opal64, [True, False])
    np.savez_compressed(os.path.join(HERE, "long_opal64_f32.npz"),
                        **{k + "_coef32": v for k, v in r32.items()},
                        **{k + "_exact": v for k, v in rex.items()})


if __name__ == "__main__":
    names = sys.argv[1:] or ["opal64"]
    for name in names:
        {"opal64": make_opal64}[name]()
