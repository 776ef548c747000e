"""The byte model behind bench.py's roofline fraction (no GPU): the
compulsory HBM bytes of one step launch are every state word read once and
written once plus the material byte (binary32: 12 field words + 1 byte per
cell, 8 CPML words per slab membership, 21 gain words per gain cell), worked
out here by hand for the benchmark workloads and compared with bench.py."""
import numpy as np

import bench
from oracle.rasterize import rasterize
from paper_0802_3775_gb300 import inputs


def test_passive_184_cubed_bytes_by_hand():
    spec = inputs.opal_planewave_f32(ncell=8, res=20, npml=12, sigma=0.06)
    assert spec.shape == (184, 184, 184) and spec.gain is None
    ncell = 184 ** 3
    fields = ncell * (6 * 4 * 2 + 1)              # six fields read and written, material read
    slabs = 3 * (24 * 184 * 184) * (4 * 4 * 2)    # per axis 24 slab planes, 4 psi words read and written
    assert fields + slabs == 383249920
    assert bench.algorithmic_bytes(spec, 0) == 383249920.0


def test_lasing_140_cubed_bytes_with_oracle_gain_cells():
    spec = inputs.opal_lasing_f32(ncell=6, res=20, npml=10, sigma=0.05, pump=1e10)
    assert spec.shape == (140, 140, 140)
    mat = rasterize(spec.shape, spec.spheres, spec.box_lo, spec.box_hi)
    gain_cells = int(np.count_nonzero(mat & 64))
    # gain in the spheres of the 120^3 interior: close to the touching-sphere fill
    # fraction pi / (3 sqrt 2) of the interior, less what the disorder and the box clip
    frac = gain_cells / 120 ** 3
    assert 0.68 < frac < np.pi / (3 * np.sqrt(2)) + 0.01
    ncell = 140 ** 3
    by_hand = ncell * 49 + 3 * (20 * 140 * 140) * 32 + gain_cells * (6 + 3 + 3 + 3 + 3 + 3) * 4
    assert bench.algorithmic_bytes(spec, gain_cells) == float(by_hand)


def test_binary64_bytes_double_the_words():
    spec = inputs.opal_planewave_f32(ncell=2, res=12, npml=8, sigma=0.0, precision="f64")
    nx, ny, nz = spec.shape
    ncell = nx * ny * nz
    slab = sum(16 * ncell // n for n in (nx, ny, nz))
    assert bench.algorithmic_bytes(spec, 0) == float(ncell * 97 + slab * 64)
