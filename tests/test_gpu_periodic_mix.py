"""Periodic axes combined with the other features, against the FP64 oracle
on the same seeded inputs: a slab of opal periodic in x and y (the paper's
crystal seen as an infinite slab; the step runs on the plain-load kernel,
the only one that wraps), with

* a gain medium in the cell coupling and in the centred coupling (pump,
  noise; the centred averages wrap across the periodic faces),
* the uniaxial PML on the non-periodic axis,

in binary64 (fields <= 1e-12 relative L2, population deviations <= 1e-9)
and binary32 (fields <= 1e-5 against the binary32-coefficient oracle)."""
import numpy as np
import pytest

from helpers import gpu_grid, oracle_grid, rel_l2
from paper_0802_3775_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0802_3775_gb300 import build
    build.build()


def _slab(precision, gain=None, absorber="cpml"):
    res, npml = 8, 6
    n = 2 * res
    shape = (n, n, n + 2 * npml + 4)
    spec = inputs.RunSpec(shape=shape, res=res, npml=(0, 0, 0, 0, npml, npml), periodic=(True, True, False),
                          eps=(11.9, 11.9, 1.0 if gain is None else 2.25), precision=precision, seed=9,
                          absorber=absorber)
    spec.box_lo, spec.box_hi = (0, 0, npml + 2), (n, n, npml + 2 + n)
    spec.spheres = inputs.fcc_opal_spheres(spec.box_lo, spec.box_hi, res, sigma=0.05, seed=19)
    spec.sources = [inputs.SourceSpec(kind="sheet", comp=0, axis=2, index=npml + 1, f0_hat=0.8, rel_bw=0.3)]
    spec.probes = inputs.probe_cells(spec.shape, spec.npml, 4, seed=10)
    spec.fluxes = [inputs.plane_flux(spec, 2, shape[2] - npml - 1)]
    spec.gain = gain
    return spec


def _gain(coupling):
    return inputs.GainSpec(n_total=1e24, fa_hat=0.8, dw_rel=0.02, tau32=100e-15, tau21=1e-9, tau10=100e-15,
                           pump=5e11, noise_amp=1e-3, init="ground", coupling=coupling)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("case", ["cell", "centred", "upml"])
def test_periodic_slab_matches_oracle(precision, case):
    spec = _slab(precision, gain=None if case == "upml" else _gain(case), absorber="upml" if case == "upml" else "cpml")
    g = gpu_grid(spec)
    o = oracle_grid(spec)
    g.step(250)
    o.step(250)
    assert g.kernel_in_use()[0] == (4 if case == "upml" else 1)
    tol = 1e-12 if precision == "f64" else 1e-5
    assert rel_l2(g.read_fields(), o.fields_memory_order()) <= tol
    assert rel_l2(g.read_flux(), o.flux_series()) <= (1e-12 if precision == "f64" else 1e-4)
    if spec.gain is not None:
        assert np.max(np.abs(o.P)) > 0
        assert rel_l2(g.read_gain(3), o.dN[1:].transpose(0, 3, 2, 1)) <= (1e-9 if precision == "f64" else 1e-6)
