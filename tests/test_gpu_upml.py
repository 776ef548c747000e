"""GPU parity of the uniaxial PML option (the paper's absorber, Sec. "Sample
and numerical approach") and of an air margin around the crystal (the
paper's 6 um box around a 4 um opal), against the FP64 oracle on the same
seeded inputs, through the C ABI.

Bars as for the CPML runs: FP64 fields, probes and flux <= 1e-12 relative
L2; FP32 (oracle fed the binary32-rounded coefficients) fields and probes
<= 1e-5, flux <= 1e-4.  A UPML grid refuses a gain medium."""
import dataclasses

import numpy as np
import pytest

from helpers import gpu_grid, oracle_grid, rel_l2, small_opal
from paper_0802_3775_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0802_3775_gb300 import build
    build.build()


def _air_margin(spec, margin=3):
    """The structure box inset by `margin` cells from the absorbing slabs, air
    (eps 1) between the crystal and the slabs and inside them."""
    lo = tuple(spec.npml[2 * d] + margin for d in range(3))
    hi = tuple(spec.shape[d] - spec.npml[2 * d + 1] - margin for d in range(3))
    out = dataclasses.replace(spec, eps=(1.0,) + tuple(spec.eps[1:]), box_lo=lo, box_hi=hi)
    out.spheres = inputs.fcc_opal_spheres(lo, hi, spec.res, sigma=0.05, seed=spec.seed)
    return out


def _check(spec, steps, tol_f, tol_t):
    g = gpu_grid(spec)
    o = oracle_grid(spec, coef32=spec.precision == "f32")
    g.step(steps)
    o.step(steps)
    assert rel_l2(g.read_fields(), o.fields_memory_order()) <= tol_f
    assert rel_l2(g.read_probes(), o.probe_series()) <= tol_f
    assert rel_l2(g.read_flux(), o.flux_series()) <= tol_t
    return g, o


@pytest.mark.parametrize("source", ["dipole", "sheet"])
def test_fp64_upml_matches_oracle(source):
    spec = small_opal(precision="f64", source=source)
    spec.absorber = "upml"
    g, o = _check(spec, 400, 1e-12, 1e-12)
    assert g.kernel_in_use()[0] == 4
    assert abs(g.field_energy() / o.energy() - 1.0) <= 1e-12


def test_fp32_upml_matches_oracle():
    spec = small_opal(precision="f32", source="sheet", sigma=0.08)
    spec.absorber = "upml"
    _check(spec, 1200, 1e-5, 1e-4)


@pytest.mark.parametrize("precision,absorber", [("f64", "cpml"), ("f32", "cpml"), ("f32", "upml")])
def test_air_margin_matches_oracle(precision, absorber):
    spec = _air_margin(small_opal(precision=precision, source="sheet"))
    spec.absorber = absorber
    o = oracle_grid(spec)
    # air around the crystal and in the slabs: the outside class is eps 1
    assert np.any(o.eps_E == 1.0) and np.any(o.eps_E == 11.9)
    tol = (1e-12, 1e-12) if precision == "f64" else (1e-5, 1e-4)
    _check(spec, 600, *tol)


def test_upml_grid_refuses_gain():
    from paper_0802_3775_gb300.fdtd import FdtdError
    spec = small_opal(precision="f32")
    spec.absorber = "upml"
    g = gpu_grid(spec)
    with pytest.raises(FdtdError) as e:
        g.set_gain(inputs.GainSpec())
    assert e.value.code == -1


def test_a_batch_refuses_a_upml_member():
    from paper_0802_3775_gb300.fdtd import Batch, FdtdError
    spec = small_opal(precision="f32")
    spec.absorber = "upml"
    a = gpu_grid(spec)
    b = gpu_grid(small_opal(precision="f32"))
    with pytest.raises(FdtdError) as e:
        Batch([a, b])
    assert e.value.code == -1


def test_upml_checkpoint_and_autotune_are_bitwise():
    """The UPML's auxiliary fields travel with a checkpoint and survive the
    autotuner's trials: a run split by save/load, or tuned mid-run, equals
    the straight run bit for bit."""
    import os
    import tempfile
    spec = small_opal(precision="f32", source="sheet")
    spec.absorber = "upml"
    a = gpu_grid(spec)
    a.step(200)
    ref = a.read_fields()
    b = gpu_grid(spec)
    b.step(120)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        b.save_state(path)
        c = gpu_grid(spec)
        c.load_state(path)
    c.step(80)
    assert np.array_equal(c.read_fields(), ref)
    t = gpu_grid(spec)
    t.step(120)
    t.autotune(trial_steps=3)
    t.step(80)
    assert np.array_equal(t.read_fields(), ref)
