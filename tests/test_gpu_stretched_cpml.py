"""GPU parity with a stretched absorbing layer (kappa_max = 3): the 1/kappa
factor of every CPML derivative (paper, Sec. "Sample and numerical approach":
absorbing layer; CPML reading) enters each step kernel through its
coefficient tables, so every kernel is compared with the oracle on a small
ragged opal whose fields the stretch changes by ~30 % in relative L2.
Bars as in the other parity tests: FP64 fields, probes and every flux plane
<= 1e-12; FP32 fields and probes <= 1e-5, transmitted flux <= 1e-4 (oracle
fed the binary32-rounded coefficients)."""
import pytest

from helpers import gpu_grid, oracle_grid, rel_l2, small_opal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0802_3775_gb300 import build
    build.build()


@pytest.mark.parametrize("kernel,precision", [("pair", "f32"), ("tma", "f32"), ("plain", "f32"),
                                              ("tma", "f64"), ("plain", "f64")])
def test_stretched_cpml_matches_oracle(kernel, precision):
    spec = small_opal(precision=precision, source="sheet", sigma=0.08)
    spec.cpml_kappa_max = 3.0
    g = gpu_grid(spec)
    g.set_kernel(kernel)
    o = oracle_grid(spec, coef32=precision == "f32")
    g.step(600)
    o.step(600)
    assert g.kernel_in_use()[0] == {"plain": 1, "tma": 2, "pair": 3}[kernel]
    if precision == "f32":
        assert rel_l2(g.read_fields(), o.fields_memory_order()) <= 1e-5
        assert rel_l2(g.read_flux(0), o.flux_series()[0]) <= 1e-4
        assert rel_l2(g.read_probes(), o.probe_series()) <= 1e-5
    else:
        assert rel_l2(g.read_fields(), o.fields_memory_order()) <= 1e-12
        assert rel_l2(g.read_flux(), o.flux_series()) <= 1e-12
        assert rel_l2(g.read_probes(), o.probe_series()) <= 1e-12
