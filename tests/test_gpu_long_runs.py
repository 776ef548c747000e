"""Binary32 parity at the passive workload's run length, and the paper's
post-processing applied to device output.

The reduced passive workload (the [111] disordered opal recipe at 2x2x2 unit
cells, 20 cells/a, 12-cell CPML: a 64^3 grid) is stepped 20000 steps on the
GPU -- as long as the passive workload runs -- and compared with the FP64
oracle's results for the same seeded inputs, stored by
tests/golden/make_long_runs.py (it calls only the oracle):

* against the oracle fed the binary32-rounded coefficient tables (the
  discrete problem an FP32 run solves): fields <= 1e-5, probe series <= 1e-5,
  flux series <= 1e-4 relative L2, the storage round-off random walk of
  20000 steps included;
* against the exact-coefficient oracle the error is reported (the rounding of
  the coefficients to binary32 changes the discrete problem itself).

Post-processing (paper, Sec. "Diffusion constant and decay times"): the
tail time constant tau0 of the transmitted power, D = L^2/(pi^2 tau0) and the
decay-time distribution g(tau) computed by the product's analysis functions
from the device's flux series agree with the same functions applied to the
oracle's series: tau0 and D within 1 %, g(tau) within 1 % relative L2.
"""
import importlib.util
import os

import numpy as np
import pytest

from helpers import rel_l2

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden_module():
    spec = importlib.util.spec_from_file_location("make_long_runs", os.path.join(HERE, "golden", "make_long_runs.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module")
def golden():
    mod = _golden_module()
    path = os.path.join(HERE, "golden", "long_opal64_f32.npz")
    return mod, dict(np.load(path))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0802_3775_gb300 import build
    build.build()


_runs = {}


def _gpu_run(mod, kernel):
    """The reduced passive workload stepped 20000 steps on one step kernel
    (cached per kernel for the module)."""
    if kernel not in _runs:
        from paper_0802_3775_gb300.fdtd import Grid
        spec = mod.opal64_spec()
        g = Grid.from_spec(spec, record_capacity=spec.steps + 16)
        if kernel != "auto":
            g.set_kernel(kernel)
        g.step(spec.steps)
        g.sync()
        F = g.read_fields()
        _runs[kernel] = dict(spec=spec, fields=F, flux=g.read_flux(0), probes=g.read_probes(),
                             energy=g.field_energy(), kind=g.kernel_in_use())
        g.close()
    return _runs[kernel]


@pytest.mark.parametrize("kernel", ["auto", "tma", "plain"])
def test_fp32_opal64_20000_steps_against_the_oracle(golden, kernel):
    mod, ref = golden
    r = _gpu_run(mod, kernel)
    spec = r["spec"]
    if kernel == "auto":
        assert r["kind"][0] == 3  # a passive binary32 grid runs on the paired kernel
    planes, cells = mod.sample_fields(r["fields"], spec.shape)
    err_planes = rel_l2(planes, ref["planes_coef32"])
    err_cells = rel_l2(cells, ref["cells_coef32"])
    err_flux = rel_l2(r["flux"], ref["flux_coef32"])
    err_probes = rel_l2(r["probes"][mod.PROBE_EVERY - 1::mod.PROBE_EVERY], ref["probes_coef32"])
    err_energy = abs(r["energy"] / float(ref["energy_coef32"][0]) - 1.0)
    exact = (rel_l2(planes, ref["planes_exact"]), rel_l2(cells, ref["cells_exact"]),
             rel_l2(r["flux"], ref["flux_exact"]))
    print(f"\n{kernel}: 20000 steps, vs coef32 oracle: planes {err_planes:.2e} cells {err_cells:.2e} "
          f"flux {err_flux:.2e} probes {err_probes:.2e} energy {err_energy:.2e}; vs exact-coefficient oracle: "
          f"planes {exact[0]:.2e} cells {exact[1]:.2e} flux {exact[2]:.2e}")
    # the comparison is of a live field: after 20000 steps the opal still
    # holds ~1e-6 of the 1 V/m pulse, far above binary32's round-off floor
    assert np.max(np.abs(ref["cells_coef32"])) > 1e-7
    assert err_planes <= 1e-5 and err_cells <= 1e-5
    assert err_probes <= 1e-5
    assert err_flux <= 1e-4
    assert err_energy <= 1e-5
    # the exact-coefficient problem differs from the rounded one by far less
    # than the field itself
    assert max(exact) < 1e-2


def test_decay_analysis_on_device_flux(golden):
    """tau0, D and g(tau) of the transmitted power, from the device's series
    and from the oracle's, through the same analysis functions."""
    from paper_0802_3775_gb300 import analysis
    mod, ref = golden
    r = _gpu_run(mod, "auto")
    spec = r["spec"]
    dt = 0.5 / np.sqrt(3.0) * (spec.a / spec.res) / 299792458.0
    T_gpu, T_ref = r["flux"], ref["flux_coef32"]
    win = analysis.trailing_edge(T_ref)
    assert analysis.trailing_edge(T_gpu) == win
    tau_gpu = analysis.tail_time_constant(T_gpu, dt)
    tau_ref = analysis.tail_time_constant(T_ref, dt)
    assert abs(tau_gpu / tau_ref - 1.0) <= 0.01
    L = (spec.box_hi[2] - spec.box_lo[2]) * spec.a / spec.res
    D_gpu, D_ref = analysis.diffusion_constant(tau_gpu, L), analysis.diffusion_constant(tau_ref, L)
    assert abs(D_gpu / D_ref - 1.0) <= 0.01
    taus = tau_ref * np.logspace(-1, 1, 24)
    g_gpu = analysis.decay_time_distribution(T_gpu, dt, taus, window=win, alpha=1e-3)
    g_ref = analysis.decay_time_distribution(T_ref, dt, taus, window=win, alpha=1e-3)
    assert np.sum(g_ref) > 0
    assert rel_l2(g_gpu, g_ref) <= 0.01
