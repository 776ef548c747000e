"""GPU parity of the centred Bloch coupling (polarization and populations at
the cell centre; paper, Sec. "Sample and numerical approach": the Bloch
variables are solved in the middle of the Yee cell) against the FP64 oracle
on the same seeded inputs, through the C ABI.

Bars: FP64 fields and polarization <= 1e-12 relative L2, population
deviations <= 1e-9; FP32 (oracle fed the binary32-rounded coefficients)
fields <= 1e-5, population deviations <= 1e-6; on every step kernel that
steps the fields (the centred kernels follow each of them).  Lasing with the
centred coupling: emitted energy and lasing frequency within 1 % of the
oracle.  A batch refuses a centred member."""
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


def _spec(precision, init="ground"):
    gain = inputs.GainSpec(n_total=1e24, fa_hat=0.8, dw_rel=0.02, tau32=100e-15, tau21=1e-9, tau10=100e-15,
                           pump=5e11, noise_amp=1e-3, init=init, coupling="centred")
    return small_opal(n_cells=2, res=8, npml=5, precision=precision, source="dipole", gain=gain)


@pytest.mark.parametrize("kernel", ["tma", "plain"])
def test_fp64_centred_coupling_matches_oracle(kernel):
    spec = _spec("f64")
    g = gpu_grid(spec)
    g.set_kernel(kernel)
    o = oracle_grid(spec)
    assert o.gain["centred"]
    g.step(300)
    o.step(300)
    assert rel_l2(g.read_fields(), o.fields_memory_order()) <= 1e-12
    assert rel_l2(g.read_gain(0), o.P.transpose(0, 3, 2, 1)) <= 1e-12
    assert rel_l2(g.read_gain(3), o.dN[1:].transpose(0, 3, 2, 1)) <= 1e-9
    assert rel_l2(g.read_flux(), o.flux_series()) <= 1e-12
    # the polarization took part
    assert np.max(np.abs(o.P)) > 1e-6 * np.max(np.abs(o.E))


@pytest.mark.parametrize("kernel", ["auto", "tma", "plain"])
def test_fp32_centred_coupling_matches_oracle(kernel):
    spec = _spec("f32")
    g = gpu_grid(spec)
    if kernel != "auto":
        g.set_kernel(kernel)
    o = oracle_grid(spec, coef32=True)
    g.step(300)
    o.step(300)
    if kernel == "auto":
        assert g.kernel_in_use()[0] == 3  # the fields step on the paired kernel
    assert rel_l2(g.read_fields(), o.fields_memory_order()) <= 1e-5
    assert rel_l2(g.read_gain(3), o.dN[1:].transpose(0, 3, 2, 1)) <= 1e-6
    assert rel_l2(g.read_flux(0), o.flux_series()[0]) <= 1e-4


def test_centred_differs_from_cell_coupling():
    spec = _spec("f64")
    a = gpu_grid(spec)
    a.step(200)
    spec.gain.coupling = "cell"
    b = gpu_grid(spec)
    b.step(200)
    assert rel_l2(a.read_fields(), b.read_fields()) > 1e-9


def test_centred_lasing_emitted_energy_and_frequency():
    from oracle import Oracle
    from paper_0802_3775_gb300 import analysis
    from paper_0802_3775_gb300.fdtd import Grid
    N, NPML, STEPS = 12, 6, 12000
    shape = (N, N, N + NPML)
    spec = inputs.RunSpec(shape=shape, res=8, npml=(0, 0, 0, 0, 0, NPML), eps=(2.25, 2.25, 2.25), precision="f32",
                          seed=5)
    spec.fluxes = [inputs.FluxSpec(axis=2, index=N, sign=1.0, u=(0, N - 1), v=(0, N - 1))]
    spec.probes = np.array([[N // 3, N // 2 + 1, N // 2 - 1]], dtype=np.int32)
    mat = np.full(shape[::-1], 0b0101010, dtype=np.uint8)
    mat[:N - 1] |= 64
    gain = inputs.GainSpec(n_total=1e24, fa_hat=0.8, dw_rel=0.02, tau32=100e-15, tau21=1e-9, tau10=100e-15,
                           pump=1e12, noise_amp=1e-6, init="steady", coupling="centred")
    g = Grid.from_spec(spec, record_capacity=STEPS)
    g.set_material(mat)
    g.set_gain(gain)
    o = Oracle.from_spec(spec, coef32=True)
    o.set_material(mat)
    o.set_gain(n_total=gain.n_total, fa_hat=gain.fa_hat, dw_rel=gain.dw_rel, tau32=gain.tau32, tau21=gain.tau21,
               tau10=gain.tau10, pump=gain.pump, noise_amp=gain.noise_amp, coupling="centred")
    g.step(STEPS)
    g.sync()
    o.step(STEPS)
    T_gpu, T_ref = g.read_flux(0), o.flux_series()[0]
    n = len(T_ref)
    assert np.mean(T_ref[n // 2:]) > 1e3 * np.mean(np.abs(T_ref[:n // 10]))
    assert abs(float(np.sum(T_gpu)) / float(np.sum(T_ref)) - 1.0) <= 0.01
    f_gpu = analysis.peak_frequency(g.read_probes(0), o.dt)
    f_ref = analysis.peak_frequency(o.probe_series()[:, 0, :], o.dt)
    assert abs(f_gpu / f_ref - 1.0) <= 0.01


def test_a_batch_refuses_a_centred_member():
    from paper_0802_3775_gb300.fdtd import Batch, FdtdError
    a = gpu_grid(_spec("f32"))
    b = gpu_grid(small_opal(n_cells=2, res=8, npml=5, precision="f32"))
    with pytest.raises(FdtdError) as e:
        Batch([a, b])
    assert e.value.code == -1


def test_centred_checkpoint_and_autotune_are_bitwise():
    """The centred coupling's gain state travels with a checkpoint and
    survives the autotuner's trials bit for bit."""
    import os
    import tempfile
    spec = _spec("f32")
    a = gpu_grid(spec)
    a.step(200)
    ref = a.read_fields(), a.read_gain(3)
    b = gpu_grid(spec)
    b.step(120)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        b.save_state(path)
        c = gpu_grid(spec)
        c.load_state(path)
    c.step(80)
    assert np.array_equal(c.read_fields(), ref[0]) and np.array_equal(c.read_gain(3), ref[1])
    t = gpu_grid(spec)
    t.step(120)
    t.autotune(trial_steps=3)
    t.step(80)
    assert np.array_equal(t.read_fields(), ref[0]) and np.array_equal(t.read_gain(3), ref[1])
