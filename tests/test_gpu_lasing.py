"""Lasing parity: a pumped four-level gain medium (paper, Sec. "3+1D
simulation of lasing": self-starting laser oscillation from spontaneous-
emission noise) in a box with PEC walls and one absorbing face, stepped
through threshold, amplification from the seeded noise and saturation.

Past threshold pointwise agreement is not the bar; the emitted energy
(time-integrated Poynting flux out through the open face) and the peak lasing
frequency (analysis.peak_frequency: Hann-windowed spectrum of the last half
of a probe series, peak refined by a parabola) must agree with the FP64
oracle within 1 %.  The oracle itself moves by ~3e-6 in emitted energy when
its coefficients are rounded to binary32, so the bar is not met by luck.

Each run must also show that it lased: the emitted power of the last half
exceeds that of the first tenth by more than 1e3 (it grows from the noise by
many orders of magnitude), and the mean inversion N2 - N1 of the gain cells
at the end lies well below its pumped start (gain saturation).

Two media: a homogeneous gain-filled box, and a gain-filled fcc opal (the
lasing workload's spheres of eps_host 2.25 in eps 11.9, 2x2x2 unit cells,
sigma 5 %) whose open face is the only exit.
"""
import numpy as np
import pytest

from paper_0802_3775_gb300 import inputs

pytestmark = pytest.mark.gpu

N, NPML, STEPS = 12, 6, 12000


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0802_3775_gb300 import build
    build.build()


def _box_spec(precision):
    shape = (N, N, N + NPML)
    spec = inputs.RunSpec(shape=shape, res=8, npml=(0, 0, 0, 0, 0, NPML), eps=(2.25, 2.25, 2.25),
                          precision=precision, seed=5)
    spec.fluxes = [inputs.FluxSpec(axis=2, index=N, sign=1.0, u=(0, N - 1), v=(0, N - 1))]
    spec.probes = np.array([[N // 3, N // 2 + 1, N // 2 - 1]], dtype=np.int32)
    mat = np.full(shape[::-1], 0b0101010, dtype=np.uint8)
    mat[:N - 1] |= 64   # gain inside the box, not in the absorbing slab
    gain = inputs.GainSpec(n_total=1e24, fa_hat=0.8, dw_rel=0.02, tau32=100e-15, tau21=1e-9, tau10=100e-15,
                           pump=1e12, noise_amp=1e-6, init="steady")
    return spec, mat, gain, STEPS


def _opal_spec(precision):
    """Gain in the spheres of a 2x2x2-unit-cell opal at 8 cells/a filling a
    PEC box, an absorbing slab behind its +z face (26000 steps: the noise
    grows ~10x per 1000 steps and saturates near step 24000)."""
    res, npml = 8, 6
    n = 2 * res
    shape = (n, n, n + npml)
    spec = inputs.RunSpec(shape=shape, res=res, npml=(0, 0, 0, 0, 0, npml), eps=(11.9, 11.9, 2.25),
                          precision=precision, box_lo=(0, 0, 0), box_hi=(n, n, n), seed=7)
    spec.spheres = inputs.fcc_opal_spheres(spec.box_lo, spec.box_hi, res, sigma=0.05, seed=2001)
    spec.gain = inputs.GainSpec(n_total=1e24, fa_hat=0.8, dw_rel=0.02, tau32=100e-15, tau21=1e-9, tau10=100e-15,
                                pump=1e12, noise_amp=1e-6, init="steady")
    spec.fluxes = [inputs.FluxSpec(axis=2, index=n, sign=1.0, u=(0, n - 1), v=(0, n - 1))]
    spec.probes = np.array([[n // 3, n // 2 + 1, n // 2 - 1]], dtype=np.int32)
    return spec, None, None, 26000


def _run(spec, mat, gain, steps):
    """The run on the GPU and in the oracle; `mat` and `gain` given: a
    material map set directly, then the gain medium."""
    from oracle import Oracle
    from paper_0802_3775_gb300.fdtd import Grid
    g = Grid.from_spec(spec, record_capacity=steps)
    o = Oracle.from_spec(spec, coef32=spec.precision == "f32")
    if mat is not None:
        g.set_material(mat)
        g.set_gain(gain)
        o.set_material(mat)
        gs = gain
        o.set_gain(n_total=gs.n_total, fa_hat=gs.fa_hat, dw_rel=gs.dw_rel, tau32=gs.tau32, tau21=gs.tau21,
                   tau10=gs.tau10, pump=gs.pump, noise_amp=gs.noise_amp)
    inv0 = float(o.gain["n_eq"][2] - o.gain["n_eq"][1])
    g.step(steps)
    g.sync()
    o.step(steps)
    return g, o, inv0


def _check(g, o, inv0):
    from paper_0802_3775_gb300 import analysis
    T_gpu, T_ref = g.read_flux(0), o.flux_series()[0]
    emitted_gpu = float(np.sum(T_gpu)) * o.dt
    emitted_ref = float(np.sum(T_ref)) * o.dt
    n = len(T_ref)
    for T in (T_gpu, T_ref):
        # threshold crossed: the output grew from the noise by orders of magnitude
        assert np.mean(T[n // 2:]) > 1e3 * np.mean(np.abs(T[:n // 10]))
    assert abs(emitted_gpu / emitted_ref - 1.0) <= 0.01
    f_gpu = analysis.peak_frequency(g.read_probes(0), o.dt)
    f_ref = analysis.peak_frequency(o.probe_series()[:, 0, :], o.dt)
    assert abs(f_gpu / f_ref - 1.0) <= 0.01
    # the lasing line sits within the gain bandwidth around f_a = 0.80 c / a
    f_a = 0.8 * 299792458.0 / 480e-9
    assert abs(f_ref / f_a - 1.0) < 0.05
    # gain saturation: the stimulated emission pulled the inversion well below its start
    mask = o.gain["mask"].transpose(2, 1, 0)
    Ng = g.read_gain(2)           # N1, N2, N3 of every node, [3, nz, ny, nx]
    inv_gpu = float(np.mean((Ng[1] - Ng[0])[mask]))
    No = o.populations()
    inv_ref = float(np.mean((No[2] - No[1])[o.gain["mask"]]))
    for inv in (inv_gpu, inv_ref):
        assert inv < 0.8 * inv0
    return emitted_ref, f_ref


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_lasing_emitted_energy_and_frequency(precision):
    g, o, inv0 = _run(*_box_spec(precision))
    _check(g, o, inv0)


def test_lasing_in_gain_filled_opal_spheres():
    g, o, inv0 = _run(*_opal_spec("f32"))
    _check(g, o, inv0)
