"""Lasing parity: a pumped four-level gain medium (paper, Sec. "3+1D
simulation of lasing": self-starting laser oscillation from spontaneous-
emission noise) in a box with PEC walls and one absorbing face, stepped
through threshold, amplification from the seeded noise and saturation.

Past threshold pointwise agreement is not the bar; the emitted energy
(time-integrated Poynting flux out through the open face) and the peak lasing
frequency (Hann-windowed spectrum of the last half of a probe series, peak
refined by a parabola) must agree with the FP64 oracle within 1 %.  The
oracle itself moves by ~3e-6 in emitted energy when its coefficients are
rounded to binary32, so the bar is not met by luck."""
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


def _spec(precision):
    shape = (N, N, N + NPML)
    spec = inputs.RunSpec(shape=shape, res=8, npml=(0, 0, 0, 0, 0, NPML), eps=(2.25, 2.25, 2.25),
                          precision=precision, seed=5)
    spec.fluxes = [inputs.FluxSpec(axis=2, index=N, sign=1.0, u=(0, N - 1), v=(0, N - 1))]
    spec.probes = np.array([[N // 3, N // 2 + 1, N // 2 - 1]], dtype=np.int32)
    mat = np.full(shape[::-1], 0b0101010, dtype=np.uint8)
    mat[:N - 1] |= 64   # gain inside the box, not in the absorbing slab
    gain = inputs.GainSpec(n_total=1e24, fa_hat=0.8, dw_rel=0.02, tau32=100e-15, tau21=1e-9, tau10=100e-15,
                           pump=1e12, noise_amp=1e-6, init="steady")
    return spec, mat, gain


def _peak_frequency(series):
    x = series[len(series) // 2:]
    x = x - x.mean(axis=0)
    w = np.hanning(len(x))[:, None]
    S = (np.abs(np.fft.rfft(x * w, axis=0)) ** 2).sum(axis=1)
    i = int(np.argmax(S[1:])) + 1
    a, b, c = np.log(S[i - 1]), np.log(S[i]), np.log(S[i + 1])
    return (i + 0.5 * (a - c) / (a - 2 * b + c)) / len(x)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_lasing_emitted_energy_and_frequency(precision):
    from oracle import Oracle
    from paper_0802_3775_gb300.fdtd import Grid
    spec, mat, gain = _spec(precision)
    g = Grid.from_spec(spec, record_capacity=STEPS)
    g.set_material(mat)
    g.set_gain(gain)
    g.step(STEPS)
    g.sync()
    o = Oracle.from_spec(spec, coef32=precision == "f32")
    o.set_material(mat)
    o.set_gain(n_total=gain.n_total, fa_hat=gain.fa_hat, dw_rel=gain.dw_rel, tau32=gain.tau32, tau21=gain.tau21,
               tau10=gain.tau10, pump=gain.pump, noise_amp=gain.noise_amp)
    o.step(STEPS)
    emitted_gpu = float(np.sum(g.read_flux(0))) * o.dt
    emitted_ref = float(np.sum(o.flux_series()[0])) * o.dt
    # the run crossed threshold: the output grew by many orders of magnitude
    assert emitted_ref > 1e-16
    assert abs(emitted_gpu / emitted_ref - 1.0) <= 0.01
    f_gpu = _peak_frequency(g.read_probes(0))
    f_ref = _peak_frequency(o.probe_series()[:, 0, :])
    assert abs(f_gpu / f_ref - 1.0) <= 0.01
    # the lasing line sits within the gain bandwidth around f_a
    f_a = 0.8 * o.S / 8
    assert abs(f_ref / f_a - 1.0) < 0.05
