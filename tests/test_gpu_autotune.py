"""Launch-shape autotuner: tuning from a mid-run state times every candidate,
restores the state, and the run continues exactly as an untuned one."""
import numpy as np
import pytest

from helpers import small_opal
from paper_0802_3775_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0802_3775_gb300 import build
    build.build()


def _state(g):
    return [g.read_fields(), g.read_probes(), g.read_flux()]


@pytest.mark.parametrize("precision,with_gain", [("f32", False), ("f32", True), ("f64", False)])
def test_grid_autotune_keeps_the_run_exact(precision, with_gain):
    from paper_0802_3775_gb300.fdtd import Grid
    gain = inputs.GainSpec(pump=5e11, noise_amp=1e-3, init="ground") if with_gain else None
    spec = small_opal(n_cells=2, res=9, npml=5, precision=precision, source="sheet", gain=gain, sigma=0.05)
    ref = Grid.from_spec(spec)
    ref.step(90)
    want = _state(ref)
    g = Grid.from_spec(spec)
    g.step(40)
    choice = g.autotune(trial_steps=6)
    assert choice["candidates"] >= 3 and choice["ms_per_step"] > 0
    assert g.steps_done == 40
    g.step(50)
    for a, b in zip(_state(g), want):
        assert np.array_equal(a, b)
    if with_gain:
        assert np.array_equal(g.read_gain(3), ref.read_gain(3))


def test_batch_autotune_keeps_members_exact():
    from paper_0802_3775_gb300.fdtd import Batch, Grid
    gain = inputs.GainSpec(pump=5e11, noise_amp=1e-3, init="ground")
    specs = [small_opal(n_cells=2, res=8, npml=5, precision="f32", source="sheet", seed=1),
             small_opal(n_cells=2, res=10, npml=6, precision="f32", source="dipole", gain=gain, seed=2),
             inputs.opal_planewave_f32(ncell=2, res=9, npml=5, sigma=0.04, realization=7)]
    alone = []
    for s in specs:
        g = Grid.from_spec(s)
        g.step(45)
        alone.append(_state(g))
    grids = [Grid.from_spec(s) for s in specs]
    b = Batch(grids)
    b.step(20)
    choice = b.autotune(trial_steps=4)
    assert choice["candidates"] >= 5
    b.step(25)
    b.sync()
    for g, ref in zip(grids, alone):
        assert g.steps_done == 45
        for x, y in zip(_state(g), ref):
            assert np.array_equal(x, y)
    b.close()
