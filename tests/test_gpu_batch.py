"""Batched stepping (many grids of mixed size in one launch per step) against
the same grids stepped alone, and CUDA-graph replay against direct launches."""
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


def _members():
    gain = inputs.GainSpec(pump=5e11, noise_amp=1e-3, init="ground")
    return [small_opal(n_cells=2, res=8, npml=5, precision="f32", source="sheet", seed=1),
            small_opal(n_cells=2, res=10, npml=6, precision="f32", source="dipole", gain=gain, seed=2),
            small_opal(n_cells=3, res=7, npml=4, precision="f32", source="sheet", gain=gain, seed=3),
            inputs.opal_planewave_f32(ncell=2, res=9, npml=5, sigma=0.04, realization=7)]


def _state(g):
    out = [g.read_fields(), g.read_probes(), g.read_flux()]
    return out


@pytest.mark.parametrize("kernel,graph", [("tma", 0), ("tma", 7), ("plain", 0), ("plain", 5), ("pair", 0), ("pair", 7),
                                          ("auto", 0), ("auto", 7)])
def test_batch_equals_members_alone(kernel, graph):
    """kernel "auto": every member on its own automatic kernel (passive
    binary32 members paired, gain members TMA), one launch per kernel."""
    from paper_0802_3775_gb300.fdtd import Batch, Grid
    specs = _members()
    alone = []
    for s in specs:
        g = Grid.from_spec(s)
        g.set_kernel(kernel)
        g.step(60)
        alone.append(_state(g))
        g.close()
    grids = [Grid.from_spec(s) for s in specs]
    b = Batch(grids)
    b.set_launch(kernel, {"pair": 16, "auto": 0}.get(kernel, 8), 0, 0)
    b.set_graph(graph)
    b.step(23)
    b.step(37)
    b.sync()
    for g, ref in zip(grids, alone):
        got = _state(g)
        for x, y in zip(got, ref):
            assert np.array_equal(x, y)
    b.close()


@pytest.mark.parametrize("kernel,by", [("tma", 4), ("pair", 16)])
def test_batch_step_limits_and_persistent_launch(kernel, by):
    from paper_0802_3775_gb300.fdtd import Batch, Grid
    specs = _members()
    grids = [Grid.from_spec(s) for s in specs]
    grids[1].set_step_limit(25)
    b = Batch(grids)
    b.set_launch(kernel, by, 9, 40)   # persistent: 40 blocks looping over the items
    b.step(50)
    b.sync()
    assert grids[1].steps_done == 25
    assert grids[0].steps_done == 50
    ref = Grid.from_spec(specs[1])
    ref.step(25)
    assert np.array_equal(grids[1].read_fields(), ref.read_fields())
    ref0 = Grid.from_spec(specs[0])
    ref0.step(50)
    assert np.array_equal(grids[0].read_fields(), ref0.read_fields())
    b.close()
