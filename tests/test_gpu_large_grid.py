"""A grid of the paper's largest size (400^3, its convergence checks; Sec.
"Sample and numerical approach") stepped on the GPU and checked, cell by
cell, in windows the oracle can compute on its own.

Every field of step n+1 depends on fields of step n at most one cell away,
so after s steps a window's interior depends only on the initial fields
within s cells of it.  The 400^3 binary32 opal (24^3 unit cells at 16
cells/a, 8-cell CPML, seeded random initial fields in every cell) takes 3
steps on the GPU; for each of four windows (the low corner with its three
absorbing slabs, the centre, two seeded interior positions) the oracle steps
the window plus a 4-cell margin from the same initial fields, its material
rasterized by the oracle from the same sphere list, its absorbing layer the
corner's own, and the window interiors must agree to the binary32 bar.  At
this size the field arrays span 4.6 GB (three sets), so every 64-bit offset
of the step and observation kernels is exercised."""
import numpy as np
import pytest

from helpers import rel_l2
from paper_0802_3775_gb300 import inputs

pytestmark = pytest.mark.gpu

STEPS, MARGIN, W = 3, 4, 20


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0802_3775_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def big():
    spec = inputs.opal_planewave_f32(ncell=24, res=16, npml=8, sigma=0.06, realization=3, steps=STEPS)
    assert spec.shape == (400, 400, 400)
    spec.sources, spec.fluxes, spec.probes = [], [], None
    F0 = inputs.random_fields(spec.shape, seed=400, scale=1.0, dtype=np.float32)
    return spec, F0


def _oracle_window(spec, F0, lo):
    """The oracle on the window [lo - MARGIN, lo + W + MARGIN) (clipped at the
    grid's low faces, where the window keeps the grid's absorbing slabs)."""
    from oracle import Oracle
    from oracle.rasterize import rasterize
    start = [max(0, l - MARGIN) for l in lo]
    stop = [l + W + MARGIN for l in lo]
    shape = tuple(b - a for a, b in zip(start, stop))
    npml = tuple(v for d in range(3) for v in ((spec.npml[2 * d] if start[d] == 0 else 0), 0))
    o = Oracle(shape, spec.res, a=spec.a, courant=spec.courant, npml=npml, eps=spec.eps, coef32=True)
    # the material of the window, rasterized in the grid's own coordinates
    # (the spheres that reach the window, over the block [0, stop))
    sph = spec.spheres
    near = np.all((sph[:, :3] + sph[:, 3:4] >= np.asarray(start) - 1) & (sph[:, :3] - sph[:, 3:4] <= np.asarray(stop) + 1),
                  axis=1)
    mat = rasterize(tuple(stop), sph[near], spec.box_lo, spec.box_hi)
    o.set_material(mat[start[2]:, start[1]:, start[0]:])
    sl = np.s_[:, start[2]:stop[2], start[1]:stop[1], start[0]:stop[0]]
    o.set_fields_memory_order(F0[sl].astype(np.float64))
    o.step(STEPS)
    inner = np.s_[:, lo[2] - start[2]:lo[2] - start[2] + W, lo[1] - start[1]:lo[1] - start[1] + W,
                  lo[0] - start[0]:lo[0] - start[0] + W]
    return o.fields_memory_order()[inner]


@pytest.mark.parametrize("kernel", ["auto", "tma"])
def test_400_cubed_windows_match_the_oracle(big, kernel):
    from paper_0802_3775_gb300.fdtd import Grid
    spec, F0 = big
    g = Grid.from_spec(spec, record_capacity=16)
    if kernel != "auto":
        g.set_kernel(kernel)
    g.write_fields(F0)
    g.step(STEPS)
    g.sync()
    F = g.read_fields()
    g.close()
    rng = np.random.Generator(np.random.PCG64(401))
    windows = [(0, 0, 0), (190, 190, 190)] + [tuple(int(v) for v in rng.integers(MARGIN, 400 - W - MARGIN, 3))
                                             for _ in range(2)]
    for lo in windows:
        ref = _oracle_window(spec, F0, lo)
        got = F[:, lo[2]:lo[2] + W, lo[1]:lo[1] + W, lo[0]:lo[0] + W]
        assert rel_l2(got, ref) <= 1e-6, lo
