"""The seeded workload generators follow their stated recipes (no GPU): the
passive and lasing opals, the 64-realization mixed batch and the served
request stream.  Only shapes, ranges and statistics are checked; the
generators hold none of the method's arithmetic."""
import math

import numpy as np

from paper_0802_3775_gb300 import inputs


def test_planewave_and_lasing_workloads():
    pw = inputs.opal_planewave_f32(ncell=8, res=20, npml=12, sigma=0.06)
    assert pw.shape == (184, 184, 184) and pw.npml == (12,) * 6 and pw.gain is None
    assert pw.eps == (11.9, 11.9, 1.0) and pw.precision == "f32"
    las = inputs.opal_lasing_f32(ncell=6, res=20, npml=10, sigma=0.05)
    assert las.shape == (140, 140, 140) and las.npml == (10,) * 6
    g = las.gain
    assert (g.n_total, g.fa_hat, g.dw_rel, g.tau32, g.tau21, g.tau10, g.noise_amp) == \
        (1e24, 0.80, 0.02, 100e-15, 1e-9, 100e-15, 1e-6)
    assert las.eps[2] == 2.25
    # sphere radius a / (2 sqrt 2) in cells, jittered by sigma: the mean stays at r0
    r0 = 20 / (2 * math.sqrt(2))
    r = np.asarray(las.spheres).reshape(-1, 4)[:, 3]
    assert abs(np.mean(r) / r0 - 1) < 0.02 and 0.02 < np.std(r / r0) < 0.08


def test_mixed_batch_recipe():
    specs = inputs.mixed_batch(64, seed=4000)
    assert len(specs) == 64
    for q, s in enumerate(specs):
        n = s.shape[0]
        assert s.shape == (n, n, n) and s.npml == (12,) * 6
        res = int(s.res)
        assert 16 <= res <= 20
        ncell = (n - 24) / res
        assert ncell == int(ncell) and 4 <= ncell <= 8
        assert (s.gain is not None) == (q % 2 == 1)
        assert s.seed == 4000 + q
    # sizes and resolutions vary across the batch
    assert len({s.shape for s in specs}) > 8 and len({s.res for s in specs}) == 5


def test_request_stream_is_poisson_at_the_stated_rate():
    stream = inputs.request_stream(400, rate_hz=4.0, seed=5000)
    t = np.array([a for a, _ in stream])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(np.mean(gaps) - 0.25) < 0.03                 # mean arrival interval 1 / (4 per s)
    assert abs(np.std(gaps) / np.mean(gaps) - 1.0) < 0.15   # exponential: coefficient of variation 1
    edges = np.array([s.shape[0] for _, s in stream])
    assert edges.min() >= 2 * 16 + 24 and edges.max() <= 200 + 20
    steps = np.array([s.steps for _, s in stream])
    assert steps.min() >= 5000 and steps.max() <= 50000
    lasing = np.mean([s.gain is not None for _, s in stream])
    assert 0.4 < lasing < 0.6


def test_sources_observers_and_seeds_of_the_workloads():
    # passive: x-polarized sheet at z = npml + 2, flux plane at z = nz - npml - 3 over the interior faces
    pw = inputs.opal_planewave_f32(ncell=4, res=10, npml=8, sigma=0.03, realization=5)
    n = pw.shape[0]
    (src,) = pw.sources
    assert (src.kind, src.comp, src.axis, src.index, src.f0_hat, src.rel_bw) == ("sheet", 0, 2, 10, 0.80, 0.10)
    (fl,) = pw.fluxes
    assert (fl.axis, fl.index, fl.sign, fl.u, fl.v) == (2, n - 11, 1.0, (8, n - 9), (8, n - 9))
    assert pw.seed == 1005 and pw.box_lo == (8,) * 3 and pw.box_hi == (n - 8,) * 3
    # probes: 8 cells of the non-absorbing interior, drawn from PCG64(seed + 1)
    assert pw.probes.shape == (8, 3)
    assert np.all(pw.probes >= 8) and np.all(pw.probes < n - 8)
    again = inputs.probe_cells(pw.shape, pw.npml, 8, seed=1006)
    assert np.array_equal(pw.probes, again)
    # lasing: six outward planes two cells inside the CPML, enclosing a closed box
    las = inputs.opal_lasing_f32(ncell=3, res=10, npml=6, realization=2)
    n = las.shape[0]
    lo, hi = 8, n - 8
    got = {(f.axis, f.index, f.sign, f.u, f.v) for f in las.fluxes}
    assert got == {(d, i, s, (lo, hi), (lo, hi)) for d in range(3) for i, s in ((lo, -1.0), (hi, 1.0))}
    assert las.sources == [] and las.seed == 2002 and las.gain.init == "steady"
    # FP64 dipole: Ez point source at the centre cell
    dp = inputs.opal_dipole_f64()
    (src,) = dp.sources
    assert dp.shape == (40, 40, 40) and dp.precision == "f64"
    assert (src.kind, src.comp, src.pos) == ("point", 2, (20, 20, 20))


def test_batch_members_per_rank_are_distinct_realizations():
    a = inputs.mixed_batch(8, seed=4000)
    b = inputs.mixed_batch(8, seed=5000)
    assert [s.seed for s in a] == list(range(4000, 4008))
    # the same member index on two ranks draws another size, resolution and disorder
    diff = [(x.shape, x.res) != (y.shape, y.res) or not np.array_equal(x.spheres, y.spheres) for x, y in zip(a, b)]
    assert all(diff)


def test_111_rotation_stacks_close_packed_layers_along_z():
    # without disorder, the [111] lattice puts the sphere centres on planes
    # normal to z spaced a / sqrt 3, each a triangular net of spacing a / sqrt 2
    res = 10.0
    sph = inputs.fcc_opal_spheres((0, 0, 0), (40, 40, 40), res, rotation="111", sigma=0.0)
    c = sph[:, :3]
    assert np.allclose(sph[:, 3], res / (2 * np.sqrt(2)))
    z = np.unique(np.round(c[:, 2], 9))
    gaps = np.diff(z)
    assert np.allclose(gaps, res / np.sqrt(3), atol=1e-9)
    # nearest neighbours in one layer sit a / sqrt 2 apart, six around an inner site
    mid = c[np.isclose(c[:, 2], z[len(z) // 2])]
    inner = mid[np.argmin(np.sum((mid[:, :2] - 20.0) ** 2, axis=1))]
    d = np.sqrt(np.sum((mid[:, :2] - inner[:2]) ** 2, axis=1))
    d = np.sort(d[d > 1e-9])
    assert np.allclose(d[:6], res / np.sqrt(2), atol=1e-9) and d[6] > res / np.sqrt(2) + 1.0
    # the identity lattice instead stacks (001) planes a / 2 apart
    sph0 = inputs.fcc_opal_spheres((0, 0, 0), (40, 40, 40), res, sigma=0.0)
    assert np.allclose(np.diff(np.unique(np.round(sph0[:, 2], 9))), res / 2)


def test_paper_disorder_moves_radii_only_uniformly():
    res, gamma = 10.0, 0.2
    ordered = inputs.fcc_opal_spheres((0, 0, 0), (60, 60, 60), res, sigma=0.0)
    paper = inputs.fcc_opal_spheres((0, 0, 0), (60, 60, 60), res, disorder="paper", gamma=gamma, seed=3)
    assert np.array_equal(paper[:, :3], ordered[:, :3])        # centres stay on the lattice
    r0 = res / (2 * np.sqrt(2))
    xi = paper[:, 3] / r0 - 1.0
    assert np.all(np.abs(xi) <= gamma / 2)
    # uniform on [-gamma/2, gamma/2]: mean 0, variance gamma^2 / 12
    assert abs(np.mean(xi)) < 0.01 and abs(np.var(xi) / (gamma ** 2 / 12) - 1) < 0.1
