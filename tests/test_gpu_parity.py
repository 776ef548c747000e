"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Bars (FP32 against the oracle fed the same binary32-rounded coefficients):
  FP64 fields: relative L2 <= 1e-12 over all six components;
  FP32 passive fields: relative L2 <= 1e-5, flux series relative L2 <= 1e-4;
  rasterization: bit for bit.
"""
import math

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


def _fields_gpu_vs_oracle(g, o):
    return rel_l2(g.read_fields(), o.fields_memory_order())


@pytest.mark.parametrize("seed", [0, 1])
def test_rasterizer_bit_exact(seed):
    from oracle.rasterize import rasterize
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (37, 29, 33)
    sph = np.column_stack([rng.uniform(-3, 40, 60), rng.uniform(-3, 32, 60), rng.uniform(-3, 36, 60),
                           rng.uniform(0.5, 6.0, 60)])
    # spheres whose surfaces pass through sample points exactly
    sph = np.vstack([sph, [[10.0, 10.0, 10.0, 2.5], [20.5, 15.0, 12.0, 3.0], [5.0, 5.5, 7.0, 0.5]]])
    lo, hi = (2, 3.5, 1), (35, 27, 31.5)
    from paper_0802_3775_gb300.fdtd import Grid
    g = Grid(shape, 12, precision="f32", eps=(1, 11.9, 1))
    g.set_eps_from_spheres(sph, lo, hi)
    assert np.array_equal(g.get_material(), rasterize(shape, sph, lo, hi))


def test_rasterizer_opal_bit_exact():
    from oracle.rasterize import rasterize
    spec = inputs.opal_planewave_f32(ncell=3, res=14, npml=6, sigma=0.06, realization=2)
    from paper_0802_3775_gb300.fdtd import Grid
    g = Grid(spec.shape, spec.res, precision="f32", eps=spec.eps)
    g.set_eps_from_spheres(spec.spheres, spec.box_lo, spec.box_hi)
    assert np.array_equal(g.get_material(), rasterize(spec.shape, spec.spheres, spec.box_lo, spec.box_hi))


def test_fp64_opal_dipole_40cubed_2000_steps():
    """The 40^3 FP64 dipole workload in full: fields and probes after 2000 steps."""
    spec = inputs.opal_dipole_f64(steps=2000)
    g = gpu_grid(spec)
    o = oracle_grid(spec)
    g.step(spec.steps)
    g.sync()
    o.step(spec.steps)
    err = _fields_gpu_vs_oracle(g, o)
    assert err <= 1e-12, err
    assert rel_l2(g.read_probes(), o.probe_series()) <= 1e-12


@pytest.mark.parametrize("source", ["dipole", "sheet"])
def test_fp64_small_opal_all_observers(source):
    spec = small_opal(precision="f64", source=source)
    g = gpu_grid(spec)
    o = oracle_grid(spec)
    g.step(400)
    o.step(400)
    assert _fields_gpu_vs_oracle(g, o) <= 1e-12
    assert rel_l2(g.read_probes(), o.probe_series()) <= 1e-12
    assert rel_l2(g.read_flux(), o.flux_series()) <= 1e-12
    assert abs(g.field_energy() - o.energy()) <= 1e-12 * o.energy()


LAUNCHES = [("tma", (32, 8, 0, 0)), ("tma", (32, 4, 7, 0)), ("tma", (32, 2, 3, 5)), ("plain", (32, 8, 0, 0)),
            ("plain", (64, 4, 7, 0)), ("plain", (32, 16, 3, 5)), ("plain", (16, 2, 0, 0)),
            ("pair", (32, 16, 0, 0)), ("pair", (32, 8, 5, 0)), ("pair", (32, 16, 3, 7))]


@pytest.mark.parametrize("kernel,launch", LAUNCHES)
def test_fp32_passive_fields_and_flux(kernel, launch):
    spec = small_opal(precision="f32", source="sheet", sigma=0.08)
    g = gpu_grid(spec)
    g.set_kernel(kernel)
    g.set_launch(*launch)
    o = oracle_grid(spec, coef32=True)
    g.step(1200)
    o.step(1200)
    assert _fields_gpu_vs_oracle(g, o) <= 1e-5
    assert rel_l2(g.read_flux(0), o.flux_series()[0]) <= 1e-4
    assert rel_l2(g.read_probes(), o.probe_series()) <= 1e-5


@pytest.mark.parametrize("kernel", ["tma", "plain"])
def test_fp64_both_kernels_match_oracle(kernel):
    gain = inputs.GainSpec(pump=5e11, noise_amp=1e-3, init="ground")
    spec = small_opal(n_cells=2, res=8, npml=5, precision="f64", source="sheet", gain=gain)
    g = gpu_grid(spec)
    g.set_kernel(kernel)
    o = oracle_grid(spec)
    g.step(250)
    o.step(250)
    assert _fields_gpu_vs_oracle(g, o) <= 1e-12
    assert rel_l2(g.read_gain(3), o.dN[1:].transpose(0, 3, 2, 1)) <= 1e-9
    assert rel_l2(g.read_flux(), o.flux_series()) <= 1e-12


def test_results_do_not_depend_on_launch_shape():
    gain = inputs.GainSpec(pump=5e11, noise_amp=1e-3, init="ground")
    spec = small_opal(precision="f32", source="dipole", gain=gain)
    out = {}
    for kernel, launch in LAUNCHES:
        g = gpu_grid(spec)
        g.set_kernel(kernel)
        g.set_launch(*launch)
        g.step(150)
        out.setdefault(kernel, []).append((g.read_fields(), g.read_probes(), g.read_gain(3), g.read_flux()))
    for kernel, runs in out.items():
        for F, P, N, T in runs[1:]:
            assert np.array_equal(F, runs[0][0])
            assert np.array_equal(P, runs[0][1])
            assert np.array_equal(N, runs[0][2])
            assert np.array_equal(T, runs[0][3])
    # the kernels share the per-node arithmetic; the paired kernel performs
    # the TMA kernel's operations lane by lane
    assert rel_l2(out["tma"][0][0], out["plain"][0][0]) <= 1e-6
    for a, b in zip(out["pair"][0], out["tma"][0]):
        assert np.array_equal(a, b)


def _ragged_spec(gain):
    """Odd grid sizes and odd absorbing-slab thicknesses: node pairs that
    straddle a slab edge, a last pair with one node off the grid, partial
    tiles in x and y."""
    spec = small_opal(n_cells=2, res=9, npml=5, precision="f32", source="sheet", gain=gain, sigma=0.07, seed=11)
    spec.npml = (5, 6, 7, 5, 5, 6)
    spec.sources.append(inputs.SourceSpec(kind="point", comp=1, pos=(9, 7, 11), f0_hat=0.75, rel_bw=0.3))
    return spec


@pytest.mark.parametrize("with_gain", [False, True])
def test_paired_kernel_is_bitwise_equal_to_tma_kernel(with_gain):
    gain = inputs.GainSpec(pump=5e11, noise_amp=1e-3, init="ground") if with_gain else None
    spec = _ragged_spec(gain)
    runs = []
    for kernel, launch in [("tma", (32, 8, 0, 0)), ("pair", (32, 16, 0, 0)), ("pair", (32, 8, 4, 3))]:
        g = gpu_grid(spec)
        g.set_kernel(kernel)
        g.set_launch(*launch)
        g.step(160)
        r = [g.read_fields(), g.read_probes(), g.read_flux(), np.array([g.field_energy()])]
        if with_gain:
            r += [g.read_gain(0), g.read_gain(1), g.read_gain(3)]
        runs.append(r)
    for other in runs[1:]:
        for a, b in zip(other, runs[0]):
            assert np.array_equal(a, b)


def test_observation_beside_the_step_equals_observation_in_line():
    """A grid frozen on the paired kernel cycles three field sets and runs the
    observation of step n on a second stream while step n+1 runs; stepped in
    uneven chunks (1, 2, 3, ... steps per call, chunk ends join the streams)
    its probes, flux series, fields and energy equal those of the same grid on
    the TMA kernel with the observation in line."""
    spec = _ragged_spec(None)
    ref = gpu_grid(spec)
    ref.set_kernel("tma")
    ref.step(120)
    g = gpu_grid(spec)
    g.set_kernel("pair")
    done = 0
    for n in [1, 2, 3, 1, 7, 40]:
        g.step(n)
        done += n
    g.step(120 - done)
    for a, b in zip([g.read_fields(), g.read_probes(), g.read_flux(), np.array([g.field_energy()])],
                    [ref.read_fields(), ref.read_probes(), ref.read_flux(), np.array([ref.field_energy()])]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("with_gain", [False, True])
def test_tma_steps_overlapping_the_observation_equal_single_step_calls(with_gain):
    """On the TMA kernel the blocks of step s+1 start while the in-line
    observation of step s still runs (three field sets); the first step of
    each call waits for everything before it.  200 steps in one call and 200
    calls of one step give the same probes, flux series, fields, energy and
    gain state, bit for bit."""
    gain = inputs.GainSpec(pump=5e11, noise_amp=1e-3, init="ground") if with_gain else None
    spec = _ragged_spec(gain)
    runs = []
    for calls in [[200], [1] * 200]:
        g = gpu_grid(spec)
        g.set_kernel("tma")
        for n in calls:
            g.step(n)
        r = [g.read_probes(), g.read_flux(), g.read_fields(), np.array([g.field_energy()])]
        if with_gain:
            r += [g.read_gain(0), g.read_gain(3)]
        runs.append(r)
    for a, b in zip(runs[0], runs[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("kernel", ["pair", "tma", "plain"])
def test_l2_residency_changes_no_result(kernel):
    """The persisting L2 window of the CPML memory is a cache placement: with
    it (the default), without it, and switched off after 60 steps, the grid
    gives the same fields, probes, flux and energy, bit for bit."""
    gain = inputs.GainSpec(pump=5e11, noise_amp=1e-3, init="ground") if kernel == "tma" else None
    spec = _ragged_spec(gain)
    runs = []
    for mode in ["on", "off", "switch"]:
        g = gpu_grid(spec)
        g.set_kernel(kernel)
        if mode == "off":
            g.set_l2_residency(False)
        g.step(60)
        if mode == "switch":
            g.set_l2_residency(False)
        g.step(60)
        runs.append([g.read_fields(), g.read_probes(), g.read_flux(), np.array([g.field_energy()])])
        g.close()
    for other in runs[1:]:
        for a, b in zip(other, runs[0]):
            assert np.array_equal(a, b)


def test_l2_window_passes_between_grids_and_batches():
    """Two grids stepped in turn take the persisting L2 window from each
    other, a batch step releases it, and a destroyed holder gives it back:
    each grid's results equal those of the same grid stepped with the window
    off, bit for bit."""
    from paper_0802_3775_gb300.fdtd import Batch
    spec_a = _ragged_spec(None)
    spec_b = small_opal(precision="f32", source="dipole", seed=5)
    ref = {}
    for name, spec in (("a", spec_a), ("b", spec_b)):
        g = gpu_grid(spec)
        g.set_l2_residency(False)
        g.step(90)
        ref[name] = [g.read_fields(), g.read_probes(), g.read_flux()]
        g.close()
    a, b, c = gpu_grid(spec_a), gpu_grid(spec_b), gpu_grid(spec_b)
    batch = Batch([c])
    for n in [30, 30]:
        a.step(n)
        b.step(n)
        batch.step(5)
    a.step(30)
    a.close()  # the holder goes away
    b.step(30)
    assert all(np.array_equal(x, y) for x, y in zip([b.read_fields(), b.read_probes(), b.read_flux()], ref["b"]))
    a2 = gpu_grid(spec_a)
    a2.step(90)
    assert all(np.array_equal(x, y) for x, y in zip([a2.read_fields(), a2.read_probes(), a2.read_flux()], ref["a"]))


def test_paired_kernel_matches_oracle_on_ragged_grid():
    gain = inputs.GainSpec(pump=5e11, noise_amp=1e-3, init="ground")
    spec = _ragged_spec(gain)
    g = gpu_grid(spec)
    g.set_kernel("pair")
    o = oracle_grid(spec, coef32=True)
    g.step(250)
    o.step(250)
    assert _fields_gpu_vs_oracle(g, o) <= 1e-5
    assert rel_l2(g.read_flux(0), o.flux_series()[0]) <= 1e-4
    assert rel_l2(g.read_gain(3), o.dN[1:].transpose(0, 3, 2, 1)) <= 1e-6
    assert abs(g.field_energy() / o.energy() - 1.0) <= 1e-5


def test_energy_after_a_grid_of_another_kernel_reused_the_memory():
    """Grids created one after another reuse the same device blocks; the field
    energy (summed over the padded layout) must not see what an earlier grid
    or kernel left in the row padding."""
    gain = inputs.GainSpec(pump=5e11, noise_amp=1e-3, init="ground")
    spec = small_opal(n_cells=2, res=10, npml=6, precision="f32", source="dipole", gain=gain, seed=2)
    out = []
    for kernel in ["pair", "tma", "pair", "plain", "pair"]:
        g = gpu_grid(spec)
        g.set_kernel(kernel)
        g.step(7)
        out.append((kernel, g.read_fields(), g.field_energy()))
        g.close()
    ref = out[0]
    for kernel, F, e in out[1:]:
        if kernel == "plain":   # the plain-load kernel is compared within 1e-6 elsewhere
            assert rel_l2(F, ref[1]) <= 1e-6
            continue
        assert np.array_equal(F, ref[1])
        assert e == ref[2]


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_periodic_plane_wave_on_gpu(precision):
    """Discrete plane-wave eigenmode of a periodic box (Yee dispersion closed form)."""
    shape = (16, 12, 20)
    spec = inputs.RunSpec(shape=shape, res=12, periodic=(True, True, True), eps=(2.0, 2.0, 2.0), precision=precision)
    from paper_0802_3775_gb300.fdtd import Grid
    g = Grid.from_spec(spec)
    g.set_material(np.full(shape[::-1], 0b010101, dtype=np.uint8))
    S = 0.5 / math.sqrt(3)
    m = (1, -2, 3)
    k = np.array([2 * math.pi * m[d] / shape[d] for d in range(3)])
    K = 2 * np.sin(k / 2)
    Eh = np.cross(K, [0.2, 1.0, -0.4])
    Eh /= np.linalg.norm(Eh)
    Om = S * np.linalg.norm(K) / math.sqrt(2.0)
    w = 2 * math.asin(Om / 2)
    Hh = (S / Om) * np.cross(K, Eh)
    NODE = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5), (0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]

    def field(c, t):
        Z, Y, X = np.meshgrid(np.arange(shape[2]) + NODE[c][2], np.arange(shape[1]) + NODE[c][1],
                              np.arange(shape[0]) + NODE[c][0], indexing="ij")
        amp = Eh[c] if c < 3 else Hh[c - 3]
        return amp * np.cos(k[0] * X + k[1] * Y + k[2] * Z - w * t)

    g.write_fields(np.stack([field(c, 0.0 if c < 3 else -0.5) for c in range(6)]))
    N = 500
    g.step(N)
    ref = np.stack([field(c, N if c < 3 else N - 0.5) for c in range(6)])
    tol = 1e-11 if precision == "f64" else 2e-5
    assert rel_l2(g.read_fields(), ref) <= tol


def test_fp64_gain_with_noise_matches_oracle():
    gain = inputs.GainSpec(n_total=1e24, fa_hat=0.8, dw_rel=0.02, tau32=100e-15, tau21=1e-9, tau10=100e-15,
                           pump=5e11, noise_amp=1e-3, init="steady")
    spec = small_opal(n_cells=2, res=8, npml=5, precision="f64", source="dipole", gain=gain)
    g = gpu_grid(spec)
    o = oracle_grid(spec)
    g.step(300)
    o.step(300)
    assert _fields_gpu_vs_oracle(g, o) <= 1e-12
    for what in range(2):
        P = g.read_gain(what)
        Po = (o.P if what == 0 else o.Pm).transpose(0, 3, 2, 1)
        assert rel_l2(P, Po) <= 1e-12
    dN = g.read_gain(3)
    assert rel_l2(dN, o.dN[1:].transpose(0, 3, 2, 1)) <= 1e-9
    N = g.read_gain(2)
    assert rel_l2(N, o.populations()[1:].transpose(0, 3, 2, 1)) <= 1e-14


@pytest.mark.parametrize("kernel", ["tma", "pair", "plain"])
def test_fp32_noise_kick_matches_oracle_deviates(kernel):
    """One step from zero fields and steady populations leaves P~^1 =
    noise_amp xi in every gain cell (xi: Box-Muller deviates of the Philox
    stream), which isolates the binary32 deviates (special-function-unit log,
    sin and cos) from the oracle's binary64 ones of the same counters: about
    1e-6 relative, up to sqrt(2 x 2^-21.41) absolute where rho is tiny."""
    gain = inputs.GainSpec(n_total=1e24, fa_hat=0.8, dw_rel=0.02, tau32=100e-15, tau21=1e-9, tau10=100e-15,
                           pump=5e11, noise_amp=1e-3, init="steady")
    spec = small_opal(n_cells=3, res=8, npml=5, precision="f32", source="dipole", gain=gain)
    g = gpu_grid(spec)
    g.set_kernel(kernel)
    o = oracle_grid(spec, coef32=True)
    g.step(1)
    o.step(1)
    P = g.read_gain(0)
    Po = o.P.transpose(0, 3, 2, 1)
    gcell = np.broadcast_to(o.gain_cell.transpose(2, 1, 0)[None], P.shape)
    assert gcell.sum() > 1000
    assert np.all(P[~gcell] == 0.0)
    xi, xo = P[gcell] / 1e-3, Po[gcell] / 1e-3
    assert rel_l2(xi, xo) <= 1e-5
    assert np.max(np.abs(xi - xo)) <= 1.5e-3
    assert abs(np.mean(xi)) < 0.02 and abs(np.std(xi) - 1.0) < 0.02


def test_fp32_gain_short_run():
    gain = inputs.GainSpec(n_total=1e24, fa_hat=0.8, dw_rel=0.02, tau32=100e-15, tau21=1e-9, tau10=100e-15,
                           pump=5e11, noise_amp=1e-3, init="ground")
    spec = small_opal(n_cells=2, res=8, npml=5, precision="f32", source="dipole", gain=gain)
    g = gpu_grid(spec)
    o = oracle_grid(spec, coef32=True)
    g.step(300)
    o.step(300)
    assert _fields_gpu_vs_oracle(g, o) <= 1e-5
    # populations relax from the ground state: deviations carried in binary32
    # with compensated sums
    assert rel_l2(g.read_gain(3), o.dN[1:].transpose(0, 3, 2, 1)) <= 1e-6


def test_full_size_planewave_grid_few_steps():
    """184^3 FP32 disordered-opal grid in the launch shape the benchmark times
    (autotuned from the same state): 4 steps from seeded random fields, every
    cell compared with the oracle."""
    spec = inputs.opal_planewave_f32(ncell=8, res=20, npml=12, sigma=0.06, realization=1)
    g = gpu_grid(spec)
    o = oracle_grid(spec, coef32=True)
    F = inputs.random_fields(spec.shape, seed=5, scale=1.0)
    g.write_fields(F)
    o.set_fields_memory_order(F.astype(np.float32).astype(np.float64))
    g.autotune(trial_steps=3)
    g.step(4)
    o.step(4)
    assert _fields_gpu_vs_oracle(g, o) <= 1e-6


def test_full_size_lasing_grid_few_steps():
    """140^3 FP32 Maxwell-Bloch lasing grid (gain in the spheres, pump, noise)
    in the autotuned launch shape: 3 steps from seeded random fields, every
    cell's fields and population deviations compared with the oracle."""
    spec = inputs.opal_lasing_f32(ncell=6, res=20, npml=10, sigma=0.05, pump=1e10, realization=1)
    g = gpu_grid(spec)
    o = oracle_grid(spec, coef32=True)
    F = inputs.random_fields(spec.shape, seed=6, scale=1.0e4)
    g.write_fields(F)
    o.set_fields_memory_order(F.astype(np.float32).astype(np.float64))
    g.autotune(trial_steps=3)
    g.step(3)
    o.step(3)
    assert _fields_gpu_vs_oracle(g, o) <= 1e-5
    assert rel_l2(g.read_gain(0), o.P.transpose(0, 3, 2, 1)) <= 1e-5
    assert rel_l2(g.read_gain(3), o.dN[1:].transpose(0, 3, 2, 1)) <= 1e-6


def test_full_size_batch_sampled_members():
    """The 64-realization mixed batch stepped together in its autotuned shape:
    a passive and a lasing member (from seeded random fields) against the
    oracle, every cell, after 2 steps."""
    from paper_0802_3775_gb300.fdtd import Batch
    specs = inputs.mixed_batch(64, seed=4000, steps=40)
    grids = [gpu_grid(s, record_capacity=64) for s in specs]
    picks = [0, 1]
    oracles = {}
    for q in picks:
        F = inputs.random_fields(specs[q].shape, seed=70 + q, scale=1.0e3)
        grids[q].write_fields(F)
        oracles[q] = oracle_grid(specs[q], coef32=True)
        oracles[q].set_fields_memory_order(F.astype(np.float32).astype(np.float64))
    b = Batch(grids)
    b.autotune(trial_steps=2)
    b.step(2)
    b.sync()
    for q in picks:
        oracles[q].step(2)
        assert _fields_gpu_vs_oracle(grids[q], oracles[q]) <= 1e-5
    b.close()
    for g in grids:
        g.close()


def test_checkpoint_restart_is_bitwise():
    spec = small_opal(precision="f32", source="dipole")
    a = gpu_grid(spec)
    a.step(200)
    ref = a.read_fields()
    b = gpu_grid(spec)
    b.step(120)
    import tempfile, os
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        b.save_state(path)
        c = gpu_grid(spec)
        c.load_state(path)
    c.step(80)
    assert np.array_equal(c.read_fields(), ref)
    assert np.array_equal(c.read_probes(t0=120, count=80), a.read_probes(t0=120, count=80))


@pytest.mark.parametrize("saver,loader", [("tma", "pair"), ("pair", "tma")])
def test_checkpoint_moves_between_kernels(saver, loader):
    """A grid on the paired kernel cycles three field sets, one on the TMA
    kernel two: a checkpoint taken on one continues bitwise on the other."""
    spec = small_opal(precision="f32", source="dipole")
    a = gpu_grid(spec)
    a.set_kernel(saver)
    a.step(200)
    ref = a.read_fields()
    b = gpu_grid(spec)
    b.set_kernel(saver)
    b.step(122)  # 122 % 3 != 122 % 2: the current set moves
    import tempfile, os
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        b.save_state(path)
        c = gpu_grid(spec)
        c.set_kernel(loader)
        c.load_state(path)
    c.step(78)
    assert c.kernel_in_use()[0] == {"tma": 2, "pair": 3}[loader]
    assert np.array_equal(c.read_fields(), ref)
    assert np.array_equal(c.read_probes(t0=122, count=78), a.read_probes(t0=122, count=78))


def test_nonfinite_values_are_reported():
    from paper_0802_3775_gb300.fdtd import FdtdError
    spec = small_opal(precision="f32", source="dipole")
    spec.sources[0].amplitude = 3e38
    g = gpu_grid(spec)
    g.step(400)
    with pytest.raises(FdtdError) as e:
        g.sync()
    assert e.value.code == -5
