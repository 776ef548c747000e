"""Shared helpers of the parity tests: build the same run on the GPU library and
on the oracle, and compare."""
import numpy as np

from paper_0802_3775_gb300 import inputs


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0))


def gpu_grid(spec, **kw):
    from paper_0802_3775_gb300.fdtd import Grid
    return Grid.from_spec(spec, **kw)


def oracle_grid(spec, coef32=None):
    from oracle import Oracle
    return Oracle.from_spec(spec, coef32=coef32)


def small_opal(n_cells=2, res=10, npml=6, precision="f64", source="dipole", gain=None, sigma=0.05, seed=3,
               rotation="identity", probes=6, flux=True):
    """A small opal run that spans several tiles with ragged edges."""
    n = n_cells * res + 2 * npml
    spec = inputs.RunSpec(shape=(n + 3, n - 2, n + 5), res=res, npml=(npml, npml + 1, npml, npml, npml + 2, npml),
                          eps=(11.9, 11.9, 1.0 if gain is None else 2.25), precision=precision, seed=seed)
    lo = (npml, npml, npml + 2)
    hi = (spec.shape[0] - npml - 1, spec.shape[1] - npml, spec.shape[2] - npml)
    spec.box_lo, spec.box_hi = lo, hi
    spec.spheres = inputs.fcc_opal_spheres(lo, hi, res, rotation=rotation, sigma=sigma, seed=seed)
    c = [s // 2 for s in spec.shape]
    if source == "dipole":
        spec.sources = [inputs.SourceSpec(kind="point", comp=2, pos=tuple(c), f0_hat=0.8, rel_bw=0.3)]
    else:
        spec.sources = [inputs.SourceSpec(kind="sheet", comp=0, axis=2, index=npml + 3, f0_hat=0.8, rel_bw=0.3,
                                          waist=6.0)]
    spec.probes = inputs.probe_cells(spec.shape, spec.npml, probes, seed=seed + 1)
    if flux:
        spec.fluxes = [inputs.plane_flux(spec, 2, spec.shape[2] - npml - 3)] + inputs.flux_box(spec, inset=1)
    spec.gain = gain
    return spec
