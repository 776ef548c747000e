"""FP64 CPU oracle of the Maxwell-Bloch FDTD time step.

Test infrastructure only: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.  It shares no code,
header, table or constant generator with the CUDA library.

What it computes (paper, Sec. "Sample and numerical approach"): the Yee
finite-difference time-domain leapfrog for Maxwell's curl equations over a
per-node permittivity map, an absorbing layer at the box faces, and -- for the
lasing runs (Sec. "3+1D simulation of lasing") -- a four-level gain medium
coupled cell by cell through a polarization oscillator per field component,
with spontaneous-emission noise entering as a random term.  Observables: field
probes (Sec. "Wide-band excitation and gap filling") and the Poynting flux
T(t) summed over the faces of a plane (Sec. "Dynamical diffusion and
localization").

Units (normalized, exact rescalings of SI):
  E in V/m; H~ = eta0 H in V/m; P~ = P / eps0 in V/m; N in m^-3.
  S = c dt / dx = courant / sqrt(3)  (courant 0.5: half the 3D stability limit).

One step n -> n+1 (plain loops over whole arrays, in this order):
  1. H~^{n+1/2} = H~^{n-1/2} - S curl_f E^n, each derivative in an absorbing
     slab replaced by d/kappa + psi,  psi <- b psi + c d   (CPML, convolutional
     form of the PML; the paper names a uniaxial PML, available as absorber="upml").
  2. flux T^n from E^n and (H~^{n-1/2} + H~^{n+1/2}) / 2.
  3. gain cells: P~^{n+1} = a1 P~^n - a2 P~^{n-1} + a3 (N1 - N2)^n E^n + noise.
  4. E^{n+1} = E^n + (S/eps_r) curl_b H~^{n+1/2} - (1/eps_r)(P~^{n+1} - P~^n + src^n),
     tangential E held at 0 on the index-0 plane of every non-periodic axis
     (the plane at index n_d is outside the arrays and reads as 0: PEC walls).
  5. gain cells: r = eps0/(hbar omega_a) sum_c (E_c^{n+1} + E_c^n)/2 (P~_c^{n+1} - P~_c^n),
     dN^{n+1} = dN^n + (M - I) dN^n + w r     (dN = N - N_eq).
  6. probes record E^{n+1}.

Readings where the paper is silent:
  * PML grading: sigma = sigma_max rho^m, kappa = 1 + (kappa_max-1) rho^m,
    alpha = alpha_max (1 - rho); sigma_max dt/eps0 = factor (m+1) S / sqrt(eps_edge),
    alpha dt/eps0 = alpha_max 2 pi f_ref dt;  b = exp(-(sigma/kappa + alpha) dt/eps0),
    c = sigma (b - 1) / (sigma kappa + kappa^2 alpha).  Depth rho(x) = (L0 - x)/L0
    below L0 and (x - (n - L1))/L1 above n - L1, x the node coordinate in cells
    (integer for E-curl terms, half-integer for H-curl terms).
  * Gain per cell ("cell" coupling): P_c(i,j,k) sits on E_c(i,j,k); the
    populations of cell (i,j,k) drive and are driven by that cell's three
    components.
  * "centred" coupling (the paper solves the Bloch variables in the middle of
    the Yee cell): P and N live at the cell centre (i+1/2, j+1/2, k+1/2); the
    oscillator is driven by the centre average E_bar = A E of the four
    E_c edges of the cell, the polarization current reaches each E_c edge
    as the average A^T dP of the four cells that share the edge, and the
    populations see r = eps0/(hbar omega_a) sum_c A((E^{n+1}+E^n)/2)_c dP_c,
    so the field-medium exchange balances exactly (A^T is A's adjoint).
  * coef32: round every update coefficient (S, S/eps_r, 1/eps_r, 1/kappa, b, c,
    a1, a2) to binary32, which defines the discrete problem an FP32 run solves.
  * absorber="upml" (the paper's uniaxial PML): the same sigma' = sigma dt/eps0
    and kappa grading as the CPML, no alpha, evaluated at each field node's own
    position on every axis (half-integer along the component's axis for E,
    integer for H, and the other way round on the other axes).  Nodes where a
    grading is non-zero keep an auxiliary field: for E_c with (d1, d2) the
    other axes in cyclic order,
      D~^{n+1} = [(k1 - s1/2) D~^n + S curl_b H~] / (k1 + s1/2)     (axis d1),
      E^{n+1} = [(k2 - s2/2) E^n + ((kc + sc/2) D~^{n+1} - (kc - sc/2) D~^n)/eps_r]
                / (k2 + s2/2)                                    (axes c, d2),
    and H~_c the same with B~, -S curl_f E and eps_r = 1 (the uniaxial tensor
    diag(s_y s_z/s_x, s_z s_x/s_y, s_x s_y/s_z) split into two first-order
    steps); every other node takes the plain Yee update.  Each coefficient is
    rounded like the others in coef32 mode.
"""
from __future__ import annotations

import math

import numpy as np

from . import gain as _gain
from .philox import gain_noise
from .rasterize import rasterize as _rasterize

C0 = 299792458.0
MU0 = 1.25663706212e-6
EPS0 = 1.0 / (MU0 * C0 * C0)
ETA0 = MU0 * C0
HBAR = 1.054571817e-34


def _r32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def _ident(x):
    return np.asarray(x, dtype=np.float64)


def waveform(n, f0_hat, rel_bw, S, res, t0_steps=0.0):
    """Gaussian-modulated sine at t = (n + 1/2) dt, all times in units of dt.

    g(t) = exp(-(t - t0)^2 / (2 tau^2)) sin(2 pi f0 (t - t0)),
    tau = sqrt(ln 2) / (pi rel_bw f0)  (rel_bw = FWHM of the power spectrum / f0),
    t0 = 5 tau unless given; f0 dt = f0_hat S / res.
    """
    f0dt = f0_hat * S / res
    tau = math.sqrt(math.log(2.0)) / (math.pi * rel_bw * f0dt)
    t0 = 5.0 * tau if t0_steps == 0 else t0_steps
    t = np.asarray(n, dtype=np.float64) + 0.5 - t0
    return np.exp(-t * t / (2.0 * tau * tau)) * np.sin(2.0 * math.pi * f0dt * t)


class Oracle:
    """Plain FP64 stepper.  Arrays are indexed [component, i, j, k]."""

    def __init__(self, shape, res, *, a=480e-9, courant=0.5, npml=(0, 0, 0, 0, 0, 0),
                 periodic=(False, False, False), eps=(1.0, 1.0, 1.0), cpml_m=3.0,
                 cpml_sigma_factor=0.8, cpml_kappa_max=1.0, cpml_alpha_max=0.05, cpml_f_hat=0.80,
                 coef32=False, seed=0, absorber="cpml"):
        if absorber not in ("cpml", "upml"):
            raise ValueError(absorber)
        self.upml = absorber == "upml"
        self.shape = tuple(int(s) for s in shape)
        nx, ny, nz = self.shape
        self.res = float(res)
        self.a = float(a)
        self.dx = self.a / self.res
        self.S = courant / math.sqrt(3.0)
        self.dt = self.S * self.dx / C0
        self.periodic = tuple(bool(p) for p in periodic)
        self.npml = tuple(int(p) for p in npml)
        for d in range(3):
            if self.periodic[d] and (self.npml[2 * d] or self.npml[2 * d + 1]):
                raise ValueError("a periodic axis has no absorbing slab")
        self.eps = np.asarray(eps, dtype=np.float64)
        self.R = _r32 if coef32 else _ident
        self.seed = int(seed)
        self.cH = float(self.R(self.S))
        self.E = np.zeros((3, nx, ny, nz))
        self.H = np.zeros((3, nx, ny, nz))
        self.n = 0
        self._cpml = dict(m=cpml_m, factor=cpml_sigma_factor, kmax=cpml_kappa_max,
                          amax=cpml_alpha_max, fhat=cpml_f_hat)
        # CPML grading coefficients (the UPML uses its own, built below)
        self.prof = None if self.upml else {"E": [self._profile(d, False) for d in range(3)],
                                              "H": [self._profile(d, True) for d in range(3)]}
        self.psi = {"E": {}, "H": {}}
        for kind in ("E", "H"):
            for c in range(3):
                for d in ((c + 1) % 3, (c + 2) % 3):
                    if self._has_pml(d):
                        self.psi[kind][(c, d)] = np.zeros((nx, ny, nz))
        if self.upml:
            self.D = np.zeros((3, nx, ny, nz))
            self.B = np.zeros((3, nx, ny, nz))
            self._upml_h = self._upml_coefficients(True)
        self.set_material(np.full((nz, ny, nx), 0b010101, dtype=np.uint8))
        self.gain = None
        self.src = np.zeros((3, nx, ny, nz))
        self.sources = []
        self.probes = []
        self.fluxes = []
        self.probe_log = []
        self.flux_log = []

    # ------------------------------------------------------------------ set-up
    @classmethod
    def from_spec(cls, spec, coef32=None):
        """Build from a run description record (attributes as in the input generators)."""
        if coef32 is None:
            coef32 = spec.precision == "f32"
        o = cls(spec.shape, spec.res, a=spec.a, courant=spec.courant, npml=spec.npml,
                periodic=spec.periodic, eps=spec.eps, cpml_m=spec.cpml_m,
                cpml_sigma_factor=spec.cpml_sigma_factor, cpml_kappa_max=spec.cpml_kappa_max,
                cpml_alpha_max=spec.cpml_alpha_max, cpml_f_hat=spec.cpml_f_hat, coef32=coef32,
                seed=spec.seed, absorber=getattr(spec, "absorber", "cpml"))
        if spec.spheres is not None:
            o.rasterize(spec.spheres, spec.box_lo, spec.box_hi)
        if spec.gain is not None:
            g = spec.gain
            o.set_gain(n_total=g.n_total, fa_hat=g.fa_hat, dw_rel=g.dw_rel, tau32=g.tau32,
                       tau21=g.tau21, tau10=g.tau10, pump=g.pump, kappa=g.kappa,
                       noise_amp=g.noise_amp, init=g.init, coupling=getattr(g, "coupling", "cell"))
        for s in spec.sources:
            o.add_source(kind=s.kind, comp=s.comp, pos=s.pos, axis=s.axis, index=s.index,
                         waist=s.waist, f0_hat=s.f0_hat, rel_bw=s.rel_bw, t0_steps=s.t0_steps,
                         amplitude=s.amplitude)
        if spec.probes is not None:
            for p in np.asarray(spec.probes).reshape(-1, 3):
                o.add_probe(*[int(v) for v in p])
        for f in spec.fluxes:
            o.add_flux(f.axis, f.index, f.sign, f.u, f.v)
        return o

    def _has_pml(self, d):
        """Axis d has CPML memory (a slab, and the absorber is the CPML)."""
        return not self.upml and (self.npml[2 * d] > 0 or self.npml[2 * d + 1] > 0)

    def _grading(self, d, half):
        """(sigma dt/eps0, kappa) at the integer (or half-integer) nodes of axis d,
        shaped to broadcast along d; the CPML's grading without alpha."""
        n = self.shape[d]
        L0, L1 = self.npml[2 * d], self.npml[2 * d + 1]
        x = np.arange(n, dtype=np.float64) + (0.5 if half else 0.0)
        rho = np.zeros(n)
        if L0 > 0:
            lo = x < L0
            rho[lo] = (L0 - x[lo]) / L0
        if L1 > 0:
            hi = x > n - L1
            rho[hi] = (x[hi] - (n - L1)) / L1
        p = self._cpml
        sig_max = p["factor"] * (p["m"] + 1.0) * self.S / math.sqrt(self.eps[0])
        sig = sig_max * rho ** p["m"]
        kap = 1.0 + (p["kmax"] - 1.0) * rho ** p["m"]
        shp = [1, 1, 1]
        shp[d] = n
        return sig.reshape(shp), kap.reshape(shp), (rho > 0).reshape(shp)

    def _upml_coefficients(self, h_side, eps_nodes=None):
        """Per-component UPML coefficients (u1, u2, v1, v2, v3) and node mask:
        aux^{n+1} = u1 aux^n + u2 (S curl), field^{n+1} = v1 field^n + v2 aux^{n+1} - v3 aux^n."""
        out = []
        for c in range(3):
            d1, d2 = (c + 1) % 3, (c + 2) % 3
            # E_c is half-integer along c, integer elsewhere; H_c the other way round
            g = [self._grading(d, (d == c) != h_side) for d in range(3)]
            s1, k1, m1 = g[d1]
            s2, k2, m2 = g[d2]
            sc, kc, mc = g[c]
            er = 1.0 if h_side else eps_nodes[c]
            den2 = k2 + 0.5 * s2
            u1 = (k1 - 0.5 * s1) / (k1 + 0.5 * s1)
            u2 = 1.0 / (k1 + 0.5 * s1)
            v1 = (k2 - 0.5 * s2) / den2
            v2 = (kc + 0.5 * sc) / (er * den2)
            v3 = (kc - 0.5 * sc) / (er * den2)
            shape = self.shape
            mask = np.broadcast_to(m1 | m2 | mc, shape)
            out.append(tuple(self.R(np.broadcast_to(v, shape)) for v in (u1, u2, v1, v2, v3)) + (mask,))
        return out

    def _profile(self, d, half):
        """(1/kappa, b, c) at the nodes of axis d, shaped to broadcast along d."""
        n = self.shape[d]
        L0, L1 = self.npml[2 * d], self.npml[2 * d + 1]
        x = np.arange(n, dtype=np.float64) + (0.5 if half else 0.0)
        rho = np.zeros(n)
        if L0 > 0:
            lo = x < L0
            rho[lo] = (L0 - x[lo]) / L0
        if L1 > 0:
            hi = x > n - L1
            rho[hi] = (x[hi] - (n - L1)) / L1
        p = self._cpml
        eps_edge = self.eps[0]
        sig_max = p["factor"] * (p["m"] + 1.0) * self.S / math.sqrt(eps_edge)
        alpha_max = p["amax"] * 2.0 * math.pi * p["fhat"] * self.S / self.res
        ik = np.ones(n)
        b = np.ones(n)
        c = np.zeros(n)
        on = rho > 0
        sig = sig_max * rho[on] ** p["m"]
        kap = 1.0 + (p["kmax"] - 1.0) * rho[on] ** p["m"]
        alp = alpha_max * (1.0 - rho[on])
        b[on] = np.exp(-(sig / kap + alp))
        c[on] = sig * (b[on] - 1.0) / (sig * kap + kap * kap * alp)
        ik[on] = 1.0 / kap
        shp = [1, 1, 1]
        shp[d] = n
        return tuple(self.R(v).reshape(shp) for v in (ik, b, c))

    def set_material(self, mat):
        """Material bytes uint8[nz, ny, nx] (x fastest), see oracle.rasterize."""
        m = np.asarray(mat, dtype=np.uint8).transpose(2, 1, 0)
        self.mat = m.copy()
        cls = np.stack([(m >> (2 * c)) & 3 for c in range(3)])
        self.eps_E = self.eps[cls]
        self.cE = self.R(self.S / self.eps_E)
        self.cP = self.R(1.0 / self.eps_E)
        self.gain_cell = ((m >> 6) & 1).astype(bool)
        if self.upml:
            self._upml_e = self._upml_coefficients(False, self.eps_E)

    def rasterize(self, spheres, box_lo, box_hi):
        self.set_material(_rasterize(self.shape, spheres, box_lo, box_hi))

    def set_gain(self, *, n_total, fa_hat, dw_rel, tau32, tau21, tau10, pump, kappa=0.0,
                 noise_amp=0.0, init="steady", coupling="cell"):
        omega_a = 2.0 * math.pi * fa_hat * C0 / self.a
        domega = dw_rel * omega_a
        if kappa == 0.0:
            kappa = _gain.default_kappa(omega_a, tau21)
        a1, a2, a3 = _gain.polarization_coefficients(omega_a, domega, kappa, self.dt)
        A = _gain.rate_matrix(pump, tau32, tau21, tau10)
        m_minus_i, w = _gain.crank_nicolson(A, self.dt)
        n_eq = _gain.equilibrium(n_total, pump, tau32, tau21, tau10)
        nx, ny, nz = self.shape
        mask = self.gain_cell
        self.gain = dict(a1=float(self.R(a1)), a2=float(self.R(a2)), a3=a3, A=A, MmI=m_minus_i, w=w,
                         n_eq=n_eq, n_total=n_total, omega_a=omega_a, domega=domega, kappa=kappa,
                         q=EPS0 / (HBAR * omega_a), noise_amp=float(noise_amp), mask=mask)
        if coupling not in ("cell", "centred"):
            raise ValueError(coupling)
        self.gain["centred"] = coupling == "centred"
        self.P = np.zeros((3, nx, ny, nz))
        self.Pm = np.zeros((3, nx, ny, nz))
        self.dN = np.zeros((4, nx, ny, nz))
        if init == "ground":
            ground = np.array([n_total, 0.0, 0.0, 0.0])
            self.dN[:] = ((ground - n_eq)[:, None, None, None]) * mask[None]
        elif init != "steady":
            raise ValueError(init)
        i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
        self._cell_index = ((k.astype(np.int64) * ny + j) * nx + i)[mask].astype(np.uint64)

    def populations(self):
        """N = N_eq + dN, float[4, nx, ny, nz] (zero outside gain cells)."""
        g = self.gain
        return (self.dN + g["n_eq"][:, None, None, None]) * g["mask"][None]

    def add_source(self, *, kind="point", comp=2, pos=(0, 0, 0), axis=2, index=0, waist=0.0,
                   f0_hat=0.8, rel_bw=0.1, t0_steps=0.0, amplitude=1.0):
        nx, ny, nz = self.shape
        w = np.zeros((nx, ny, nz))
        if kind == "point":
            w[tuple(pos)] = amplitude
        elif kind == "sheet":
            d1, d2 = (axis + 1) % 3, (axis + 2) % 3
            lo1, hi1 = self.npml[2 * d1], self.shape[d1] - self.npml[2 * d1 + 1]
            lo2, hi2 = self.npml[2 * d2], self.shape[d2] - self.npml[2 * d2 + 1]
            u = np.arange(lo1, hi1, dtype=np.float64)
            v = np.arange(lo2, hi2, dtype=np.float64)
            if waist > 0:
                uc, vc = 0.5 * (lo1 + hi1 - 1), 0.5 * (lo2 + hi2 - 1)
                prof = np.exp(-(((u - uc) ** 2)[:, None] + ((v - vc) ** 2)[None, :]) / (waist * waist))
            else:
                prof = np.ones((u.size, v.size))
            idx = [None, None, None]
            idx[axis] = index
            idx[d1] = slice(lo1, hi1)
            idx[d2] = slice(lo2, hi2)
            # assign with the (d1, d2) profile laid out in array-axis order
            sub = w[tuple(idx)]
            sub[...] = amplitude * (prof if d1 < d2 else prof.T)
        else:
            raise ValueError(kind)
        self.sources.append(dict(comp=comp, w=w, f0_hat=f0_hat, rel_bw=rel_bw, t0_steps=t0_steps))

    def add_probe(self, i, j, k):
        self.probes.append((i, j, k))

    def add_flux(self, axis, index, sign=1.0, u=(0, 0), v=(0, 0)):
        d1, d2 = (axis + 1) % 3, (axis + 2) % 3
        if not (1 <= index <= self.shape[axis] - 1):
            raise ValueError("flux plane index out of range")
        if not (0 <= u[0] <= u[1] <= self.shape[d1] - 1 and 0 <= v[0] <= v[1] <= self.shape[d2] - 1):
            raise ValueError("flux face range out of range")
        self.fluxes.append(dict(axis=axis, index=index, sign=sign, u=tuple(u), v=tuple(v)))

    # ------------------------------------------------------------ the operator
    def _fwd(self, F, d):
        """F[idx + 1] - F[idx] along axis d; beyond the last node reads 0 (or wraps)."""
        if self.periodic[d]:
            return np.roll(F, -1, axis=d) - F
        pad = np.zeros_like(np.take(F, [0], axis=d))
        return np.diff(np.concatenate([F, pad], axis=d), axis=d)

    def _bwd(self, F, d):
        """F[idx] - F[idx - 1] along axis d; before the first node reads 0 (or wraps)."""
        if self.periodic[d]:
            return F - np.roll(F, 1, axis=d)
        pad = np.zeros_like(np.take(F, [0], axis=d))
        return np.diff(np.concatenate([pad, F], axis=d), axis=d)

    def _nb(self, F, d, s):
        """F at the neighbour idx + s along axis d (s = +1 or -1); outside the
        arrays it reads 0, or wraps on a periodic axis."""
        if self.periodic[d]:
            return np.roll(F, -s, axis=d)
        out = np.zeros_like(F)
        src = [slice(None)] * 3
        dst = [slice(None)] * 3
        if s > 0:
            src[d], dst[d] = slice(1, None), slice(0, -1)
        else:
            src[d], dst[d] = slice(0, -1), slice(1, None)
        out[tuple(dst)] = F[tuple(src)]
        return out

    def to_cells(self, E):
        """A: the centre average of each E component over the four edges of
        its orientation around cell (i, j, k): for E_c with (d1, d2) the other
        two axes in cyclic order, 1/4 ((E + E[+d1]) + (E[+d2] + E[+d1+d2]))."""
        out = np.empty_like(E)
        for c in range(3):
            d1, d2 = (c + 1) % 3, (c + 2) % 3
            F = E[c]
            F2 = self._nb(F, d2, +1)
            out[c] = 0.25 * ((F + self._nb(F, d1, +1)) + (F2 + self._nb(F2, d1, +1)))
        return out

    def to_edges(self, P):
        """A^T: at each E_c edge, 1/4 of the sum of the cell values of the four
        cells sharing it, 1/4 ((P + P[-d1]) + (P[-d2] + P[-d1-d2]))."""
        out = np.empty_like(P)
        for c in range(3):
            d1, d2 = (c + 1) % 3, (c + 2) % 3
            F = P[c]
            F2 = self._nb(F, d2, -1)
            out[c] = 0.25 * ((F + self._nb(F, d1, -1)) + (F2 + self._nb(F2, d1, -1)))
        return out

    def _term(self, D, d, comp, kind):
        """Difference D along d as seen by component `comp`: D/kappa + psi inside slabs."""
        if not self._has_pml(d):
            return D
        ik, b, c = self.prof[kind][d]
        psi = b * self.psi[kind][(comp, d)] + c * D
        self.psi[kind][(comp, d)] = psi
        return ik * D + psi

    def curl_E(self, E):
        out = np.empty_like(E)
        for c in range(3):
            c1, c2 = (c + 1) % 3, (c + 2) % 3
            out[c] = self._term(self._fwd(E[c2], c1), c1, c, "H") - self._term(self._fwd(E[c1], c2), c2, c, "H")
        return out

    def curl_H(self, H):
        out = np.empty_like(H)
        for c in range(3):
            c1, c2 = (c + 1) % 3, (c + 2) % 3
            out[c] = self._term(self._bwd(H[c2], c1), c1, c, "E") - self._term(self._bwd(H[c1], c2), c2, c, "E")
        return out

    def _pec(self, E):
        for d in range(3):
            if self.periodic[d]:
                continue
            for c in range(3):
                if c != d:
                    idx = [slice(None)] * 3
                    idx[d] = 0
                    E[c][tuple(idx)] = 0.0

    def step(self, count=1):
        for _ in range(int(count)):
            self._step_once()

    def _step_once(self):
        n = self.n
        E_n = self.E
        H_old = self.H
        # 1. magnetic half step
        if self.upml:
            cE_n = self.curl_E(E_n)
            H_new = H_old - self.cH * cE_n
            for c in range(3):
                u1, u2, v1, v2, v3, mask = self._upml_h[c]
                B_new = u1 * self.B[c] - u2 * (self.cH * cE_n[c])
                H_new[c] = np.where(mask, v1 * H_old[c] + v2 * B_new - v3 * self.B[c], H_new[c])
                self.B[c] = np.where(mask, B_new, self.B[c])
        else:
            H_new = H_old - self.cH * self.curl_E(E_n)
        # 2. flux through the planes at time n
        flux_vals = [self._flux(f, E_n, 0.5 * (H_old + H_new)) for f in self.fluxes]
        # 3. polarization
        g = self.gain
        dP = np.zeros_like(E_n)
        if g is not None:
            N = self.populations()
            dn12 = (N[1] - N[2])
            # the field that drives the oscillator: on the cell's own nodes, or
            # averaged to the cell centre
            E_drive = self.to_cells(E_n) if g["centred"] else E_n
            P_new = g["a1"] * self.P - g["a2"] * self.Pm + g["a3"] * dn12[None] * E_drive
            if g["noise_amp"] != 0.0:
                xi = gain_noise(self.seed, n, self._cell_index)
                for c in range(3):
                    P_new[c][g["mask"]] += g["noise_amp"] * xi[c]
            P_new *= g["mask"][None]
            dP = P_new - self.P
            # the polarization current on the E nodes
            dP_nodes = self.to_edges(dP) if g["centred"] else dP
        # 4. electric step
        src = np.zeros_like(E_n)
        for s in self.sources:
            src[s["comp"]] += s["w"] * float(waveform(n, s["f0_hat"], s["rel_bw"], self.S, self.res, s["t0_steps"]))
        cH_new = self.curl_H(H_new)
        E_new = E_n + self.cE * cH_new - self.cP * ((dP_nodes if g is not None else dP) + src)
        if self.upml:
            for c in range(3):
                u1, u2, v1, v2, v3, mask = self._upml_e[c]
                D_new = u1 * self.D[c] + u2 * (self.cH * cH_new[c])
                E_new[c] = np.where(mask, v1 * E_n[c] + v2 * D_new - v3 * self.D[c], E_new[c])
                self.D[c] = np.where(mask, D_new, self.D[c])
        self._pec(E_new)
        # 5. populations
        if g is not None:
            E_half = 0.5 * (E_new + E_n)
            if g["centred"]:
                E_half = self.to_cells(E_half)
            r = g["q"] * np.sum(E_half * dP, axis=0)
            inc = np.einsum("ab,bijk->aijk", g["MmI"], self.dN) + g["w"][:, None, None, None] * r[None]
            self.dN = (self.dN + inc) * g["mask"][None]
            self.Pm = self.P
            self.P = P_new
        self.E = E_new
        self.H = H_new
        self.n = n + 1
        # 6. observers
        if self.probes:
            self.probe_log.append([self.E[:, i, j, k].copy() for (i, j, k) in self.probes])
        if self.fluxes:
            self.flux_log.append((n, flux_vals))

    def _flux(self, f, E, Havg):
        """sign * dx^2 * sum over faces of (E x H).n with H = H~/eta0 (SI watts).

        Faces sit at the cell-face centres of the plane `index` along `axis`;
        with (d, d1, d2) cyclic and [p, u, v] the array index in that order:
          E1 averaged over v, v+1;  E2 over u, u+1;
          H2 over (p-1, p) x (v, v+1);  H1 over (p-1, p) x (u, u+1);
          S_d = E1 H2 - E2 H1.
        """
        d = f["axis"]
        d1, d2 = (d + 1) % 3, (d + 2) % 3
        order = (d, d1, d2)
        E1, E2 = E[d1].transpose(order), E[d2].transpose(order)
        H1, H2 = Havg[d1].transpose(order), Havg[d2].transpose(order)
        p = f["index"]
        u0, u1 = f["u"]
        v0, v1 = f["v"]
        U = slice(u0, u1)
        Up = slice(u0 + 1, u1 + 1)
        V = slice(v0, v1)
        Vp = slice(v0 + 1, v1 + 1)
        e1 = 0.5 * (E1[p, U, V] + E1[p, U, Vp])
        e2 = 0.5 * (E2[p, U, V] + E2[p, Up, V])
        h2 = 0.25 * (H2[p - 1, U, V] + H2[p, U, V] + H2[p - 1, U, Vp] + H2[p, U, Vp])
        h1 = 0.25 * (H1[p - 1, U, V] + H1[p, U, V] + H1[p - 1, Up, V] + H1[p, Up, V])
        return f["sign"] * self.dx * self.dx * float(np.sum(e1 * h2 - e2 * h1)) / ETA0

    # -------------------------------------------------------------- read-outs
    def energy(self):
        """Field energy 1/2 eps0 dx^3 (sum eps_r E^2 + sum H~^2) in joules (E^n, H~^{n-1/2})."""
        return 0.5 * EPS0 * self.dx ** 3 * (float(np.sum(self.eps_E * self.E * self.E)) + float(np.sum(self.H * self.H)))

    def fields_memory_order(self):
        """float64[6, nz, ny, nx]: Ex, Ey, Ez, H~x, H~y, H~z with x fastest."""
        return np.ascontiguousarray(np.concatenate([self.E, self.H]).transpose(0, 3, 2, 1))

    def set_fields_memory_order(self, F):
        F = np.asarray(F, dtype=np.float64).transpose(0, 3, 2, 1)
        self.E = F[:3].copy()
        self.H = F[3:].copy()

    def probe_series(self):
        """float64[steps, n_probes, 3]: E^{n+1} at each probe after update n."""
        return np.asarray(self.probe_log, dtype=np.float64).reshape(len(self.probe_log), len(self.probes), 3)

    def flux_series(self):
        """float64[n_planes, steps]: T^n of each plane (watts)."""
        return np.asarray([vals for (_, vals) in self.flux_log], dtype=np.float64).T.reshape(len(self.fluxes), -1)
