"""Python binding of the request server (fdtd_server_* / fdtd_submit /
fdtd_poll in include/fdtd.h): argument marshalling only.

The server's worker thread admits runs against an HBM budget and a slot
count, keeps them resident and steps them together (continuous batching);
see the C header for the semantics.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .fdtd import (FP32, FP64, FdtdError, GainParams, GridDesc, SourceDesc, check, load_library)

_P = C.c_void_p
_D = C.POINTER(C.c_double)


class ServerDesc(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_slots", C.c_int32), ("steps_per_chunk", C.c_int32),
                ("precision", C.c_int32), ("graph", C.c_int32)]


class FluxDesc(C.Structure):
    _fields_ = [("axis", C.c_int32), ("index", C.c_int32), ("u0", C.c_int32), ("u1", C.c_int32), ("v0", C.c_int32),
                ("v1", C.c_int32), ("sign", C.c_double)]


class Request(C.Structure):
    _fields_ = [("grid", GridDesc), ("spheres", _D), ("n_spheres", C.c_int64), ("box_lo", C.c_double * 3),
                ("box_hi", C.c_double * 3), ("gain", C.POINTER(GainParams)), ("sources", C.POINTER(SourceDesc)),
                ("n_sources", C.c_int32), ("probes", C.POINTER(C.c_int32)), ("n_probes", C.c_int32),
                ("fluxes", C.POINTER(FluxDesc)), ("n_fluxes", C.c_int32), ("steps", C.c_int64)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("steps", C.c_int64), ("submit_s", C.c_double), ("admit_s", C.c_double),
                ("done_s", C.c_double), ("field_energy", C.c_double), ("n_probes", C.c_int32),
                ("n_fluxes", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("chunks", C.c_int64), ("cell_updates", C.c_int64), ("resident", C.c_int32), ("queued", C.c_int32),
                ("used_bytes", C.c_int64)]


_SIGS = {
    "fdtd_server_create": [C.POINTER(ServerDesc), _P, C.POINTER(_P)],
    "fdtd_server_destroy": [_P],
    "fdtd_submit": [_P, C.POINTER(Request), C.POINTER(C.c_uint64)],
    "fdtd_poll": [_P, C.c_uint64, C.POINTER(Result), C.c_int32],
    "fdtd_result_probes": [_P, C.c_uint64, _D],
    "fdtd_result_flux": [_P, C.c_uint64, _D],
    "fdtd_result_release": [_P, C.c_uint64],
    "fdtd_server_get_stats": [_P, C.POINTER(Stats)],
}


def _lib():
    lib = load_library()
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    return lib


def grid_desc(spec, record_capacity):
    d = GridDesc()
    d.nx, d.ny, d.nz = [int(v) for v in spec.shape]
    for q in range(6):
        d.npml[q] = int(spec.npml[q])
    for q in range(3):
        d.periodic[q] = int(bool(spec.periodic[q]))
        d.eps[q] = float(spec.eps[q])
    d.precision = FP32 if spec.precision == "f32" else FP64
    d.res, d.a, d.courant = float(spec.res), float(spec.a), float(spec.courant)
    d.cpml_m, d.cpml_sigma_factor, d.cpml_kappa_max = spec.cpml_m, spec.cpml_sigma_factor, spec.cpml_kappa_max
    d.cpml_alpha_max, d.cpml_f_hat = spec.cpml_alpha_max, spec.cpml_f_hat
    d.seed = int(spec.seed) & 0xFFFFFFFFFFFFFFFF
    d.record_capacity = int(record_capacity)
    return d


class Server:
    """Continuous-batching request server on the current CUDA device."""

    def __init__(self, hbm_budget_bytes=150 << 30, max_slots=64, steps_per_chunk=500, precision="f32", graph=True):
        self._lib = _lib()
        d = ServerDesc(int(hbm_budget_bytes), int(max_slots), int(steps_per_chunk),
                       FP32 if precision == "f32" else FP64, int(bool(graph)))
        h = C.c_void_p()
        check(self._lib.fdtd_server_create(C.byref(d), None, C.byref(h)))
        self.h = h
        self._meta = {}

    def submit(self, spec, steps=None):
        """Queue one run record; returns its ticket."""
        steps = int(steps if steps is not None else spec.steps)
        keep = []
        r = Request()
        r.grid = grid_desc(spec, steps)
        sp = np.ascontiguousarray(np.asarray(spec.spheres if spec.spheres is not None else np.zeros((0, 4)),
                                             dtype=np.float64).reshape(-1, 4))
        keep.append(sp)
        r.spheres = sp.ctypes.data_as(_D)
        r.n_spheres = sp.shape[0]
        for q in range(3):
            r.box_lo[q] = float(spec.box_lo[q])
            r.box_hi[q] = float(spec.box_hi[q])
        if spec.gain is not None:
            g = spec.gain
            gp = GainParams(g.n_total, g.fa_hat, g.dw_rel, g.tau32, g.tau21, g.tau10, g.pump, g.kappa, g.noise_amp,
                            0 if g.init == "steady" else 1)
            keep.append(gp)
            r.gain = C.pointer(gp)
        srcs = (SourceDesc * max(1, len(spec.sources)))()
        for q, s in enumerate(spec.sources):
            srcs[q] = SourceDesc(0 if s.kind == "point" else 1, s.comp, *[int(v) for v in s.pos], s.axis, s.index,
                                 s.waist, s.f0_hat, s.rel_bw, s.t0_steps, s.amplitude)
        keep.append(srcs)
        r.sources = C.cast(srcs, C.POINTER(SourceDesc))
        r.n_sources = len(spec.sources)
        pr = np.ascontiguousarray(np.asarray(spec.probes if spec.probes is not None else np.zeros((0, 3)),
                                             dtype=np.int32).reshape(-1, 3))
        keep.append(pr)
        r.probes = pr.ctypes.data_as(C.POINTER(C.c_int32))
        r.n_probes = pr.shape[0]
        fl = (FluxDesc * max(1, len(spec.fluxes)))()
        for q, f in enumerate(spec.fluxes):
            fl[q] = FluxDesc(f.axis, f.index, f.u[0], f.u[1], f.v[0], f.v[1], f.sign)
        keep.append(fl)
        r.fluxes = C.cast(fl, C.POINTER(FluxDesc))
        r.n_fluxes = len(spec.fluxes)
        r.steps = steps
        t = C.c_uint64()
        check(self._lib.fdtd_submit(self.h, C.byref(r), C.byref(t)))
        self._meta[t.value] = (steps, pr.shape[0], len(spec.fluxes))
        return t.value

    def poll(self, ticket, timeout_ms=0):
        """Result record; status -6 (E_BUSY) while pending."""
        out = Result()
        code = self._lib.fdtd_poll(self.h, C.c_uint64(ticket), C.byref(out), int(timeout_ms))
        if code not in (0, -6, -7):
            check(code)
        return out

    def wait(self, ticket, timeout_s=600.0):
        out = self.poll(ticket, int(timeout_s * 1000))
        if out.status != 0:
            raise FdtdError(out.status, f"run {ticket} ended with status {out.status}")
        return out

    def probes(self, ticket):
        steps, np_, _ = self._meta[ticket]
        out = np.empty((steps, np_, 3))
        check(self._lib.fdtd_result_probes(self.h, C.c_uint64(ticket), out.ctypes.data_as(_D)))
        return out

    def flux(self, ticket):
        steps, _, nf = self._meta[ticket]
        out = np.empty((nf, steps))
        check(self._lib.fdtd_result_flux(self.h, C.c_uint64(ticket), out.ctypes.data_as(_D)))
        return out

    def release(self, ticket):
        check(self._lib.fdtd_result_release(self.h, C.c_uint64(ticket)))
        self._meta.pop(ticket, None)

    def stats(self):
        s = Stats()
        check(self._lib.fdtd_server_get_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def close(self):
        if getattr(self, "h", None):
            self._lib.fdtd_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
