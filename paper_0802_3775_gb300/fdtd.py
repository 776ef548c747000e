"""Python binding of libfdtd.so (the C ABI in include/fdtd.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  There is no CPU fallback: if the shared library is missing or no
CUDA device is usable, the calls raise.

PyTorch supplies device memory (its caching allocator, through the C ABI's
allocator callback) and the CUDA stream the grid is stepped on.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfdtd.so")

FDTD_OK = 0
ERRORS = {-1: "E_INVAL", -2: "E_NOMEM", -3: "E_CUDA", -4: "E_STATE", -5: "E_NONFINITE", -6: "E_BUSY",
          -7: "E_TIMEOUT", -8: "E_BUDGET"}
FP32, FP64 = 0, 1


class FdtdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("npml", C.c_int32 * 6),
                ("periodic", C.c_int32 * 3), ("precision", C.c_int32), ("reserved", C.c_int32),
                ("res", C.c_double), ("a", C.c_double), ("courant", C.c_double), ("eps", C.c_double * 3),
                ("cpml_m", C.c_double), ("cpml_sigma_factor", C.c_double), ("cpml_kappa_max", C.c_double),
                ("cpml_alpha_max", C.c_double), ("cpml_f_hat", C.c_double), ("seed", C.c_uint64),
                ("record_capacity", C.c_int64)]


class GainParams(C.Structure):
    _fields_ = [("n_total", C.c_double), ("fa_hat", C.c_double), ("dw_rel", C.c_double), ("tau32", C.c_double),
                ("tau21", C.c_double), ("tau10", C.c_double), ("pump", C.c_double), ("kappa", C.c_double),
                ("noise_amp", C.c_double), ("init", C.c_int32)]


class SourceDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("comp", C.c_int32), ("i", C.c_int32), ("j", C.c_int32), ("k", C.c_int32),
                ("axis", C.c_int32), ("index", C.c_int32), ("waist", C.c_double), ("f0_hat", C.c_double),
                ("rel_bw", C.c_double), ("t0_steps", C.c_double), ("amplitude", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class TuneResult(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("bx", C.c_int32), ("by", C.c_int32), ("zdepth", C.c_int32),
                ("grid_blocks", C.c_int32), ("candidates", C.c_int32), ("ms_per_step", C.c_double),
                ("order", C.c_int32)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
SIGNATURES = {
    "fdtd_create_grid": [C.POINTER(GridDesc), C.POINTER(Allocator), _P, C.POINTER(_P)],
    "fdtd_destroy_grid": [_P],
    "fdtd_set_eps_from_spheres": [_P, _D, C.c_int64, _D, _D],
    "fdtd_set_material": [_P, C.POINTER(C.c_uint8)],
    "fdtd_get_material": [_P, C.POINTER(C.c_uint8)],
    "fdtd_set_gain": [_P, C.POINTER(GainParams)],
    "fdtd_add_source": [_P, C.POINTER(SourceDesc), C.POINTER(C.c_int32)],
    "fdtd_add_probe": [_P, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_int32)],
    "fdtd_add_flux_plane": [_P, C.c_int32, C.c_int32, C.c_double, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                            C.POINTER(C.c_int32)],
    "fdtd_set_launch": [_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32],
    "fdtd_set_kernel": [_P, C.c_int32],
    "fdtd_set_l2_residency": [_P, C.c_int32],
    "fdtd_kernel_in_use": [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
    "fdtd_autotune": [_P, C.c_int32, C.POINTER(TuneResult)],
    "fdtd_batch_autotune": [_P, C.c_int32, C.POINTER(TuneResult)],
    "fdtd_step_n": [_P, C.c_int64],
    "fdtd_sync": [_P],
    "fdtd_steps_done": [_P, C.POINTER(C.c_int64)],
    "fdtd_read_probes": [_P, C.c_int32, C.c_int64, C.c_int64, _D],
    "fdtd_read_flux": [_P, C.c_int32, C.c_int64, C.c_int64, _D],
    "fdtd_read_fields": [_P, C.c_int32, _D],
    "fdtd_write_fields": [_P, C.c_int32, _D],
    "fdtd_read_gain": [_P, C.c_int32, _D],
    "fdtd_field_energy": [_P, _D],
    "fdtd_set_timing": [_P, C.c_int32],
    "fdtd_kernel_time": [_P, _D, C.POINTER(C.c_int64)],
    "fdtd_set_step_limit": [_P, C.c_int64],
    "fdtd_set_wait_limit": [_P, C.c_int64],
    "fdtd_set_gain_coupling": [_P, C.c_int32],
    "fdtd_set_item_order": [_P, C.c_int32],
    "fdtd_set_absorber": [_P, C.c_int32],
    "fdtd_batch_create": [C.POINTER(_P), C.c_int32, _P, C.POINTER(_P)],
    "fdtd_batch_destroy": [_P],
    "fdtd_batch_set_launch": [_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32],
    "fdtd_batch_set_graph": [_P, C.c_int32],
    "fdtd_batch_step_n": [_P, C.c_int64],
    "fdtd_batch_sync": [_P],
    "fdtd_batch_set_timing": [_P, C.c_int32],
    "fdtd_batch_kernel_time": [_P, _D, C.POINTER(C.c_int64)],
    "fdtd_save_state": [_P, C.c_char_p],
    "fdtd_load_state": [_P, C.c_char_p],
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libfdtd.so and declare the exported signatures (raises if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FdtdError(-3, f"{path} is missing: build it with paper_0802_3775_gb300.build.build() "
                            "(the CUDA library is required; there is no CPU path)")
    lib = C.CDLL(path)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.fdtd_last_error.restype = C.c_char_p
    lib.fdtd_last_error.argtypes = []
    lib.fdtd_version.restype = C.c_char_p
    lib.fdtd_version.argtypes = []
    _lib = lib
    return lib


def check(code):
    if code != FDTD_OK:
        raise FdtdError(code, _lib.fdtd_last_error().decode())
    return code


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


class TorchAllocator:
    """Device memory from torch's caching allocator on a given stream."""

    def __init__(self, device=None, stream=None):
        import torch
        self.torch = torch
        self.device = torch.cuda.current_device() if device is None else device
        self.stream = stream
        self._sizes = {}

        def _alloc(nbytes, _stream, _ctx):
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
            except Exception:  # out of memory: the library reports FDTD_E_NOMEM
                return None
            return p

        def _free(ptr, _nbytes, _stream, _ctx):
            if ptr:
                torch.cuda.caching_allocator_delete(ptr)

        self._cb_alloc = ALLOC_FN(_alloc)
        self._cb_free = FREE_FN(_free)
        self.struct = Allocator(self._cb_alloc, self._cb_free, None)


class Grid:
    """One FDTD grid on the GPU (see include/fdtd.h for the semantics)."""

    def __init__(self, shape, res, *, a=480e-9, courant=0.5, npml=(0,) * 6, periodic=(False,) * 3,
                 precision="f32", eps=(1.0, 1.0, 1.0), cpml_m=3.0, cpml_sigma_factor=0.8, cpml_kappa_max=1.0,
                 cpml_alpha_max=0.05, cpml_f_hat=0.8, seed=0, record_capacity=1 << 16, stream=None,
                 allocator="torch"):
        self._lib = load_library()
        self.shape = tuple(int(s) for s in shape)
        self.precision = precision
        d = GridDesc()
        d.nx, d.ny, d.nz = self.shape
        for q in range(6):
            d.npml[q] = int(npml[q])
        for q in range(3):
            d.periodic[q] = int(bool(periodic[q]))
            d.eps[q] = float(eps[q])
        d.precision = FP32 if precision == "f32" else FP64
        d.reserved = 0
        d.res, d.a, d.courant = float(res), float(a), float(courant)
        d.cpml_m, d.cpml_sigma_factor, d.cpml_kappa_max = float(cpml_m), float(cpml_sigma_factor), float(cpml_kappa_max)
        d.cpml_alpha_max, d.cpml_f_hat = float(cpml_alpha_max), float(cpml_f_hat)
        d.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        d.record_capacity = int(record_capacity)
        self.desc = d
        self._alloc = None
        alloc_ptr = None
        st = None
        if stream is not None:
            st = int(getattr(stream, "cuda_stream", stream))
        if allocator == "torch":
            import torch
            if stream is None:
                stream = torch.cuda.current_stream()
                st = int(stream.cuda_stream)
            self._alloc = TorchAllocator(stream=stream)
            alloc_ptr = C.byref(self._alloc.struct)
        self.stream_ptr = st
        h = C.c_void_p()
        check(self._lib.fdtd_create_grid(C.byref(d), alloc_ptr, C.c_void_p(st) if st else None, C.byref(h)))
        self.h = h
        self.nprobe = 0
        self.nflux = 0

    # -- set-up
    @classmethod
    def from_spec(cls, spec, precision=None, **kw):
        """Grid + geometry + gain + sources + observers from a run record."""
        g = cls(spec.shape, spec.res, a=spec.a, courant=spec.courant, npml=spec.npml, periodic=spec.periodic,
                precision=precision or spec.precision, eps=spec.eps, cpml_m=spec.cpml_m,
                cpml_sigma_factor=spec.cpml_sigma_factor, cpml_kappa_max=spec.cpml_kappa_max,
                cpml_alpha_max=spec.cpml_alpha_max, cpml_f_hat=spec.cpml_f_hat, seed=spec.seed, **kw)
        if getattr(spec, "absorber", "cpml") != "cpml":
            g.set_absorber(spec.absorber)
        if spec.spheres is not None:
            g.set_eps_from_spheres(spec.spheres, spec.box_lo, spec.box_hi)
        if spec.gain is not None:
            g.set_gain(spec.gain)
        for s in spec.sources:
            g.add_source(s)
        if spec.probes is not None:
            for p in np.asarray(spec.probes).reshape(-1, 3):
                g.add_probe(*[int(v) for v in p])
        for f in spec.fluxes:
            g.add_flux(f.axis, f.index, f.sign, f.u, f.v)
        return g

    def set_eps_from_spheres(self, spheres, box_lo, box_hi):
        sp = np.ascontiguousarray(np.asarray(spheres, dtype=np.float64).reshape(-1, 4))
        lo = np.ascontiguousarray(box_lo, dtype=np.float64)
        hi = np.ascontiguousarray(box_hi, dtype=np.float64)
        check(self._lib.fdtd_set_eps_from_spheres(self.h, _dptr(sp), sp.shape[0], _dptr(lo), _dptr(hi)))

    def set_material(self, mat):
        m = np.ascontiguousarray(mat, dtype=np.uint8)
        check(self._lib.fdtd_set_material(self.h, m.ctypes.data_as(C.POINTER(C.c_uint8))))

    def get_material(self):
        nx, ny, nz = self.shape
        m = np.empty((nz, ny, nx), dtype=np.uint8)
        check(self._lib.fdtd_get_material(self.h, m.ctypes.data_as(C.POINTER(C.c_uint8))))
        return m

    def set_gain(self, g):
        p = GainParams(g.n_total, g.fa_hat, g.dw_rel, g.tau32, g.tau21, g.tau10, g.pump, g.kappa, g.noise_amp,
                       0 if g.init == "steady" else 1)
        check(self._lib.fdtd_set_gain(self.h, C.byref(p)))
        coupling = getattr(g, "coupling", "cell")
        if coupling != "cell":
            self.set_gain_coupling(coupling)

    def set_gain_coupling(self, coupling):
        """"cell" (P on each cell's own E nodes) or "centred" (P at the cell centre)."""
        check(self._lib.fdtd_set_gain_coupling(self.h, {"cell": 0, "centred": 1}[coupling]))

    def add_source(self, s):
        d = SourceDesc(0 if s.kind == "point" else 1, s.comp, *[int(v) for v in s.pos], s.axis, s.index,
                       s.waist, s.f0_hat, s.rel_bw, s.t0_steps, s.amplitude)
        i = C.c_int32()
        check(self._lib.fdtd_add_source(self.h, C.byref(d), C.byref(i)))
        return i.value

    def add_probe(self, i, j, k):
        out = C.c_int32()
        check(self._lib.fdtd_add_probe(self.h, int(i), int(j), int(k), C.byref(out)))
        self.nprobe += 1
        return out.value

    def add_flux(self, axis, index, sign=1.0, u=(0, 0), v=(0, 0)):
        out = C.c_int32()
        check(self._lib.fdtd_add_flux_plane(self.h, int(axis), int(index), float(sign), int(u[0]), int(u[1]),
                                            int(v[0]), int(v[1]), C.byref(out)))
        self.nflux += 1
        return out.value

    def set_launch(self, bx=32, by=8, zdepth=0, grid_blocks=0):
        check(self._lib.fdtd_set_launch(self.h, int(bx), int(by), int(zdepth), int(grid_blocks)))

    def set_absorber(self, absorber):
        """"cpml" (default) or "upml" (uniaxial PML on the same grading; passive grids)."""
        check(self._lib.fdtd_set_absorber(self.h, {"cpml": 0, "upml": 1}[absorber]))

    def set_item_order(self, order):
        """"costliest" (slab items first) or "z" (plain z order) for the single-node kernels."""
        check(self._lib.fdtd_set_item_order(self.h, {"costliest": 0, "z": 1}[order]))

    def set_kernel(self, kind):
        """0 automatic, 1 plain-load step kernel, 2 TMA-staged step kernel,
        3 paired TMA-staged kernel (binary32 grids)."""
        kinds = {"auto": 0, "plain": 1, "tma": 2, "pair": 3}
        check(self._lib.fdtd_set_kernel(self.h, int(kinds.get(kind, kind))))

    def set_l2_residency(self, on):
        """Keep the CPML memory in a persisting L2 window (default on)."""
        check(self._lib.fdtd_set_l2_residency(self.h, 1 if on else 0))

    def autotune(self, trial_steps=10):
        """Time the candidate launch shapes from the current state (restored
        after every trial) and keep the fastest; returns the choice."""
        r = TuneResult()
        check(self._lib.fdtd_autotune(self.h, int(trial_steps), C.byref(r)))
        return {k: getattr(r, k) for k, _ in TuneResult._fields_}

    def kernel_in_use(self):
        """(kind, rows): the step kernel of the grid's launches (1 plain, 2 TMA,
        3 paired) and the rows of its tile; valid after the first step."""
        kind, rows = C.c_int32(), C.c_int32()
        check(self._lib.fdtd_kernel_in_use(self.h, C.byref(kind), C.byref(rows)))
        return int(kind.value), int(rows.value)

    def set_step_limit(self, limit):
        check(self._lib.fdtd_set_step_limit(self.h, int(limit)))

    def set_wait_limit(self, ns):
        """Limit (ns) of the TMA step kernels' bounded waits; 0 gives up at once."""
        check(self._lib.fdtd_set_wait_limit(self.h, int(ns)))

    # -- stepping
    def step(self, n=1):
        check(self._lib.fdtd_step_n(self.h, int(n)))

    def sync(self):
        check(self._lib.fdtd_sync(self.h))

    @property
    def steps_done(self):
        n = C.c_int64()
        check(self._lib.fdtd_steps_done(self.h, C.byref(n)))
        return n.value

    def set_timing(self, on=True, every=1):
        """Bracket every `every`-th step-kernel launch with CUDA events (off: on=False)."""
        check(self._lib.fdtd_set_timing(self.h, int(every) if on else 0))

    def kernel_time(self):
        """(summed step-kernel milliseconds, launches) since timing was switched on."""
        ms = C.c_double()
        n = C.c_int64()
        check(self._lib.fdtd_kernel_time(self.h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    # -- read-backs
    def read_probes(self, pid=None, t0=0, count=None):
        """float64[count, 3] for one probe, or [count, nprobe, 3] for all."""
        n = self.steps_done
        if count is None:
            count = n - t0
        if pid is None:
            out = np.empty((count, self.nprobe, 3))
            for p in range(self.nprobe):
                out[:, p, :] = self.read_probes(p, t0, count)
            return out
        out = np.empty((count, 3))
        check(self._lib.fdtd_read_probes(self.h, int(pid), int(t0), int(count), _dptr(out)))
        return out

    def read_flux(self, fid=None, t0=0, count=None):
        """float64[count] for one plane, or [nflux, count] for all."""
        n = self.steps_done
        if count is None:
            count = n - t0
        if fid is None:
            return np.stack([self.read_flux(f, t0, count) for f in range(self.nflux)]) if self.nflux else np.empty((0, count))
        out = np.empty(count)
        check(self._lib.fdtd_read_flux(self.h, int(fid), int(t0), int(count), _dptr(out)))
        return out

    def read_fields(self):
        """float64[6, nz, ny, nx]: Ex, Ey, Ez, H~x, H~y, H~z."""
        nx, ny, nz = self.shape
        out = np.empty((6, nz, ny, nx))
        for c in range(6):
            check(self._lib.fdtd_read_fields(self.h, c, _dptr(out[c])))
        return out

    def write_fields(self, F):
        F = np.ascontiguousarray(F, dtype=np.float64)
        for c in range(6):
            check(self._lib.fdtd_write_fields(self.h, c, _dptr(np.ascontiguousarray(F[c]))))

    def read_gain(self, what):
        nx, ny, nz = self.shape
        out = np.empty((3, nz, ny, nx))
        check(self._lib.fdtd_read_gain(self.h, int(what), _dptr(out)))
        return out

    def field_energy(self):
        v = C.c_double()
        check(self._lib.fdtd_field_energy(self.h, C.byref(v)))
        return v.value

    def save_state(self, path):
        check(self._lib.fdtd_save_state(self.h, str(path).encode()))

    def load_state(self, path):
        check(self._lib.fdtd_load_state(self.h, str(path).encode()))

    def close(self):
        if getattr(self, "h", None):
            self._lib.fdtd_destroy_grid(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


KERNELS = {"auto": 0, "plain": 1, "tma": 2, "pair": 3}


class Batch:
    """Many grids stepped together: one step-kernel launch per time step over
    the work items of every member (see fdtd_batch_* in include/fdtd.h)."""

    def __init__(self, grids, stream=None):
        self._lib = load_library()
        self.grids = list(grids)
        if stream is None:
            stream = self.grids[0].stream_ptr
        st = int(getattr(stream, "cuda_stream", stream)) if stream else None
        arr = (_P * len(self.grids))(*[g.h.value for g in self.grids])
        h = C.c_void_p()
        check(self._lib.fdtd_batch_create(arr, len(self.grids), C.c_void_p(st) if st else None, C.byref(h)))
        self.h = h

    def set_launch(self, kernel="auto", by=0, zdepth=0, grid_blocks=0):
        check(self._lib.fdtd_batch_set_launch(self.h, int(KERNELS.get(kernel, kernel)), int(by), int(zdepth),
                                              int(grid_blocks)))

    def set_graph(self, steps_per_graph):
        check(self._lib.fdtd_batch_set_graph(self.h, int(steps_per_graph)))

    def autotune(self, trial_steps=5):
        """As Grid.autotune over the batch's launch shapes (every member restored)."""
        r = TuneResult()
        check(self._lib.fdtd_batch_autotune(self.h, int(trial_steps), C.byref(r)))
        return {k: getattr(r, k) for k, _ in TuneResult._fields_}

    def step(self, n=1):
        check(self._lib.fdtd_batch_step_n(self.h, int(n)))

    def sync(self):
        check(self._lib.fdtd_batch_sync(self.h))

    def set_timing(self, on=True, every=1):
        """Bracket every `every`-th step-kernel launch with CUDA events (off: on=False)."""
        check(self._lib.fdtd_batch_set_timing(self.h, int(every) if on else 0))

    def kernel_time(self):
        ms = C.c_double()
        n = C.c_int64()
        check(self._lib.fdtd_batch_kernel_time(self.h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def close(self):
        if getattr(self, "h", None):
            self._lib.fdtd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
