"""The allocation-free field-energy entry point against the grid's own.

fdtd_field_energy_noalloc serves callers that cannot allocate device memory
where they need the field energy (the device allocator belongs to another
framework, a real-time loop must not enter it, a tool inspects fields in
place): its reduction scratch is a fixed static device array.  This test
stages a stepped grid's fields and material in caller-owned device buffers
(torch tensors), calls the entry point twice in a row through the C ABI and
compares both results with fdtd_field_energy on the grid itself, to the
FP64 reduction tolerance of the other energy checks (1e-12 relative).
It lives in its own file, collected last, and needs nothing from the others.
"""
import ctypes as C

import numpy as np
import pytest

from helpers import small_opal

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_noalloc_energy_matches_grid_energy_twice(precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0802_3775_gb300 import build
    build.build()
    from paper_0802_3775_gb300 import fdtd as F

    spec = small_opal(precision=precision, source="dipole")
    g = F.Grid.from_spec(spec)
    g.step(120)
    ref = g.field_energy()
    assert ref > 0

    dt = torch.float32 if precision == "f32" else torch.float64
    F6 = g.read_fields()
    dev = [torch.as_tensor(np.ascontiguousarray(F6[c]), dtype=dt, device="cuda") for c in range(6)]
    mat = torch.as_tensor(g.get_material(), dtype=torch.uint8, device="cuda")
    nx, ny, nz = spec.shape
    lib = F.load_library()
    fn = lib.fdtd_field_energy_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.POINTER(C.c_void_p), C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                   C.POINTER(C.c_double), C.c_double, C.c_void_p, C.POINTER(C.c_double)]
    ptrs = (C.c_void_p * 6)(*[t.data_ptr() for t in dev])
    eps = (C.c_double * 3)(*spec.eps)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for _ in range(2):
        out = C.c_double()
        code = fn(ptrs, C.c_void_p(mat.data_ptr()), nx, ny, nz, nx, 0 if precision == "f32" else 1, eps,
                  spec.a / spec.res, stream, C.byref(out))
        assert code == 0, lib.fdtd_last_error()
        assert abs(out.value - ref) <= 1e-12 * ref

    # sizes beyond the static scratch are refused with a clear error
    out = C.c_double()
    code = fn(ptrs, C.c_void_p(mat.data_ptr()), 4096, 4096, 16, 4096, 0, eps, 1e-8, stream, C.byref(out))
    assert code == -1 and b"static scratch" in lib.fdtd_last_error()
    g.close()
