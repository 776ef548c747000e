"""The C ABI library loads and exports every function that include/fdtd.h
declares; argument checks that need no GPU return the documented codes."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in ("fdtd.h",):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(fdtd_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_0802_3775_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fdtd_create_grid", "fdtd_set_eps_from_spheres", "fdtd_set_gain", "fdtd_add_source",
                     "fdtd_step_n", "fdtd_read_probes"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_null_and_range_checks_without_gpu(lib):
    from paper_0802_3775_gb300 import fdtd as F
    L = F.load_library()
    # null arguments are rejected before any device work
    assert L.fdtd_create_grid(None, None, None, None) == -1
    assert L.fdtd_step_n(None, 1) == -1
    assert b"null" in L.fdtd_last_error()
    d = F.GridDesc()
    d.nx = d.ny = d.nz = 8
    d.res, d.a, d.courant = 10.0, 480e-9, 0.5
    d.eps[0] = d.eps[1] = d.eps[2] = 1.0
    d.cpml_kappa_max = 1.0
    d.record_capacity = 16
    d.periodic[0] = 1
    d.npml[0] = 2
    h = ctypes.c_void_p()
    assert L.fdtd_create_grid(ctypes.byref(d), None, None, ctypes.byref(h)) == -1  # slab on a periodic axis
    d.periodic[0] = 0
    d.npml[0] = 8
    assert L.fdtd_create_grid(ctypes.byref(d), None, None, ctypes.byref(h)) == -1  # slab fills the axis
    d.npml[0] = 2
    d.courant = 1.5
    assert L.fdtd_create_grid(ctypes.byref(d), None, None, ctypes.byref(h)) == -1  # unstable step
    assert L.fdtd_destroy_grid(None) == 0
    assert L.fdtd_version().startswith(b"fdtd-gb300")
    # the variant and launch options reject a null grid before looking at anything else
    for fn, arg in (("fdtd_set_gain_coupling", 1), ("fdtd_set_absorber", 1), ("fdtd_set_item_order", 1),
                    ("fdtd_set_wait_limit", 0), ("fdtd_set_l2_residency", 1)):
        assert getattr(L, fn)(None, arg) == -1, fn
        assert b"null" in L.fdtd_last_error()
    # the allocation-free energy checks its arguments before touching the device
    six = (ctypes.c_void_p * 6)(*([None] * 6))
    eps = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    out = ctypes.c_double()
    assert L.fdtd_field_energy_noalloc(six, None, 8, 8, 8, 8, 0, eps, ctypes.c_double(1e-8), None,
                                       ctypes.byref(out)) == -1


def test_create_without_device_fails_loudly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_0802_3775_gb300 import fdtd as F
    with pytest.raises(F.FdtdError) as e:
        F.Grid((8, 8, 8), 10, allocator=None)
    assert e.value.code == -3


def test_batch_and_server_checks_without_gpu(lib):
    import ctypes as C

    from paper_0802_3775_gb300 import fdtd as F
    from paper_0802_3775_gb300 import serve as S
    L = S._lib()
    h = C.c_void_p()
    # batches: null handles and empty member lists
    assert L.fdtd_batch_create(None, 0, None, C.byref(h)) == -1
    assert L.fdtd_batch_set_launch(None, 0, 0, 0, 0) == -1
    assert L.fdtd_batch_step_n(None, 1) == -1
    assert L.fdtd_batch_sync(None) == -1
    assert L.fdtd_batch_destroy(None) == 0
    # server: null arguments and a description that admits nothing
    assert L.fdtd_server_create(None, None, C.byref(h)) == -1
    for bad in (S.ServerDesc(0, 4, 10, F.FP32, 0), S.ServerDesc(1 << 30, 0, 10, F.FP32, 0),
                S.ServerDesc(1 << 30, 4, 0, F.FP32, 0)):
        assert L.fdtd_server_create(C.byref(bad), None, C.byref(h)) == -1
        assert b"positive" in L.fdtd_last_error()
    t = C.c_uint64()
    res = S.Result()
    assert L.fdtd_submit(None, None, C.byref(t)) == -1
    assert L.fdtd_poll(None, 0, C.byref(res), 0) == -1
    assert L.fdtd_result_probes(None, 0, None) == -1
    assert L.fdtd_result_flux(None, 0, None) == -1
    assert L.fdtd_result_release(None, 0) == -1
    assert L.fdtd_server_get_stats(None, None) == -1
    assert L.fdtd_server_destroy(None) == 0


def test_server_without_device_fails_loudly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_0802_3775_gb300 import fdtd as F
    from paper_0802_3775_gb300.serve import Server
    with pytest.raises(F.FdtdError) as e:
        Server(hbm_budget_bytes=1 << 30, max_slots=2, steps_per_chunk=10)
    assert e.value.code == -3
