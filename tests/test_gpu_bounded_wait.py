"""The step kernels' bounded waits, made to run out on a healthy run.

Every wait of the TMA-staged step kernels for a staged plane has a time
limit; when one runs out the kernel lets its copies in flight land, stops its
block and flags the grid, and the host reports FDTD_E_TIMEOUT at the next
synchronization -- no trap, no hang, and the CUDA context stays usable.  A
wait limit of 0 makes every wait give up at once without looking at the copy,
so this test drives that path with no fault of any kind: the grid reports the
timeout, and a fresh grid stepped afterwards in the same process still
matches a grid stepped before."""
import numpy as np
import pytest

from helpers import gpu_grid, small_opal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0802_3775_gb300 import build
    build.build()


@pytest.mark.parametrize("kernel", ["pair", "tma"])
def test_a_wait_that_runs_out_is_reported_and_the_context_survives(kernel):
    from paper_0802_3775_gb300.fdtd import FdtdError
    spec = small_opal(precision="f32", source="sheet")
    ref = gpu_grid(spec)
    ref.set_kernel(kernel)
    ref.step(20)
    F_ref = ref.read_fields()
    ref.close()

    g = gpu_grid(spec)
    g.set_kernel(kernel)
    g.set_wait_limit(0)
    g.step(3)
    with pytest.raises(FdtdError) as e:
        g.sync()
    assert e.value.code == -7  # FDTD_E_TIMEOUT
    g.close()

    h = gpu_grid(spec)
    h.set_kernel(kernel)
    h.set_wait_limit(2_000_000_000)
    h.step(20)
    h.sync()
    assert np.array_equal(h.read_fields(), F_ref)
    h.close()
