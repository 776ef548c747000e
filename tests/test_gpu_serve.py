"""Request server: continuous batching under an HBM budget.

A run's results are the same whether it runs alone or shares the GPU with
other runs admitted while it is resident; admission respects the budget and
slot count; requests that can never fit are refused."""
import time

import numpy as np
import pytest

from helpers import small_opal
from paper_0802_3775_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0802_3775_gb300 import build
    build.build()


def _mix():
    gain = inputs.GainSpec(pump=5e11, noise_amp=1e-3, init="ground")
    return [small_opal(n_cells=2, res=8, npml=5, precision="f32", source="sheet", seed=1),
            small_opal(n_cells=2, res=10, npml=6, precision="f32", source="dipole", gain=gain, seed=2),
            small_opal(n_cells=3, res=7, npml=4, precision="f32", source="sheet", gain=gain, seed=3),
            inputs.opal_planewave_f32(ncell=2, res=9, npml=5, sigma=0.04, realization=7)]


def test_result_alone_equals_result_in_the_mix():
    from paper_0802_3775_gb300.serve import Server
    specs = _mix()
    steps = [130, 70, 95, 160]
    srv = Server(hbm_budget_bytes=8 << 30, max_slots=8, steps_per_chunk=40)
    t = srv.submit(specs[1], steps=steps[1])
    srv.wait(t)
    alone = (srv.probes(t), srv.flux(t), srv.poll(t).field_energy)
    srv.close()

    srv = Server(hbm_budget_bytes=8 << 30, max_slots=8, steps_per_chunk=40)
    tickets = [srv.submit(specs[0], steps=steps[0])]
    time.sleep(0.05)
    tickets.append(srv.submit(specs[2], steps=steps[2]))
    tickets.append(srv.submit(specs[1], steps=steps[1]))   # joins while others are resident
    tickets.append(srv.submit(specs[3], steps=steps[3]))
    for t in tickets:
        srv.wait(t)
    mixed = (srv.probes(tickets[2]), srv.flux(tickets[2]), srv.poll(tickets[2]).field_energy)
    assert np.array_equal(mixed[0], alone[0])
    assert np.array_equal(mixed[1], alone[1])
    assert mixed[2] == alone[2]
    st = srv.stats()
    assert st["completed"] == 4 and st["failed"] == 0 and st["used_bytes"] == 0
    srv.close()


def test_admission_respects_budget_and_slots():
    from paper_0802_3775_gb300.serve import Server
    specs = _mix()
    srv = Server(hbm_budget_bytes=8 << 30, max_slots=2, steps_per_chunk=25)
    tickets = [srv.submit(s, steps=60) for s in specs + specs]
    seen_resident = 0
    while True:
        st = srv.stats()
        seen_resident = max(seen_resident, st["resident"])
        assert st["resident"] <= 2
        if st["completed"] + st["failed"] == len(tickets):
            break
        time.sleep(0.01)
    assert srv.stats()["failed"] == 0
    for t in tickets:
        r = srv.poll(t)
        assert r.status == 0 and r.admit_s >= r.submit_s and r.done_s >= r.admit_s
    srv.close()


def test_request_that_never_fits_is_refused():
    from paper_0802_3775_gb300.fdtd import FdtdError
    from paper_0802_3775_gb300.serve import Server
    srv = Server(hbm_budget_bytes=1 << 20, max_slots=4, steps_per_chunk=10)
    with pytest.raises(FdtdError) as e:
        srv.submit(_mix()[0], steps=10)
    assert e.value.code == -8
    srv.close()


def test_poll_pending_and_timeout():
    from paper_0802_3775_gb300.serve import Server
    spec = inputs.opal_planewave_f32(ncell=3, res=16, npml=8, sigma=0.02, realization=1)
    srv = Server(hbm_budget_bytes=8 << 30, max_slots=4, steps_per_chunk=200)
    t = srv.submit(spec, steps=4000)
    r = srv.poll(t, 0)
    assert r.status == -6
    r = srv.wait(t, timeout_s=300)
    assert r.status == 0 and r.steps == 4000
    srv.close()
