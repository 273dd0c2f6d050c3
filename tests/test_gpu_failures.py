"""Failure detection without a GPU fault: the bounded device wait of the
tensor-core kernels gives up and reports PM_ETIMEOUT (a barrier that nothing
arrives at), an allocation failure injected on the host gives PM_ENOMEM
with everything freed, and a solve held to too few V-cycles gives
PM_ENOCONV; after each the GPU and the library stay usable."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1709_04703_gb300 import ics  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_04703_gb300 import build
    from paper_1709_04703_gb300 import _lib as L
    build.build()
    return L.load()


def _deposit_ok():
    from oracle import pm as opm
    from paper_1709_04703_gb300.sim import deposit, pack
    pos, _, _ = ics.random_particles(5000, 16, 1)
    p4, _ = pack(pos, np.zeros_like(pos))
    rho, _ = deposit(torch.from_numpy(p4).cuda(), 16)
    np.testing.assert_array_equal(rho.cpu().numpy(), opm.deposit(pos, 16, 0, 16, True)[0])


def test_bounded_wait_gives_up_and_reports_timeout(lib):
    from paper_1709_04703_gb300 import _lib as L
    assert lib.pm_selftest_wait(1, 1000, None) == L.PM_OK
    assert lib.pm_selftest_wait(0, 1000, None) == L.PM_ETIMEOUT
    assert b"gave up" in lib.pm_last_error(None)
    assert lib.pm_selftest_wait(0, 0, None) == L.PM_EINVAL
    _deposit_ok()


@pytest.mark.parametrize("k", [1, 4, 9, 17])
def test_injected_allocation_failure(lib, monkeypatch, k):
    from paper_1709_04703_gb300 import _lib as L
    from paper_1709_04703_gb300.sim import Sim
    pos, mom, ids = ics.zeldovich(16, -1.5, 0.5, 1, 0.5)
    Sim(pos, mom, ids, 16, 500.0, 0.5, 1.0, 4).close()  # modules loaded, pools warm
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    monkeypatch.setenv("PM_FAULT_ALLOC", str(k))
    with pytest.raises(L.PmError) as e:
        Sim(pos, mom, ids, 16, 500.0, 0.5, 1.0, 4)
    assert e.value.code == L.PM_ENOMEM and "injected" in str(e.value)
    monkeypatch.delenv("PM_FAULT_ALLOC")
    torch.cuda.synchronize()
    # what the failed pm_init allocated was freed
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20)
    sim = Sim(pos, mom, ids, 16, 500.0, 0.5, 1.0, 4)
    sim.step(4)
    assert sim.stats()["step"] == 4
    sim.close()


def test_solve_without_enough_vcycles_reports_noconv(lib):
    from paper_1709_04703_gb300 import _lib as L
    from paper_1709_04703_gb300.sim import Sim
    pos, mom, ids = ics.zeldovich(32, -1.5, 0.5, 2, 0.1)
    sim = Sim(pos, mom, ids, 32, 500.0, 0.1, 1.0, 8, rtol=1e-13, max_vcycles=1)
    with pytest.raises(L.PmError) as e:
        sim.step(1)
    assert e.value.code == L.PM_ENOCONV and "after 1 V-cycles" in str(e.value)
    st = sim.stats()
    assert st["resid_last"] > 1e-13 and st["vcycles_last"] == 1
    sim.close()
    _deposit_ok()
