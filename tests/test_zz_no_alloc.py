"""pm_shrink_static, the compaction entry point for callers that cannot
allocate device memory (hosts that fix the library's memory budget, loops
that cannot afford cudaMalloc's implicit synchronisation), gives the same
survivors and leavers as pm_shrink, call after call.

Collected last on purpose, so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1709_04703_gb300 import _lib as L  # noqa: E402
from paper_1709_04703_gb300 import ics  # noqa: E402

OM, OL = 0.3, 0.7


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_04703_gb300 import build
    build.build()
    return L.load()


def _ctx_shrink(pos, mom, ids, n, box, a):
    """Survivors and leavers from the existing entry point, pm_shrink."""
    from paper_1709_04703_gb300.sim import Sim
    sim = Sim(pos, mom, ids, n, box, 0.5, 1.0, 10)
    kept = sim.shrink(a)
    sp, sm, si = sim.particles()
    lp, lm, li, la = sim.lightcone()
    sim.close()
    return kept, (sp, sm, si), (lp, lm, li, la)


def _static_shrink(lib, pos, mom, ids, n, box, a):
    from paper_1709_04703_gb300.sim import pack, unpack
    p4, m4 = pack(pos, mom, ids)
    N = len(pos)
    dp, dm = torch.from_numpy(p4).cuda(), torch.from_numpy(m4).cuda()
    kp, km = torch.empty_like(dp), torch.empty_like(dm)
    lp, lm = torch.empty_like(dp), torch.empty_like(dm)
    torch.cuda.synchronize()
    nk = C.c_int64(-1)
    code = lib.pm_shrink_static(C.c_void_p(dp.data_ptr()), C.c_void_p(dm.data_ptr()), N, n,
                                box, OM, OL, 1.0, a, C.c_void_p(kp.data_ptr()),
                                C.c_void_p(km.data_ptr()), C.c_void_p(lp.data_ptr()),
                                C.c_void_p(lm.data_ptr()), C.byref(nk), None)
    assert code == L.PM_OK, lib.pm_shrink_static_error()
    k = nk.value
    keep = unpack(kp[:k].cpu().numpy(), km[:k].cpu().numpy())
    leave = unpack(lp[:N - k].cpu().numpy(), lm[:N - k].cpu().numpy())
    return k, keep, leave


def test_static_compaction_matches_pm_shrink_twice(lib):
    n, box = 64, 8000.0
    for call, (N, seed, a) in enumerate([(300001, 11, 0.7), (123457, 12, 0.85)]):
        pos, mom, ids = ics.random_particles(N, n, seed)
        kept, (sp, sm, si), (lp, lm, li, la) = _ctx_shrink(pos, mom, ids, n, box, a)
        k, keep, leave = _static_shrink(lib, pos, mom, ids, n, box, a)
        assert 0 < k < N, call
        assert k == kept
        # bit-exact, the tolerance of every compaction test
        np.testing.assert_array_equal(keep[0], sp)
        np.testing.assert_array_equal(keep[1], sm)
        np.testing.assert_array_equal(keep[2], si)
        np.testing.assert_array_equal(leave[0], lp)
        np.testing.assert_array_equal(leave[1], lm)
        np.testing.assert_array_equal(leave[2], li)
        np.testing.assert_array_equal(leave[3], la)


def test_static_compaction_rejects_oversized_input(lib):
    nk = C.c_int64(-1)
    big = L.PM_SHRINK_STATIC_MAX_PARTICLES + 1
    dummy = torch.zeros(4, device="cuda")
    ptr = C.c_void_p(dummy.data_ptr())
    code = lib.pm_shrink_static(ptr, ptr, big, 64, 8000.0, OM, OL, 1.0, 0.7, ptr, ptr, ptr,
                                ptr, C.byref(nk), None)
    assert code == L.PM_EINVAL
    assert b"exceeds the static scratch limit" in lib.pm_shrink_static_error()
    assert nk.value == -1
