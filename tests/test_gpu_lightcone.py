"""The fixed-box run with a lightcone record (PM_SHRINK_RECORD, the run the
paper compares the shrinking one with, Sec. 3.3) on the GPU: against the
oracle's record-only run, and against the shrinking run when gravity is off
(then the two catalogues are the same)."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import cosmology as cz  # noqa: E402
from oracle import pm as opm  # noqa: E402
from paper_1709_04703_gb300 import ics  # noqa: E402

OM, OL = 0.3, 0.7


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_04703_gb300 import build
    build.build()


def _run(pos, mom, ids, n, box, a0, steps, shrink, bc, om=OM, rtol=1e-8):
    from paper_1709_04703_gb300.sim import Sim
    sim = Sim(pos, mom, ids, n, box, a0, 1.0, steps, rtol=rtol, shrink=shrink, bc=bc,
              omega_m=om, omega_l=1 - om)
    sim.step(steps)
    st = sim.stats()
    act = sim.particles()
    lc = sim.lightcone()
    sim.close()
    return st, act, lc


def test_record_matches_oracle():
    """32^3 Zel'dovich particles, 4000 Mpc/h, a 0.5 -> 1 in 8 steps (open from
    the first step): the catalogue matches the oracle's, particle for particle
    but for the few within float rounding of the keep boundary."""
    n, box, a0, steps = 32, 4000.0, 0.5, 8
    pos, mom, ids = ics.zeldovich(n, -2.0, None, 5, a0)
    st, (gp, gm, gi), (cp, cm, ci, ca) = _run(pos, mom, ids, n, box, a0, steps, "record",
                                              "periodic")
    assert st["n_active"] == n**3 and st["n_lightcone"] == len(ci)
    assert len(np.unique(ci)) == len(ci)
    np.testing.assert_array_equal(gi, ids)            # nobody moves in the active set
    sched = cz.schedule(n, box, OM, OL, a0, 1.0, steps)
    out = opm.run(pos, mom, ids, sched, n, OM, 1.0, record_only=True)
    common, gi_idx, oi_idx = np.intersect1d(ci, out["lc_ids"], return_indices=True)
    assert len(ci) - len(common) <= 3 and len(out["lc_ids"]) - len(common) <= 3
    assert len(common) > n**3 // 2
    # the record's a is the oracle's for the common particles but for
    # boundary cases; positions agree to the step's force tolerance
    same_a = ca[gi_idx] == out["lc_a"][oi_idx].astype(np.float32)
    assert same_a.mean() > 0.999
    d = np.abs(cp[gi_idx][same_a].astype(np.float64) - out["lc_pos"][oi_idx][same_a])
    d = np.minimum(d, n - d)
    assert d.max() < 1e-3
    # the ids in each record step come in index order
    for a in np.unique(ca):
        assert np.all(np.diff(ci[ca == a]) > 0)


def test_record_equals_shrink_without_gravity():
    """Omega_m = 1e-6: the source, and with it the kick, is a millionth of
    the usual one, so trajectories do not depend on the boundary: the
    fixed-box catalogue is the shrinking run's lightcone (same particles and
    a but for float ties at the keep boundary, positions to float rounding)."""
    n, box, a0, steps, om = 32, 4000.0, 0.5, 10, 1e-6
    pos, mom, ids = ics.zeldovich(n, -2.0, None, 6, a0, om=om, ol=1 - om)
    mom = mom + np.float32(0.02) * np.sign(pos - n / 2).astype(np.float32)
    _, _, (sp, sm, si, sa) = _run(pos, mom, ids, n, box, a0, steps, True, "paper", om=om)
    _, _, (rp, rm, ri, ra) = _run(pos, mom, ids, n, box, a0, steps, "record", "periodic",
                                  om=om)
    assert len(si) > n**3 // 4
    common, i_s, i_r = np.intersect1d(si, ri, return_indices=True)
    assert len(si) - len(common) <= 2 and len(ri) - len(common) <= 2
    assert np.mean(sa[i_s] == ra[i_r]) > 0.999
    same = sa[i_s] == ra[i_r]
    np.testing.assert_allclose(rp[i_r][same], sp[i_s][same], rtol=0, atol=1e-4)
    np.testing.assert_allclose(rm[i_r][same], sm[i_s][same], rtol=0, atol=1e-6)


def test_record_marks_cleared_at_init_kept_by_set_particles():
    """pm_init clears mom.w in the record mode (every particle can be
    recorded once); pm_set_particles takes the marks as given."""
    from paper_1709_04703_gb300 import _lib as L
    from paper_1709_04703_gb300.sim import Sim, pack
    n, box, a0, steps = 16, 8000.0, 0.6, 4
    pos, mom, ids = ics.zeldovich(n, -2.0, None, 7, a0)
    marked = pack(pos, mom, ids, extra=np.full(len(pos), 0.25, np.float32))
    ref = Sim(pos, mom, ids, n, box, a0, 1.0, steps, shrink="record", bc="periodic")
    lib = ref._lib
    # the same configuration initialised from marked records
    ctx = C.c_void_p()
    s = torch.cuda.Stream()
    L.check(lib.pm_init(C.byref(ref.cfg), marked[0].ctypes.data, marked[1].ctypes.data, 1,
                        C.c_void_p(s.cuda_stream), C.byref(ctx)), None)
    L.check(lib.pm_step(ctx, steps), ctx)
    st = L.PmStats()
    L.check(lib.pm_stats(ctx, C.byref(st)), ctx)
    lib.pm_destroy(ctx)
    ref.step(steps)
    n_ref = ref.stats()["n_lightcone"]
    assert n_ref > 0 and st.n_lightcone == n_ref
    ref.close()
    # marks set through pm_set_particles: nothing is recorded
    sim = Sim(pos, mom, ids, n, box, a0, 1.0, steps, shrink="record", bc="periodic")
    L.check(lib.pm_set_particles(sim._ctx, marked[0].ctypes.data, marked[1].ctypes.data,
                                 len(pos), 1), sim._ctx)
    sim.step(steps)
    assert sim.stats()["n_lightcone"] == 0
    sim.close()


def test_batch_rejects_the_record_mode():
    from paper_1709_04703_gb300 import _lib as L
    from paper_1709_04703_gb300.sim import _config, pack
    lib = L.load()
    n = 16
    pos, mom, ids = ics.zeldovich(n, -2.0, None, 8, 0.5)
    cfg = _config(n, n**3, 1000.0, 0.5, 1.0, 4, shrink="record", bc="periodic")
    cfgs = (L.PmConfig * 1)(cfg)
    p4, m4 = pack(pos, mom, ids)
    pp = (C.c_void_p * 1)(p4.ctypes.data)
    mm = (C.c_void_p * 1)(m4.ctypes.data)
    b = C.c_void_p()
    s = torch.cuda.Stream()
    code = lib.pm_batch_init(1, cfgs, pp, mm, 1, C.c_void_p(s.cuda_stream), C.byref(b))
    assert code == L.PM_EINVAL
