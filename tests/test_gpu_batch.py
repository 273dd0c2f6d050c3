"""Batched step (pm_batch_*): many realisations of different mesh sizes,
boxes and lightcone schedules advanced by one launch per phase must give,
bit for bit, what separate contexts give for each realisation."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1709_04703_gb300 import ics  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_04703_gb300 import build
    build.build()


def _realisation(n, box, seed, a0):
    pos, mom, ids = ics.zeldovich(n, -1.5, 0.5, seed, a0)
    return dict(pos=pos, mom=mom, ids=ids, n_mesh=n, box=box)


def _single(re, a0, a1, steps, rtol, k=None):
    from paper_1709_04703_gb300.sim import Sim
    sim = Sim(re["pos"], re["mom"], re["ids"], re["n_mesh"], re["box"], a0, a1, steps,
              rtol=rtol)
    sim.step(steps if k is None else k)
    out = sim.particles(), sim.lightcone(), sim.stats()
    sim.close()
    return out


def _compare(batch, r, ref):
    (sp, sm, si), (lp, lm, li, la), st = ref
    bp, bm, bi = batch.particles(r)
    np.testing.assert_array_equal(bi, si)
    np.testing.assert_array_equal(bp, sp)
    np.testing.assert_array_equal(bm, sm)
    cp, cm, ci, ca = batch.lightcone(r)
    np.testing.assert_array_equal(ci, li)
    np.testing.assert_array_equal(cp, lp)
    np.testing.assert_array_equal(ca, la)
    bs = batch.stats(r)
    for key in ("n_active", "n_lightcone", "cube_side", "periodic"):
        assert bs[key] == st[key], (key, bs[key], st[key])
    # the batch decides convergence on the device after every V-cycle; a
    # single context first runs one V-cycle fewer than its previous solve
    # took before it reads a residual, so it may run one more per step (a
    # correction far below what the FP32 particles resolve: same bits)
    extra = st["vcycles_total"] - bs["vcycles_total"]
    assert 0 <= extra <= st["step"], (bs["vcycles_total"], st["vcycles_total"])


def test_batch_matches_separate_contexts_bitwise():
    from paper_1709_04703_gb300.sim import Batch
    a0, a1, steps, rtol = 0.02, 1.0, 6, 1e-7
    reals = [_realisation(16, 4000.0, 100, a0), _realisation(32, 8000.0, 101, a0),
             _realisation(48, 1000.0, 102, a0), _realisation(64, 12000.0, 103, a0)]
    batch = Batch(reals, a0, a1, steps, rtol=rtol)
    batch.step(steps)
    shrank = 0
    for r, re in enumerate(reals):
        ref = _single(re, a0, a1, steps, rtol)
        _compare(batch, r, ref)
        shrank += batch.stats(r)["n_lightcone"] > 0
    assert shrank >= 2   # the schedule includes shrinking steps
    batch.close()


def test_batched_workload_sample_matches():
    """The first six realisations of the 48-realisation workload (mesh sizes
    32..128, boxes 200-1500 Mpc/h), 8 of its 50 steps."""
    from paper_1709_04703_gb300.sim import Batch
    cfgs = ics.batched_workload(range(100, 106))
    a0, a1, steps = cfgs[0]["a_init"], cfgs[0]["a_final"], cfgs[0]["steps"]
    reals = [_realisation(c["n"], c["box"], c["seed"], a0) for c in cfgs]
    batch = Batch(reals, a0, a1, steps, rtol=cfgs[0]["rtol"])
    batch.step(8)
    for r in (0, len(reals) - 1):
        from paper_1709_04703_gb300.sim import Sim
        re = reals[r]
        sim = Sim(re["pos"], re["mom"], re["ids"], re["n_mesh"], re["box"], a0, a1, steps,
                  rtol=cfgs[0]["rtol"])
        sim.step(8)
        ref = sim.particles(), sim.lightcone(), sim.stats()
        sim.close()
        _compare(batch, r, ref)
    batch.close()


def test_many_open_realisations():
    """40 realisations, all in the open phase (two boundary entries each in
    the batched tables), compared with separate contexts."""
    from paper_1709_04703_gb300.sim import Batch
    a0, a1, steps = 0.5, 1.0, 3
    reals = [_realisation(16, 9000.0 + 100.0 * r, 200 + r, a0) for r in range(40)]
    batch = Batch(reals, a0, a1, steps)
    batch.step(steps)
    for r in (0, 17, 39):
        assert batch.stats(r)["periodic"] == 0
        _compare(batch, r, _single(reals[r], a0, a1, steps, 1e-7))
    batch.close()


def test_fused_finest_level_matches_batched_passes():
    """At n = 192 a single context smooths its finest level with the fused
    two-sweep pass; the batched step uses one-colour passes: the same bits,
    in the periodic and in the open phase."""
    from paper_1709_04703_gb300.sim import Batch
    a0, a1, steps, rtol = 0.4, 1.0, 8, 1e-7
    reals = [_realisation(192, 6000.0, 300, a0)]
    batch = Batch(reals, a0, a1, steps, rtol=rtol)
    batch.step(4)   # periodic 192, open 192, open 192, open 128
    ref = _single(reals[0], a0, a1, steps, rtol, 4)
    _compare(batch, 0, ref)
    assert ref[2]["periodic"] == 0
    batch.close()


def _rel_rms(a, b):
    return np.sqrt(((a - b) ** 2).sum() / (b**2).sum())


def test_batch_against_oracle():
    """The batched step against the FP64 oracle directly: three
    realisations (a periodic 48^3, an open 32^3 that shrinks every step and
    one of the 48-realisation workload's), each step's forces recomputed by
    the oracle from the batch's own float32 particles (relative RMS <= 1e-5),
    and each shrink reproduced bit for bit by the oracle's keep rule and
    stable partition on the batch's float32 positions (Sec. 2.4)."""
    from oracle import cosmology as cz
    from oracle import pm as opm
    from paper_1709_04703_gb300.sim import Batch
    a0, a1, steps, rtol = 0.5, 1.0, 6, 1e-7
    w = ics.batched_workload([101])[0]
    reals = [_realisation(48, 1500.0, 110, a0), _realisation(32, 8000.0, 111, a0),
             _realisation(w["n"], w["box"], w["seed"], a0)]
    scheds = [cz.schedule(re["n_mesh"], re["box"], 0.3, 0.7, a0, a1, steps) for re in reals]
    batch = Batch(reals, a0, a1, steps, rtol=rtol, store_forces=True)
    phases = set()
    shrunk = 0
    for k in range(steps):
        before = [batch.particles(r) for r in range(len(reals))]
        lc0 = [batch.stats(r)["n_lightcone"] for r in range(len(reals))]
        batch.step(1)
        for r, re in enumerate(reals):
            n, sched = re["n_mesh"], scheds[r]
            p0, m0, i0 = before[r]
            st = batch.stats(r)
            F = batch.forces(r)
            _, _, info = opm.step(p0.astype(np.float64), m0.astype(np.float64), k, sched, n,
                                  0.3, 1.0, want=True, drift32=True)
            assert (st["cube_lo"], st["cube_side"], st["periodic"]) == \
                (info["lo"], info["s"], int(info["periodic"])), (r, k)
            phases.add(bool(info["periodic"]))
            ok = info["F"].any(axis=1)
            assert _rel_rms(F[ok], info["F"][ok]) <= 1e-5, (r, k)
            # the shrink: survivors and new records, put back in the order the
            # step began with, must be the oracle's stable partition of them
            p1, m1, i1 = batch.particles(r)
            lp, lm, li, la = batch.lightcone(r)
            lp, lm, li, la = lp[lc0[r]:], lm[lc0[r]:], li[lc0[r]:], la[lc0[r]:]
            assert len(i1) + len(li) == len(i0)
            where = {int(v): q for q, v in enumerate(i0)}
            post_p = np.empty_like(p0)
            post_m = np.empty_like(m0)
            for arr_p, arr_m, arr_i in ((p1, m1, i1), (lp, lm, li)):
                idx = np.array([where[int(v)] for v in arr_i], dtype=np.int64)
                post_p[idx] = arr_p
                post_m[idx] = arr_m
            if opm.is_open(sched["R"][k + 1], n):
                keep = opm.keep_mask(post_p, sched["R"][k + 1], n)
            else:
                keep = np.ones(len(i0), bool)
            (sp, sm, si), (op, om_, oi) = opm.shrink([post_p, post_m, i0], keep)
            np.testing.assert_array_equal(i1, si)
            np.testing.assert_array_equal(p1, sp)
            np.testing.assert_array_equal(m1, sm)
            np.testing.assert_array_equal(li, oi)
            np.testing.assert_array_equal(lp, op)
            assert np.all(la == np.float32(sched["a"][k + 1])) if len(la) else True
            shrunk += len(li) > 0
    batch.close()
    assert phases == {True, False}
    assert shrunk >= 3


def test_persistent_solve_matches_graph_solve():
    """The two device-decided solves, the persistent cooperative kernel and
    the graph whose V-cycle loop is a conditional while node, give the same
    bits and V-cycle counts, in both phases; the persistent step makes at
    most 8 launches (deposit, source, boundary, predict, solve, gather,
    scan, scatter)."""
    from paper_1709_04703_gb300 import _lib as L
    from paper_1709_04703_gb300.sim import Batch
    a0, a1, steps, rtol = 0.02, 1.0, 6, 1e-7
    reals = [_realisation(32, 8000.0, 120, a0), _realisation(48, 1000.0, 121, a0),
             _realisation(64, 12000.0, 122, a0)]
    lib = L.load()
    per = Batch(reals, a0, a1, steps, rtol=rtol)
    per.set_solve(persistent=True)
    counts, phases = [], set()
    for _ in range(steps):
        l0 = lib.pm_launch_count()
        per.step(1)
        counts.append(lib.pm_launch_count() - l0)
        phases |= {per.stats(r)["periodic"] for r in range(len(reals))}
    gra = Batch(reals, a0, a1, steps, rtol=rtol)
    g0 = lib.pm_launch_count()
    gra.step(steps)
    g_launches = lib.pm_launch_count() - g0
    for r in range(len(reals)):
        ref = gra.particles(r), gra.lightcone(r), gra.stats(r)
        _compare(per, r, ref)
        assert per.stats(r)["vcycles_total"] == ref[2]["vcycles_total"]
    assert phases == {0, 1}
    assert max(counts) <= 8, counts
    assert g_launches > sum(counts)
    per.close()
    gra.close()


def test_persistent_barrier_wait_runs_out():
    """A grid barrier that waits for an arrival that never comes gives up
    after its limit: the step returns PM_ETIMEOUT after about that long, and
    the GPU stays usable (a new batch then steps as a separate context)."""
    import time
    from paper_1709_04703_gb300 import _lib as L
    from paper_1709_04703_gb300.sim import Batch
    a0, a1, steps, rtol = 0.02, 1.0, 6, 1e-7
    reals = [_realisation(16, 4000.0, 100, a0), _realisation(32, 8000.0, 101, a0)]
    b = Batch(reals, a0, a1, steps, rtol=rtol)
    b.set_solve(persistent=True, wait_seconds=0.25, extra_arrivals=1)
    t0 = time.time()
    with pytest.raises(L.PmError) as ei:
        b.step(1)
    dt = time.time() - t0
    assert ei.value.code == L.PM_ETIMEOUT, ei.value
    assert 0.2 <= dt < 20.0, dt
    b.close()
    b = Batch(reals, a0, a1, steps, rtol=rtol)
    b.step(2)
    _compare(b, 1, _single(reals[1], a0, a1, steps, rtol, 2))
    b.close()
