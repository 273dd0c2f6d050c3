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
    for key in ("n_active", "n_lightcone", "vcycles_total", "cube_side", "periodic"):
        assert bs[key] == st[key], (key, bs[key], st[key])


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
