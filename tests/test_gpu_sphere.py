"""The spherical keep region of Table 1 (PM_DOMAIN_SPHERE) on the GPU
against the FP64 oracle: the radial keep rule and stable compaction bit for
bit, one open-phase step's forces (the source carries the CIC image of the
ball) and a whole run's P(k)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import cosmology as cz  # noqa: E402
from oracle import pm as opm  # noqa: E402
from oracle.pk import power_spectrum as opk  # noqa: E402
from paper_1709_04703_gb300 import ics  # noqa: E402

OM, OL = 0.3, 0.7


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_04703_gb300 import build
    build.build()


@pytest.mark.parametrize("N", [1, 1000, 300001])
def test_sphere_shrink_bitexact(N):
    from paper_1709_04703_gb300.sim import Sim
    n = 64
    pos, mom, ids = ics.random_particles(N, n, 21)
    sim = Sim(pos, mom, ids, n, 8000.0, 0.5, 1.0, 10, domain="sphere")
    a = 0.7
    kept = sim.shrink(a)
    R = cz.chi(a, OM, OL) / (8000.0 / n) + 1.0
    keep = opm.keep_mask(pos, R, n, "sphere")
    (sp, sm, si), (lp, lm, li) = opm.shrink([pos, mom, ids], keep)
    assert kept == len(si)
    gp, gm, gi = sim.particles()
    np.testing.assert_array_equal(gi, si)
    np.testing.assert_array_equal(gp, sp)
    cp, cm, ci, ca = sim.lightcone()
    np.testing.assert_array_equal(ci, li)
    sim.close()
    if N > 1000:   # a uniform set keeps the ball's share of the cube
        cube = opm.keep_mask(pos, R, n).sum()
        assert abs(kept / cube - math.pi / 6) < 0.01


def test_sphere_step_forces_open_phase():
    from paper_1709_04703_gb300.sim import Sim
    n, box, a0, steps = 32, 8000.0, 0.5, 10
    pos, mom, ids = ics.zeldovich(n, -2.0, None, 1, a0)
    sched = cz.schedule(n, box, OM, OL, a0, 1.0, steps)
    sim = Sim(pos, mom, ids, n, box, a0, 1.0, steps, rtol=1e-10, store_forces=True,
              max_vcycles=60, domain="sphere")
    sim.step(1)
    F = sim.forces()
    st = sim.stats()
    sim.close()
    _, _, info = opm.step(pos.astype(np.float64), mom.astype(np.float64), 0, sched, n, OM, 1.0,
                          want=True, drift32=True, domain="sphere")
    assert st["periodic"] == 0 and (st["cube_lo"], st["cube_side"]) == (info["lo"], info["s"])
    ok = info["F"].any(axis=1)
    r = np.sqrt(((F - info["F"])[ok] ** 2).sum() / (info["F"][ok] ** 2).sum())
    assert r <= 1e-5, r


def test_sphere_run_pm32_power_spectrum_matches_oracle():
    from paper_1709_04703_gb300.sim import Sim, pack, power_spectrum
    cfg = ics.WORKLOADS["pm32"]
    n = cfg["n"]
    pos, mom, ids = ics.workload_ics("pm32")
    sim = Sim(pos, mom, ids, n, cfg["box"], cfg["a_init"], cfg["a_final"], cfg["steps"],
              rtol=cfg["rtol"], domain="sphere")
    sim.step(cfg["steps"])
    st = sim.stats()
    gp, _, _ = sim.particles()
    cp, _, _, _ = sim.lightcone()
    sim.close()
    sched = cz.schedule(n, cfg["box"], OM, OL, cfg["a_init"], cfg["a_final"], cfg["steps"])
    out = opm.run(pos, mom, ids, sched, n, OM, 1.0, domain="sphere")
    assert st["n_active"] + st["n_lightcone"] == n**3
    assert abs(st["n_active"] - len(out["ids"])) < 20
    p4, _ = pack((np.concatenate([gp, cp]) % n).astype(np.float32),
                 np.zeros((n**3, 3), np.float32))
    _, pg, _ = power_spectrum(torch.from_numpy(p4).cuda(), cfg["box"], n, n // 2)
    _, po, _ = opk(np.concatenate([out["pos"], out["lc_pos"]]) % n, n, cfg["box"], n // 2)
    rel = np.abs(pg[: n // 4] / po[: n // 4] - 1)
    assert rel.max() <= 5e-3, rel


def test_sphere_needs_cic():
    from paper_1709_04703_gb300 import _lib as L
    from paper_1709_04703_gb300.sim import Sim
    pos, mom, ids = ics.zeldovich(16, -2.0, None, 0, 0.5)
    with pytest.raises(L.PmError):
        Sim(pos, mom, ids, 16, 100.0, 0.5, 1.0, 2, assignment="tsc", domain="sphere")
