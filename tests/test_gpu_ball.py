"""The ball solve (PM_DOMAIN_BALL, the spherical domain of Table 1 solved on
the ball's cells only) on the GPU against the FP64 oracle's masked system
(oracle.pm.solve_ball): one open-phase step's forces, several steps with
each step's forces recomputed by the oracle from the GPU's own float
particles and each shrink reproduced bit for bit, and a whole run's P(k)."""
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


def _rel(a, b):
    ok = b.any(axis=1)
    return np.sqrt(((a - b)[ok] ** 2).sum() / (b[ok] ** 2).sum())


@pytest.mark.parametrize("n,box,a0", [(32, 8000.0, 0.5), (48, 6000.0, 0.45)])
def test_ball_step_forces_open_phase(n, box, a0):
    from paper_1709_04703_gb300.sim import Sim
    steps = 10
    pos, mom, ids = ics.zeldovich(n, -2.0, None, 1, a0)
    sched = cz.schedule(n, box, OM, OL, a0, 1.0, steps)
    sim = Sim(pos, mom, ids, n, box, a0, 1.0, steps, rtol=1e-10, store_forces=True,
              max_vcycles=200, domain="ball")
    sim.step(1)
    F = sim.forces()
    st = sim.stats()
    sim.close()
    _, _, info = opm.step(pos.astype(np.float64), mom.astype(np.float64), 0, sched, n, OM, 1.0,
                          want=True, drift32=True, domain="ball")
    assert st["periodic"] == 0 and (st["cube_lo"], st["cube_side"]) == (info["lo"], info["s"])
    assert _rel(F, info["F"]) <= 1e-5


def test_ball_steps_match_oracle_and_shrink_bitexact():
    """Six open-phase steps of a 48^3 run whose ball shrinks every step."""
    from paper_1709_04703_gb300.sim import Sim
    n, box, a0, steps = 48, 6000.0, 0.45, 6
    pos, mom, ids = ics.zeldovich(n, -2.0, None, 4, a0)
    sched = cz.schedule(n, box, OM, OL, a0, 1.0, steps)
    # (rtol 1e-9: as the ball shrinks, the potential's multipole part grows
    # against the source and the double-float defect's floor nears 1e-10)
    sim = Sim(pos, mom, ids, n, box, a0, 1.0, steps, rtol=1e-9, store_forces=True,
              max_vcycles=200, domain="ball")
    shrunk = 0
    for k in range(steps):
        p0, m0, i0 = sim.particles()
        lc0 = sim.stats()["n_lightcone"]
        sim.step(1)
        F = sim.forces()
        _, _, info = opm.step(p0.astype(np.float64), m0.astype(np.float64), k, sched, n, OM, 1.0,
                              want=True, drift32=True, domain="ball")
        st = sim.stats()
        assert (st["cube_lo"], st["cube_side"], st["periodic"]) == (info["lo"], info["s"], 0)
        assert _rel(F, info["F"]) <= 1e-5, k
        p1, m1, i1 = sim.particles()
        lp, lm, li, la = sim.lightcone()
        lp, lm, li = lp[lc0:], lm[lc0:], li[lc0:]
        where = {int(v): q for q, v in enumerate(i0)}
        post_p = np.empty_like(p0)
        post_m = np.empty_like(m0)
        for arr_p, arr_m, arr_i in ((p1, m1, i1), (lp, lm, li)):
            idx = np.array([where[int(v)] for v in arr_i], dtype=np.int64)
            post_p[idx] = arr_p
            post_m[idx] = arr_m
        keep = opm.keep_mask(post_p, sched["R"][k + 1], n, "ball")
        (sp, sm, si), (op, om_, oi) = opm.shrink([post_p, post_m, i0], keep)
        np.testing.assert_array_equal(i1, si)
        np.testing.assert_array_equal(p1, sp)
        np.testing.assert_array_equal(li, oi)
        shrunk += len(li) > 0
    sim.close()
    assert shrunk >= 3


def test_ball_run_power_spectrum_matches_oracle():
    """A 32^3 run from a = 0.3 in a 6000 Mpc/h box (open from the first
    steps, the ball shrinking to a few cells): the P(k) of lightcone plus
    survivors within 0.5 % of the oracle's for k <= k_Ny/2."""
    from paper_1709_04703_gb300.sim import Sim, pack, power_spectrum
    n, box, a0, steps, rtol = 32, 6000.0, 0.3, 20, 1e-8
    pos, mom, ids = ics.zeldovich(n, -2.0, None, 7, a0)
    sim = Sim(pos, mom, ids, n, box, a0, 1.0, steps, rtol=rtol, max_vcycles=200, domain="ball")
    sim.step(steps)
    st = sim.stats()
    gp, _, _ = sim.particles()
    cp, _, _, _ = sim.lightcone()
    sim.close()
    sched = cz.schedule(n, box, OM, OL, a0, 1.0, steps)
    out = opm.run(pos, mom, ids, sched, n, OM, 1.0, domain="ball")
    assert st["n_active"] + st["n_lightcone"] == n**3
    assert st["n_lightcone"] > n**3 // 2
    # trajectories near the keep radius may cross it at different steps
    assert abs(st["n_active"] - len(out["ids"])) < 20
    p4, _ = pack((np.concatenate([gp, cp]) % n).astype(np.float32),
                 np.zeros((n**3, 3), np.float32))
    _, pg, _ = power_spectrum(torch.from_numpy(p4).cuda(), box, n, n // 2)
    _, po, _ = opk(np.concatenate([out["pos"], out["lc_pos"]]) % n, n, box, n // 2)
    rel = np.abs(pg[: n // 4] / po[: n // 4] - 1)
    assert rel.max() <= 5e-3, rel


@pytest.mark.parametrize("kw", [dict(precision="fp32"), dict(precision="fp64"),
                                dict(gravity="diffusion"), dict(assignment="tsc")])
def test_ball_needs_the_mixed_poisson_cic_solve(kw):
    from paper_1709_04703_gb300 import _lib as L
    from paper_1709_04703_gb300.sim import Sim
    pos, mom, ids = ics.zeldovich(16, -2.0, None, 0, 0.5)
    with pytest.raises(L.PmError):
        Sim(pos, mom, ids, 16, 100.0, 0.5, 1.0, 2, domain="ball", **kw)
