"""Mixed precision with an FP64 outer loop (precision "mixed64",
PM_MIXED_FP64): FP32 V-cycles inside a defect correction whose residual
r = f - A Phi and update Phi += e run in FP64 on an FP64 potential.  Against
the FP64 oracle: the exact discrete potential of Eq. 3 (open and periodic,
odd bottoms), one step's forces in both boundary phases, a whole 32^3 run's
P(k), and the run against the double-float path; checkpoints resume bit
for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import crossings  # noqa: E402
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


def _err(got, ref):
    return np.sqrt(np.mean((got - ref) ** 2) / np.mean(ref**2))


def _rel_rms(a, b):
    return np.sqrt(((a - b) ** 2).sum() / (b**2).sum())


def _sim(n, rtol=1e-11, **kw):
    from paper_1709_04703_gb300.sim import Sim
    pos, mom, ids = ics.random_particles(8, n, 0)
    return Sim(pos, mom, ids, n, 100.0, 0.5, 1.0, 4, rtol=rtol, precision="mixed64",
               max_vcycles=80, **kw)


# 12, 24 and 48 coarsen to an odd 3^3 bottom
@pytest.mark.parametrize("n", [12, 16, 24, 32, 48, 64])
def test_open_solve_matches_oracle(n):
    rng = np.random.default_rng(17 + n)
    delta = rng.standard_normal((n, n, n))
    delta[: n // 3] = 0.0
    sim = _sim(n)
    _, phi64, vc, res = sim.solve_potential(delta, 0.5, "open")
    S = opm.source_S(0.5, OM)
    f = S * delta
    ref = opm.solve_open(f, opm.open_ghost_potential(f, S, 0, n))[1:-1, 1:-1, 1:-1]
    assert res <= 1e-11 and vc <= 40
    assert _err(phi64.cpu().numpy(), ref) < 1e-9
    sim.close()


@pytest.mark.parametrize("n", [12, 24, 32, 48])
def test_periodic_solve_matches_oracle(n):
    rng = np.random.default_rng(300 + n)
    delta = rng.standard_normal((n, n, n))
    delta -= delta.mean()
    sim = _sim(n)
    _, phi64, vc, res = sim.solve_potential(delta, 0.7, "periodic")
    ref = opm.solve_periodic(opm.source_S(0.7, OM) * delta)
    assert res <= 1e-11 and vc <= 40
    assert _err(phi64.cpu().numpy(), ref) < 1e-9
    sim.close()


def _one_step(n, box, a0, steps, seed):
    from paper_1709_04703_gb300.sim import Sim
    pos, mom, ids = ics.zeldovich(n, -2.0, None, seed, a0)
    sched = cz.schedule(n, box, OM, OL, a0, 1.0, steps)
    sim = Sim(pos, mom, ids, n, box, a0, 1.0, steps, rtol=1e-10, store_forces=True,
              max_vcycles=80, precision="mixed64")
    sim.step(1)
    F = sim.forces()
    st = sim.stats()
    sim.close()
    _, _, info = opm.step(pos.astype(np.float64), mom.astype(np.float64), 0, sched, n, OM, 1.0,
                          want=True, drift32=True)
    return F, info, st


def test_step_forces_periodic_phase():
    F, info, st = _one_step(32, 250.0, 0.02, 20, 0)
    assert st["periodic"] == 1
    assert _rel_rms(F, info["F"]) <= 1e-5


def _a_for_side(n, box, side):
    for a in np.linspace(0.3, 0.995, 4000):
        R = cz.chi(a, OM, OL) / (box / n) + 1.0
        lo, s, per = opm.active_cube(R, n)
        if not per and s == side:
            return a
    raise AssertionError(side)


@pytest.mark.parametrize("n,side", [(32, None), (64, 56), (64, 40), (64, 20)])
def test_step_forces_open_phase(n, side):
    a0 = 0.5 if side is None else _a_for_side(n, 8000.0, side)
    F, info, st = _one_step(n, 8000.0, a0, 10, 1)
    assert st["periodic"] == 0 and st["cube_side"] == info["s"]
    ok = info["F"].any(axis=1)
    assert _rel_rms(F[ok], info["F"][ok]) <= 1e-5


def test_run_pm32_power_spectrum_matches_oracle():
    """The 32^3 workload (250 Mpc/h, a 0.02 -> 1 in 20 steps, rtol 1e-8):
    final P(k) of lightcone + survivors within 0.5 % of the oracle's run."""
    from paper_1709_04703_gb300.sim import Sim, pack, power_spectrum
    cfg = ics.WORKLOADS["pm32"]
    n = cfg["n"]
    pos, mom, ids = ics.workload_ics("pm32")
    sim = Sim(pos, mom, ids, n, cfg["box"], cfg["a_init"], cfg["a_final"], cfg["steps"],
              rtol=cfg["rtol"], precision="mixed64")
    sim.step(cfg["steps"])
    st = sim.stats()
    gp, _, gi = sim.particles()
    cp, _, ci, ca = sim.lightcone()
    sim.close()
    sched = cz.schedule(n, cfg["box"], OM, OL, cfg["a_init"], cfg["a_final"], cfg["steps"])
    out = opm.run(pos, mom, ids, sched, n, OM, 1.0)
    assert st["n_active"] + st["n_lightcone"] == n**3
    a_g, x_g = crossings.table(n**3, gi, gp, ci, cp, ca)
    a_o, x_o = crossings.table(n**3, out["ids"], out["pos"], out["lc_ids"], out["lc_pos"],
                               out["lc_a"])
    crossings.check_crossings(a_g, x_g, a_o, x_o, sched, n)
    allg = (np.concatenate([gp, cp]) % n).astype(np.float32)
    p4, _ = pack(allg, np.zeros_like(allg))
    _, pg, _ = power_spectrum(torch.from_numpy(p4).cuda(), cfg["box"], n, n // 2)
    _, po, _ = opk(np.concatenate([out["pos"], out["lc_pos"]]) % n, n, cfg["box"], n // 2)
    sel = slice(0, n // 4)
    assert np.abs(pg[sel] / po[sel] - 1).max() <= 5e-3


def test_run_agrees_with_the_double_float_path():
    """12 steps through both boundary phases solved to 1e-10 with the FP64
    and the double-float defect: the same particles to float32 rounding, the
    same lightcone."""
    from paper_1709_04703_gb300.sim import Sim
    n = 32
    pos, mom, ids = ics.zeldovich(n, -1.5, 0.5, 3, 0.3, rms_disp=0.5)
    out = []
    for prec in ("mixed", "mixed64"):
        sim = Sim(pos, mom, ids, n, 6000.0, 0.3, 1.0, 12, rtol=1e-10, precision=prec,
                  max_vcycles=80)
        sim.step(12)
        p, m, i = sim.particles()
        li = sim.lightcone()[2]
        st = sim.stats()
        sim.close()
        out.append((p, m, i, np.sort(li), st["n_active"]))
    (p0, m0, i0, l0, n0), (p1, m1, i1, l1, n1) = out
    assert n0 == n1 and n0 < n**3
    np.testing.assert_array_equal(i0, i1)
    np.testing.assert_array_equal(l0, l1)
    np.testing.assert_allclose(p1, p0, rtol=0, atol=1e-4)
    np.testing.assert_allclose(m1, m0, rtol=0, atol=1e-4 * np.abs(m0).max())


@pytest.mark.parametrize("cut", [5, 11])
def test_checkpoint_resume_is_bitwise(tmp_path, cut):
    from paper_1709_04703_gb300.sim import Sim
    n, steps = 32, 16
    pos, mom, ids = ics.zeldovich(n, -1.5, 0.5, 6, 0.2, rms_disp=0.6)

    def new():
        return Sim(pos, mom, ids, n, 6000.0, 0.2, 1.0, steps, precision="mixed64")
    ref = new()
    ref.step(steps)
    want = ref.particles(), ref.lightcone(), ref.stats()
    ref.close()
    a = new()
    a.step(cut)
    a.save(tmp_path / "c.ckpt")
    a.close()
    b = new()
    b.load(tmp_path / "c.ckpt")
    b.step(steps - cut)
    got = b.particles(), b.lightcone(), b.stats()
    b.close()
    for u, v in zip(got[0] + got[1], want[0] + want[1]):
        np.testing.assert_array_equal(u, v)
    for f in ("n_active", "n_lightcone", "vcycles_total", "resid_last"):
        assert got[2][f] == want[2][f], f


def test_rejects_diffusion_and_learned_guess():
    from paper_1709_04703_gb300 import _lib as L
    from paper_1709_04703_gb300.sim import Sim
    pos, mom, ids = ics.random_particles(8, 16, 0)
    for kw in (dict(gravity="diffusion"), dict(guess="learned")):
        with pytest.raises(L.PmError) as e:
            Sim(pos, mom, ids, 16, 100.0, 0.5, 1.0, 4, precision="mixed64", **kw)
        assert e.value.code == L.PM_EINVAL
