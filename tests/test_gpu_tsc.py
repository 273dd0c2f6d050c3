"""The TSC assignment (Sec. 2.4 footnote: CIC or TSC, one scheme for the
density and the force) on the GPU against the FP64 oracle: the integer
deposit bit for bit, one step's forces in both boundary phases and a whole
run's P(k)."""
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


def _dev4(pos, mom=None):
    from paper_1709_04703_gb300.sim import pack
    p4, m4 = pack(pos, np.zeros_like(pos) if mom is None else mom)
    return torch.from_numpy(p4).cuda(), torch.from_numpy(m4).cuda()


@pytest.mark.parametrize("n,N,seed", [(16, 16**3, 0), (48, 100003, 1), (8, 1, 2)])
def test_tsc_deposit_bitexact_periodic(n, N, seed):
    from paper_1709_04703_gb300.sim import deposit
    if N == n**3:
        pos, _, _ = ics.zeldovich(n, -2.0, None, seed, 0.5, rms_disp=0.4)
    else:
        pos, _, _ = ics.random_particles(N, n, seed)
    p4, _ = _dev4(pos)
    rho, esc = deposit(p4, n, assignment="tsc")
    ref, resc = opm.deposit_tsc(pos, n, 0, n, True)
    assert esc == resc == 0
    np.testing.assert_array_equal(rho.cpu().numpy(), ref)


@pytest.mark.parametrize("lo,s", [(4, 24), (10, 12)])
def test_tsc_deposit_bitexact_open_cube_with_escapes(lo, s):
    from paper_1709_04703_gb300.sim import deposit
    n = 32
    pos, _, _ = ics.random_particles(50000, n, 3)
    p4, _ = _dev4(pos)
    rho, esc = deposit(p4, n, lo, s, periodic=False, assignment="tsc")
    ref, resc = opm.deposit_tsc(pos, n, lo, s, False)
    assert esc == resc > 0
    np.testing.assert_array_equal(rho.cpu().numpy(), ref)


def _one_step(n, box, a0, steps, seed):
    from paper_1709_04703_gb300.sim import Sim
    pos, mom, ids = ics.zeldovich(n, -2.0, None, seed, a0)
    sched = cz.schedule(n, box, OM, OL, a0, 1.0, steps)
    sim = Sim(pos, mom, ids, n, box, a0, 1.0, steps, rtol=1e-10, store_forces=True,
              max_vcycles=60, assignment="tsc")
    sim.step(1)
    F = sim.forces()
    st = sim.stats()
    sim.close()
    _, _, info = opm.step(pos.astype(np.float64), mom.astype(np.float64), 0, sched, n, OM, 1.0,
                          want=True, drift32=True, assign="tsc")
    return F, st, info


def _rel_rms(a, b):
    return np.sqrt(((a - b) ** 2).sum() / (b**2).sum())


def test_tsc_step_forces_periodic_phase():
    F, st, info = _one_step(32, 250.0, 0.02, 20, 0)
    assert st["periodic"] == 1
    assert _rel_rms(F, info["F"]) <= 1e-5


def test_tsc_step_forces_open_phase():
    F, st, info = _one_step(32, 8000.0, 0.5, 10, 1)
    assert st["periodic"] == 0 and (st["cube_lo"], st["cube_side"]) == (info["lo"], info["s"])
    ok = info["F"].any(axis=1)
    assert ok.sum() > 0
    assert _rel_rms(F[ok], info["F"][ok]) <= 1e-5


def test_tsc_run_pm32_power_spectrum_matches_oracle():
    from paper_1709_04703_gb300.sim import Sim, power_spectrum
    cfg = ics.WORKLOADS["pm32"]
    n = cfg["n"]
    pos, mom, ids = ics.workload_ics("pm32")
    sim = Sim(pos, mom, ids, n, cfg["box"], cfg["a_init"], cfg["a_final"], cfg["steps"],
              rtol=cfg["rtol"], assignment="tsc")
    sim.step(cfg["steps"])
    st = sim.stats()
    gp, _, _ = sim.particles()
    cp, _, _, _ = sim.lightcone()
    sim.close()
    sched = cz.schedule(n, cfg["box"], OM, OL, cfg["a_init"], cfg["a_final"], cfg["steps"])
    out = opm.run(pos, mom, ids, sched, n, OM, 1.0, assign="tsc")
    assert st["n_active"] + st["n_lightcone"] == n**3
    p4, _ = _dev4((np.concatenate([gp, cp]) % n).astype(np.float32))
    _, pg, _ = power_spectrum(p4, cfg["box"], n, n // 2)
    _, po, _ = opk(np.concatenate([out["pos"], out["lc_pos"]]) % n, n, cfg["box"], n // 2)
    rel = np.abs(pg[: n // 4] / po[: n // 4] - 1)
    assert rel.max() <= 5e-3, rel


def test_tsc_needs_poisson_gravity():
    from paper_1709_04703_gb300 import _lib as L
    from paper_1709_04703_gb300.sim import Sim
    pos, mom, ids = ics.zeldovich(16, -2.0, None, 0, 0.5)
    with pytest.raises(L.PmError):
        Sim(pos, mom, ids, 16, 100.0, 0.5, 1.0, 2, gravity="diffusion", assignment="tsc")
