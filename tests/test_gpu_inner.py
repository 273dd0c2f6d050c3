"""Mixed precision with several FP32 V-cycles per defect (pm_config
inner_vcycles > 1): the V-cycles the solver runs before it first reads the
residual share one correction equation A e = r, and the defect r = f - A Phi
(double-float or FP64) is evaluated only between those groups.  Results
against the FP64 oracle: one step's forces in both boundary phases, and the
32^3 workload's whole run (final P(k), lightcone crossings)."""
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


def _rel_rms(a, b):
    return np.sqrt(((a - b) ** 2).sum() / (b**2).sum())


@pytest.mark.parametrize("precision", ["mixed", "mixed64"])
@pytest.mark.parametrize("box,a0", [(250.0, 0.02), (8000.0, 0.5)])
def test_forces_after_warm_steps(precision, box, a0):
    """Four steps (so that the warm start predicts several V-cycles and the
    inner groups form), then the fifth step's forces against the oracle's
    step from the GPU's own particles."""
    from paper_1709_04703_gb300.sim import Sim
    n = 32
    pos, mom, ids = ics.zeldovich(n, -2.0, None, 4, a0)
    sched = cz.schedule(n, box, OM, OL, a0, 1.0, 12)
    sim = Sim(pos, mom, ids, n, box, a0, 1.0, 12, rtol=1e-9, store_forces=True,
              max_vcycles=80, precision=precision, inner_vcycles=4)
    sim.step(4)
    assert sim.stats()["vcycles_last"] >= 3      # the inner groups were used
    p, m, _ = sim.particles()
    sim.step(1)
    F = sim.forces()
    st = sim.stats()
    sim.close()
    _, _, info = opm.step(p.astype(np.float64), m.astype(np.float64), 4, sched, n, OM, 1.0,
                          want=True, drift32=True)
    assert st["periodic"] == int(info["periodic"])
    ok = info["F"].any(axis=1)
    assert _rel_rms(F[ok], info["F"][ok]) <= 1e-5


@pytest.mark.parametrize("precision", ["mixed", "mixed64"])
def test_run_pm32_matches_oracle(precision):
    from paper_1709_04703_gb300.sim import Sim, pack, power_spectrum
    cfg = ics.WORKLOADS["pm32"]
    n = cfg["n"]
    pos, mom, ids = ics.workload_ics("pm32")
    sim = Sim(pos, mom, ids, n, cfg["box"], cfg["a_init"], cfg["a_final"], cfg["steps"],
              rtol=cfg["rtol"], precision=precision, inner_vcycles=4)
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


def test_inner_one_is_the_default_iteration():
    """inner_vcycles = 0 and 1 both run one V-cycle per defect: the same bits."""
    from paper_1709_04703_gb300.sim import Sim
    n = 32
    pos, mom, ids = ics.zeldovich(n, -1.5, 0.5, 3, 0.3, rms_disp=0.5)
    out = []
    for inner in (0, 1):
        sim = Sim(pos, mom, ids, n, 6000.0, 0.3, 1.0, 8, rtol=1e-8, inner_vcycles=inner)
        sim.step(8)
        out.append(sim.particles() + (sim.stats()["vcycles_total"],))
        sim.close()
    for u, v in zip(out[0], out[1]):
        np.testing.assert_array_equal(u, v)


def test_batch_rejects_inner_groups():
    from paper_1709_04703_gb300 import _lib as L
    from paper_1709_04703_gb300.sim import Batch
    pos, mom, ids = ics.random_particles(64, 16, 0)
    re = dict(pos=pos, mom=mom, ids=ids, n_mesh=16, box=500.0)
    with pytest.raises(L.PmError) as e:
        Batch([re], 0.5, 1.0, 4, inner_vcycles=4)
    assert e.value.code == L.PM_EINVAL
