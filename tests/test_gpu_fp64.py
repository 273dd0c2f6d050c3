"""The FP64-everywhere solve (precision "fp64", PM_FP64_PLAIN) against the
FP64 oracle: the exact discrete potential of Eq. 3 with open (multipole
Dirichlet) and periodic boundaries, including multigrid hierarchies whose
bottom is an odd side; one step's forces in both boundary phases; and a
short run against the mixed double-float path."""
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


def _sim(n, rtol=1e-11, **kw):
    from paper_1709_04703_gb300.sim import Sim
    pos, mom, ids = ics.random_particles(8, n, 0)
    return Sim(pos, mom, ids, n, 100.0, 0.5, 1.0, 4, rtol=rtol, precision="fp64",
               max_vcycles=80, **kw)


def _err(got, ref):
    return np.sqrt(np.mean((got - ref) ** 2) / np.mean(ref**2))


# 12, 24 and 48 coarsen to an odd 3^3 bottom
@pytest.mark.parametrize("n", [12, 16, 24, 32, 48, 64])
def test_open_solve_matches_oracle(n):
    rng = np.random.default_rng(7 + n)
    delta = rng.standard_normal((n, n, n))
    delta[: n // 3] = 0.0
    sim = _sim(n)
    phi32, phi64, vc, res = sim.solve_potential(delta, 0.5, "open")
    S = opm.source_S(0.5, OM)
    f = S * delta
    ref = opm.solve_open(f, opm.open_ghost_potential(f, S, 0, n))[1:-1, 1:-1, 1:-1]
    assert res <= 1e-11 and vc <= 40
    assert _err(phi64.cpu().numpy(), ref) < 1e-9
    sim.close()


@pytest.mark.parametrize("n", [12, 24, 32, 48])
def test_periodic_solve_matches_oracle(n):
    rng = np.random.default_rng(200 + n)
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
              max_vcycles=80, precision="fp64")
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
    assert np.sqrt(((F - info["F"]) ** 2).sum() / (info["F"] ** 2).sum()) <= 1e-5


def test_step_forces_open_phase():
    F, info, st = _one_step(32, 8000.0, 0.5, 10, 1)
    assert st["periodic"] == 0 and st["cube_side"] == info["s"]
    ok = info["F"].any(axis=1)
    assert np.sqrt(((F[ok] - info["F"][ok]) ** 2).sum() / (info["F"][ok] ** 2).sum()) <= 1e-5


def _a_for_side(n, box, side):
    for a in np.linspace(0.3, 0.995, 4000):
        R = cz.chi(a, OM, OL) / (box / n) + 1.0
        lo, s, per = opm.active_cube(R, n)
        if not per and s == side:
            return a
    raise AssertionError(side)


@pytest.mark.parametrize("side", [56, 40, 20])
def test_step_forces_open_cubes_with_odd_bottoms(side):
    """Open cubes of side 7 * 2^j and 5 * 2^j: FP64 levels down to a 7^3 or
    5^3 bottom."""
    a0 = _a_for_side(64, 8000.0, side)
    F, info, st = _one_step(64, 8000.0, a0, 10, 2)
    assert st["periodic"] == 0 and st["cube_side"] == side == info["s"]
    ok = info["F"].any(axis=1)
    assert np.sqrt(((F[ok] - info["F"][ok]) ** 2).sum() / (info["F"][ok] ** 2).sum()) <= 1e-5


def test_run_agrees_with_the_mixed_path():
    """The same 12 steps through both boundary phases, solved to 1e-10 in
    FP64 and by the double-float defect correction: the same particles to
    float32 rounding, the same lightcone."""
    from paper_1709_04703_gb300.sim import Sim
    n = 32
    pos, mom, ids = ics.zeldovich(n, -1.5, 0.5, 3, 0.3, rms_disp=0.5)
    out = []
    for prec in ("mixed", "fp64"):
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


def test_fp64_rejects_diffusion_gravity():
    from paper_1709_04703_gb300 import _lib as L
    from paper_1709_04703_gb300.sim import Sim
    pos, mom, ids = ics.random_particles(8, 16, 0)
    with pytest.raises(L.PmError):
        Sim(pos, mom, ids, 16, 100.0, 0.5, 1.0, 4, precision="fp64", gravity="diffusion")
