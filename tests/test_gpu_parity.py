"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  Bars: bit-exact for the integer deposit and the
compaction; per-step relative force RMS <= 1e-5; potential within the
solver tolerance; P(k) within 0.5 % per bin for k <= k_Ny / 2."""
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


def _dev4(pos, mom=None, ids=None):
    from paper_1709_04703_gb300.sim import pack
    p4, m4 = pack(pos, np.zeros_like(pos) if mom is None else mom, ids)
    return torch.from_numpy(p4).cuda(), torch.from_numpy(m4).cuda()


# --------------------------------------------------------------- deposit

@pytest.mark.parametrize("n,N,seed", [(32, 32**3, 0), (48, 12345, 1), (8, 1, 2), (16, 0, 3),
                                      (96, 200003, 4)])
def test_deposit_bitexact_periodic(n, N, seed):
    from paper_1709_04703_gb300.sim import deposit
    pos, _, _ = ics.random_particles(N, n, seed)
    if N > 3:
        pos[0] = [0.5, 0.5, 0.5]
        pos[1] = [1.0, 2.0, 3.0]
        pos[2] = [0.0, np.float32(n) - np.float32(1e-5), 0.25]
    p4, _ = _dev4(pos)
    rho, esc = deposit(p4, n)
    ref, _ = opm.deposit(pos, n, 0, n, True)
    assert esc == 0
    np.testing.assert_array_equal(rho.cpu().numpy(), ref)
    assert int(ref.astype(object).sum()) == N * 2**48   # exact, no int64 overflow


def test_deposit_bitexact_zeldovich_lattice():
    from paper_1709_04703_gb300.sim import deposit
    n = 64
    pos, mom, ids = ics.zeldovich(n, -1.5, 0.5, 1, 0.02)
    p4, _ = _dev4(pos)
    rho, _ = deposit(p4, n)
    ref, _ = opm.deposit(pos, n, 0, n, True)
    np.testing.assert_array_equal(rho.cpu().numpy(), ref)


@pytest.mark.parametrize("n,lo,s", [(64, 16, 32), (48, 12, 24), (32, 0, 32)])
def test_deposit_bitexact_open_cube_with_escapes(n, lo, s):
    from paper_1709_04703_gb300.sim import deposit
    pos, _, _ = ics.random_particles(50000, n, 5, lo=lo - 2.0, hi=lo + s + 2.0)
    p4, _ = _dev4(pos)
    rho, esc = deposit(p4, n, lo, s, periodic=False)
    ref, esc_ref = opm.deposit(pos, n, lo, s, False)
    assert esc == esc_ref > 0
    np.testing.assert_array_equal(rho.cpu().numpy(), ref)


@pytest.mark.parametrize("periodic", [True, False])
def test_fused_drift_deposit_bitexact(periodic):
    """The fused half drift is float32 x = fl(x + fl(p c)); the oracle takes
    the same float32 decision before its integer deposit."""
    from paper_1709_04703_gb300.sim import deposit
    n = 32
    pos, mom, ids = ics.random_particles(40000, n, 7, lo=4.0 if not periodic else 0.0,
                                         hi=28.0 if not periodic else None, vmax=3.0)
    c = 0.37
    p4, m4 = _dev4(pos, mom, ids)
    lo, s = (0, n) if periodic else (4, 24)
    rho, esc = deposit(p4, n, lo, s, periodic=periodic, mom4_dev=m4, drift_coef=c)
    x32 = opm.drift_fp32(pos, mom, c, n, periodic)
    np.testing.assert_array_equal(p4[:, :3].cpu().numpy(), x32)
    ref, esc_ref = opm.deposit(x32, n, lo, s, periodic)
    assert esc == esc_ref
    np.testing.assert_array_equal(rho.cpu().numpy(), ref)


# --------------------------------------------------------------- schedule

def test_schedule_matches_oracle():
    from paper_1709_04703_gb300.sim import Sim
    n = 16
    pos, mom, ids = ics.zeldovich(n, -2.0, None, 0, 0.01)
    sim = Sim(pos, mom, ids, n, 2000.0, 0.01, 1.0, 37)
    got = sim.schedule()
    ref = cz.schedule(n, 2000.0, OM, OL, 0.01, 1.0, 37)
    np.testing.assert_allclose(got["a"], ref["a"], rtol=1e-15)
    np.testing.assert_allclose(got["dtau"][:-1], ref["dtau"], rtol=1e-12)
    np.testing.assert_allclose(got["a_half"][:-1], ref["a_half"], rtol=1e-12)
    np.testing.assert_allclose(got["chi"], ref["chi"], rtol=1e-12, atol=1e-9)
    sim.close()


# --------------------------------------------------------------- Poisson solve

def _sim_for_solve(n, precision="mixed", rtol=1e-10):
    from paper_1709_04703_gb300.sim import Sim
    pos, mom, ids = ics.random_particles(8, n, 0)
    return Sim(pos, mom, ids, n, 100.0, 0.5, 1.0, 4, rtol=rtol, precision=precision,
               max_vcycles=60)


# 192 and up: the finest level is smoothed by the fused two-sweep pass
@pytest.mark.parametrize("n", [16, 32, 48, 64, 192])
def test_open_solve_matches_oracle(n):
    rng = np.random.default_rng(n)
    delta = rng.standard_normal((n, n, n))
    delta[: n // 4] = 0.0
    sim = _sim_for_solve(n)
    phi32, phi64, vc, res = sim.solve_potential(delta, 0.5, "open")
    S = opm.source_S(0.5, OM)
    f = S * delta
    ref = opm.solve_open(f, opm.open_ghost_potential(f, S, 0, n))[1:-1, 1:-1, 1:-1]
    got = phi64.cpu().numpy()
    err = np.sqrt(np.mean((got - ref) ** 2) / np.mean(ref**2))
    assert res <= 1e-10 and vc <= 16
    assert err < 1e-8, err
    np.testing.assert_allclose(phi32.cpu().numpy(), got.astype(np.float32), rtol=0, atol=0)
    sim.close()


@pytest.mark.parametrize("n", [32, 48, 192])
def test_periodic_solve_matches_oracle(n):
    rng = np.random.default_rng(100 + n)
    delta = rng.standard_normal((n, n, n))
    delta -= delta.mean()
    sim = _sim_for_solve(n)
    _, phi64, vc, res = sim.solve_potential(delta, 0.7, "periodic")
    ref = opm.solve_periodic(opm.source_S(0.7, OM) * delta)
    got = phi64.cpu().numpy()
    err = np.sqrt(np.mean((got - ref) ** 2) / np.mean(ref**2))
    assert res <= 1e-10 and vc <= 16
    assert err < 1e-8, err
    sim.close()


def test_gaussian_closed_form_through_gpu():
    from math import erf, pi, sqrt
    n = 64
    sigma = n / 10
    g = np.arange(n) + 0.5 - n / 2
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    r = np.sqrt(X**2 + Y**2 + Z**2)
    delta = np.exp(-r**2 / (2 * sigma**2))
    sim = _sim_for_solve(n)
    _, phi64, _, _ = sim.solve_potential(delta, 0.5, "open")
    S = opm.source_S(0.5, OM)
    exact = -(S / (4 * pi)) * (2 * pi * sigma**2) ** 1.5 * np.vectorize(erf)(
        r / (sqrt(2) * sigma)) / r
    err = np.sqrt(np.mean((phi64.cpu().numpy() - exact) ** 2) / np.mean(exact**2))
    assert err < 5e-3
    sim.close()


@pytest.mark.parametrize("n", [32, 192])
def test_plain_fp32_solve_reaches_its_tolerance(n):
    rng = np.random.default_rng(3)
    delta = rng.standard_normal((n, n, n))
    sim = _sim_for_solve(n, precision="fp32", rtol=1e-4)
    _, phi64, vc, res = sim.solve_potential(delta, 0.5, "open")
    assert res <= 1e-4
    S = opm.source_S(0.5, OM)
    f = S * delta
    ref = opm.solve_open(f, opm.open_ghost_potential(f, S, 0, n))[1:-1, 1:-1, 1:-1]
    err = np.sqrt(np.mean((phi64.cpu().numpy() - ref) ** 2) / np.mean(ref**2))
    assert err < 1e-3
    sim.close()


# --------------------------------------------------------------- one full step

def _one_step(n, box, a0, a1, steps, seed, alpha=-2.0, cutoff=None, take=0):
    from paper_1709_04703_gb300.sim import Sim
    pos, mom, ids = ics.zeldovich(n, alpha, cutoff, seed, a0)
    sched = cz.schedule(n, box, OM, OL, a0, a1, steps)
    sim = Sim(pos, mom, ids, n, box, a0, a1, steps, rtol=1e-10, store_forces=True,
              max_vcycles=60)
    sim.step(1)
    F = sim.forces()
    st = sim.stats()
    p_gpu, m_gpu, id_gpu = sim.particles()
    sim.close()
    p_o, m_o, info = opm.step(pos.astype(np.float64), mom.astype(np.float64), 0, sched, n,
                              OM, 1.0, want=True, drift32=True)
    return F, info, st, (p_gpu, m_gpu, id_gpu), (p_o, m_o), sched, mom


def _rel_rms(a, b):
    return np.sqrt(((a - b) ** 2).sum() / (b**2).sum())


def test_step_forces_periodic_phase():
    F, info, st, (p, m, ids), (po, mo), _, m0 = _one_step(32, 250.0, 0.02, 1.0, 20, 0)
    assert st["periodic"] == 1 and st["cube_side"] == 32
    assert _rel_rms(F, info["F"]) <= 1e-5
    # kick: the momentum change carries the force error (<= 1e-5) plus float32
    # rounding of p; the drift adds float32 rounding of x (|x| < 32)
    dp, dpo = m - m0, mo - m0
    assert _rel_rms(dp, dpo) <= 2e-5
    d = np.abs(((p - po) + 16) % 32 - 16).max()
    assert d < 2e-5
    np.testing.assert_array_equal(ids, np.arange(32**3))


def test_step_forces_open_phase():
    # box so large that the lightcone is inside the mesh from the start
    F, info, st, (p, m, ids), (po, mo), sched, _ = _one_step(32, 8000.0, 0.5, 1.0, 10, 1)
    assert st["periodic"] == 0 and info["periodic"] is False
    assert (st["cube_lo"], st["cube_side"]) == (info["lo"], info["s"])
    ok = info["F"].any(axis=1)
    assert _rel_rms(F[ok], info["F"][ok]) <= 1e-5


def _a_for_side(n, box, side):
    """First a in [0.3, 0.995] whose keep radius gives an open cube of this side."""
    for a in np.linspace(0.3, 0.995, 4000):
        R = cz.chi(a, OM, OL) / (box / n) + 1.0
        lo, s, per = opm.active_cube(R, n)
        if not per and s == side:
            return a
    raise AssertionError(side)


@pytest.mark.parametrize("side", [56, 40, 28, 20, 14, 10])
def test_step_forces_open_cubes_of_factor_5_and_7(side):
    """Open cubes of side 5 * 2^j and 7 * 2^j: the levels halve down to a
    5^3 or 7^3 bottom solved by red-black SOR in one CTA."""
    a0 = _a_for_side(64, 8000.0, side)
    F, info, st, _, _, _, _ = _one_step(64, 8000.0, a0, 1.0, 10, 2)
    assert st["periodic"] == 0 and st["cube_side"] == side == info["s"]
    ok = info["F"].any(axis=1)
    assert ok.sum() > 0
    assert _rel_rms(F[ok], info["F"][ok]) <= 1e-5


def test_step_forces_full_size_sampled():
    """256^3 mesh and particles (the benchmarked launch configuration): the
    oracle recomputes the step's forces at a sample of particles."""
    n = 256
    from paper_1709_04703_gb300.sim import Sim
    pos, mom, ids = ics.workload_ics("pm256")
    sched = cz.schedule(n, 2000.0, OM, OL, 0.01, 1.0, 200)
    sim = Sim(pos, mom, ids, n, 2000.0, 0.01, 1.0, 200, rtol=1e-9, store_forces=True)
    sim.step(1)
    F = sim.forces()
    sim.close()
    k = 0
    lo, s, per = opm.active_cube(sched["R"][k], n)
    # the same float32 half drift as the kernel, so both deposit identical
    # particles; from there on the oracle is FP64
    x = opm.drift_fp32(pos, mom, sched["dtau"][k] / (2 * sched["a"][k]), n,
                       per).astype(np.float64)
    rho, _ = opm.deposit(x, n, lo, s, per)
    f, phi = opm.solve_step_potential(rho, n, lo, s, per, 1.0, sched["R"][k],
                                      sched["a_half"][k], OM)
    sample = np.random.default_rng(0).choice(n**3, 4000, replace=False)
    Fo, _ = opm.gather_force(phi, x[sample], n, lo, s, per)
    assert _rel_rms(F[sample], Fo) <= 1e-5


# --------------------------------------------------------------- shrink

@pytest.mark.parametrize("N", [1, 1000, 300001])
def test_shrink_bitexact(N):
    from paper_1709_04703_gb300.sim import Sim, pack
    n = 64
    pos, mom, ids = ics.random_particles(N, n, 11)
    sim = Sim(pos, mom, ids, n, 8000.0, 0.5, 1.0, 10)
    a = 0.7
    kept = sim.shrink(a)
    chi = cz.chi(a, OM, OL)
    R = chi / (8000.0 / n) + 1.0
    keep = opm.keep_mask(pos, R, n)
    (sp, sm, si), (lp, lm, li) = opm.shrink([pos, mom, ids], keep)
    assert kept == len(si)
    gp, gm, gi = sim.particles()
    np.testing.assert_array_equal(gi, si)
    np.testing.assert_array_equal(gp, sp)
    np.testing.assert_array_equal(gm, sm)
    cp, cm, ci, ca = sim.lightcone()
    np.testing.assert_array_equal(ci, li)
    np.testing.assert_array_equal(cp, lp)
    np.testing.assert_array_equal(cm, lm)
    assert np.all(ca == np.float32(a))
    sim.close()


def test_cell_count_overflow_is_reported():
    """More than 2^14 particles in one cell push its Q16 count past 2^62: the
    step reports PM_EOVERFLOW (the flag is read back with the solve's
    residual, not by a read of its own)."""
    from paper_1709_04703_gb300 import _lib as L
    from paper_1709_04703_gb300.sim import Sim
    n, N = 16, 20000
    pos = np.full((N, 3), 8.5, np.float32)
    mom = np.zeros((N, 3), np.float32)
    sim = Sim(pos, mom, np.arange(N, dtype=np.int32), n, 1000.0, 0.5, 1.0, 4)
    with pytest.raises(L.PmError) as err:
        sim.step(1)
    assert err.value.code == L.PM_EOVERFLOW, str(err.value)
    sim.close()


def test_all_particles_leave_and_empty_steps_run():
    from paper_1709_04703_gb300.sim import Sim
    n = 16
    pos, mom, ids = ics.zeldovich(n, -2.0, None, 2, 0.9)
    sim = Sim(pos, mom, ids, n, 60000.0, 0.9, 1.0, 4)
    sim.step(4)
    st = sim.stats()
    gp, _, gi = sim.particles()
    sim.close()
    assert st["n_active"] + st["n_lightcone"] == n**3
    # at a = 1 only the particles within the 1-cell buffer of the observer stay
    sched = cz.schedule(n, 60000.0, OM, OL, 0.9, 1.0, 4)
    assert sched["R"][-1] == 1.0
    assert st["n_active"] <= 27
    assert np.all(np.abs(gp.astype(np.float64) - n / 2).max(axis=1) <= 1.0)
    out = opm.run(pos, mom, ids, sched, n, OM, 1.0)
    assert set(gi) <= set(out["ids"]) | set(out["lc_ids"])
    assert abs(len(out["ids"]) - st["n_active"]) <= 2


# --------------------------------------------------------------- power spectrum

@pytest.mark.parametrize("n,N,shot", [(32, 32**3, False), (48, 100000, True)])
def test_power_spectrum_matches_oracle(n, N, shot):
    from paper_1709_04703_gb300.sim import power_spectrum
    if N == n**3:
        pos, _, _ = ics.zeldovich(n, -2.0, None, 0, 0.5, rms_disp=0.5)
    else:
        pos, _, _ = ics.random_particles(N, n, 9)
    p4, _ = _dev4(pos)
    k, p, m = power_spectrum(p4, 300.0, n, n // 2, subtract_shot=shot)
    ko, po, mo = opk(pos, n, 300.0, n // 2, shot_noise=shot)
    np.testing.assert_array_equal(m, mo)
    np.testing.assert_allclose(k, ko, rtol=1e-12)
    scale = np.abs(po).max()
    np.testing.assert_allclose(p, po, rtol=2e-4, atol=2e-5 * scale)


@pytest.mark.parametrize("n,N,shot", [(32, 32**3, False), (48, 100000, True)])
def test_power_spectrum_jing_matches_oracle(n, N, shot):
    """The alias-corrected estimator (Jing 2005) against the FP64 oracle:
    same slopes, same passes, P per bin to the FP32 FFT's precision."""
    from oracle.pk import power_spectrum_jing as opkj
    from paper_1709_04703_gb300.sim import power_spectrum_jing
    pos, _, _ = ics.zeldovich(n, -2.0, None, 3, 0.5, rms_disp=0.5)
    if N < n**3:
        pos = pos[np.random.default_rng(4).choice(n**3, N, replace=False)]
    p4, _ = _dev4(pos)
    k, p, m, nu, passes = power_spectrum_jing(p4, 300.0, n, n // 2, subtract_shot=shot)
    ko, po, mo, nuo, passo = opkj(pos, n, 300.0, n // 2, shot_noise=shot)
    np.testing.assert_array_equal(m, mo)
    np.testing.assert_allclose(k, ko, rtol=1e-12)
    np.testing.assert_allclose(nu, nuo, rtol=0, atol=2e-3)
    assert abs(passes - passo) <= 2
    scale = np.abs(po).max()
    np.testing.assert_allclose(p, po, rtol=3e-4, atol=3e-5 * scale)


# --------------------------------------------------------------- whole run

def test_run_pm32_power_spectrum_matches_oracle():
    """32^3 particles, 32^3 mesh, 250 Mpc/h, a 0.02 -> 1 in 20 steps,
    rtol 1e-8: final P(k) of lightcone + survivors within 0.5 %."""
    from paper_1709_04703_gb300.sim import Sim, pack, power_spectrum
    cfg = ics.WORKLOADS["pm32"]
    n = cfg["n"]
    pos, mom, ids = ics.workload_ics("pm32")
    sim = Sim(pos, mom, ids, n, cfg["box"], cfg["a_init"], cfg["a_final"], cfg["steps"],
              rtol=cfg["rtol"])
    sim.step(cfg["steps"])
    st = sim.stats()
    gp, gm, gi = sim.particles()
    cp, cm, ci, ca = sim.lightcone()
    sim.close()
    sched = cz.schedule(n, cfg["box"], OM, OL, cfg["a_init"], cfg["a_final"], cfg["steps"])
    out = opm.run(pos, mom, ids, sched, n, OM, 1.0)
    assert st["n_active"] + st["n_lightcone"] == n**3
    # the FP32 and FP64 trajectories differ by a small distance, so a particle
    # that ends a step that close to the keep cube's face may leave one step
    # earlier in one run; every differing crossing must be such a particle
    a_g, x_g = crossings.table(n**3, gi, gp, ci, cp, ca)
    a_o, x_o = crossings.table(n**3, out["ids"], out["pos"], out["lc_ids"], out["lc_pos"],
                               out["lc_a"])
    crossings.check_crossings(a_g, x_g, a_o, x_o, sched, n)
    allg = np.concatenate([gp, cp]).astype(np.float32) % n
    allo = np.concatenate([out["pos"], out["lc_pos"]]) % n
    p4, _ = _dev4(allg.astype(np.float32))
    k, pg, _ = power_spectrum(p4, cfg["box"], n, n // 2)
    _, po, _ = opk(allo, n, cfg["box"], n // 2)
    sel = slice(0, n // 4)   # k <= k_Ny / 2
    rel = np.abs(pg[sel] / po[sel] - 1)
    assert rel.max() <= 5e-3, rel
