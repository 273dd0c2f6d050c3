"""Pins of the oracle's PM step against exact arithmetic, closed forms,
brute force and conservation laws (no GPU)."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy.special import erf

from oracle import cosmology as cz
from oracle import pm
from paper_1709_04703_gb300 import ics

OM, OL = 0.3, 0.7


# ---------------------------------------------------------------- deposit

def _rational_cic(pos, n):
    """CIC weights from exact rational arithmetic on the float32 value:
    nodes at cell centres, weight 1 - |u - node| per axis, quantised down to
    multiples of 2^-16 on the upper node."""
    rho = {}
    for p in pos:
        axes = []
        for u in p:
            v = Fraction(float(u)) - Fraction(1, 2)
            i = math.floor(v)
            frac = v - i
            dq = math.floor(frac * 65536)
            axes.append(((i % n, 65536 - dq), ((i + 1) % n, dq)))
        for (x, wx), (y, wy), (z, wz) in itertools.product(*axes):
            rho[(z, y, x)] = rho.get((z, y, x), 0) + wx * wy * wz
    return rho


def test_deposit_matches_rational_brute_force():
    n = 8
    pos, _, _ = ics.random_particles(40, n, seed=3)
    pos[0] = [0.5, 0.5, 0.5]          # exactly on a node
    pos[1] = [1.0, 2.0, 3.0]          # on cell faces: equal split
    pos[2] = [0.1, 7.9, 0.25]         # wraps in x and y
    rho, esc = pm.deposit(pos, n, 0, n, True)
    ref = _rational_cic(pos, n)
    assert esc == 0
    dense = np.zeros_like(rho)
    for k, v in ref.items():
        dense[k] = v
    np.testing.assert_array_equal(rho, dense)


def test_deposit_mass_is_exact():
    n = 16
    pos, _, _ = ics.random_particles(5000, n, seed=1)
    rho, _ = pm.deposit(pos, n, 0, n, True)
    assert int(rho.sum()) == 5000 * 2**48
    one, _ = pm.deposit(np.array([[3.5, 4.5, 5.5]], np.float32), n, 0, n, True)
    assert one[5, 4, 3] == 2**48 and int(one.sum()) == 2**48
    corner, _ = pm.deposit(np.array([[4.0, 4.0, 4.0]], np.float32), n, 0, n, True)
    np.testing.assert_array_equal(corner[3:5, 3:5, 3:5], np.full((2, 2, 2), 2**45))


def test_deposit_open_counts_escapes():
    n, lo, s = 32, 8, 16
    pos = np.array([[16.0, 16.0, 16.0],     # inside
                    [8.6, 16.0, 16.0],      # node 8 and 9: inside
                    [8.4, 16.0, 16.0],      # node 7: outside
                    [23.5, 23.5, 23.5],     # nodes 23, 24 -> 24 outside... 23.5-0.5=23 -> 23,24
                    [23.4, 20.0, 20.0]],    # nodes 22, 23: inside
                   np.float32)
    rho, esc = pm.deposit(pos, n, lo, s, False)
    assert esc == 2
    assert int(rho.sum()) == 3 * 2**48
    assert int(rho[:lo].sum()) == 0 and int(rho[lo + s:].sum()) == 0


# ---------------------------------------------------------------- solve

def test_periodic_single_mode_exact():
    n = 16
    x = np.arange(n)
    m = (1, 3, 2)
    f = (np.cos(2 * np.pi * m[0] * x / n)[None, None, :]
         * np.cos(2 * np.pi * m[1] * x / n)[None, :, None]
         * np.cos(2 * np.pi * m[2] * x / n)[:, None, None])
    lam = -4 * sum(math.sin(math.pi * k / n) ** 2 for k in m)
    np.testing.assert_allclose(pm.solve_periodic(f), f / lam, atol=1e-13)


def _dense_open_solve(f, ghost):
    s = f.shape[0]
    N = s**3
    A = np.zeros((N, N))
    b = f.ravel().copy()
    idx = lambda z, y, x: (z * s + y) * s + x
    for z, y, x in itertools.product(range(s), repeat=3):
        r = idx(z, y, x)
        A[r, r] = -6.0
        for dz, dy, dx in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0),
                           (0, 0, 1), (0, 0, -1)]:
            zz, yy, xx = z + dz, y + dy, x + dx
            if 0 <= zz < s and 0 <= yy < s and 0 <= xx < s:
                A[r, idx(zz, yy, xx)] = 1.0
            else:
                b[r] -= ghost[zz + 1, yy + 1, xx + 1]
    return np.linalg.solve(A, b).reshape(s, s, s)


def test_open_solve_matches_dense_solve():
    rng = np.random.default_rng(5)
    s = 7
    f = rng.standard_normal((s, s, s))
    ghost = rng.standard_normal((s + 2,) * 3)
    out = pm.solve_open(f, ghost)
    np.testing.assert_allclose(out[1:-1, 1:-1, 1:-1], _dense_open_solve(f, ghost),
                               rtol=1e-11, atol=1e-12)
    # ghosts are left untouched
    g = ghost.copy()
    g[1:-1, 1:-1, 1:-1] = out[1:-1, 1:-1, 1:-1]
    np.testing.assert_array_equal(out, g)


def test_multipole_boundary_matches_direct_sum():
    n, lo, s, S = 32, 0, 32, 2.0
    delta = np.zeros((s, s, s))
    delta[16, 16, 19] = 3.0      # off-centre: dipole and quadrupole matter
    delta[14, 17, 15] = -1.0
    delta[15, 15, 16] = 0.5
    ghost = pm.open_ghost_potential(S * delta, S, lo, n)
    coords = np.arange(lo - 1, lo + s + 1) + 0.5 - n / 2
    src = np.argwhere(delta != 0)
    err_max, scale = 0.0, 0.0
    for (gz, gy, gx) in [(0, 5, 7), (20, 0, 33), (33, 33, 33), (10, 33, 1)]:
        p = np.array([coords[gx], coords[gy], coords[gz]])
        direct = 0.0
        for (z, y, x) in src:
            q = np.array([x, y, z]) + lo + 0.5 - n / 2
            direct += -S / (4 * math.pi) * delta[z, y, x] / np.linalg.norm(p - q)
        err_max = max(err_max, abs(ghost[gz, gy, gx] - direct))
        scale = max(scale, abs(direct))
    # octupole remainder ~ (source extent / distance)^3 ~ (3.5/16)^3
    assert err_max < 2e-2 * scale


def _gaussian_problem(s, om=OM, a=0.5):
    n = s
    sigma = s / 10.0
    c = n / 2
    g = np.arange(s) + 0.5 - c
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    r = np.sqrt(X**2 + Y**2 + Z**2)
    A = 1.0
    delta = A * np.exp(-r**2 / (2 * sigma**2))
    S = pm.source_S(a, om)
    f = S * delta
    phi = pm.solve_open(f, pm.open_ghost_potential(f, S, 0, n))
    exact = -(S / (4 * math.pi)) * A * (2 * math.pi * sigma**2) ** 1.5 * erf(
        r / (math.sqrt(2) * sigma)) / r
    return phi[1:-1, 1:-1, 1:-1], exact


def test_gaussian_potential_converges_second_order():
    errs = []
    for s in (16, 32, 64):
        phi, exact = _gaussian_problem(s)
        errs.append(np.sqrt(np.mean((phi - exact) ** 2)) / np.sqrt(np.mean(exact**2)))
    assert errs[2] < 5e-3
    assert 3.0 < errs[0] / errs[1] < 5.0
    assert 3.0 < errs[1] / errs[2] < 5.0


def test_uniform_sphere_potential():
    s = 64
    c = s / 2
    R = 10.0
    g = np.arange(s) + 0.5 - c
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    r = np.sqrt(X**2 + Y**2 + Z**2)
    d0 = 1.0
    delta = np.where(r <= R, d0, 0.0)
    S = 1.0
    phi = pm.solve_open(S * delta, pm.open_ghost_potential(S * delta, S, 0, s))
    phi = phi[1:-1, 1:-1, 1:-1]
    M = delta.sum()                           # discrete mass of the sphere
    Reff = (3 * M / (4 * math.pi)) ** (1 / 3)  # radius holding that mass
    exact = np.where(r <= Reff, S * d0 * (r**2 - 3 * Reff**2) / 6,
                     -S * d0 * Reff**3 / (3 * r))
    far = r > 1.5 * R
    inner = r < 0.5 * R
    assert np.max(np.abs(phi[far] - exact[far]) / np.abs(exact[far])) < 3e-3
    assert np.max(np.abs(phi[inner] - exact[inner]) / np.abs(exact[inner])) < 3e-2


# ---------------------------------------------------------------- forces

def _forces(pos, n, periodic, R=None, a=0.5, lo=None, s=None):
    if periodic:
        lo, s = 0, n
        R = n
    rho, _ = pm.deposit(pos, n, lo, s, periodic)
    f, phi = pm.solve_step_potential(rho, n, lo, s, periodic, 1.0, R, a, OM)
    F, esc = pm.gather_force(phi, pos, n, lo, s, periodic)
    return F, esc


def test_single_particle_feels_no_self_force():
    n = 16
    pos = np.array([[3.3, 7.8, 11.1]], np.float32)
    F, _ = _forces(pos, n, True)
    np.testing.assert_allclose(F, 0.0, atol=1e-13)


def test_two_particles_antisymmetric_and_attractive_periodic():
    n = 16
    pos = np.array([[5.25, 8.0, 8.0], [10.75, 8.0, 8.0]], np.float32)
    F, _ = _forces(pos, n, True)
    np.testing.assert_allclose(F[0], -F[1], atol=1e-14)
    # Phi has its well at each particle, so grad Phi at particle 0 points
    # away from particle 1; the kick -a grad(Phi) dtau then attracts
    assert F[0, 0] < 0 and F[1, 0] > 0


def test_two_particle_inverse_square_law_open():
    n = 64
    S = pm.source_S(0.5, OM)
    R, lo, s = 30.5, 0, 64
    out = []
    for d in (4.0, 6.0, 8.0, 12.0):
        pos = np.array([[32.0 - d / 2 + 0.5, 32.5, 32.5],
                        [32.0 + d / 2 + 0.5, 32.5, 32.5]], np.float32)
        rho, _ = pm.deposit(pos, n, lo, s, False)
        # no background: source of two unit masses only
        f = S * rho[lo:lo + s, lo:lo + s, lo:lo + s].astype(np.float64) / 2**48
        phi = pm.solve_open(f, pm.open_ghost_potential(f, S, lo, n))
        F, _ = pm.gather_force(phi, pos, n, lo, s, False)
        expected = S / (4 * math.pi * d * d)   # |grad Phi| of a unit mass
        assert F[0, 0] < 0 and F[1, 0] > 0
        out.append(-F[0, 0] / expected)
    # discretisation error of the 7-point Green's function + centred
    # gradient falls off as 1/d^2 relative to the inverse-square force
    for d, x in zip((4.0, 6.0, 8.0, 12.0), out):
        assert abs(x - 1) < 2.5 / d**2, out
    assert abs(out[-1] - 1) < 0.02


def test_lattice_feels_no_force_and_momentum_conserved():
    n = 8
    g = np.arange(n) + 0.5
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    lat = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1).astype(np.float32)
    F, _ = _forces(lat, n, True)
    np.testing.assert_allclose(F, 0.0, atol=1e-12)
    pos, _, _ = ics.random_particles(300, n, seed=9)
    F, _ = _forces(pos, n, True)
    assert np.abs(F.sum(axis=0)).max() < 1e-11 * np.abs(F).sum()


# ---------------------------------------------------------------- geometry + shrink

def test_active_cube_rules():
    assert pm.active_cube(200.0, 256) == (0, 256, True)
    assert pm.is_open(127.0, 256) and not pm.is_open(127.01, 256)
    lo, s, per = pm.active_cube(60.2, 256)       # m = 62 -> 2m = 124 -> 128
    assert (lo, s, per) == (64, 128, False)
    lo, s, per = pm.active_cube(40.0, 256)       # m = 41 -> 82 -> 96
    assert (lo, s, per) == (80, 96, False)
    lo, s, per = pm.active_cube(1.0, 32)         # m = 2 -> 4
    assert (lo, s, per) == (14, 4, False)
    lo, s, per = pm.active_cube(50.0, 256)       # m = 51 -> 102 -> 112 = 7 * 16
    assert (lo, s, per) == (72, 112, False)
    lo, s, per = pm.active_cube(35.0, 256)       # m = 36 -> 72 -> 80 = 5 * 16
    assert (lo, s, per) == (88, 80, False)
    lo, s, per = pm.active_cube(1.5, 32)         # m = 3 -> 6
    assert (lo, s, per) == (13, 6, False)
    # the cube holds the keep cube plus the CIC reach on both sides
    for R in np.linspace(1.0, 126.9, 500):
        lo, s, per = pm.active_cube(R, 256)
        m = math.ceil(R) + 1
        assert lo <= 128 - m and lo + s >= 128 + m
        q = s
        while q % 2 == 0:
            q //= 2
        assert q in (1, 3, 5, 7)


def test_shrink_is_stable_partition():
    rng = np.random.default_rng(0)
    n = 32
    pos = rng.uniform(0, n, (1000, 3))
    ids = np.arange(1000)
    R = 9.3
    keep = pm.keep_mask(pos, R, n)
    (sp, si), (lp, li) = pm.shrink([pos, ids], keep)
    ref_keep = [i for i in range(1000)
                if max(abs(pos[i, d] - 16.0) for d in range(3)) <= R]
    assert list(si) == ref_keep
    assert list(li) == [i for i in range(1000) if i not in set(ref_keep)]
    assert len(si) + len(li) == 1000


def test_keep_boundary_is_inclusive():
    pos = np.array([[16 + 9.5, 16.0, 16.0], [16 - 9.5, 16, 16],
                    [np.nextafter(np.float32(25.5), np.float32(30)), 16, 16]],
                   np.float32)
    assert list(pm.keep_mask(pos, 9.5, 32)) == [True, True, False]


def test_background_weights_partition_the_keep_interval():
    """The tents of all cells sum to one at every point, so the weights of
    the keep interval [c - R, c + R] sum to its length 2R, whatever R."""
    n = 64
    for R in (1.0, 3.5, 7.25, 12.0, 19.999):
        lo, s, _ = pm.active_cube(R, n)
        w = pm.background_weights(R, n, lo, s, False)
        assert abs(w.sum() - 2 * R) < 1e-12, R
        assert w.min() >= 0 and w.max() <= 1
        np.testing.assert_allclose(w, w[::-1], rtol=0, atol=1e-14)   # centred on c = n/2
        x = np.arange(lo, lo + s) + 0.5
        assert np.all(w[np.abs(x - n / 2) <= R - 1] == 1.0)
        assert np.all(w[np.abs(x - n / 2) >= R + 1] == 0.0)
    assert np.all(pm.background_weights(5.0, 32, 0, 32, True) == 1.0)
    # tent integral: 0, 1/2 at the node, 1, and the quadratic pieces
    np.testing.assert_allclose(pm.tent_integral([-2.0, -1.0, -0.5, 0.0, 0.5, 1.0, 3.0]),
                               [0.0, 0.0, 0.125, 0.5, 0.875, 1.0, 1.0], rtol=0, atol=0)


def test_uniform_density_has_zero_contrast_on_every_cell():
    """Particles filling the keep cube uniformly: delta sums to zero exactly
    (the deposit conserves mass, the background sums to (2R)^3) and its
    mean over each plane of cells, the edge planes included, is zero to the
    sampling noise."""
    n, R, N = 32, 9.3, 3_000_000
    rng = np.random.default_rng(12)
    pos = n / 2 + rng.uniform(-R, R, (N, 3))
    lo, s, per = pm.active_cube(R, n)
    rho, esc = pm.deposit(pos, n, lo, s, per)
    assert esc == 0
    nbar = N / (2 * R) ** 3                      # the density inside the cube
    d = pm.delta_cube(rho, n, lo, s, nbar, R, per)
    assert abs(d.sum()) < 1e-9 * (2 * R) ** 3
    layer = d.mean(axis=(0, 1)) * s * s / np.count_nonzero(
        pm.background_weights(R, n, lo, s, per)) ** 2
    assert np.abs(layer).max() < 0.02, layer


# ---------------------------------------------------------------- dynamics

def test_free_particle_drift_integrates_schedule():
    n = 16
    sched = cz.schedule(n, 100.0, OM, OL, 0.02, 0.1, 10)
    pos = np.array([[3.0, 5.0, 7.0]])
    mom = np.array([[0.01, -0.02, 0.005]])
    out = pm.run(pos, mom, np.array([0]), sched, n, OM, 1.0 / n**3)
    coef = sum(sched["dtau"][k] * (0.5 / sched["a"][k] + 0.5 / sched["a"][k + 1])
               for k in range(10))
    np.testing.assert_allclose(out["pos"], pos + mom * coef, rtol=1e-12)
    np.testing.assert_allclose(out["mom"], mom, atol=1e-15)


def test_momentum_conserved_and_mass_bookkept():
    n = 16
    pos, mom, ids = ics.zeldovich(n, -2.0, None, 4, 0.02)
    sched = cz.schedule(n, 250.0, OM, OL, 0.02, 1.0, 8)
    out = pm.run(pos, mom, ids, sched, n, OM, 1.0, steps=4)
    p0 = mom.astype(np.float64).sum(axis=0)
    assert np.abs(out["mom"].sum(axis=0) - p0).max() < 1e-12 * np.abs(out["mom"]).sum()
    assert len(out["ids"]) + len(out["lc_ids"]) == n**3


def _plane_wave_growth(n, steps, a0=0.02, a1=0.3, eps=1e-3):
    g = np.arange(n) + 0.5
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    q = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    psi = eps * np.sin(2 * np.pi * q[:, 0] / n)
    pos = q.copy()
    pos[:, 0] += psi
    mom = np.zeros_like(pos)
    mom[:, 0] = a0**2 * cz.E(a0, OM, OL) * cz.growth_f(a0, OM, OL) * psi
    sched = cz.schedule(n, 250.0, OM, OL, a0, a1, steps)
    out = pm.run(pos, mom, np.arange(len(pos)), sched, n, OM, 1.0)
    sel = np.abs(psi) > 0.5 * eps
    growth = np.median((out["pos"][sel, 0] - q[sel, 0]) / psi[sel])
    return 1 - growth / (cz.growth_D(a1, OM, OL) / cz.growth_D(a0, OM, OL))


def test_zeldovich_plane_wave_growth_converges_to_linear_theory():
    """A small plane-wave displacement grows like D(a) (Zel'dovich regime);
    the PM deficit of the fundamental mode vanishes as h^2."""
    d16 = _plane_wave_growth(16, 100)
    d32 = _plane_wave_growth(32, 100)
    assert 0 < d32 < 0.03
    assert 3.0 < d16 / d32 < 5.0


def test_shrinking_run_bookkeeping():
    n = 16
    pos, mom, ids = ics.zeldovich(n, -2.0, None, 2, 0.5)
    # tiny box so that the lightcone crosses it mid-run
    sched = cz.schedule(n, 4000.0, OM, OL, 0.5, 1.0, 6)
    out = pm.run(pos, mom, ids, sched, n, OM, 1.0)
    assert len(out["ids"]) + len(out["lc_ids"]) == n**3
    assert np.all(np.diff(out["n_active"]) <= 0)
    assert sorted(np.concatenate([out["ids"], out["lc_ids"]])) == list(range(n**3))
    R = sched["R"][-1]
    assert np.all(np.abs(out["pos"] - n / 2).max(axis=1) <= R)


def test_fixed_box_record_bookkeeping():
    """Without shrinking every particle stays active; each one is catalogued
    at most once, at the end of a step after which it lies outside the keep
    cube, and in index order within a step."""
    n = 16
    pos, mom, ids = ics.zeldovich(n, -2.0, None, 2, 0.5)
    sched = cz.schedule(n, 4000.0, OM, OL, 0.5, 1.0, 6)
    out = pm.run(pos, mom, ids, sched, n, OM, 1.0, record_only=True)
    assert len(out["ids"]) == n**3 and np.all(out["n_active"] == n**3)
    assert len(np.unique(out["lc_ids"])) == len(out["lc_ids"]) == out["recorded"].sum()
    assert set(out["lc_ids"]) == set(out["ids"][out["recorded"]])
    for a in np.unique(out["lc_a"]):
        k1 = int(np.argmin(np.abs(sched["a"] - a)))
        sel = out["lc_a"] == a
        assert np.all(np.abs(out["lc_pos"][sel] - n / 2).max(axis=1) > sched["R"][k1])
        assert np.all(np.diff(out["lc_ids"][sel]) > 0)     # ids are the index order here
    # a particle never catalogued is inside the final keep cube, or was
    # inside at every check (R shrinks, so it is inside now)
    rest = ~out["recorded"]
    assert np.all(np.abs(out["pos"][rest] - n / 2).max(axis=1) <= sched["R"][-1])


def test_fixed_box_record_equals_shrink_without_forces():
    """With gravity switched off (Omega_m -> 0: no source) trajectories do
    not depend on the boundary, so the catalogue of the fixed-box record
    is the shrinking run's lightcone: same particles, order, a, positions."""
    n, om = 16, 1e-12
    pos, mom, ids = ics.zeldovich(n, -2.0, None, 3, 0.5, om=om, ol=1 - om)
    mom = mom + np.float32(0.02) * np.sign(pos - n / 2).astype(np.float32)   # outward streaming
    sched = cz.schedule(n, 4000.0, om, 1 - om, 0.5, 1.0, 8)
    shr = pm.run(pos, mom, ids, sched, n, om, 1.0)
    rec = pm.run(pos, mom, ids, sched, n, om, 1.0, record_only=True)
    assert len(shr["lc_ids"]) > n**3 // 4
    np.testing.assert_array_equal(rec["lc_ids"], shr["lc_ids"])
    np.testing.assert_array_equal(rec["lc_a"], shr["lc_a"])
    np.testing.assert_allclose(rec["lc_pos"], shr["lc_pos"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(rec["lc_mom"], shr["lc_mom"], rtol=0, atol=1e-12)


def test_drift_fp32_exact_cases_and_wrap():
    """drift_fp32 follows float32 arithmetic: exact where float32 is exact,
    and the periodic wrap lands in [0, n)."""
    n = 16
    pos = np.array([[1.0, 15.75, 0.25], [8.0, 8.0, 8.0]], np.float32)
    mom = np.array([[0.5, 0.5, -1.0], [2.0 ** -10, -3.0, 0.0]], np.float32)
    x = pm.drift_fp32(pos, mom, 0.5, n, True)
    np.testing.assert_array_equal(x, np.array([[1.25, 0.0, 15.75],
                                               [8.0 + 2.0 ** -11, 6.5, 8.0]], np.float32))
    assert x.dtype == np.float32
    # a tiny negative step rounds to n in float32 and must wrap to 0
    y = pm.drift_fp32(np.array([[0.0, 1.0, 1.0]], np.float32),
                       np.array([[-1e-9, 0, 0]], np.float32), 1.0, n, True)
    assert 0.0 <= y[0, 0] < n
    # one rounding per operation: 1 + 2^-24 rounds to 1 in float32
    z = pm.drift_fp32(np.array([[1.0, 1.0, 1.0]], np.float32),
                       np.array([[2.0 ** -24, 0, 0]], np.float32), 1.0, n, False)
    assert z[0, 0] == np.float32(1.0)


# ---------------------------------------------------------------- TSC variant

def test_tsc_weights_are_exact_and_sum_to_one():
    """Q16 TSC weights from exact rational arithmetic on the float position:
    q = floor(2^16 u) - 2^16 i, outer nodes floor((2^16 - q)^2 / 2^17) and
    floor(q^2 / 2^17), the centre the remainder; within 3 * 2^-16 of the
    kernel 3/4 - d^2 at the exact offset d = u - (i + 1/2)."""
    rng = np.random.default_rng(3)
    pos = rng.uniform(0, 16, (200, 3)).astype(np.float32)
    i, w = pm.tsc_index(pos)
    assert np.all(w.sum(axis=-1) == 2**16)
    for p, ii, ww in zip(pos[:50], i[:50], w[:50]):
        for ax in range(3):
            u = Fraction(float(p[ax]))
            c = math.floor(u)
            q = math.floor(u * 2**16) - c * 2**16
            d = u - c - Fraction(1, 2)
            wm = math.floor(Fraction((2**16 - q) ** 2, 2**17))
            wp = math.floor(Fraction(q * q, 2**17))
            assert ii[ax] == c and ww[ax, 0] == wm and ww[ax, 2] == wp
            assert abs(ww[ax, 1] / 2**16 - float(Fraction(3, 4) - d * d)) <= 3 * 2.0**-16


def test_tsc_deposit_conserves_mass_and_a_lattice_is_uniform():
    n = 8
    pos, _, _ = ics.random_particles(500, n, seed=4)
    rho, esc = pm.deposit_tsc(pos, n, 0, n, True)
    assert esc == 0 and int(rho.astype(object).sum()) == 500 * 2**48
    g = np.arange(n) + 0.5
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    lat = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1).astype(np.float32)
    rho, _ = pm.deposit_tsc(lat, n, 0, n, True)
    assert np.all(rho == 2**48)


def test_tsc_background_partitions_the_keep_interval():
    np.testing.assert_allclose(pm.tsc_integral([-2, -1.5, -0.5, 0, 0.5, 1.5, 2]),
                               [0, 0, 1 / 6, 0.5, 5 / 6, 1, 1], rtol=0, atol=1e-15)
    u = np.linspace(-1.6, 1.6, 3201)
    c = pm.tsc_integral(u)
    assert np.all(np.diff(c) >= 0) and np.max(np.abs(np.diff(c))) < 1e-3   # continuous
    n = 64
    for R in (2.0, 7.3, 15.5):
        lo, s, _ = pm.active_cube(R, n, 2)
        w = pm.background_weights(R, n, lo, s, False, "tsc")
        assert abs(w.sum() - 2 * R) < 1e-12


def test_tsc_forces_conserve_momentum_and_follow_the_inverse_square():
    n = 16
    pos, _, _ = ics.random_particles(300, n, seed=9)
    rho, _ = pm.deposit_tsc(pos, n, 0, n, True)
    f = pm.source_S(0.5, OM) * (rho / (300 * 2**48 / n**3) - 1.0)
    F, _ = pm.gather_force_tsc(pm.solve_periodic(f), pos, n, 0, n, True)
    assert np.abs(F.sum(axis=0)).max() < 1e-11 * np.abs(F).sum()
    n = 64
    S = pm.source_S(0.5, OM)
    for d in (8.0, 12.0):
        p2 = np.array([[32.0 - d / 2 + 0.5, 32.5, 32.5], [32.0 + d / 2 + 0.5, 32.5, 32.5]],
                      np.float32)
        rho, _ = pm.deposit_tsc(p2, n, 0, n, False)
        f = S * rho.astype(np.float64) / 2**48
        phi = pm.solve_open(f, pm.open_ghost_potential(f, S, 0, n))
        F, _ = pm.gather_force_tsc(phi, p2, n, 0, n, False)
        ratio = -F[0, 0] / (S / (4 * math.pi * d * d))
        assert abs(ratio - 1) < 2.5 / d**2, (d, ratio)


# ---------------------------------------------------------------- spherical domain

def test_sphere_keep_rule_is_exact():
    rng = np.random.default_rng(13)
    n, R = 32, 9.3
    pos = (n / 2 + rng.uniform(-10, 10, (2000, 3))).astype(np.float32)
    got = pm.keep_mask(pos, R, n, "sphere")
    Rf = Fraction(R)
    ref = [sum((Fraction(float(v)) - n // 2) ** 2 for v in p) <= Rf * Rf for p in pos]
    assert list(got) == ref
    assert 0 < got.sum() < len(pos)


def test_ball_background_has_the_ball_volume_and_its_symmetry():
    n = 32
    for R, tol in ((3.2, 3e-4), (9.3, 5e-5), (14.0, 5e-5)):   # the rule's error ~ 1/R^2
        lo, s, _ = pm.active_cube(R, n)
        W = pm.background_ball(R, n, lo, s)
        assert abs(W.sum() / (4 / 3 * math.pi * R**3) - 1) < tol, R
        assert W.min() >= -1e-12 and W.max() <= 1 + 1e-12
        np.testing.assert_allclose(W, W[::-1, ::-1, ::-1], rtol=0, atol=1e-12)
        np.testing.assert_allclose(W, W.transpose(0, 2, 1), rtol=0, atol=1e-12)
        # z is integrated in closed form, x and y by the rule, whose error per
        # cell (the chord length has a square-root edge) is below 1e-2
        np.testing.assert_allclose(W, W.transpose(2, 1, 0), rtol=0, atol=1e-2)


def test_uniform_density_in_the_ball_has_zero_contrast():
    n, R, N = 32, 9.3, 3_000_000
    rng = np.random.default_rng(14)
    v = rng.normal(size=(N, 3))
    v *= (R * rng.uniform(0, 1, N) ** (1 / 3) / np.linalg.norm(v, axis=1))[:, None]
    pos = n / 2 + v
    lo, s, per = pm.active_cube(R, n)
    rho, esc = pm.deposit(pos, n, lo, s, per)
    assert esc == 0
    nbar = N / (4 / 3 * math.pi * R**3)
    d = pm.delta_cube(rho, n, lo, s, nbar, R, per, domain="sphere")
    assert abs(d.sum()) < 1e-4 * 4 / 3 * math.pi * R**3
    a1 = np.arange(lo, lo + s) + 0.5 - n / 2
    AZ, AY, AX = np.meshgrid(a1, a1, a1, indexing="ij")
    r = np.sqrt(AX**2 + AY**2 + AZ**2)
    for r0 in np.arange(R - 2.0, R + 1.5, 0.5):    # shells across the surface
        sel = (r >= r0) & (r < r0 + 0.5)
        assert abs(d[sel].mean()) < 0.03, (r0, d[sel].mean())


def test_cell_order_worked_example():
    """A hand-sorted case: cells of the CIC base node, z slowest, x fastest,
    ties in input order, wrap of floor(u - 1/2) = -1 to n - 1."""
    n = 4
    pos = np.array([[1.7, 0.5, 0.5],    # cell (1, 0, 0): key 1
                    [0.5, 0.5, 0.5],    # (0, 0, 0): key 0
                    [0.4, 0.5, 0.5],    # x cell -1 -> 3: key 3
                    [1.5, 2.6, 0.5],    # (1, 2, 0): key 9
                    [1.9, 0.6, 0.99],   # (1, 0, 0): key 1, after particle 0
                    [0.5, 0.5, 1.5],    # (0, 0, 1): key 16
                    [3.6, 3.6, 3.6],    # (3, 3, 3): key 63
                    [0.5, 0.5, 0.2]])   # z cell -1 -> 3: key 48
    np.testing.assert_array_equal(pm.cell_order(pos, n), [1, 0, 4, 2, 3, 5, 7, 6])


def test_cell_order_is_a_stable_sort_by_cell():
    """Keys non-decreasing along the order, input order kept among equal
    keys, every particle once; keys read from the CIC base node."""
    rng = np.random.default_rng(21)
    n = 16
    centres = rng.integers(0, n, (40, 3)) + 0.5
    pos = (centres[rng.integers(0, 40, 3000)] + rng.uniform(-0.4, 0.4, (3000, 3))) % n
    o = pm.cell_order(pos.astype(np.float32), n)
    assert sorted(o.tolist()) == list(range(3000))
    i, _ = pm.cic_index(pos.astype(np.float32))
    i %= n
    key = (i[:, 2] * n + i[:, 1]) * n + i[:, 0]
    k = key[o]
    assert np.all(np.diff(k) >= 0)
    assert np.all(np.diff(o)[np.diff(k) == 0] > 0)
    # non-finite coordinates count as cell 0
    bad = np.array([[np.nan, 1.5, 1.5], [np.inf, 0.5, 0.5], [0.5, 0.5, 0.5]], np.float32)
    assert pm.cell_order(bad, n).tolist() == [1, 2, 0]
