"""Pins of the diffusion-gravity oracle (oracle/diffusion.py): the shifted
solves against closed forms, dense linear algebra and the Poisson limits,
and the backward-Euler substep against the exact decay of a mode."""
import numpy as np
import pytest

from oracle import cosmology as cz
from oracle import diffusion as df
from oracle import pm

OM, OL = 0.3, 0.7


def _mode(n, kx=1):
    x = np.arange(n)
    return np.broadcast_to(np.cos(2 * np.pi * kx * x / n)[None, None, :], (n, n, n)).copy()


def test_single_mode_decay_is_the_closed_form():
    n, sig = 16, 0.37
    phi_old = _mode(n, 2)
    lam = -4.0 * np.sin(np.pi * 2 / n) ** 2
    got = df.substep(phi_old, np.zeros((n, n, n)), sig, True)
    np.testing.assert_allclose(got, phi_old * sig / (sig - lam), rtol=1e-12, atol=1e-13)


def test_backward_euler_converges_to_the_exact_decay():
    """dPhi/dtau = (c^2 / 3H) lam Phi for a mode; one BE step of length dt
    has error O(dt^2): halving dt quarters the error."""
    n, c2, H = 16, 3.0, 0.8
    lam = -4.0 * np.sin(np.pi * 1 / n) ** 2
    phi0 = _mode(n, 1)
    errs = []
    for dt in (0.2, 0.1, 0.05):
        sig = 3 * H / (c2 * dt)
        got = df.substep(phi0, np.zeros((n, n, n)), sig, True)
        exact = phi0 * np.exp(c2 * lam * dt / (3 * H))
        errs.append(np.abs(got - exact).max())
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


def test_open_shifted_solve_matches_a_dense_solve():
    s, sig = 4, 0.6
    rng = np.random.default_rng(1)
    g = rng.standard_normal((s, s, s))
    ghost = rng.standard_normal((s + 2,) * 3)
    got = df.solve_open_shifted(g, ghost, sig)[1:-1, 1:-1, 1:-1]
    # dense matrix of sum_nb - (6 + sig) with the ghost values moved right
    N = s ** 3
    A = np.zeros((N, N))
    b = g.reshape(-1).copy()
    idx = lambda z, y, x: (z * s + y) * s + x  # noqa: E731
    for z in range(s):
        for y in range(s):
            for x in range(s):
                r = idx(z, y, x)
                A[r, r] = -6.0 - sig
                for dz, dy, dx in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1),
                                   (0, 0, -1)):
                    zz, yy, xx = z + dz, y + dy, x + dx
                    if 0 <= zz < s and 0 <= yy < s and 0 <= xx < s:
                        A[r, idx(zz, yy, xx)] = 1.0
                    else:
                        b[r] -= ghost[zz + 1, yy + 1, xx + 1]
    ref = np.linalg.solve(A, b).reshape(s, s, s)
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-12)


def test_repeated_substeps_reach_the_static_solution():
    """The fixed point of (A - sig) Phi = f - sig Phi is A Phi = f."""
    s = 8
    rng = np.random.default_rng(2)
    f = rng.standard_normal((s, s, s))
    ghost = np.zeros((s + 2,) * 3)
    ghost[0] = 0.3
    ref = pm.solve_open(f, ghost)
    phi = np.zeros((s, s, s))
    for _ in range(400):
        phi = df.substep(phi, f, 0.05, False, ghost)[1:-1, 1:-1, 1:-1]
    np.testing.assert_allclose(phi, ref[1:-1, 1:-1, 1:-1], rtol=0,
                               atol=1e-9 * np.abs(ref).max())


def test_small_shift_is_the_poisson_solve():
    n = 16
    rng = np.random.default_rng(3)
    f = rng.standard_normal((n, n, n))
    f -= f.mean()
    phi_old = rng.standard_normal((n, n, n))
    got = df.substep(phi_old, f, 1e-9, True)
    ref = pm.solve_periodic(f) + phi_old.mean()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-6 * np.abs(ref).max())


def test_c_eff_in_cells_is_independent_of_the_cell_size():
    assert df.c_eff_cells() == pytest.approx(0.019 * cz.C_OVER_H0)
    # sig: 3 H / (c^2 dtau), H = a E(a)
    a = 0.5
    assert df.sigma(a, 0.01, OM, OL, 10.0) == pytest.approx(
        3 * a * np.sqrt(OM / a**3 + OL) / (100.0 * 0.01))


def test_fast_light_step_is_the_poisson_step():
    """With c_eff -> infinity (sig -> 0) a diffusion step's kick equals the
    static step's."""
    n = 16
    rng = np.random.default_rng(4)
    pos = rng.uniform(0, n, (200, 3))
    mom = rng.uniform(-0.1, 0.1, (200, 3))
    sched = cz.schedule(n, 200.0, OM, OL, 0.5, 1.0, 4)
    nbar = 200 / n**3
    phi0, geo = df.initial_field(pos, sched, n, OM, nbar)
    p1, m1, _, info = df.step(pos.copy(), mom.copy(), (phi0, geo), 0, sched, n, OM, OL, nbar,
                              c_cells=1e9, want=True)
    p2, m2, info2 = pm.step(pos.copy(), mom.copy(), 0, sched, n, OM, nbar, want=True)
    np.testing.assert_allclose(info["F"], info2["F"], rtol=0, atol=1e-8 * np.abs(info2["F"]).max())
    np.testing.assert_allclose(m1, m2, rtol=0, atol=1e-10)


# ---------------------------------------------------------------- ADE scheme

def _ade_dense(phi_old, f, lam, upward, periodic, ghost=None):
    """The ADE sweep as one linear solve: cell c (flat lexicographic index)
    is coupled to its neighbours with a smaller index (upward; larger
    downward) at the new level, to the others at the old level."""
    n = f.shape[0]
    N = n**3
    A = np.zeros((N, N))
    b = np.zeros(N)
    flat = lambda z, y, x: (z * n + y) * n + x  # noqa: E731
    for z in range(n):
        for y in range(n):
            for x in range(n):
                c = flat(z, y, x)
                rhs = -lam * f[z, y, x]
                m_new = 0
                for ax in range(3):
                    for sg in (-1, 1):
                        q = [z, y, x]
                        q[ax] += sg
                        inside = 0 <= q[ax] < n
                        if periodic:
                            q[ax] %= n
                            inside = True
                        if inside:
                            qc = flat(*q)
                            new = qc < c if upward else qc > c
                            if new:
                                A[c, qc] -= lam
                            else:
                                rhs += lam * phi_old[q[0], q[1], q[2]]
                        else:
                            g = ghost[q[0] + 1, q[1] + 1, q[2] + 1]
                            new = (q[ax] < 0) if upward else (q[ax] >= n)
                            rhs += lam * g
                        m_new += 1 if new else 0
                A[c, c] += 1 + lam * m_new
                b[c] = rhs + (1 - lam * (6 - m_new)) * phi_old[z, y, x]
    return np.linalg.solve(A, b).reshape(n, n, n)


@pytest.mark.parametrize("periodic,upward", [(False, True), (False, False), (True, True),
                                             (True, False)])
def test_ade_sweep_is_its_triangular_system(periodic, upward):
    n, lam = 4, 0.7
    rng = np.random.default_rng(5)
    phi = rng.standard_normal((n, n, n))
    f = rng.standard_normal((n, n, n))
    ghost = None if periodic else rng.standard_normal((n + 2,) * 3)
    got = df.ade_substep(phi, f, lam, upward, periodic, ghost)
    if not periodic:
        np.testing.assert_array_equal(got[0], ghost[0])
        got = got[1:-1, 1:-1, 1:-1]
    ref = _ade_dense(phi, f, lam, upward, periodic, ghost)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_ade_sweeps_converge_to_the_poisson_solution():
    """The fixed point of an ADE sweep is lap Phi = f: alternating sweeps
    with a fixed source reach the static solution (open and periodic)."""
    s = 6
    rng = np.random.default_rng(6)
    f = rng.standard_normal((s, s, s))
    ghost = np.zeros((s + 2,) * 3)
    ghost[0] = 0.2
    ghost[:, -1] = -0.1
    ref = pm.solve_open(f, ghost)[1:-1, 1:-1, 1:-1]
    phi = np.zeros((s, s, s))
    for it in range(120):
        phi = df.ade_substep(phi, f, 1.0, it % 2 == 0, False, ghost)[1:-1, 1:-1, 1:-1]
    np.testing.assert_allclose(phi, ref, rtol=0, atol=1e-8 * np.abs(ref).max())
    fp = f - f.mean()
    refp = pm.solve_periodic(fp)
    phi = np.zeros((s, s, s))
    for it in range(160):
        phi = df.ade_substep(phi, fp, 1.0, it % 2 == 0, True)
    np.testing.assert_allclose(phi - phi.mean(), refp, rtol=0, atol=1e-8 * np.abs(refp).max())


def test_ade_small_step_follows_the_diffusion_equation():
    """For a smooth mode with no source, one up + down pair with lam -> 0
    approaches the exact decay exp(2 lam lap_k); the error shrinks as lam does."""
    n = 12
    phi0 = _mode(n, 1)
    lapk = -4.0 * np.sin(np.pi / n) ** 2
    errs = []
    for lam in (0.2, 0.1, 0.05):
        u = df.ade_substep(phi0, np.zeros((n, n, n)), lam, True, True)
        u = df.ade_substep(u, np.zeros((n, n, n)), lam, False, True)
        errs.append(np.abs(u - phi0 * np.exp(2 * lam * lapk)).max())
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.01, errs
