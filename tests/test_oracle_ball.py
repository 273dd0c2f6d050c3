"""Pins of the oracle's masked solve on the ball (domain "ball"): the
unknowns are the cells within R + 2 of the centre, the cells next to them
hold Dirichlet values.  The pins are independent of the oracle's sparse
assembly: a loop-built mask, quadratic potentials that the 7-point stencil
differentiates exactly, and a dense solve of a loop-built system."""
import itertools
import math

import numpy as np

from oracle import pm


def test_ball_mask_matches_a_loop():
    n, lo, s, R = 16, 2, 12, 3.7
    m = pm.ball_mask(R, n, lo, s)
    for k, j, i in itertools.product(range(s), repeat=3):
        d2 = sum((lo + q + 0.5 - n / 2) ** 2 for q in (i, j, k))
        assert m[k, j, i] == (d2 <= (R + 2.0) ** 2)
    assert m.sum() > 0 and not m.all()


def _ghost_field(fn, n, lo, s):
    """fn(x, y, z) at every cell centre of the padded cube (relative to c)."""
    a = np.arange(lo - 1, lo + s + 1) + 0.5 - n / 2
    Z, Y, X = np.meshgrid(a, a, a, indexing="ij")
    return fn(X, Y, Z)


def test_quadratic_potentials_are_exact():
    """sum_nb - 6 Phi of x^2 + y^2 + z^2 is exactly 6 (h = 1); of the
    harmonic x^2 - y^2 + 3 z it is 0.  With those sources and the same
    function as ghost values, the masked solution is the function itself."""
    n, lo, s, R = 24, 4, 16, 4.3
    mask = pm.ball_mask(R, n, lo, s)
    for fn, src in ((lambda x, y, z: x * x + y * y + z * z, 6.0),
                    (lambda x, y, z: x * x - y * y + 3.0 * z, 0.0)):
        g = _ghost_field(fn, n, lo, s)
        f = np.where(mask, src, 0.0)
        phi = pm.solve_ball(f, g, mask)
        exact = g[1:-1, 1:-1, 1:-1]
        np.testing.assert_allclose(phi[1:-1, 1:-1, 1:-1][mask], exact[mask], rtol=0,
                                   atol=1e-9 * np.abs(exact).max())
        out = np.ones_like(g, dtype=bool)
        out[1:-1, 1:-1, 1:-1] = ~mask
        np.testing.assert_array_equal(phi[out], g[out])


def test_dense_loop_system_agrees():
    """A dense system assembled cell by cell with Python loops, solved by
    numpy, against the sparse solve, for a random source and ghost field."""
    n, lo, s, R = 12, 1, 10, 2.2
    rng = np.random.default_rng(5)
    mask = pm.ball_mask(R, n, lo, s)
    f = np.where(mask, rng.standard_normal((s, s, s)), 0.0)
    g = rng.standard_normal((s + 2,) * 3)
    cells = [(k, j, i) for k, j, i in itertools.product(range(s), repeat=3) if mask[k, j, i]]
    where = {c: q for q, c in enumerate(cells)}
    A = np.zeros((len(cells), len(cells)))
    b = np.zeros(len(cells))
    for q, (k, j, i) in enumerate(cells):
        A[q, q] = -6.0
        b[q] = f[k, j, i]
        for dk, dj, di in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            nb = (k + dk, j + dj, i + di)
            if nb in where:
                A[q, where[nb]] = 1.0
            else:
                b[q] -= g[nb[0] + 1, nb[1] + 1, nb[2] + 1]
    u = np.linalg.solve(A, b)
    phi = pm.solve_ball(f, g, mask)
    got = np.array([phi[k + 1, j + 1, i + 1] for k, j, i in cells])
    np.testing.assert_allclose(got, u, rtol=0, atol=1e-11 * max(1.0, np.abs(u).max()))


def test_ball_cube_holds_mask_and_ghosts():
    """With reach 3 the mask lies in the cube's interior (never in its outer
    layer), and the kept particles' CIC support (R + sqrt 3) lies inside
    it, for a range of radii."""
    n = 256
    for R in np.linspace(5.0, 120.0, 37):
        lo, s, per = pm.active_cube(R, n, pm.BALL_REACH)
        if per:
            continue
        mask = pm.ball_mask(R, n, lo, s)
        assert not mask[0].any() and not mask[-1].any()
        assert not mask[:, 0].any() and not mask[:, :, 0].any()
        a = np.arange(lo, lo + s) + 0.5 - n / 2
        d2 = (a[:, None, None] ** 2 + a[None, :, None] ** 2) + a[None, None, :] ** 2
        assert mask[d2 <= (R + math.sqrt(3.0)) ** 2].all()


def test_conjugate_gradient_branch_matches_the_direct_solve(monkeypatch):
    """Above DIRECT_MAX unknowns the oracle solves by conjugate gradients:
    on a system small enough for both, the two agree."""
    n, lo, s, R = 20, 2, 16, 4.5
    rng = np.random.default_rng(9)
    mask = pm.ball_mask(R, n, lo, s)
    f = np.where(mask, rng.standard_normal((s, s, s)), 0.0)
    g = rng.standard_normal((s + 2,) * 3)
    a = pm.solve_ball(f, g, mask)
    monkeypatch.setattr(pm, "DIRECT_MAX", 0)
    b = pm.solve_ball(f, g, mask)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-10 * np.abs(a).max())
