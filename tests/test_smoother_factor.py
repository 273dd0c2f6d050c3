"""The multigrid smoother's over-relaxation factor (PM_MG_OMEGA in
include/pmshrink.h).  A plain numpy model of the solver's V(2,2) cycle on a
periodic cell-centred grid: red-black SOR sweeps, the residual averaged over
the 8 children, trilinear (3/4, 1/4) prolongation, a many-sweep bottom.  It
checks the reason the factor was chosen: it cuts the residual per V-cycle at
least twice as hard as Gauss-Seidel (factor 1), whose per-cycle reduction
the model puts near 0.1, as the GPU solver's iteration counts do."""
import numpy as np

from paper_1709_04703_gb300 import _lib as L


def _nb(u):
    return sum(np.roll(u, sh, ax) for ax in range(3) for sh in (1, -1))


def _resid(u, b, h2):
    return b - (_nb(u) - 6.0 * u) / h2


def _sweeps(u, b, h2, omega, n=2):
    colour = np.indices(u.shape).sum(0) % 2
    for _ in range(n):
        for c in (0, 1):
            m = colour == c
            g = (_nb(u) - h2 * b) / 6.0
            u[m] += omega * (g[m] - u[m])


def _restrict(r):
    c = r.shape[0] // 2
    return r.reshape(c, 2, c, 2, c, 2).mean(axis=(1, 3, 5))


def _prolong(uc):
    out = uc
    for ax in range(3):
        even = 0.75 * out + 0.25 * np.roll(out, 1, ax)
        odd = 0.75 * out + 0.25 * np.roll(out, -1, ax)
        shape = list(out.shape)
        shape[ax] *= 2
        f = np.empty(shape)
        sl = [slice(None)] * 3
        sl[ax] = slice(0, None, 2)
        f[tuple(sl)] = even
        sl[ax] = slice(1, None, 2)
        f[tuple(sl)] = odd
        out = f
    return out


def _vcycle(u, b, h2, omega):
    if u.shape[0] <= 4:
        for _ in range(100):
            _sweeps(u, b, h2, 1.0, 1)
            u -= u.mean()
        return
    _sweeps(u, b, h2, omega)
    bc = _restrict(_resid(u, b, h2))
    uc = np.zeros_like(bc)
    _vcycle(uc, bc, 4.0 * h2, omega)
    u += _prolong(uc)
    _sweeps(u, b, h2, omega)


def _reduction(omega, n=32, cycles=6):
    """Geometric mean of the residual reduction over the last 4 cycles."""
    b = np.random.default_rng(0).standard_normal((n, n, n))
    b -= b.mean()
    u = np.zeros_like(b)
    r = [np.linalg.norm(_resid(u, b, 1.0))]
    for _ in range(cycles):
        _vcycle(u, b, 1.0, omega)
        u -= u.mean()
        r.append(np.linalg.norm(_resid(u, b, 1.0)))
    q = np.array(r[1:]) / np.array(r[:-1])
    return float(np.exp(np.log(q[-4:]).mean()))


def test_model_reproduces_the_gauss_seidel_cycle():
    assert 0.05 < _reduction(1.0) < 0.15


def test_overrelaxation_factor_at_least_halves_the_reduction():
    assert 1.0 < L.PM_MG_OMEGA < 2.0
    assert _reduction(L.PM_MG_OMEGA) < 0.5 * _reduction(1.0)
