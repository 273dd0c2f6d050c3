"""The paper's diffusion-equation gravity in FP64 (oracle; test
infrastructure only).

Sec. 2.3 replaces Poisson's equation by the diffusion equation (Eq. 4)
    3 H dPhi/dtau - c^2 lap(Phi) = -c^2 S(a) delta,
H the conformal Hubble rate a E(a) (H0 = 1), solved in two half-substeps per
step, ordered as in Table 2 (right column): half drift, density at t+dt/2,
Phi from t to t+dt/2, gradient + kick, half drift, Phi from t+dt/2 to t+dt,
lightcone shrink.  The speed of light of the gravity solve is reduced to
c_eff = 0.019 h c with h the comoving cell size in Mpc/h (Sec. 3.1.1).

Readings (the paper evolves Eq. 4 with an explicit ADE scheme and leaves
implicit methods for future work; its boundary values and initial field are
not spelled out):
* each half-substep is one backward-Euler step of length dtau/2:
      3 H_e (Phi - Phi_old) / (dtau/2) - c_eff^2 A Phi = -c_eff^2 f,
  i.e. (A - sig) Phi = f - sig Phi_old with sig = 3 H_e / (c_eff^2 dtau/2),
  H_e and f = S delta taken at the substep's end (a_half, then a_{n+1});
  the second substep reuses the density deposited at t+dt/2;
* in cell units c_eff = 0.019 * (c/H0 in Mpc/h) cells per 1/H0, whatever the
  cell size (h cancels);
* open cubes take the same Dirichlet ghost values as the static solve (the
  multipole field of the substep's source); the cube of a later step is a
  sub-cube of the earlier one, so Phi_old is restricted to it;
* the field starts from the static (Poisson) solution of the first step's
  density (linear theory, Table 1);
* the paper's own scheme (Sec. 2.3), alternating-direction explicit, is
  ade_substep: the Saul'yev form, an in-place lexicographic sweep upward in
  the first half-substep and downward in the second ("two consecutive
  steps with alternate directions"), with the same lam = 1/sig, f, ghosts
  and initial field as the implicit reading.
Pins: tests/test_oracle_diffusion.py (single-mode decay in closed form, the
sig -> 0 and steady-state limits against the Poisson solve, a dense solve;
for the ADE sweep its lower/upper-triangular system solved densely, its
fixed point = the Poisson solution, and small-lam consistency).
"""
import numpy as np
from scipy import fft as sfft

from . import cosmology as cz
from . import pm

C_OVER_H0 = cz.C_OVER_H0
CEFF_FACTOR = 0.019


def c_eff_cells(factor=CEFF_FACTOR):
    """c_eff in cells per 1/H0: factor * h * (c/H0) / h."""
    return factor * C_OVER_H0


def sigma(a_end, dtau_sub, om, ol, c_cells):
    """sig = 3 H(a_end) / (c_eff^2 dtau_sub), H = a E(a) (H0 = 1)."""
    return 3.0 * a_end * cz.E(a_end, om, ol) / (c_cells * c_cells * dtau_sub)


def solve_periodic_shifted(g, sig):
    """(sum_nb - 6 - sig) Phi = g on a periodic grid (sig > 0: unique)."""
    lam = pm.laplacian_eig_periodic(g.shape[0]) - sig
    return np.real(np.fft.ifftn(np.fft.fftn(g) / lam))


def solve_open_shifted(g, ghost, sig):
    """(sum_nb - 6 - sig) Phi = g on an s^3 cube with Dirichlet ghost values."""
    s = g.shape[0]
    rhs = g.copy()
    rhs[0, :, :] -= ghost[0, 1:-1, 1:-1]
    rhs[-1, :, :] -= ghost[-1, 1:-1, 1:-1]
    rhs[:, 0, :] -= ghost[1:-1, 0, 1:-1]
    rhs[:, -1, :] -= ghost[1:-1, -1, 1:-1]
    rhs[:, :, 0] -= ghost[1:-1, 1:-1, 0]
    rhs[:, :, -1] -= ghost[1:-1, 1:-1, -1]
    lam = pm.laplacian_eig_dirichlet(s) - sig
    u = sfft.idstn(sfft.dstn(rhs, type=1) / lam, type=1)
    out = ghost.copy()
    out[1:-1, 1:-1, 1:-1] = u
    return out


def substep(phi_old, f, sig, periodic, ghost=None):
    """One backward-Euler half-substep: (A - sig) Phi = f - sig Phi_old.
    periodic: phi_old, f are n^3; open: phi_old is the interior s^3 and
    ghost the padded (s+2)^3 Dirichlet array.  Returns Phi (n^3, or padded)."""
    g = f - sig * phi_old
    if periodic:
        return solve_periodic_shifted(g, sig)
    return solve_open_shifted(g, ghost, sig)


def ade_substep(phi_old, f, lam, upward, periodic, ghost=None):
    """One half-substep by the alternating-direction explicit scheme of
    Sec. 2.3 (Saul'yev form): dPhi/dtau = D (lap Phi - f), lam = D dtau_sub
    (= 1 / sig).  The cells are swept in place in lexicographic order (z
    slowest, x fastest), upward or downward; every neighbour difference
    (Phi_q - Phi_c) takes the centre at the time level of the neighbour's
    value as it stands in memory: new for neighbours already swept, old for
    the others.  With m_new neighbours already swept,
        Phi_new (1 + lam m_new) = Phi_old (1 - lam (6 - m_new)) + lam (sum_q Phi_q - f).
    Open cubes: ghost values are fixed; a ghost counts as swept when it lies
    on the side the sweep comes from.  Periodic grids wrap, so the neighbour
    across the wrap of the first cell of a row is swept only at the end.
    Returns the new field (n^3 periodic, or the padded array with ghost's
    values on its ghost layer).  Plain loops: small grids only."""
    if periodic:
        n = phi_old.shape[0]
        u = phi_old.astype(np.float64).copy()
    else:
        n = phi_old.shape[0]
        u = ghost.astype(np.float64).copy()
        u[1:-1, 1:-1, 1:-1] = phi_old
    order = range(n) if upward else range(n - 1, -1, -1)

    def idx(z, y, x):
        return (z, y, x) if periodic else (z + 1, y + 1, x + 1)

    for z in order:
        for y in order:
            for x in order:
                c = idx(z, y, x)
                tot, m_new = 0.0, 0
                for ax in range(3):
                    for sgn in (-1, 1):
                        q = [z, y, x]
                        q[ax] += sgn
                        v = q[ax]
                        if periodic:
                            q[ax] %= n
                        # swept before (z, y, x)?  Upward: the lower side
                        # (including the lower ghost, or, across the wrap,
                        # the upper neighbour of the last cell); downward:
                        # the mirror
                        if periodic:
                            before = (q[ax] < [z, y, x][ax]) if upward else (q[ax] > [z, y, x][ax])
                        else:
                            before = (v < [z, y, x][ax]) if upward else (v > [z, y, x][ax])
                        m_new += 1 if before else 0
                        tot += u[idx(*q)] if periodic else u[q[0] + 1, q[1] + 1, q[2] + 1]
                u[c] = ((1.0 - lam * (6 - m_new)) * u[c] + lam * (tot - f[z, y, x])) / (
                    1.0 + lam * m_new)
    return u


def restrict_field(phi, lo_old, s_old, periodic_old, lo, s):
    """The previous step's field on the current cube [lo, lo+s)^3 (interior)."""
    a = phi if periodic_old else phi[1:-1, 1:-1, 1:-1]
    off = lo - (0 if periodic_old else lo_old)
    return a[off:off + s, off:off + s, off:off + s].copy()


def initial_field(pos, sched, n, om, nbar):
    """Static solution for the density of the first step's half drift."""
    x = pm.drift(np.asarray(pos, np.float64), np.zeros_like(pos, np.float64), 0.0, n, True)
    lo, s, per = pm.active_cube(sched["R"][0], n)
    rho, _ = pm.deposit(x, n, lo, s, per)
    _, phi = pm.solve_step_potential(rho, n, lo, s, per, nbar, sched["R"][0], sched["a"][0], om)
    return phi, (lo, s, per)


def step(pos, mom, state, k, sched, n, om, ol, nbar, c_cells=None, want=False, drift32=False,
         scheme="implicit"):
    """Advance (pos, mom) and the field state (phi, (lo, s, periodic)) by
    step k in the Table 2 order.  Returns (pos, mom, state, info).
    drift32: the first half drift in the float32 arithmetic the CUDA kernel
    documents (pm.drift_fp32), so that both deposit the same positions.
    scheme: "implicit" (backward Euler half-substeps) or "ade" (the paper's
    alternating-direction explicit scheme: an upward sweep for the first
    half-substep, a downward one for the second)."""
    c_cells = c_eff_cells() if c_cells is None else c_cells
    if scheme == "ade":
        def half(phi_old, f, sig, periodic, ghost, first):
            return ade_substep(phi_old, f, 1.0 / sig, first, periodic, ghost)
    else:
        def half(phi_old, f, sig, periodic, ghost, first):
            return substep(phi_old, f, sig, periodic, ghost)
    a0, a1 = sched["a"][k], sched["a"][k + 1]
    dtau, ah = sched["dtau"][k], sched["a_half"][k]
    lo, s, per = pm.active_cube(sched["R"][k], n)
    phi_prev, (lo_p, s_p, per_p) = state
    phi_old = restrict_field(phi_prev, lo_p, s_p, per_p, lo, s)
    # 1-2. half drift, density at t + dt/2
    if drift32:
        pos = pm.drift_fp32(np.asarray(pos, np.float32), np.asarray(mom, np.float32),
                            dtau / (2 * a0), n, per).astype(np.float64)
    else:
        pos = pm.drift(pos, mom, dtau / (2 * a0), n, per)
    x_half = pos
    rho, esc = pm.deposit(pos, n, lo, s, per)
    delta = pm.delta_cube(rho, n, lo, s, nbar, sched["R"][k], per)
    # 3. Phi from t to t + dt/2
    S1 = pm.source_S(ah, om)
    f1 = S1 * delta
    sig1 = sigma(ah, 0.5 * dtau, om, ol, c_cells)
    ghost1 = None if per else pm.open_ghost_potential(f1, S1, lo, n)
    phi_h = half(phi_old, f1, sig1, per, ghost1, True)
    # 4-5. gradient + kick, half drift
    F, _ = pm.gather_force(phi_h, pos, n, lo, s, per)
    mom = mom - ah * dtau * F
    pos = pm.drift(pos, mom, dtau / (2 * a1), n, per)
    # 6. Phi from t + dt/2 to t + dt (same density, S and H at a_{n+1})
    S2 = pm.source_S(a1, om)
    f2 = S2 * delta
    sig2 = sigma(a1, 0.5 * dtau, om, ol, c_cells)
    ghost2 = None if per else pm.open_ghost_potential(f2, S2, lo, n)
    phi_h_int = phi_h if per else phi_h[1:-1, 1:-1, 1:-1]
    phi_1 = half(phi_h_int, f2, sig2, per, ghost2, False)
    info = dict(lo=lo, s=s, periodic=per, escaped=esc, sig=(sig1, sig2))
    if want:
        info.update(F=F, phi_half=phi_h, phi_end=phi_1, x_half=x_half, f=f1)
    return pos, mom, (phi_1, (lo, s, per)), info


def run(pos, mom, ids, sched, n, om, ol, nbar, steps=None, c_cells=None, scheme="implicit"):
    """Whole run with shrinking (as pm.run, with the diffusion field)."""
    pos = np.asarray(pos, dtype=np.float64).copy()
    mom = np.asarray(mom, dtype=np.float64).copy()
    ids = np.asarray(ids).copy()
    lc = [np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, dtype=ids.dtype), np.zeros(0)]
    state = initial_field(pos, sched, n, om, nbar)
    nsteps = len(sched["dtau"]) if steps is None else steps
    for k in range(nsteps):
        pos, mom, state, _ = step(pos, mom, state, k, sched, n, om, ol, nbar, c_cells,
                                  scheme=scheme)
        R1 = sched["R"][k + 1]
        if pm.is_open(R1, n):
            keep = pm.keep_mask(pos, R1, n)
            (pos, mom, ids), (lp, lm, li) = pm.shrink([pos, mom, ids], keep)
            lc = [np.concatenate([lc[0], lp]), np.concatenate([lc[1], lm]),
                  np.concatenate([lc[2], li]),
                  np.concatenate([lc[3], np.full(len(li), sched["a"][k + 1])])]
    return dict(pos=pos, mom=mom, ids=ids, lc_pos=lc[0], lc_mom=lc[1], lc_ids=lc[2],
                lc_a=lc[3])
