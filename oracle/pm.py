"""One shrinking-domain PM step in FP64 (oracle; test infrastructure only).

Units: positions in cells of the n^3 mesh, measured from the mesh corner, so
cell (i,j,k) has its centre at (i+0.5, j+0.5, k+0.5); conformal time in 1/H0;
momentum p = a dx/dtau in cells*H0; potential in (cells*H0)^2.  With H0 = 1
and the cell as length unit, Poisson's equation (Sec. 2.1, Eq. 3) reads
    sum_nb(Phi) - 6 Phi = S(a) delta,    S(a) = 3 Om / (2 a),
and the equations of motion (Sec. 2.1, Eqs. 1-2) are dx/dtau = p/a,
dp/dtau = -a grad(Phi).  (The printed Eq. 2 has +a grad(Phi), which with the
printed Poisson sign would make gravity repulsive; the attractive sign is
taken.)

Grid arrays are indexed [z, y, x] (x fastest); particle arrays are (N, 3) in
(x, y, z) order.

Step order follows Table 2 (usual-algorithm column for the static Poisson
solve, plus the shrinking row of the right-hand column):
  1. x += p dtau / (2 a_n)                       (Sec. 2.2, first DKD line)
  2. CIC deposit of delta at t + dt/2            (Sec. 2.4 footnote: CIC)
  3. solve Poisson for Phi(t + dt/2)             (Sec. 2.1, Eq. 3)
  4. gradient + CIC gather (same weights as 2)   (Sec. 2.4 footnote)
  5. p += -a_half grad(Phi) dtau                 (Sec. 2.2, second DKD line)
  6. x += p dtau / (2 a_{n+1})                   (Sec. 2.2, third DKD line)
  7. eliminate particles outside the lightcone   (Sec. 2.4, active cells and
     particle pointers recomputed at the end of every step)

Readings taken where the paper is silent (each also applies to the CUDA
library, which implements them independently):
* Domain shape: the implementation restricts loop bounds (Sec. 2.4), i.e. a
  cube, centred on the observer at the box centre c = n/2.  Keep half-width
  R = chi(a)/cell + buffer (1 cell).  Keep iff max_d |x_d - c| <= R.  The
  sphere of Table 1 is the variant domain="sphere": keep iff |x - c| <= R,
  solved on the same cube, its mean-density term the CIC image of the ball
  (background_ball).  domain="ball" keeps and weighs as "sphere" but solves
  only on the ball's cells: the unknowns are the cells whose centre lies
  within R + 2 of c (the CIC support of every kept particle and of the ball
  image lies inside), every other cell of the cube and its ghost layer
  takes the multipole value (the ones next to the mask are its Dirichlet
  ghosts; the rest give the force of particles beyond the mask in the step
  before they leave), and the cube reaches 3 cells beyond R so that the
  mask lies in the cube's interior.
* Boundary conditions: periodic until the lightcone reaches the box border
  (Sec. 3), read as R > n/2 - 1; afterwards open (Table 1) with Dirichlet
  values from a monopole + dipole + quadrupole expansion of the source about
  c at the centres of one ghost-cell layer.
* Active mesh cube in the open phase: half-width m = ceil(R) + 1 cells, side
  the smallest q*2^j >= 2m with q in {1, 3, 5, 7} (halves down to a side of
  at most 7 for the multigrid), at most n.
* Density contrast: delta = rho/rho_mean - W with the cosmic mean N/n^3 and
  W the mean density's own CIC image: the keep cube [c-R, c+R]^3 filled
  uniformly and assigned with the deposit's tent, i.e. per axis
  w_i = T(c + R - x_i) - T(c - R - x_i), T the integral of the tent
  max(0, 1 - |t|), x_i = i + 0.5, and W = w_x w_y w_z (W = 1 everywhere in
  the periodic phase).  A uniform density inside the keep cube then has
  zero mean contrast on every cell, the edge cells included; cells of the
  mesh cube beyond the lightcone carry no source; and sum W = (2R)^3, the
  keep cube's volume, changes smoothly as R shrinks.
* Fixed-point CIC (not in the paper): on the float position u,
  v = u - 0.5, i = floor(v), dq = floor(v*2^16) - i*2^16 in [0, 2^16);
  per-axis weights (2^16 - dq, dq); the product (<= 2^48) is added to an
  int64 cell count.  Each particle adds exactly 2^48 in total.
* Gradient: centred difference (Phi_{i+1} - Phi_{i-1}) / 2 at the 8 CIC
  nodes, gathered with the deposit's weights dq / 2^16.
* A particle whose CIC nodes are not all inside the active cube (open phase)
  is counted as escaped: it deposits nothing and feels no force.
"""
import math

import numpy as np
from scipy import fft as sfft

Q16 = 65536
MASS_UNIT = 2 ** 48


# --------------------------------------------------------------------------
# geometry of the active region (Sec. 2.4 and Sec. 3, readings above)
# --------------------------------------------------------------------------

def is_open(R, n):
    """Open phase once the keep cube no longer wraps the box (Sec. 3)."""
    return R <= n / 2 - 1


def _mg_size(m):
    """Smallest q*2^j (q = 1, 3, 5 or 7) that is >= m."""
    sizes = sorted({q * 2 ** j for q in (1, 3, 5, 7) for j in range(40)})
    return next(x for x in sizes if x >= m)


def active_cube(R, n, reach=1):
    """(lo, s, periodic) of the mesh cube worked on while the keep radius is R;
    reach: cells the assignment extends beyond a particle's cell (CIC 1,
    TSC 2)."""
    if not is_open(R, n):
        return 0, n, True
    m = math.ceil(R) + reach
    s = min(_mg_size(2 * m), n)
    return n // 2 - s // 2, s, False


def tent_integral(u):
    """T(u): integral of the CIC tent max(0, 1 - |t|) over t < u."""
    u = np.asarray(u, dtype=np.float64)
    return np.where(u <= -1.0, 0.0,
                    np.where(u <= 0.0, 0.5 * (u + 1.0) * (u + 1.0),
                             np.where(u <= 1.0, 1.0 - 0.5 * (1.0 - u) * (1.0 - u), 1.0)))


def tsc_integral(u):
    """Integral over t < u of the TSC kernel, 3/4 - t^2 on |t| <= 1/2 and
    (3/2 - |t|)^2 / 2 on 1/2 <= |t| <= 3/2."""
    u = np.asarray(u, dtype=np.float64)
    lo = (1.5 + u) ** 3 / 6.0
    mid = 1.0 / 6.0 + 0.75 * (u + 0.5) - (u ** 3 + 0.125) / 3.0
    hi = 1.0 - (1.5 - u) ** 3 / 6.0
    return np.where(u <= -1.5, 0.0, np.where(u <= -0.5, lo, np.where(
        u <= 0.5, mid, np.where(u <= 1.5, hi, 1.0))))


def background_weights(R, n, lo, s, periodic, assign="cic"):
    """Per-axis weight w_i of the mean density on cells lo..lo+s-1: the
    image of the keep interval [c - R, c + R] under the assignment kernel
    (CIC tent or TSC; all ones when periodic)."""
    if periodic:
        return np.ones(s)
    c = n / 2
    x = np.arange(lo, lo + s) + 0.5
    cdf = tsc_integral if assign == "tsc" else tent_integral
    return cdf((c + R) - x) - cdf((c - R) - x)


# --------------------------------------------------------------------------
# CIC with fixed-point weights
# --------------------------------------------------------------------------

def cic_index(pos):
    """Base node i and Q16 weight dq per axis.  Exact in FP64 for float32 or
    float64 positions |u| < 2^36."""
    v = np.asarray(pos, dtype=np.float64) - 0.5
    i = np.floor(v)
    dq = np.floor(v * Q16) - i * Q16
    return i.astype(np.int64), dq.astype(np.int64)


def cell_order(pos, n):
    """Permutation that orders particles by the mesh cell of their CIC base
    node, stably (equal cells keep their input order).  Not a step of the
    paper's method but a data layout of the library (its sort_every option):
    key ((k n + j) n + i), i = floor(u_x - 1/2) mod n with the subtraction in
    float32 (exact below 2^23), likewise j and k; a non-finite coordinate or
    one beyond 1e9 counts as cell 0."""
    u = np.asarray(pos, dtype=np.float32)
    with np.errstate(invalid="ignore"):
        v = np.floor(u - np.float32(0.5)).astype(np.float64)
        ok = np.isfinite(v) & (np.abs(v) <= 1.0e9)
    c = np.mod(np.where(ok, v, 0.0).astype(np.int64), n)
    key = (c[:, 2] * n + c[:, 1]) * n + c[:, 0]
    return np.argsort(key, kind="stable")


def _valid(i, lo, s):
    return np.all((i >= lo) & (i + 1 <= lo + s - 1), axis=1)


def deposit(pos, n, lo, s, periodic):
    """Integer CIC mass counts rho[z,y,x] (int64), and the escaped count."""
    i, dq = cic_index(pos)
    rho = np.zeros((n, n, n), dtype=np.int64)
    if periodic:
        ok = np.ones(len(i), dtype=bool)
    else:
        ok = _valid(i, lo, s)
    i, dq = i[ok], dq[ok]
    w = [Q16 - dq, dq]
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                ix, iy, iz = i[:, 0] + cx, i[:, 1] + cy, i[:, 2] + cz
                if periodic:
                    ix, iy, iz = ix % n, iy % n, iz % n
                wt = w[cx][:, 0] * w[cy][:, 1] * w[cz][:, 2]
                np.add.at(rho, (iz, iy, ix), wt)
    return rho, int((~ok).sum())


# --------------------------------------------------------------------------
# source and boundary values (Sec. 2.1 Eq. 3; Table 1 open boundaries)
# --------------------------------------------------------------------------

def source_S(a, om):
    """S(a) = 3 Om / (2a), the Poisson source factor in H0 = 1 units."""
    return 1.5 * om / a


BALL_GL = 16  # Gauss-Legendre points per axis and quadrant of the ball image


def background_ball(R, n, lo, s):
    """Mean-density term for a spherical keep region: the CIC image of the
    ball |x - c| <= R on the cells of [lo, lo+s)^3 (float64, [z,y,x]).
    Per cell with centre p (a = p - c): the z integral of the tent over the
    ball's chord is exact, T(h - a_z) - T(-h - a_z) with
    h = sqrt(R^2 - X^2 - Y^2); the x-y integral of the tents runs over the
    four quadrants of [-1, 1]^2 by BALL_GL-point Gauss-Legendre rules.
    Cells with |a| + sqrt(3) <= R are 1, with |a| - sqrt(3) >= R are 0."""
    c = n / 2
    a1 = np.arange(lo, lo + s) + 0.5 - c
    AZ, AY, AX = np.meshgrid(a1, a1, a1, indexing="ij")
    r = np.sqrt(AX * AX + AY * AY + AZ * AZ)
    W = np.where(r + math.sqrt(3.0) <= R, 1.0, 0.0)
    shell = (r + math.sqrt(3.0) > R) & (r - math.sqrt(3.0) < R)
    ax, ay, az = AX[shell], AY[shell], AZ[shell]
    xg, wg = np.polynomial.legendre.leggauss(BALL_GL)
    xi = 0.5 * (xg + 1.0)
    om = 0.5 * wg * (1.0 - xi)          # rule on [0, 1] times the tent 1 - xi
    tot = np.zeros(len(ax))
    for qx in (-1.0, 1.0):
        for qy in (-1.0, 1.0):
            X = ax[:, None, None] + qx * xi[None, :, None]
            Y = ay[:, None, None] + qy * xi[None, None, :]
            h2 = R * R - X * X - Y * Y
            h = np.sqrt(np.maximum(h2, 0.0))
            Z = np.where(h2 > 0.0, tent_integral(h - az[:, None, None])
                         - tent_integral(-h - az[:, None, None]), 0.0)
            tot += np.einsum("cij,i,j->c", Z, om, om)
    W[shell] = tot
    return W


def delta_cube(rho, n, lo, s, nbar, R, periodic, assign="cic", domain="cube"):
    """Density contrast on the active cube [z,y,x] (s^3, float64)."""
    sub = rho[lo:lo + s, lo:lo + s, lo:lo + s].astype(np.float64)
    d = sub / (MASS_UNIT * nbar)
    if domain in ("sphere", "ball") and not periodic:
        return d - background_ball(R, n, lo, s)
    w = background_weights(R, n, lo, s, periodic, assign)
    return d - w[:, None, None] * w[None, :, None] * w[None, None, :]


def multipoles(delta, lo, n):
    """Monopole, dipole and traceless quadrupole of delta about the box centre.

    Q0 = sum delta,  D_a = sum delta y_a,  Q_ab = sum delta (3 y_a y_b - y^2 d_ab)
    with y the cell centre relative to c = n/2 (cell volume 1).
    """
    s = delta.shape[0]
    y1 = np.arange(lo, lo + s) + 0.5 - n / 2
    Z, Y, X = np.meshgrid(y1, y1, y1, indexing="ij")
    comps = [X, Y, Z]
    q0 = delta.sum()
    dip = np.array([(delta * c).sum() for c in comps])
    r2 = X * X + Y * Y + Z * Z
    quad = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            t = 3 * comps[a] * comps[b] - (r2 if a == b else 0.0)
            quad[a, b] = (delta * t).sum()
    return q0, dip, quad


def multipole_potential(points, S, q0, dip, quad):
    """Phi at points (M,3) relative to c:  -(S/4pi)[Q0/r + D.r/r^3 + r.Q.r/(2 r^5)]."""
    r2 = (points * points).sum(axis=1)
    r = np.sqrt(r2)
    dr = points @ dip
    qr = np.einsum("ma,ab,mb->m", points, quad, points)
    return -(S / (4 * math.pi)) * (q0 / r + dr / (r * r2) + 0.5 * qr / (r2 * r2 * r))


def open_ghost_potential(f_cube, S, lo, n, full=False):
    """Padded (s+2)^3 array whose ghost layer holds the Dirichlet values
    (full: the multipole potential at every cell of the padded cube)."""
    s = f_cube.shape[0]
    delta = f_cube / S
    q0, dip, quad = multipoles(delta, lo, n)
    g = np.zeros((s + 2,) * 3)
    coords = np.arange(lo - 1, lo + s + 1) + 0.5 - n / 2
    Z, Y, X = np.meshgrid(coords, coords, coords, indexing="ij")
    ghost = np.ones((s + 2,) * 3, dtype=bool)
    if not full:
        ghost[1:-1, 1:-1, 1:-1] = False
    pts = np.stack([X[ghost], Y[ghost], Z[ghost]], axis=1)
    g[ghost] = multipole_potential(pts, S, q0, dip, quad)
    return g


# --------------------------------------------------------------------------
# Poisson solve: the exact discrete solution of the 7-point system
# --------------------------------------------------------------------------

def laplacian_eig_periodic(n):
    k = np.arange(n)
    lam1 = -4.0 * np.sin(np.pi * k / n) ** 2
    return lam1[:, None, None] + lam1[None, :, None] + lam1[None, None, :]


def solve_periodic(f):
    """sum_nb - 6 Phi = f on a periodic n^3 grid; gauge mean(Phi) = 0.

    The discrete Laplacian is diagonal in the DFT basis with eigenvalue
    -4 sum_d sin^2(pi k_d / n); the k = 0 mode is set to zero."""
    n = f.shape[0]
    fk = np.fft.fftn(f)
    lam = laplacian_eig_periodic(n)
    lam[0, 0, 0] = 1.0
    phik = fk / lam
    phik[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(phik))


def laplacian_eig_dirichlet(s):
    m = np.arange(1, s + 1)
    lam1 = -4.0 * np.sin(np.pi * m / (2.0 * (s + 1))) ** 2
    return lam1[:, None, None] + lam1[None, :, None] + lam1[None, None, :]


def solve_open(f, ghost):
    """sum_nb - 6 Phi = f on an s^3 cube with Dirichlet values at the ghost
    cell centres (ghost: padded (s+2)^3 array, interior ignored).

    Ghost neighbours move to the right-hand side; the remaining operator with
    zero values one cell outside is diagonalised by the type-I DST."""
    s = f.shape[0]
    rhs = f.copy()
    rhs[0, :, :] -= ghost[0, 1:-1, 1:-1]
    rhs[-1, :, :] -= ghost[-1, 1:-1, 1:-1]
    rhs[:, 0, :] -= ghost[1:-1, 0, 1:-1]
    rhs[:, -1, :] -= ghost[1:-1, -1, 1:-1]
    rhs[:, :, 0] -= ghost[1:-1, 1:-1, 0]
    rhs[:, :, -1] -= ghost[1:-1, 1:-1, -1]
    rh = sfft.dstn(rhs, type=1)
    u = sfft.idstn(rh / laplacian_eig_dirichlet(s), type=1)
    out = ghost.copy()
    out[1:-1, 1:-1, 1:-1] = u
    return out


BALL_MARGIN = 2.0   # mask radius R + 2: beyond the CIC reach (sqrt 3) of every kept particle
BALL_REACH = 3      # the ball's cube reaches ceil(R) + 3 cells
DIRECT_MAX = 20000  # unknowns up to which solve_ball factorises the system


def ball_mask(R, n, lo, s):
    """The unknowns of the ball solve: cells of [lo, lo+s)^3 ([z,y,x] bool)
    whose centre lies within R + BALL_MARGIN of c = n/2 (FP64; the squared
    distances of cell centres are exact)."""
    a = np.arange(lo, lo + s) + 0.5 - n / 2
    d2 = (a[:, None, None] ** 2 + a[None, :, None] ** 2) + a[None, None, :] ** 2
    return d2 <= (R + BALL_MARGIN) ** 2


def ball_ghosts(mask):
    """Padded (s+2)^3 bool array of the ghost cells: outside the mask, next
    (along an axis) to a cell of it."""
    s = mask.shape[0]
    pm = np.zeros((s + 2,) * 3, dtype=bool)
    pm[1:-1, 1:-1, 1:-1] = mask
    near = np.zeros_like(pm)
    for ax in range(3):
        for sh in (1, -1):
            near |= np.roll(pm, sh, axis=ax)   # the padding keeps rolls from wrapping mask cells
    return near & ~pm


def solve_ball(f, ghost, mask):
    """sum_nb Phi - 6 Phi = f on the cells of `mask` (s^3), with Dirichlet
    values at the ghost cells (ghost: padded (s+2)^3, read where
    ball_ghosts is true).  The masked 7-point system is solved directly
    (sparse LU) up to DIRECT_MAX unknowns, by conjugate gradients on its
    negative (symmetric positive definite) to a relative residual of 1e-13
    above.  Returns the padded potential: the solution on the mask, `ghost`
    everywhere else (outside the mask the potential is the multipole field,
    felt by particles beyond the mask before they leave)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.linalg import cg, spsolve
    s = f.shape[0]
    gmask = ball_ghosts(mask)
    pm = np.zeros((s + 2,) * 3, dtype=bool)
    pm[1:-1, 1:-1, 1:-1] = mask
    cells = np.argwhere(pm)                 # padded coordinates of the unknowns
    idx = -np.ones((s + 2,) * 3, dtype=np.int64)
    idx[tuple(cells.T)] = np.arange(len(cells))
    rows, cols, vals = [np.arange(len(cells))], [np.arange(len(cells))], [np.full(len(cells), -6.0)]
    rhs = f[mask].astype(np.float64).copy()   # argwhere and boolean indexing share C order
    for ax in range(3):
        for sh in (1, -1):
            nb = cells.copy()
            nb[:, ax] += sh
            t = tuple(nb.T)
            inside = pm[t]
            rows.append(np.nonzero(inside)[0])
            cols.append(idx[t][inside])
            vals.append(np.ones(int(inside.sum())))
            g = gmask[t]
            rhs[g] -= ghost[t][g]
    A = coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                   shape=(len(cells), len(cells))).tocsc()
    if len(cells) <= DIRECT_MAX:
        u = spsolve(A, rhs)
    else:
        u, info = cg(-A, -rhs, rtol=1e-13, atol=0.0, maxiter=100000)
        if info != 0 or np.linalg.norm(A @ u - rhs) > 1e-12 * max(np.linalg.norm(rhs), 1e-300):
            raise RuntimeError("solve_ball: conjugate gradients did not converge")
    out = np.array(ghost, dtype=np.float64, copy=True)
    out[tuple(cells.T)] = u
    return out


def apply_laplacian_padded(phi_pad):
    """7-point operator on the interior of a padded array (h = 1)."""
    p = phi_pad
    c = p[1:-1, 1:-1, 1:-1]
    return (p[2:, 1:-1, 1:-1] + p[:-2, 1:-1, 1:-1] + p[1:-1, 2:, 1:-1]
            + p[1:-1, :-2, 1:-1] + p[1:-1, 1:-1, 2:] + p[1:-1, 1:-1, :-2]
            - 6.0 * c)


def apply_laplacian_periodic(phi):
    return (sum(np.roll(phi, sh, axis=ax) for ax in range(3) for sh in (1, -1))
            - 6.0 * phi)


def solve_step_potential(rho, n, lo, s, periodic, nbar, R, a_half, om, assign="cic",
                         domain="cube"):
    """Source and potential of one step.  Returns (f_cube, phi) where phi is
    n^3 (periodic) or padded (s+2)^3 (open, ghosts included)."""
    S = source_S(a_half, om)
    f = S * delta_cube(rho, n, lo, s, nbar, R, periodic, assign, domain)
    if periodic:
        return f, solve_periodic(f)
    if domain == "ball":
        return f, solve_ball(f, open_ghost_potential(f, S, lo, n, full=True),
                             ball_mask(R, n, lo, s))
    return f, solve_open(f, open_ghost_potential(f, S, lo, n))


# --------------------------------------------------------------------------
# gradient + CIC gather (Sec. 2.4 footnote: same scheme as the deposit)
# --------------------------------------------------------------------------

def gather_force(phi, pos, n, lo, s, periodic):
    """grad(Phi) interpolated to the particles; escaped particles get 0."""
    i, dq = cic_index(pos)
    N = len(i)
    F = np.zeros((N, 3))
    ok = np.ones(N, dtype=bool) if periodic else _valid(i, lo, s)
    w = [(Q16 - dq) / Q16, dq / Q16]

    if periodic:
        def val(ix, iy, iz):
            return phi[iz % n, iy % n, ix % n]
        base = i
    else:
        def val(ix, iy, iz):
            return phi[iz, iy, ix]
        base = i - lo + 1  # padded local index
        base = np.where(ok[:, None], base, 1)

    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                x, y, z = base[:, 0] + cx, base[:, 1] + cy, base[:, 2] + cz
                wt = w[cx][:, 0] * w[cy][:, 1] * w[cz][:, 2]
                gx = 0.5 * (val(x + 1, y, z) - val(x - 1, y, z))
                gy = 0.5 * (val(x, y + 1, z) - val(x, y - 1, z))
                gz = 0.5 * (val(x, y, z + 1) - val(x, y, z - 1))
                F[:, 0] += wt * gx
                F[:, 1] += wt * gy
                F[:, 2] += wt * gz
    F[~ok] = 0.0
    return F, int((~ok).sum())


# --------------------------------------------------------------------------
# TSC with fixed-point weights (Sec. 2.4 footnote: CIC or TSC, the same
# scheme for the density and the force)
# --------------------------------------------------------------------------

def tsc_index(pos):
    """Cell i (the node nearest the particle) and Q16 weights of nodes
    i-1, i, i+1 per axis.  The position within the cell is taken in Q16,
    frac = floor(2^16 u) - 2^16 i (exact), and d = frac - 2^15 is the offset
    from the cell centre; the outer weights are floor((2^15 -+ d)^2 / 2^17)
    (the kernel's (1/2 -+ d)^2 / 2 in Q16) and the centre takes the rest, so
    every axis sums to exactly 2^16."""
    u = np.asarray(pos, dtype=np.float64)
    i = np.floor(u)
    frac = np.floor(u * Q16) - i * Q16
    d = frac - Q16 // 2
    a = Q16 // 2 - d
    b = Q16 // 2 + d
    wm = np.floor(a * a / 2.0 ** 17)
    wp = np.floor(b * b / 2.0 ** 17)
    w0 = Q16 - wm - wp
    return i.astype(np.int64), np.stack([wm, w0, wp], axis=-1).astype(np.int64)


def _valid_tsc(i, lo, s):
    return np.all((i - 1 >= lo) & (i + 1 <= lo + s - 1), axis=1)


def deposit_tsc(pos, n, lo, s, periodic):
    """Integer TSC mass counts rho[z,y,x] (int64), and the escaped count."""
    i, w = tsc_index(pos)
    rho = np.zeros((n, n, n), dtype=np.int64)
    ok = np.ones(len(i), dtype=bool) if periodic else _valid_tsc(i, lo, s)
    i, w = i[ok], w[ok]
    for cz in range(3):
        for cy in range(3):
            for cx in range(3):
                x = i[:, 0] + cx - 1
                y = i[:, 1] + cy - 1
                z = i[:, 2] + cz - 1
                if periodic:
                    x, y, z = x % n, y % n, z % n
                np.add.at(rho, (z, y, x), w[:, 0, cx] * w[:, 1, cy] * w[:, 2, cz])
    return rho, int((~ok).sum())


def gather_force_tsc(phi, pos, n, lo, s, periodic):
    """grad(Phi) at the particles with the TSC weights; escaped get 0."""
    i, w = tsc_index(pos)
    N = len(i)
    F = np.zeros((N, 3))
    ok = np.ones(N, dtype=bool) if periodic else _valid_tsc(i, lo, s)
    wf = w / Q16

    if periodic:
        def val(ix, iy, iz):
            return phi[iz % n, iy % n, ix % n]
        base = i
    else:
        def val(ix, iy, iz):
            return phi[iz, iy, ix]
        base = np.where(ok[:, None], i - lo + 1, 2)  # padded local index
    for cz in range(3):
        for cy in range(3):
            for cx in range(3):
                x = base[:, 0] + cx - 1
                y = base[:, 1] + cy - 1
                z = base[:, 2] + cz - 1
                wt = wf[:, 0, cx] * wf[:, 1, cy] * wf[:, 2, cz]
                F[:, 0] += wt * 0.5 * (val(x + 1, y, z) - val(x - 1, y, z))
                F[:, 1] += wt * 0.5 * (val(x, y + 1, z) - val(x, y - 1, z))
                F[:, 2] += wt * 0.5 * (val(x, y, z + 1) - val(x, y, z - 1))
    F[~ok] = 0.0
    return F, int((~ok).sum())


# --------------------------------------------------------------------------
# drift, kick, shrink
# --------------------------------------------------------------------------

def wrap(pos, n):
    x = np.where(pos < 0, pos + n, pos)
    return np.where(x >= n, x - n, x)


def drift(pos, mom, coef, n, periodic):
    """x += p * coef (FP64); periodic wrap in the periodic phase."""
    x = pos + mom * coef
    return wrap(x, n) if periodic else x


def drift_fp32(pos32, mom32, coef, n, periodic):
    """The same drift evaluated as the CUDA kernel documents it, in float32:
    x' = fl(x + fl(p * fl(coef))), then the float32 wrap.  Used where a float
    result decides an integer (the fixed-point CIC nodes)."""
    c = np.float32(coef)
    x = (pos32.astype(np.float32) + (mom32.astype(np.float32) * c)).astype(np.float32)
    if periodic:
        n32 = np.float32(n)
        x = np.where(x < 0, (x + n32).astype(np.float32), x)
        x = np.where(x >= n32, (x - n32).astype(np.float32), x)
    return x.astype(np.float32)


def keep_mask(pos, R, n, domain="cube"):
    """Keep iff max_d |x_d - c| <= R (cube), or iff
    ((x - c)^2 + (y - c)^2) + (z - c)^2 <= R^2 (sphere), in FP64 on the
    position (Sec. 2.4 / Table 1)."""
    d = np.asarray(pos, dtype=np.float64) - n / 2
    if domain in ("sphere", "ball"):
        return (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2] <= R * R
    return np.abs(d).max(axis=1) <= R


def shrink(arrays, keep):
    """Order-preserving partition: (survivors..., leavers...) of each array."""
    surv = [a[keep] for a in arrays]
    leave = [a[~keep] for a in arrays]
    return surv, leave


# --------------------------------------------------------------------------
# the whole step and the whole run
# --------------------------------------------------------------------------

def step(pos, mom, k, sched, n, om, nbar, want=False, drift32=False, fixed_box=False,
         assign="cic", domain="cube"):
    """Advance FP64 state (pos, mom) by step k.  Returns (pos, mom, info).

    drift32=True takes the first half drift in the CUDA kernel's documented
    float32 arithmetic (drift_fp32) so that both sides deposit the same float
    positions; everything after it stays FP64.  fixed_box=True solves on the
    whole periodic box at every step (the run without shrinking).  assign:
    "cic" or "tsc" (density assignment and force interpolation alike).
    domain: "cube" or "sphere" keep region (its mean-density term), or
    "ball": the sphere solved on the ball's cells only (solve_ball)."""
    a0, a1 = sched["a"][k], sched["a"][k + 1]
    dtau, ah = sched["dtau"][k], sched["a_half"][k]
    R0 = sched["R"][k]
    tsc = assign == "tsc"
    reach = BALL_REACH if domain == "ball" else (2 if tsc else 1)
    lo, s, periodic = (0, n, True) if fixed_box else active_cube(R0, n, reach)
    if drift32:
        pos = drift_fp32(np.asarray(pos, np.float32), np.asarray(mom, np.float32),
                         dtau / (2 * a0), n, periodic).astype(np.float64)
    else:
        pos = drift(pos, mom, dtau / (2 * a0), n, periodic)
    pos_half = pos
    rho, esc = (deposit_tsc if tsc else deposit)(pos, n, lo, s, periodic)
    f, phi = solve_step_potential(rho, n, lo, s, periodic, nbar, R0, ah, om, assign, domain)
    F, _ = (gather_force_tsc if tsc else gather_force)(phi, pos, n, lo, s, periodic)
    mom = mom - ah * dtau * F
    pos = drift(pos, mom, dtau / (2 * a1), n, periodic)
    info = dict(lo=lo, s=s, periodic=periodic, escaped=esc)
    if want:
        info.update(rho=rho, f=f, phi=phi, F=F, x_half=pos_half)
    return pos, mom, info


def run(pos, mom, ids, sched, n, om, nbar, steps=None, record_only=False, assign="cic",
        domain="cube"):
    """Whole run with shrinking.  Returns survivors, lightcone, per-step n_active.

    record_only=True is the run without shrinking that the paper compares
    with (Sec. 3.3): every particle stays active on the whole periodic box,
    and a particle enters the lightcone catalogue, with the step's a_{n+1},
    at the end of the first step after which it lies outside the keep cube
    (same rule and index order as the shrink).  `recorded` then marks the
    catalogued particles."""
    pos = np.asarray(pos, dtype=np.float64).copy()
    mom = np.asarray(mom, dtype=np.float64).copy()
    ids = np.asarray(ids).copy()
    lc = [np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, dtype=ids.dtype),
          np.zeros(0)]
    recorded = np.zeros(len(pos), dtype=bool)
    n_active = []
    nsteps = len(sched["dtau"]) if steps is None else steps
    for k in range(nsteps):
        n_active.append(len(pos))
        pos, mom, _ = step(pos, mom, k, sched, n, om, nbar, fixed_box=record_only,
                           assign=assign, domain=domain)
        R1 = sched["R"][k + 1]
        if is_open(R1, n):
            keep = keep_mask(pos, R1, n, domain)
            if record_only:
                new = ~keep & ~recorded
                lp, lm, li = pos[new], mom[new], ids[new]
                recorded |= new
            else:
                (pos, mom, ids), (lp, lm, li) = shrink([pos, mom, ids], keep)
            lc = [np.concatenate([lc[0], lp]), np.concatenate([lc[1], lm]),
                  np.concatenate([lc[2], li]),
                  np.concatenate([lc[3], np.full(len(li), sched["a"][k + 1])])]
    return dict(pos=pos, mom=mom, ids=ids, lc_pos=lc[0], lc_mom=lc[1],
                lc_ids=lc[2], lc_a=lc[3], n_active=np.array(n_active), recorded=recorded)
