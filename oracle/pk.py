"""Matter power spectrum of a particle set, FP64 (oracle; test use only).

The paper's code measures P(k) with a discreteness correction (Sec. 2.4,
power-spectrum calculator with the Jing 2005 correction).  This oracle takes
the first-order form of that correction:
    P(k) = |delta_k|^2 L^3 / Ng^6 / W(k)^2 - L^3 / N,
    W(k) = prod_d sinc^2(k_d h / 2)   (CIC window, h = L / Ng),
with delta_k the unnormalised DFT of the CIC density contrast on an Ng^3
periodic mesh.  Bins are linear in |k| with width k_f = 2 pi / L, bin b
holding modes with |k|/k_f in [b + 0.5, b + 1.5).  Returns, per bin, the mean
|k|, the mean P and the number of modes (both signs of k counted).
"""
import numpy as np

from . import pm


def power_spectrum(pos, n_mesh, box, n_bins, shot_noise=True):
    """pos: (N,3) positions in cells of the n_mesh^3 mesh, inside [0, n_mesh).

    shot_noise=False omits the L^3/N term (for lattice-based particle sets,
    which carry no Poisson noise)."""
    pos = np.asarray(pos)
    N = len(pos)
    rho, _ = pm.deposit(pos, n_mesh, 0, n_mesh, True)
    mean = N * pm.MASS_UNIT / n_mesh**3
    delta = rho.astype(np.float64) / mean - 1.0
    dk = np.fft.rfftn(delta)
    p_raw = (dk.real**2 + dk.imag**2) * box**3 / float(n_mesh) ** 6

    kf = 2 * np.pi / box
    h = box / n_mesh
    kx = np.fft.rfftfreq(n_mesh, d=1.0 / n_mesh) * kf
    ky = np.fft.fftfreq(n_mesh, d=1.0 / n_mesh) * kf
    KZ, KY, KX = np.meshgrid(ky, ky, kx, indexing="ij")

    def sinc(x):
        return np.where(x == 0, 1.0, np.sin(x) / np.where(x == 0, 1.0, x))

    W = (sinc(KX * h / 2) * sinc(KY * h / 2) * sinc(KZ * h / 2)) ** 2
    p = p_raw / (W * W) - (box**3 / N if shot_noise else 0.0)
    kmag = np.sqrt(KX**2 + KY**2 + KZ**2)

    # rfft keeps x-frequencies 0..Ng/2: planes 0 and Ng/2 appear once, the
    # others stand for a +k / -k pair.
    wt = np.full(kx.shape, 2.0)
    wt[0] = 1.0
    if n_mesh % 2 == 0:
        wt[-1] = 1.0
    wt = np.broadcast_to(wt, kmag.shape)

    b = np.floor(kmag / kf + 0.5).astype(np.int64) - 1
    sel = (b >= 0) & (b < n_bins)
    cnt = np.bincount(b[sel], weights=wt[sel], minlength=n_bins)
    ksum = np.bincount(b[sel], weights=(wt * kmag)[sel], minlength=n_bins)
    psum = np.bincount(b[sel], weights=(wt * p)[sel], minlength=n_bins)
    with np.errstate(invalid="ignore", divide="ignore"):
        return ksum / cnt, psum / cnt, cnt


# --------------------------------------------------------------------------
# Full aliasing correction (Jing 2005), FP64.
#
# The FFT of the CIC-assigned density at k (|k_d| <= k_N = pi / h) carries
# every alias k + 2 k_N n (n integer vector), each weighted by the window:
#     P_obs(k) = sum_n W^2(k + 2k_N n) P(|k + 2k_N n|) + (L^3/N) C1(k),
#     C1(k)    = sum_n W^2(k + 2k_N n) = prod_d [1 - (2/3) sin^2(k_d h / 2)]
# (CIC: W = prod_d sinc^2(k_d h / 2); the closed form of C1 is the CIC
# case of Jing's window sums).  Taking P locally as a power law of slope nu,
# P(|k + 2k_N n|) = P(|k|) (|k + 2k_N n| / |k|)^nu, gives
#     P(k) = (P_obs(k) - (L^3/N) C1(k)) / C2(k, nu),
#     C2   = sum_n W^2(k + 2k_N n) (|k + 2k_N n| / |k|)^nu,
# with nu found by iteration: start from the slope of the first-order
# estimate, correct, re-measure the slope of the corrected binned spectrum,
# repeat until it settles.
#
# Readings (the paper names the method only): the alias sum runs over
# n in [-m, m]^3 (m = 3 by default); each mode is corrected with the slope
# of its bin, then modes are averaged per bin (the bins of power_spectrum);
# the slope of bin b is the centred difference of ln P against ln k over
# bins b-1 and b+1 (one-sided at the ends), kept from the previous pass
# where a P involved is not positive, and clipped to [-6, 4].
# --------------------------------------------------------------------------

def cic_alias_c1(x):
    """sum over aliases of the squared CIC window, per axis x = k_d h / 2,
    in closed form: prod_d [1 - (2/3) sin^2 x_d]."""
    out = 1.0
    for xd in x:
        out = out * (1.0 - (2.0 / 3.0) * np.sin(xd) ** 2)
    return out


def _sinc4_shift(xd, nd):
    """sinc^4(x + pi n) per element, = 1 at x + pi n = 0."""
    y = xd + np.pi * nd
    s = np.sin(xd)
    with np.errstate(invalid="ignore", divide="ignore"):
        v = (s * s) ** 2 / (y * y) ** 2
    return np.where(y == 0.0, 1.0, v)


def cic_alias_c2(x, nu, m):
    """C2 = sum_{n in [-m, m]^3} W^2(k + 2k_N n) (|k + 2k_N n| / |k|)^nu for
    modes with per-axis x = (x_x, x_y, x_z), x_d = k_d h / 2 (arrays),
    slope nu (array broadcast with x, or scalar)."""
    xx, xy, xz = x
    r0 = xx * xx + xy * xy + xz * xz
    tot = np.zeros(np.broadcast(xx, xy, xz).shape)
    fx = {n: _sinc4_shift(xx, n) for n in range(-m, m + 1)}
    fy = {n: _sinc4_shift(xy, n) for n in range(-m, m + 1)}
    fz = {n: _sinc4_shift(xz, n) for n in range(-m, m + 1)}
    for nx in range(-m, m + 1):
        for ny in range(-m, m + 1):
            for nz in range(-m, m + 1):
                r = ((xx + np.pi * nx) ** 2 + (xy + np.pi * ny) ** 2
                     + (xz + np.pi * nz) ** 2)
                with np.errstate(invalid="ignore", divide="ignore"):
                    ratio = np.where(r0 > 0, (r / np.where(r0 > 0, r0, 1.0)) ** (0.5 * nu), 1.0)
                tot = tot + fx[nx] * fy[ny] * fz[nz] * ratio
    return tot


def mode_grid(n_mesh, box):
    """Wavevectors of the R2C layout [kz, ky, kx] (kx = 0..n/2), |k|, the
    +-k multiplicity of each stored mode and its bin index (b = round(|k|/k_f) - 1)."""
    kf = 2 * np.pi / box
    kx = np.fft.rfftfreq(n_mesh, d=1.0 / n_mesh) * kf
    ky = np.fft.fftfreq(n_mesh, d=1.0 / n_mesh) * kf
    KZ, KY, KX = np.meshgrid(ky, ky, kx, indexing="ij")
    kmag = np.sqrt(KX**2 + KY**2 + KZ**2)
    wt = np.full(kx.shape, 2.0)
    wt[0] = 1.0
    if n_mesh % 2 == 0:
        wt[-1] = 1.0
    wt = np.broadcast_to(wt, kmag.shape)
    b = np.floor(kmag / kf + 0.5).astype(np.int64) - 1
    return (KX, KY, KZ), kmag, wt, b


def _bin(values, kmag, wt, b, n_bins):
    sel = (b >= 0) & (b < n_bins)
    cnt = np.bincount(b[sel], weights=wt[sel], minlength=n_bins)
    ksum = np.bincount(b[sel], weights=(wt * kmag)[sel], minlength=n_bins)
    vsum = np.bincount(b[sel], weights=(wt * values)[sel], minlength=n_bins)
    with np.errstate(invalid="ignore", divide="ignore"):
        return ksum / cnt, vsum / cnt, cnt


def _slopes(k, p, prev):
    nb = len(p)
    out = prev.copy()
    for b in range(nb):
        lo, hi = max(b - 1, 0), min(b + 1, nb - 1)
        if hi == lo:
            continue
        if p[lo] > 0 and p[hi] > 0 and k[lo] > 0 and k[hi] > 0:
            out[b] = np.log(p[hi] / p[lo]) / np.log(k[hi] / k[lo])
    return np.clip(out, -6.0, 4.0)


def jing_correct(p_obs, n_mesh, box, n_bins, shot, m=3, max_iter=30, tol=1e-6):
    """Per-mode observed power p_obs (R2C layout, (Mpc/h)^3) -> binned
    (k, P, modes, nu, passes) with the alias correction above; shot = L^3/N
    (0 for lattice-like sets without Poisson noise)."""
    (KX, KY, KZ), kmag, wt, b = mode_grid(n_mesh, box)
    h = box / n_mesh
    x = (KX * h / 2, KY * h / 2, KZ * h / 2)
    c1 = cic_alias_c1(x)
    W2 = _sinc4_shift(x[0], 0) * _sinc4_shift(x[1], 0) * _sinc4_shift(x[2], 0)
    k0, p0, cnt = _bin(p_obs / W2 - shot, kmag, wt, b, n_bins)
    nu = _slopes(k0, p0, np.full(n_bins, -1.0))
    bb = np.clip(b, 0, n_bins - 1)
    passes = 0
    for passes in range(1, max_iter + 1):
        c2 = cic_alias_c2(x, nu[bb], m)
        k1, p1, cnt = _bin((p_obs - shot * c1) / c2, kmag, wt, b, n_bins)
        nu_new = _slopes(k1, p1, nu)
        done = np.max(np.abs(nu_new - nu)) < tol
        nu = nu_new
        if done:
            break
    return k1, p1, cnt, nu, passes


def observed_power(pos, n_mesh, box):
    """Per-mode |delta_k|^2 L^3 / Ng^6 of the CIC density (R2C layout)."""
    pos = np.asarray(pos)
    N = len(pos)
    rho, _ = pm.deposit(pos, n_mesh, 0, n_mesh, True)
    mean = N * pm.MASS_UNIT / n_mesh**3
    delta = rho.astype(np.float64) / mean - 1.0
    dk = np.fft.rfftn(delta)
    return (dk.real**2 + dk.imag**2) * box**3 / float(n_mesh) ** 6


def power_spectrum_jing(pos, n_mesh, box, n_bins, shot_noise=True, m=3, max_iter=30,
                        tol=1e-6):
    """P(k) of a particle set with the full alias correction; returns
    (k, P, modes, nu, passes) per bin."""
    N = len(pos)
    shot = box**3 / N if shot_noise else 0.0
    return jing_correct(observed_power(pos, n_mesh, box), n_mesh, box, n_bins, shot, m,
                        max_iter, tol)
