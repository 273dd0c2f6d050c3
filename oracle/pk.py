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
