"""Seeded synthetic inputs: Zel'dovich initial conditions and workload presets.

This module generates inputs only; it holds none of the PM step's arithmetic
and imports neither the CUDA library nor the oracle, so that both can be fed
identical particles.

Initial conditions (Sec. 3 of the paper uses Zel'dovich ICs from a COSMICS
spectrum, which is not available; power laws stand in for it):
  * white noise  w = default_rng(seed).standard_normal((n, n, n))  [z, y, x]
  * delta_k = rfftn(w)_k sqrt(P(k)),  P(k) = k^alpha exp(-k^2 / (2 k_c^2))
    with k in rad/cell, k_c = cutoff * pi (no cutoff when cutoff is None);
    the k = 0 mode and every Nyquist plane are zeroed
  * displacement psi_k = i k delta_k / k^2 (so div psi = -delta), normalised
    to a 3-D rms |psi| of ``rms_disp`` cells
  * particles on the lattice of cell centres q = (i+.5, j+.5, k+.5):
    x = q + psi(q) (wrapped into [0, n)),  p = a^2 E(a) f(a) psi
    (p = a dx/dtau, conformal time, H0 = 1)
Positions and momenta are returned as float32, ids as int32 in lattice order
(id = (k n + j) n + i).
"""
import math

import numpy as np
from scipy import integrate

# Workload presets.  Sizes, boxes (Mpc/h), spectra, seeds, step counts and
# tolerances of the five standard workloads; cosmology Om = 0.3, OL = 0.7.
WORKLOADS = {
    "pm32": dict(n=32, box=250.0, alpha=-2.0, cutoff=None, seed=0,
                 a_init=0.02, a_final=1.0, steps=20, rtol=1e-8),
    "pm128": dict(n=128, box=1000.0, alpha=-1.5, cutoff=0.5, seed=1,
                  a_init=0.02, a_final=1.0, steps=100, rtol=1e-7),
    "pm256": dict(n=256, box=2000.0, alpha=-1.5, cutoff=0.5, seed=1,
                  a_init=0.01, a_final=1.0, steps=200, rtol=1e-7),
    "pm512": dict(n=512, box=3000.0, alpha=-1.5, cutoff=0.5, seed=1,
                  a_init=0.02, a_final=1.0, steps=100, rtol=1e-7),
}
OMEGA_M, OMEGA_L = 0.3, 0.7
RMS_DISP = 0.1


def batched_workload(seeds=range(100, 148)):
    """Per-realisation (n, box) of the batched workload: n uniform over
    {32, 48, 64, 96, 128}, box uniform in [200, 1500] Mpc/h, both drawn from
    default_rng(seed)."""
    out = []
    for s in seeds:
        rng = np.random.default_rng(s)
        n = int(rng.choice([32, 48, 64, 96, 128]))
        box = float(rng.uniform(200.0, 1500.0))
        out.append(dict(n=n, box=box, alpha=-1.5, cutoff=0.5, seed=int(s),
                        a_init=0.02, a_final=1.0, steps=50, rtol=1e-7))
    return out


def _E(a, om, ol):
    return math.sqrt(om / a**3 + ol)


def _growth_rate(a, om, ol):
    """f = dlnD/dlna of the Heath (1977) growing mode."""
    val, _ = integrate.quad(lambda x: x**1.5 / (om + ol * x**3) ** 1.5,
                            0.0, a, epsabs=0.0, epsrel=1e-13, limit=200)
    e = _E(a, om, ol)
    return -1.5 * om / (a**3 * e * e) + a / ((a * e) ** 3 * val)


def displacement_field(n, alpha, cutoff, seed, rms_disp=RMS_DISP):
    """psi[z, y, x, d] (float64, cells) of a Gaussian field; see module doc."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((n, n, n))
    wk = np.fft.rfftn(w)
    kz = 2 * np.pi * np.fft.fftfreq(n)
    kx = 2 * np.pi * np.fft.rfftfreq(n)
    KZ, KY, KX = np.meshgrid(kz, kz, kx, indexing="ij")
    k2 = KX**2 + KY**2 + KZ**2
    k2s = np.where(k2 == 0, 1.0, k2)
    pk = k2s ** (alpha / 2)
    if cutoff is not None:
        kc = cutoff * np.pi
        pk = pk * np.exp(-k2s / (2 * kc * kc))
    dk = wk * np.sqrt(pk)
    dk[0, 0, 0] = 0
    if n % 2 == 0:
        dk[n // 2, :, :] = 0
        dk[:, n // 2, :] = 0
        dk[:, :, n // 2] = 0
    psi = np.empty((n, n, n, 3))
    for d, K in enumerate((KX, KY, KZ)):
        psi[..., d] = np.fft.irfftn(1j * K * dk / k2s, s=(n, n, n), axes=(0, 1, 2))
    rms = math.sqrt((psi**2).sum(axis=-1).mean())
    return psi * (rms_disp / rms)


def zeldovich(n, alpha, cutoff, seed, a_init, om=OMEGA_M, ol=OMEGA_L,
              rms_disp=RMS_DISP):
    """(pos, mom, ids): float32 (n^3, 3), float32 (n^3, 3), int32 (n^3,)."""
    psi = displacement_field(n, alpha, cutoff, seed, rms_disp).reshape(-1, 3)
    g = np.arange(n) + 0.5
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    q = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    x = q + psi
    x = np.where(x < 0, x + n, x)
    x = np.where(x >= n, x - n, x)
    vfac = a_init**2 * _E(a_init, om, ol) * _growth_rate(a_init, om, ol)
    pos = x.astype(np.float32)
    # float32 rounding of x + n can land exactly on n
    pos[pos >= np.float32(n)] = np.float32(0.0)
    mom = (vfac * psi).astype(np.float32)
    ids = np.arange(n**3, dtype=np.int32)
    return pos, mom, ids


def workload_ics(name_or_cfg):
    cfg = WORKLOADS[name_or_cfg] if isinstance(name_or_cfg, str) else name_or_cfg
    return zeldovich(cfg["n"], cfg["alpha"], cfg["cutoff"], cfg["seed"],
                     cfg["a_init"])


def random_particles(n_particles, n, seed, lo=0.0, hi=None, vmax=0.5):
    """Uniform random float32 positions in [lo, hi)^3 and momenta in
    [-vmax, vmax)^3 (unit tests of single kernels)."""
    rng = np.random.default_rng(seed)
    hi = float(n) if hi is None else hi
    pos = rng.uniform(lo, hi, size=(n_particles, 3)).astype(np.float32)
    pos[pos >= np.float32(hi)] = np.float32(lo)
    mom = rng.uniform(-vmax, vmax, size=(n_particles, 3)).astype(np.float32)
    ids = np.arange(n_particles, dtype=np.int32)
    return pos, mom, ids
