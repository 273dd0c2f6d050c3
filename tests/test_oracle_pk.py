"""Pins of the oracle's power-spectrum estimator (no GPU)."""
import itertools
import math

import numpy as np

from oracle import pm
from oracle.pk import power_spectrum
from paper_1709_04703_gb300 import ics


def test_lattice_has_zero_power_minus_shot_noise():
    n, box = 8, 100.0
    g = np.arange(n) + 0.5
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    lat = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1).astype(np.float32)
    k, p, cnt = power_spectrum(lat, n, box, 4)
    np.testing.assert_allclose(p, -box**3 / n**3, rtol=1e-12)
    _, p0, _ = power_spectrum(lat, n, box, 4, shot_noise=False)
    np.testing.assert_allclose(p0, 0.0, atol=1e-20)


def test_brute_force_dft_and_binning():
    """Direct triple-sum DFT on a 6^3 mesh, modes enumerated over the full
    k-cube, binned by |k|/k_f in [b+.5, b+1.5)."""
    n, box, nb = 6, 60.0, 3
    pos, _, _ = ics.random_particles(50, n, seed=11)
    k, p, cnt = power_spectrum(pos, n, box, nb)

    rho, _ = pm.deposit(pos, n, 0, n, True)
    delta = rho.astype(np.float64) / (50 * 2**48 / n**3) - 1
    kf, h = 2 * math.pi / box, box / n
    acc = np.zeros(nb)
    ksum = np.zeros(nb)
    num = np.zeros(nb)
    xs = np.arange(n)
    for mz, my, mx in itertools.product(range(n), repeat=3):
        m = [(v if v <= n // 2 else v - n) for v in (mx, my, mz)]
        phase = np.exp(-2j * math.pi * (
            m[0] * xs[None, None, :] + m[1] * xs[None, :, None]
            + m[2] * xs[:, None, None]) / n)
        dk = (delta * phase).sum()
        kv = [kf * v for v in m]
        kmag = math.sqrt(sum(v * v for v in kv))
        b = math.floor(kmag / kf + 0.5) - 1
        if not 0 <= b < nb:
            continue
        # the rfft half-space keeps m_x = -n/2 folded onto +n/2: count the
        # full cube once per distinct (m_x mod n) as the estimator does
        W = 1.0
        for v in kv:
            x = v * h / 2
            W *= (math.sin(x) / x) ** 2 if x != 0 else 1.0
        pk = abs(dk) ** 2 * box**3 / n**6 / W**2 - box**3 / 50
        acc[b] += pk
        ksum[b] += kmag
        num[b] += 1
    np.testing.assert_allclose(cnt, num)
    np.testing.assert_allclose(k, ksum / num, rtol=1e-12)
    np.testing.assert_allclose(p, acc / num, rtol=1e-9)


def test_poisson_sample_is_shot_noise_free_at_low_k():
    n, box, N = 32, 500.0, 200000
    pos, _, _ = ics.random_particles(N, n, seed=2)
    k, p, cnt = power_spectrum(pos, n, box, 6)
    shot = box**3 / N
    # mean over the first bins ~ 0 within the sample noise shot*sqrt(2/modes)
    noise = shot * np.sqrt(2.0 / cnt[:6].sum())
    assert abs(np.sum(p[:6] * cnt[:6]) / cnt[:6].sum()) < 5 * noise + 0.02 * shot
