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


# ------------------------------------------------------------ alias correction

from oracle import pk  # noqa: E402


def test_cic_window_alias_sum_has_its_closed_form():
    """sum over all aliases of the squared CIC window = prod [1 - 2/3 sin^2]:
    the brute alias sum (nu = 0) with a long range reaches it."""
    rng = np.random.default_rng(1)
    x = tuple(rng.uniform(-np.pi / 2, np.pi / 2, 20) for _ in range(3))
    np.testing.assert_allclose(pk.cic_alias_c2(x, 0.0, 60), pk.cic_alias_c1(x), rtol=1e-6)


def test_alias_sum_with_slope_matches_direct_terms():
    """C2 for a few modes against an explicit loop over alias vectors with
    the window written as sinc^2 of each shifted component."""
    h = 2.0
    for kvec, nu in [((0.3, -0.7, 1.1), -1.5), ((1.4, 0.0, -0.2), -2.5), ((0.5, 0.5, 0.5), 0.7)]:
        k = np.array(kvec) / h * 2            # x = k h / 2 = kvec
        kn = np.pi / h
        tot = 0.0
        for n in itertools.product(range(-3, 4), repeat=3):
            q = k + 2 * kn * np.array(n)
            w = 1.0
            for qd in q:
                u = qd * h / 2
                w *= (math.sin(u) / u) ** 2 if u != 0 else 1.0
            tot += w * w * (np.linalg.norm(q) / np.linalg.norm(k)) ** nu
        got = pk.cic_alias_c2(tuple(np.array([v]) for v in kvec), nu, 3)[0]
        assert abs(got - tot) <= 1e-12 * tot, (kvec, got, tot)


def _power_law_observed(n, box, A, nu0, shot, M=8):
    (KX, KY, KZ), kmag, wt, b = pk.mode_grid(n, box)
    h = box / n
    x = (KX * h / 2, KY * h / 2, KZ * h / 2)
    with np.errstate(divide="ignore"):
        ptrue = np.where(kmag > 0, A * kmag ** nu0, 0.0)
    return ptrue * pk.cic_alias_c2(x, nu0, M) + shot * pk.cic_alias_c1(x), ptrue, kmag, wt, b


def test_alias_correction_recovers_a_power_law_up_to_nyquist():
    """Observed power of P = A k^nu (aliases to |n| <= 8, plus shot noise):
    the correction with m = 3 finds the slope and recovers P to 0.5 % in
    every bin up to k_N, where the first-order estimate is off by > 10 %."""
    n, box, nu0, A = 32, 100.0, -1.5, 50.0
    shot = box**3 / 40000
    pobs, ptrue, kmag, wt, b = _power_law_observed(n, box, A, nu0, shot)
    k, p, cnt, nu, passes = pk.jing_correct(pobs, n, box, n // 2, shot)
    _, pt, _ = pk._bin(ptrue, kmag, wt, b, n // 2)
    assert passes < 30
    np.testing.assert_allclose(p, pt, rtol=5e-3)
    np.testing.assert_allclose(nu[2:-2], nu0, atol=0.05)
    # first order (deconvolve W^2, subtract L^3/N) fails near Nyquist
    (KX, KY, KZ), _, _, _ = pk.mode_grid(n, box)
    h = box / n
    W2 = (pk._sinc4_shift(KX * h / 2, 0) * pk._sinc4_shift(KY * h / 2, 0)
          * pk._sinc4_shift(KZ * h / 2, 0))
    _, p1, _ = pk._bin(pobs / W2 - shot, kmag, wt, b, n // 2)
    assert np.max(np.abs(p1 / pt - 1)) > 0.1


def test_alias_correction_of_poisson_noise_is_zero():
    """Uniform random particles have P = 0: after the correction every bin
    is zero within 6 sigma of its mode count (the first-order estimate
    leaves the shot noise's aliases near Nyquist)."""
    n, box, N = 32, 100.0, 200000
    pos, _, _ = ics.random_particles(N, n, seed=21)
    shot = box**3 / N
    k, p, cnt, nu, passes = pk.power_spectrum_jing(pos, n, box, n // 2)
    (KX, KY, KZ), kmag, wt, b = pk.mode_grid(n, box)
    h = box / n
    x = (KX * h / 2, KY * h / 2, KZ * h / 2)
    ratio = pk.cic_alias_c1(x) / pk.cic_alias_c2(x, -1.0, 3)
    _, r_b, _ = pk._bin(ratio, kmag, wt, b, n // 2)
    sigma = shot * r_b / np.sqrt(cnt / 2)
    assert np.all(np.abs(p) < 6 * sigma), p / sigma
    k1, p1, _ = power_spectrum(pos, n, box, n // 2)
    assert p1[-1] > 10 * sigma[-1]
