"""Background cosmology and the time-step schedule, FP64 (oracle; test use only).

Units: H0 = 1, so conformal time tau is in 1/H0.  Distances are returned in
Mpc/h using c/H0 = 2997.92458 Mpc/h.  Flat LCDM: E(a)^2 = Om a^-3 + OL.

Paper passages followed
-----------------------
* Sec. 2.1, Eqs. (1)-(3): dots are conformal-time derivatives, H = a'/a.
* Sec. 3 (test set-up): steps uniform in the expansion factor a, conformal
  time as the integration variable.
* Sec. 2.4, the lightcone equation r_lc = c (t - t0): garbled (the radius must
  shrink).  Reading: r_lc(a) = chi(a) = (c/H0) [tau(1) - tau(a)], the comoving
  distance light travels from conformal time tau(a) to the z=0 observer.
* Sec. 2.2, synchronised leapfrog: a(t+dt/2) is read as the expansion factor
  at the conformal-time midpoint of the step.
"""
import math

import numpy as np
from scipy import integrate

C_OVER_H0 = 2997.92458  # Mpc/h


def E(a, om, ol):
    """Dimensionless Hubble rate H(a)/H0 for a flat background."""
    return np.sqrt(om / a**3 + ol)


def tau(a, om, ol):
    """Conformal time tau(a) = int_0^a da' / (a'^2 E(a')), H0 = 1.

    Substituting a' = u^2 removes the 1/sqrt(a') end-point singularity:
    tau = int_0^sqrt(a) 2 du / sqrt(om + ol u^6).
    """
    val, _ = integrate.quad(lambda u: 2.0 / math.sqrt(om + ol * u**6),
                            0.0, math.sqrt(a), epsabs=0.0, epsrel=1e-13,
                            limit=200)
    return val


def chi(a, om, ol):
    """Comoving lightcone distance from the z=0 observer at expansion a, Mpc/h."""
    return C_OVER_H0 * (tau(1.0, om, ol) - tau(a, om, ol))


def a_of_tau(t, om, ol, lo=1e-12, hi=4.0):
    """Invert tau(a) = t by bisection in FP64 (tau is monotone in a)."""
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if tau(mid, om, ol) < t:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 4e-16 * hi:
            break
    return 0.5 * (lo + hi)


def growth_D(a, om, ol):
    """Linear growth factor, Heath (1977) integral, normalised to D -> a early.

    D(a) = (5 om / 2) E(a) int_0^a da' / (a' E(a'))^3.
    """
    integrand = lambda x: x**1.5 / (om + ol * x**3) ** 1.5
    val, _ = integrate.quad(integrand, 0.0, a, epsabs=0.0, epsrel=1e-13,
                            limit=200)
    return 2.5 * om * E(a, om, ol) * val


def growth_f(a, om, ol):
    """Growth rate f = dlnD/dlna = -3 om/(2 a^3 E^2) + a / ((aE)^3 I(a))."""
    integrand = lambda x: x**1.5 / (om + ol * x**3) ** 1.5
    val, _ = integrate.quad(integrand, 0.0, a, epsabs=0.0, epsrel=1e-13,
                            limit=200)
    e = E(a, om, ol)
    return -1.5 * om / (a**3 * e * e) + a / ((a * e) ** 3 * val)


def schedule(n_mesh, box, om, ol, a_init, a_final, n_steps, buffer_cells=1.0):
    """Per-step scalars of a run with steps uniform in a (Sec. 3).

    Returns a dict of float64 arrays over k = 0..n_steps:
      a[k]        expansion factor at the start of step k (a[n_steps] = a_final)
      dtau[k]     conformal step tau(a[k+1]) - tau(a[k])       (k < n_steps)
      a_half[k]   a at tau(a[k]) + dtau[k]/2                    (k < n_steps)
      chi[k]      lightcone distance chi(a[k]), Mpc/h
      R[k]        keep half-width in cells: chi/cell + buffer_cells
    """
    a = a_init + (a_final - a_init) * np.arange(n_steps + 1) / n_steps
    t = np.array([tau(x, om, ol) for x in a])
    dtau = t[1:] - t[:-1]
    a_half = np.array([a_of_tau(t[k] + 0.5 * dtau[k], om, ol)
                       for k in range(n_steps)])
    ch = np.array([chi(x, om, ol) for x in a])
    cell = box / n_mesh
    R = ch / cell + buffer_cells
    return dict(a=a, tau=t, dtau=dtau, a_half=a_half, chi=ch, R=R)
