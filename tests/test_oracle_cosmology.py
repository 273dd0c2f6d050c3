"""Pins of the oracle's background cosmology against closed forms.

tau(a) of flat LCDM is a Gauss hypergeometric function,
    tau(a) = 2 sqrt(a/Om) 2F1(1/6, 1/2; 7/6; -(OL/Om) a^3),
and the growing mode is D(a) = a 2F1(1/3, 1; 11/6; -(OL/Om) a^3).
Einstein-de Sitter (Om = 1) has tau = 2 sqrt(a), chi = 2 (c/H0)(1 - sqrt a),
D = a, f = 1.
"""
import math

import numpy as np
import pytest
from scipy.special import hyp2f1

from oracle import cosmology as cz

OM, OL = 0.3, 0.7


def tau_closed(a, om, ol):
    return 2 * math.sqrt(a / om) * hyp2f1(1 / 6, 1 / 2, 7 / 6, -(ol / om) * a**3)


def D_closed(a, om, ol):
    return a * hyp2f1(1 / 3, 1.0, 11 / 6, -(ol / om) * a**3)


@pytest.mark.parametrize("a", [0.005, 0.01, 0.02, 0.1, 0.5, 0.8, 1.0])
def test_tau_matches_hypergeometric(a):
    assert cz.tau(a, OM, OL) == pytest.approx(tau_closed(a, OM, OL), rel=1e-12)


@pytest.mark.parametrize("a", [0.01, 0.25, 0.7, 1.0])
def test_eds_closed_forms(a):
    assert cz.tau(a, 1.0, 0.0) == pytest.approx(2 * math.sqrt(a), rel=1e-13)
    assert cz.chi(a, 1.0, 0.0) == pytest.approx(
        2 * cz.C_OVER_H0 * (1 - math.sqrt(a)), rel=1e-12, abs=1e-9)
    assert cz.growth_D(a, 1.0, 0.0) == pytest.approx(a, rel=1e-12)
    assert cz.growth_f(a, 1.0, 0.0) == pytest.approx(1.0, rel=1e-10)


@pytest.mark.parametrize("a", [0.02, 0.3, 0.5, 1.0])
def test_growth_matches_hypergeometric(a):
    assert cz.growth_D(a, OM, OL) == pytest.approx(D_closed(a, OM, OL), rel=1e-11)
    # f = dlnD/dlna by a central difference of the closed form
    h = 1e-5
    fd = (math.log(D_closed(a * (1 + h), OM, OL))
          - math.log(D_closed(a * (1 - h), OM, OL))) / (
        math.log(1 + h) - math.log(1 - h))
    assert cz.growth_f(a, OM, OL) == pytest.approx(fd, rel=1e-8)


def test_chi_vanishes_today_and_decreases():
    assert cz.chi(1.0, OM, OL) == 0.0
    a = np.linspace(0.01, 1.0, 30)
    c = [cz.chi(x, OM, OL) for x in a]
    assert all(x > y for x, y in zip(c, c[1:]))


def test_a_half_eds_closed_form():
    # EdS: tau = 2 sqrt(a) so the conformal midpoint is ((sqrt a0 + sqrt a1)/2)^2
    s = cz.schedule(32, 250.0, 1.0, 0.0, 0.02, 1.0, 20)
    ah = ((np.sqrt(s["a"][:-1]) + np.sqrt(s["a"][1:])) / 2) ** 2
    np.testing.assert_allclose(s["a_half"], ah, rtol=1e-13)


def test_schedule_lcdm_consistency():
    s = cz.schedule(256, 2000.0, OM, OL, 0.01, 1.0, 200)
    assert s["dtau"].sum() == pytest.approx(
        tau_closed(1.0, OM, OL) - tau_closed(0.01, OM, OL), rel=1e-12)
    for k in (0, 57, 199):
        t_mid = tau_closed(s["a"][k], OM, OL) + 0.5 * s["dtau"][k]
        assert tau_closed(s["a_half"][k], OM, OL) == pytest.approx(t_mid, rel=1e-12)
    np.testing.assert_allclose(s["R"], s["chi"] / (2000.0 / 256) + 1.0, rtol=1e-15)
    assert s["a"][0] == 0.01 and s["a"][-1] == 1.0
    assert np.all(np.diff(s["a"]) > 0)
