"""Comparison of two runs' lightcone catalogues (test helper).

A particle leaves the active set at the end of the first step after which it
lies outside the keep cube (Sec. 2.4, Table 2's last row).  Two runs that
integrate the same particles in different arithmetic (FP32 on the GPU, FP64
in the oracle) follow trajectories a small distance apart, so a particle that
ends a step within that distance of the cube's face can leave one step
earlier in one run than in the other.  That is the only admissible
difference: check_crossings() asserts it for every particle whose crossing
differs, with the distance measured from the particles whose crossings agree.
"""
import numpy as np


def table(N, ids_act, x_act, ids_lc, x_lc, a_lc):
    """Per particle id: a_cross (0 for a survivor) and the recorded position
    (lightcone record, or the final position of a survivor)."""
    a = np.zeros(N)
    x = np.full((N, 3), np.nan)
    a[np.asarray(ids_lc)] = np.asarray(a_lc, np.float64)
    x[np.asarray(ids_lc)] = np.asarray(x_lc, np.float64)
    x[np.asarray(ids_act)] = np.asarray(x_act, np.float64)
    return a, x


def check_crossings(a_g, x_g, a_o, x_o, sched, n, slack=1.0, max_frac=None):
    """Every particle of run g whose crossing differs from run o's must have
    been, on the side that dropped it first, outside the keep cube by no more
    than slack x the largest distance between the two runs' positions of the
    particles recorded at the same time.  Returns (mismatches, that distance)."""
    a_sched = np.asarray(sched["a"])
    R_sched = np.asarray(sched["R"])
    c = 0.5 * n
    same = a_g == a_o
    # the GPU stores a_cross as float32: match it to the schedule's entries
    a_g = np.where(a_g > 0, a_sched[np.abs(a_sched[None, :] - a_g[:, None]).argmin(1)], 0.0)
    same = same | (a_g == a_o)
    ok = same & np.isfinite(x_g).all(1) & np.isfinite(x_o).all(1)
    assert ok.any()
    delta = float(np.abs(x_g[ok] - x_o[ok]).max())
    bad = np.flatnonzero(~same)
    if max_frac is not None:
        assert len(bad) <= max_frac * len(a_g), (len(bad), len(a_g))
    for i in bad:
        ag, ao = a_g[i], a_o[i]
        # the run that recorded the particle first (0 = never recorded)
        if ao == 0 or (ag != 0 and ag < ao):
            a_star, x_star = ag, x_g[i]
        else:
            a_star, x_star = ao, x_o[i]
        k = int(np.abs(a_sched - a_star).argmin())
        out = float(np.abs(x_star - c).max() - R_sched[k])
        assert 0.0 < out <= slack * delta + 1e-6, (int(i), ag, ao, out, delta)
    return len(bad), delta
