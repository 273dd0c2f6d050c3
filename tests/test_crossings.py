"""The lightcone-crossing comparison used by the whole-run parity tests,
on hand-made catalogues: a crossing one step apart on a particle at the
keep cube's face passes; one far inside the cube, or further out than the
two runs' measured divergence, fails."""
import numpy as np
import pytest

import crossings

N_MESH = 16
SCHED = {"a": np.array([0.5, 0.6, 0.7, 0.8]), "R": np.array([9.0, 6.0, 4.0, 2.0])}


def _pair():
    # four particles; both runs record 0 at a=0.6 and keep 3; 1 and 2 at a=0.7
    ids = np.arange(4)
    a = np.array([0.6, 0.7, 0.7, 0.0])
    x = np.array([[8 + 6.5, 8, 8], [8, 8 + 4.2, 8], [8 - 4.3, 8, 8], [8.5, 8, 8]])
    return ids, a, x


def test_identical_runs_agree():
    ids, a, x = _pair()
    m, d = crossings.check_crossings(a, x, a.copy(), x.copy(), SCHED, N_MESH)
    assert (m, d) == (0, 0.0)


def test_one_step_earlier_at_the_face_passes():
    ids, a, x = _pair()
    a_g, x_g = a.copy(), x.copy() + 1e-3
    # run g drops particle 1 at a=0.6, just outside R=6 (by 1e-4), run o one step later
    a_g[1] = 0.6
    x_g[1] = [8, 8 + 6.0001, 8]
    m, d = crossings.check_crossings(a_g, x_g, a, x, SCHED, N_MESH)
    assert m == 1 and d == pytest.approx(1e-3)


def test_crossing_far_from_the_face_fails():
    ids, a, x = _pair()
    a_g, x_g = a.copy(), x.copy() + 1e-3
    a_g[1] = 0.6
    x_g[1] = [8, 8 + 6.5, 8]      # 0.5 cells outside: far beyond the divergence
    with pytest.raises(AssertionError):
        crossings.check_crossings(a_g, x_g, a, x, SCHED, N_MESH)


def test_survivor_against_record_uses_the_record():
    ids, a, x = _pair()
    a_o, x_o = a.copy(), x.copy()
    a_g, x_g = a.copy(), x.copy() + 1e-3
    # run o records the survivor 3 at a=0.8 just outside R=2; run g keeps it
    a_o[3] = 0.8
    x_o[3] = [8 + 2.0005, 8, 8]
    m, _ = crossings.check_crossings(a_g, x_g, a_o, x_o, SCHED, N_MESH)
    assert m == 1
    x_o[3] = [8 + 1.5, 8, 8]        # recorded while inside the cube: impossible
    with pytest.raises(AssertionError):
        crossings.check_crossings(a_g, x_g, a_o, x_o, SCHED, N_MESH)


def test_float32_crossings_match_the_schedule():
    ids, a, x = _pair()
    a_g = a.astype(np.float32).astype(np.float64)
    m, _ = crossings.check_crossings(a_g, x.copy(), a, x.copy(), SCHED, N_MESH)
    assert m == 0
