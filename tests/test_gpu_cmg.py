"""The coarse multigrid levels in one thread-block cluster (k_cmg.cu): the
levels of side <= 64 live in the cluster's distributed shared memory and
each smoothing pass, restriction and prolongation is a phase between
cluster barriers.  It applies the per-level kernels' arithmetic, so the
potential of Eq. 3 must come out bit for bit as with one CTA per launch
(PM_CMG_CLUSTER = 16 or 8 against PM_NO_CLUSTER: levels above 16^3 launched
one kernel per phase, the rest in one CTA), for open and periodic meshes whose hierarchies put the cluster's
top at 64, 48 and 24 and the bottom at 4 and 3; and a run through both
boundary phases, whose open cubes of sides 5 * 2^j and 7 * 2^j put the top
at 56, 40, 28, ... and the bottom at 7 and 5, gives the same particles
either way."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1709_04703_gb300 import ics  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_04703_gb300 import build
    build.build()


def _with_cluster(on, fn, size="16"):
    old = {k: os.environ.pop(k, None) for k in ("PM_NO_CLUSTER", "PM_CMG_CLUSTER")}
    if on:
        os.environ["PM_CMG_CLUSTER"] = size
    else:
        os.environ["PM_NO_CLUSTER"] = "1"
    try:
        return fn()
    finally:
        for k, v in old.items():
            os.environ.pop(k, None)
            if v is not None:
                os.environ[k] = v


def _potential(n, bc, seed, rtol=1e-9):
    from paper_1709_04703_gb300 import _lib as L
    from paper_1709_04703_gb300.sim import Sim
    pos, mom, ids = ics.random_particles(8, n, 0)
    sim = Sim(pos, mom, ids, n, 100.0, 0.5, 1.0, 4, rtol=rtol, max_vcycles=60)
    cl = L.load().pm_mg_cluster_size()
    rng = np.random.default_rng(seed)
    delta = rng.standard_normal((n, n, n))
    if bc == "periodic":
        delta -= delta.mean()
    else:
        delta[: n // 4] = 0.0
    phi32, phi64, vc, res = sim.solve_potential(delta, 0.5, bc)
    out = phi64.cpu().numpy(), vc, res, cl
    sim.close()
    return out


@pytest.mark.parametrize("size", ["16", "8"])
@pytest.mark.parametrize("n,bc", [(64, "open"), (64, "periodic"), (128, "periodic"),
                                  (128, "open"), (96, "periodic"), (96, "open"),
                                  (48, "open"), (24, "periodic")])
def test_cluster_potential_is_bitwise(n, bc, size):
    a, va, ra, cl_on = _with_cluster(True, lambda: _potential(n, bc, n), size)
    b, vb, rb, cl_off = _with_cluster(False, lambda: _potential(n, bc, n))
    assert cl_off == 1
    assert cl_on == int(size)
    assert va == vb and ra == rb
    np.testing.assert_array_equal(a.view(np.uint64), b.view(np.uint64))


def test_cluster_sizes_on_this_gpu():
    """A GB300 holds clusters of 16 CTAs with the 64^3 layout (~160 KB of
    shared memory each); one CTA is the default."""
    _, _, _, cl = _with_cluster(True, lambda: _potential(16, "periodic", 0))
    assert cl == 16
    old = {k: os.environ.pop(k, None) for k in ("PM_NO_CLUSTER", "PM_CMG_CLUSTER")}
    try:
        _, _, _, cl = _potential(16, "periodic", 0)
    finally:
        for k, v in old.items():
            if v is not None:
                os.environ[k] = v
    assert cl == 1


def test_cluster_run_is_bitwise():
    """A 64^3 run through the periodic phase into shrinking open cubes
    (cluster tops 64, 56, 48, 40, 32, ...): the same particles and lightcone."""
    from paper_1709_04703_gb300.sim import Sim
    n = 64
    pos, mom, ids = ics.zeldovich(n, -1.5, 0.5, 9, 0.35, rms_disp=0.5)

    def run():
        sim = Sim(pos, mom, ids, n, 7000.0, 0.35, 1.0, 14, rtol=1e-7)
        sim.step(14)
        out = sim.particles() + sim.lightcone()[:3] + (sim.stats()["vcycles_total"],)
        sim.close()
        return out
    a = _with_cluster(True, run)
    b = _with_cluster(False, run)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)


def _with_generic(on, fn):
    old = os.environ.pop("PM_CMG_GENERIC", None)
    if on:
        os.environ["PM_CMG_GENERIC"] = "1"
    try:
        return fn()
    finally:
        os.environ.pop("PM_CMG_GENERIC", None)
        if old is not None:
            os.environ["PM_CMG_GENERIC"] = old


@pytest.mark.parametrize("n,bc", [(64, "periodic"), (64, "open"), (96, "periodic"),
                                  (96, "open"), (48, "open"), (24, "periodic"),
                                  (16, "open"), (16, "periodic"), (12, "open"),
                                  (12, "periodic"), (8, "open"), (6, "periodic"),
                                  (4, "open"), (4, "periodic")])
def test_constant_side_coarse_form_is_bitwise(n, bc):
    """The one-CTA coarse levels with compile-time sides and ghost halos
    (cmg_fast.cuh) against the generic one-CTA form (PM_CMG_GENERIC): tops
    16, 12, 8, 6 and 4, bottoms 4 and 3, the top as the whole mesh (n <= 16:
    the Dirichlet data in the top's halo) or a coarse level."""
    a, va, ra, _ = _with_cluster(False, lambda: _with_generic(False,
                                                              lambda: _potential(n, bc, n)))
    b, vb, rb, _ = _with_cluster(False, lambda: _with_generic(True,
                                                              lambda: _potential(n, bc, n)))
    assert va == vb and ra == rb
    np.testing.assert_array_equal(a.view(np.uint64), b.view(np.uint64))


def test_constant_side_coarse_form_run_is_bitwise():
    """A 64^3 run through the periodic phase into shrinking open cubes whose
    coarse tops include 14 and 10 (bottoms 7 and 5): the same particles,
    lightcone and V-cycle counts with either one-CTA form."""
    from paper_1709_04703_gb300.sim import Sim
    n = 64
    pos, mom, ids = ics.zeldovich(n, -1.5, 0.5, 9, 0.35, rms_disp=0.5)

    def run():
        sim = Sim(pos, mom, ids, n, 7000.0, 0.35, 1.0, 14, rtol=1e-7)
        sim.step(14)
        out = sim.particles() + sim.lightcone()[:3] + (sim.stats()["vcycles_total"],)
        sim.close()
        return out
    a = _with_cluster(False, lambda: _with_generic(False, run))
    b = _with_cluster(False, lambda: _with_generic(True, run))
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
