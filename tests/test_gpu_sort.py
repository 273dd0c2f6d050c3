"""Particle order by mesh cell (sort_every, pm_sort_particles): the GPU
radix sort against the oracle's stable cell order, record for record; the
deposit's in-warp merging of same-cell runs bit for bit against the oracle
deposit; and whole runs with and without reordering, equal particle by
particle (the order changes no result of a step)."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import pm as opm  # noqa: E402
from paper_1709_04703_gb300 import ics  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_04703_gb300 import build
    build.build()


def _dev4(pos, mom=None, ids=None):
    from paper_1709_04703_gb300.sim import pack
    p4, m4 = pack(pos, np.zeros_like(pos) if mom is None else mom, ids)
    return p4, m4, torch.from_numpy(p4).cuda(), torch.from_numpy(m4).cuda()


def _clustered(N, n, seed, n_centres, spread):
    """Particles around a few cell centres (runs of one cell, many per warp)."""
    rng = np.random.default_rng(seed)
    c = rng.integers(0, n, (n_centres, 3)) + 0.5
    pos = c[rng.integers(0, n_centres, N)] + rng.uniform(-spread, spread, (N, 3))
    pos = np.mod(pos, n).astype(np.float32)
    pos[pos >= np.float32(n)] = 0.0
    mom = rng.uniform(-0.5, 0.5, (N, 3)).astype(np.float32)
    return pos, mom


CASES = [(32, 1, "uniform"), (32, 4095, "uniform"), (32, 4097, "clustered"),
         (96, 100003, "clustered"), (256, 300001, "uniform"), (1024, 70001, "uniform"),
         (8, 20000, "clustered"), (64, 50000, "edge")]


@pytest.mark.parametrize("n,N,kind", CASES)
@pytest.mark.parametrize("with_mom", [True, False])
def test_sort_matches_the_oracle_order(n, N, kind, with_mom):
    from paper_1709_04703_gb300.sim import sort_particles
    if kind == "clustered":
        pos, mom = _clustered(N, n, N, max(1, N // 500), 0.7)
    else:
        pos, mom, _ = ics.random_particles(N, n, N + n)
    if kind == "edge":
        # outside the box, negative, non-finite: wrapped, or cell 0
        pos[::7] -= np.float32(n)
        pos[1::11] += np.float32(3 * n)
        pos[2::13, 0] = np.nan
        pos[3::17, 1] = np.inf
        pos[4::19, 2] = -np.inf
        pos[5::23, 0] = np.float32(-0.25)
    p4, m4, dp, dm = _dev4(pos, mom)
    po, mo = sort_particles(dp, dm if with_mom else None, n)
    o = opm.cell_order(pos, n)
    np.testing.assert_array_equal(po.cpu().numpy().view(np.uint32), p4[o].view(np.uint32))
    if with_mom:
        np.testing.assert_array_equal(mo.cpu().numpy().view(np.uint32), m4[o].view(np.uint32))


def test_sort_argument_checks():
    from paper_1709_04703_gb300 import _lib as L
    lib = L.load()
    p = torch.zeros((16, 4), device="cuda")
    q = torch.zeros((16, 4), device="cuda")
    ptr = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    assert lib.pm_sort_particles(ptr(p), None, 0, 8, ptr(q), None, None) == L.PM_OK
    assert lib.pm_sort_particles(ptr(p), None, 16, 8, ptr(p), None, None) == L.PM_EINVAL
    assert lib.pm_sort_particles(ptr(p), ptr(q), 16, 8, ptr(q), ptr(p), None) == L.PM_EINVAL
    assert lib.pm_sort_particles(ptr(p), None, 16, 0, ptr(q), None, None) == L.PM_EINVAL
    assert lib.pm_sort_particles(ptr(p), None, 16, 2048, ptr(q), None, None) == L.PM_EINVAL


@pytest.mark.parametrize("periodic,lo,s", [(True, 0, 48), (False, 8, 30)])
@pytest.mark.parametrize("drift", [False, True])
def test_deposit_of_cell_runs_is_bitexact(periodic, lo, s, drift):
    """Cell-sorted clustered particles: runs of one cell within and across
    warps, x-neighbouring runs, escaped particles inside runs (open cube)."""
    from paper_1709_04703_gb300.sim import deposit
    n = 48
    pos, mom = _clustered(200003, n, 7, 300, 0.9)
    o = opm.cell_order(pos, n)
    pos, mom = pos[o], mom[o]
    p4, m4, dp, dm = _dev4(pos, mom)
    coef = 0.37 if drift else 0.0
    rho, esc = deposit(dp, n, lo, s, periodic, mom4_dev=dm if drift else None, drift_coef=coef)
    x = opm.drift_fp32(pos, mom, coef, n, periodic) if drift else pos
    ref, resc = opm.deposit(x, n, lo, s, periodic)
    assert esc == resc
    assert periodic or resc > 0
    np.testing.assert_array_equal(rho.cpu().numpy(), ref)
    if drift:
        np.testing.assert_array_equal(dp.cpu().numpy()[:, :3], x.astype(np.float32))


def _run(n, box, a0, steps, sort_every, **kw):
    from paper_1709_04703_gb300.sim import Sim
    pos, mom, ids = ics.zeldovich(n, -1.5, 0.5, 4, a0, rms_disp=0.6)
    sim = Sim(pos, mom, ids, n, box, a0, 1.0, steps, sort_every=sort_every, **kw)
    sim.step(steps)
    st = sim.stats()
    p, m, i = sim.particles()
    lp, lm, li, la = sim.lightcone()
    sim.close()
    oa, ol = np.argsort(i), np.argsort(li)
    return st, (p[oa], m[oa], i[oa]), (lp[ol], lm[ol], li[ol], la[ol])


@pytest.mark.parametrize("kw", [dict(), dict(assignment="tsc"), dict(domain="sphere"),
                                dict(shrink="record", bc="periodic")])
@pytest.mark.parametrize("every", [1, 5])
def test_sorted_run_equals_the_unsorted_run(kw, every):
    """Reordering changes the order of the arrays, nothing else: every
    particle and lightcone record bit for bit (matched by id), the counts
    and the solver's work."""
    n, box, a0, steps = 32, 6000.0, 0.2, 24
    s0, a0_, l0 = _run(n, box, a0, steps, 0, **kw)
    s1, a1_, l1 = _run(n, box, a0, steps, every, **kw)
    assert s1["n_lightcone"] == s0["n_lightcone"] > 0
    for f in ("n_active", "vcycles_total", "escaped", "cube_side", "resid_last"):
        assert s1[f] == s0[f], f
    for u, v in zip(a1_ + l1, a0_ + l0):
        np.testing.assert_array_equal(u, v)


def test_sorted_steps_equal_unsorted_steps_full_size():
    """The 256^3 workload in the benchmarked launch configuration, three
    steps sorted before each and not: the same particles bit for bit."""
    from paper_1709_04703_gb300.sim import Sim
    cfg = ics.WORKLOADS["pm256"]
    pos, mom, ids = ics.workload_ics("pm256")
    out = []
    for every in (0, 1):
        sim = Sim(pos, mom, ids, cfg["n"], cfg["box"], cfg["a_init"], cfg["a_final"],
                  cfg["steps"], rtol=2.4e-4, max_vcycles=100, sort_every=every)
        sim.step(3)
        p, m, i = sim.particles()
        st = sim.stats()
        sim.close()
        o = np.argsort(i)
        out.append((st["vcycles_total"], p[o], m[o], i[o]))
    assert out[0][0] == out[1][0]
    for u, v in zip(out[0][1:], out[1][1:]):
        np.testing.assert_array_equal(u, v)


def test_batch_rejects_sorting():
    from paper_1709_04703_gb300 import _lib as L
    from paper_1709_04703_gb300.sim import _config, pack
    lib = L.load()
    pos, mom, ids = ics.zeldovich(16, -1.5, 0.5, 1, 0.3)
    cfgs = (L.PmConfig * 1)()
    cfgs[0] = _config(16, len(pos), 500.0, 0.3, 1.0, 4)
    cfgs[0].sort_every = 2
    p4, m4 = pack(pos, mom, ids)
    dp, dm = torch.from_numpy(p4).cuda(), torch.from_numpy(m4).cuda()
    pp = (C.c_void_p * 1)(dp.data_ptr())
    mp = (C.c_void_p * 1)(dm.data_ptr())
    st = torch.cuda.Stream()
    b = C.c_void_p()
    code = lib.pm_batch_init(1, cfgs, pp, mp, 0, C.c_void_p(st.cuda_stream), C.byref(b))
    assert code == L.PM_EINVAL and not b.value
