"""The multigrid smoother (two red-black SOR sweeps, factor PM_MG_OMEGA, of
the 7-point system of Eq. 3): the fused one-pass kernel against the four
one-colour passes (same bits) and against an FP64 statement of the
sweeps."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1709_04703_gb300 import _lib as L  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_04703_gb300 import build
    build.build()
    return L.load()


def _p(t):
    return C.c_void_p(t.data_ptr())


def _smooth(lib, u, b, s, periodic, h2, gam, zero, fused, zchunk=0):
    out = torch.full_like(u, float("nan")) if (fused and not zero) else u.clone()
    uin = u if not zero else None
    code = lib.pm_mg_smooth(_p(uin) if uin is not None else None, _p(out), _p(b), s,
                            int(periodic), C.c_float(h2), C.c_float(gam), int(zero), int(fused),
                            int(zchunk), None)
    assert code == L.PM_OK, lib.pm_last_error(None)
    return out


def _inputs(s, seed):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((s + 2,) * 3).astype(np.float32)
    b = rng.standard_normal((s + 2,) * 3).astype(np.float32)
    return torch.from_numpy(u).cuda(), torch.from_numpy(b).cuda()


CASES = [(s, per, gam) for s in (8, 24, 32, 48, 64, 100) for per, gam in
         ((0, 0.0), (1, 0.0), (0, 3.0 / 5.0))]


@pytest.mark.parametrize("s,periodic,gam", CASES)
@pytest.mark.parametrize("zero", [0, 1])
@pytest.mark.parametrize("tile", [1, 24, 32])
def test_fused_pass_gives_the_same_bits(lib, s, periodic, gam, zero, tile):
    """Every tile height (1: the default 16) against the one-colour passes;
    the sides span several tiles and ragged last tiles in x, y and z."""
    u, b = _inputs(s, 10 * s + periodic + zero)
    h2 = 4.0 if gam else 1.0
    ref = _smooth(lib, u, b, s, periodic, h2, gam, zero, fused=0)
    for zc in (0, 5, 16):
        got = _smooth(lib, u, b, s, periodic, h2, gam, zero, fused=tile, zchunk=zc)
        a = got[1:-1, 1:-1, 1:-1].cpu().numpy()
        r = ref[1:-1, 1:-1, 1:-1].cpu().numpy()
        assert np.array_equal(a.view(np.uint32), r.view(np.uint32)), (zc, np.abs(a - r).max())


def _sweeps_fp64(u, b, s, periodic, h2, gam, zero):
    """Red then black, twice, in FP64 (ghosts read as stored; periodic
    wraps): each cell moves from its old value towards the Gauss-Seidel
    value by the factor PM_MG_OMEGA."""
    u = np.zeros_like(u, dtype=np.float64) if zero else u.astype(np.float64)
    b = b.astype(np.float64)
    idx = np.arange(s)
    Z, Y, X = np.meshgrid(idx, idx, idx, indexing="ij")
    nghost = sum((c == e).astype(np.int64) for c in (X, Y, Z) for e in (0, s - 1))
    diag = 6.0 + (0.0 if periodic else gam) * nghost
    for _ in range(2):
        for colour in (0, 1):
            v = u[1:-1, 1:-1, 1:-1]
            if periodic:
                nb = sum(np.roll(v, sh, axis=ax) for ax in range(3) for sh in (1, -1))
            else:
                nb = (u[2:, 1:-1, 1:-1] + u[:-2, 1:-1, 1:-1] + u[1:-1, 2:, 1:-1]
                      + u[1:-1, :-2, 1:-1] + u[1:-1, 1:-1, 2:] + u[1:-1, 1:-1, :-2])
            new = (nb - h2 * b[1:-1, 1:-1, 1:-1]) / diag
            m = (X + Y + Z) % 2 == colour
            v[m] = v[m] + L.PM_MG_OMEGA * (new[m] - v[m])
    return u


@pytest.mark.parametrize("s,periodic,gam", [(8, 0, 0.0), (12, 1, 0.0), (16, 0, 1.0 / 3.0)])
@pytest.mark.parametrize("zero", [0, 1])
def test_fused_pass_matches_fp64_sweeps(lib, s, periodic, gam, zero):
    u, b = _inputs(s, 7 + s)
    if zero:
        u = torch.zeros_like(u)
    got = _smooth(lib, u, b, s, periodic, 2.0, gam, zero, fused=1)
    ref = _sweeps_fp64(u.cpu().numpy(), b.cpu().numpy(), s, periodic, 2.0, gam, zero)
    np.testing.assert_allclose(got[1:-1, 1:-1, 1:-1].cpu().numpy(), ref[1:-1, 1:-1, 1:-1],
                               rtol=1e-5, atol=1e-5 * np.abs(ref).max())


# ------------------------------------------------------------ transfers

def _restrict_fp64(u, b, s, periodic, h2, gam):
    """1/8 of the sum over the 8 children of b - (sum_nb u - diag u)/h2, in
    FP64 (ghosts read as stored; periodic wraps)."""
    u = u.astype(np.float64)
    b = b.astype(np.float64)[1:-1, 1:-1, 1:-1]
    v = u[1:-1, 1:-1, 1:-1]
    if periodic:
        nb = sum(np.roll(v, sh, axis=ax) for ax in range(3) for sh in (1, -1))
        diag = 6.0
    else:
        nb = (u[2:, 1:-1, 1:-1] + u[:-2, 1:-1, 1:-1] + u[1:-1, 2:, 1:-1]
              + u[1:-1, :-2, 1:-1] + u[1:-1, 1:-1, 2:] + u[1:-1, 1:-1, :-2])
        idx = np.arange(s)
        Z, Y, X = np.meshgrid(idx, idx, idx, indexing="ij")
        diag = 6.0 + gam * sum((c == e).astype(np.float64) for c in (X, Y, Z) for e in (0, s - 1))
    r = b - (nb - diag * v) / h2
    sc = s // 2
    return r.reshape(sc, 2, sc, 2, sc, 2).mean(axis=(1, 3, 5))


def _prolong_fp64(uc, u, s, periodic, gam_c):
    """u + P uc: per axis 3/4 of the parent and 1/4 of the next coarse cell
    (below for an even child, above for an odd one), wrapped, or (open)
    -gam_c times the parent outside the coarse grid."""
    sc = s // 2
    q = uc.astype(np.float64)[1:-1, 1:-1, 1:-1]
    i = np.arange(s)
    par = i // 2
    nxt = np.where(i % 2 == 1, par + 1, par - 1)
    fac = np.ones(s)
    if periodic:
        nxt %= sc
    else:
        out = (nxt < 0) | (nxt >= sc)
        nxt = np.where(out, par, nxt)
        fac = np.where(out, -gam_c, 1.0)
    terms = [(par, np.full(s, 0.75)), (nxt, 0.25 * fac)]
    val = np.zeros((s, s, s))
    for zi, wz in terms:
        for yi, wy in terms:
            for xi, wx in terms:
                val += (wz[:, None, None] * wy[None, :, None] * wx[None, None, :]
                        * q[np.ix_(zi, yi, xi)])
    return u.astype(np.float64)[1:-1, 1:-1, 1:-1] + val


TCASES = [(s, per, gam) for s in (8, 24, 64, 100) for per, gam in
          ((1, 0.0), (0, 0.0), (0, 1.0 / 3.0), (0, 3.0 / 5.0))]


@pytest.mark.parametrize("s,periodic,gam", TCASES)
def test_restriction_matches_its_definition(lib, s, periodic, gam):
    u, b = _inputs(s, 300 + s)
    sc = s // 2
    uc = torch.full(((sc + 2),) * 3, 7.0, device="cuda")
    bc = torch.zeros(((sc + 2),) * 3, device="cuda")
    h2 = 4.0 if gam else 1.0
    code = lib.pm_mg_restrict(_p(u), _p(b), s, periodic, C.c_float(h2), C.c_float(gam), _p(uc),
                              _p(bc), None)
    assert code == L.PM_OK, lib.pm_last_error(None)
    ref = _restrict_fp64(u.cpu().numpy(), b.cpu().numpy(), s, periodic, h2, gam)
    got = bc[1:-1, 1:-1, 1:-1].cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-6 * np.abs(ref).max() + 1e-6)
    assert np.all(uc[1:-1, 1:-1, 1:-1].cpu().numpy() == 0.0)
    assert np.all(uc[0].cpu().numpy() == 7.0)   # ghosts untouched


@pytest.mark.parametrize("s,periodic,gam", TCASES)
def test_prolongation_matches_its_definition(lib, s, periodic, gam):
    u, _ = _inputs(s, 400 + s)
    sc = s // 2
    uc = torch.randn(((sc + 2),) * 3, device="cuda")
    before = u.clone()
    code = lib.pm_mg_prolong(_p(uc), _p(u), s, periodic, C.c_float(gam), None)
    assert code == L.PM_OK, lib.pm_last_error(None)
    ref = _prolong_fp64(uc.cpu().numpy(), before.cpu().numpy(), s, periodic, gam)
    got = u[1:-1, 1:-1, 1:-1].cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-6 * np.abs(ref).max())
    assert torch.equal(u[0], before[0])          # ghosts untouched


def test_fused_pass_rejects_other_tile_heights(lib):
    u, b = _inputs(8, 1)
    out = u.clone()
    for fused in (2, 8, 48, -1):
        code = lib.pm_mg_smooth(_p(u), _p(out), _p(b), 8, 0, C.c_float(1.0), C.c_float(0.0), 0,
                                fused, 0, None)
        assert code == L.PM_EINVAL


@pytest.mark.parametrize("domain", ["cube", "ball"])
def test_smoother_tiles_tuned_per_level_side(lib, domain):
    """pm_init times the fused pass's launch shapes on every level side of at
    least 192 that the run's cubes give (the 256^3 schedule: 256 periodic,
    then shrinking open cubes); the ball solve keeps tile height 16."""
    from paper_1709_04703_gb300 import ics
    from paper_1709_04703_gb300.sim import Sim
    n = 256
    pos, mom, ids = ics.random_particles(8, n, 0)
    kw = dict(domain="ball", precision="mixed") if domain == "ball" else {}
    sim = Sim(pos, mom, ids, n, 2000.0, 0.01, 1.0, 200, **kw)
    try:
        cnt = C.c_int32(-1)
        assert lib.pm_smoother_tiles(sim._ctx, None, None, None, 0, C.byref(cnt)) == L.PM_OK
        m = cnt.value
        if domain == "ball":
            assert m == 0
            return
        assert m >= 1
        sides = (C.c_int32 * m)()
        ty = (C.c_int32 * m)()
        zc = (C.c_int32 * m)()
        assert lib.pm_smoother_tiles(sim._ctx, sides, ty, zc, m, C.byref(cnt)) == L.PM_OK
        assert 256 in list(sides)
        assert len(set(sides)) == m
        for i in range(m):
            assert 192 <= sides[i] <= n and sides[i] % 2 == 0
            assert ty[i] in (16, 24, 32)
            assert 1 <= zc[i] <= 128
    finally:
        sim.close()
