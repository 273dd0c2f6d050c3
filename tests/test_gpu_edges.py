"""Edge positions on the GPU against the oracle: particles exactly on cell
faces and on CIC nodes, at the periodic wrap, on the last nodes inside an
open cube and just beyond (deposit bit for bit, escape counts equal), and
exactly on the lightcone keep boundary |x_d - c| = R, where the keep rule's
"<=" decides (shrink bit for bit, cube and sphere)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import cosmology as cz  # noqa: E402
from oracle import pm as opm  # noqa: E402
from paper_1709_04703_gb300 import ics  # noqa: E402

OM, OL = 0.3, 0.7


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_04703_gb300 import build
    build.build()


def _edge_positions(n, lo, s, seed):
    """Per axis a value from: cell faces i, nodes i + 1/2, the float32
    neighbours of both, 0, the largest float below n, and the first and last
    positions whose CIC nodes lie in [lo, lo + s) and their neighbours."""
    f32 = np.float32
    vals = []
    for i in range(n):
        for v in (f32(i), f32(i + 0.5)):
            vals += [v, np.nextafter(v, f32(-1e9)), np.nextafter(v, f32(1e9))]
    vals += [f32(0.0), np.nextafter(f32(n), f32(0))]
    # CIC nodes i, i+1 with i = floor(u - 1/2): inside iff lo <= i and i + 1 <= lo + s - 1
    for edge in (f32(lo + 0.5), f32(lo + s - 0.5)):
        vals += [edge, np.nextafter(edge, f32(-1e9)), np.nextafter(edge, f32(1e9))]
    vals = np.array([v for v in vals if 0 <= v < n], np.float32)
    rng = np.random.default_rng(seed)
    return vals[rng.integers(0, len(vals), (60000, 3))]


@pytest.mark.parametrize("periodic,lo,s", [(True, 0, 32), (False, 6, 20), (False, 0, 32)])
def test_deposit_of_edge_positions_is_bitexact(periodic, lo, s):
    from paper_1709_04703_gb300.sim import deposit, pack
    n = 32
    pos = _edge_positions(n, lo, s, 5 + lo)
    p4, _ = pack(pos, np.zeros_like(pos))
    rho, esc = deposit(torch.from_numpy(p4).cuda(), n, lo, s, periodic)
    ref, resc = opm.deposit(pos, n, lo, s, periodic)
    assert esc == resc
    assert periodic or resc > 0
    np.testing.assert_array_equal(rho.cpu().numpy(), ref)


@pytest.mark.parametrize("domain", ["cube", "sphere"])
def test_keep_boundary_is_decided_like_the_oracle(domain):
    """Positions on and one float32 step either side of c +- R per axis
    (cube) or along the axes and diagonals at radius R (sphere)."""
    from paper_1709_04703_gb300.sim import Sim
    n, box, a = 64, 8000.0, 0.7
    R = cz.chi(a, OM, OL) / (box / n) + 1.0
    c = n / 2
    f32 = np.float32
    rng = np.random.default_rng(9)
    base = rng.uniform(c - 0.5 * R, c + 0.5 * R, (4000, 3)).astype(np.float32)
    pts = []
    for sgn in (-1.0, 1.0):
        e = f32(c + sgn * R)
        for v in (e, np.nextafter(e, f32(-1e9)), np.nextafter(e, f32(1e9))):
            for d in range(3):
                q = base[rng.integers(0, len(base), 200)].copy()
                if domain == "sphere":  # on an axis through the centre
                    q[:] = f32(c)
                q[:, d] = v
                pts.append(q)
    if domain == "sphere":
        # points on the diagonal at radius R, rounded to float32, and neighbours
        t = f32(c + R / np.sqrt(3.0))
        for v in (t, np.nextafter(t, f32(-1e9)), np.nextafter(t, f32(1e9))):
            pts.append(np.full((50, 3), v, np.float32))
    pos = np.concatenate([base] + pts).astype(np.float32)
    mom = np.zeros_like(pos)
    ids = np.arange(len(pos), dtype=np.int32)
    sim = Sim(pos, mom, ids, n, box, 0.5, 1.0, 10, domain=domain)
    kept = sim.shrink(a)
    keep = opm.keep_mask(pos, R, n, domain)
    assert 0 < keep.sum() < len(pos)
    assert kept == keep.sum()
    gp, gm, gi = sim.particles()
    np.testing.assert_array_equal(gi, ids[keep])
    np.testing.assert_array_equal(gp, pos[keep])
    ci = sim.lightcone()[2]
    np.testing.assert_array_equal(ci, ids[~keep])
    sim.close()
