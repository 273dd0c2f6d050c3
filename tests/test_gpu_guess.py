"""Learned initial guess on the GPU: the tensor-core forward and backward
passes against the FP64 network oracle (with the same BF16 roundings), Adam,
training progress, and the solver with the network attached."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import convnet as cn  # noqa: E402
from paper_1709_04703_gb300 import ics  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_04703_gb300 import build
    build.build()


def _net(L, params, out_scale):
    from paper_1709_04703_gb300.guess import GuessNet
    return GuessNet(L, params=params, out_scale=out_scale)


def _inputs(L, S, B, seed, periodic=False):
    rng = np.random.default_rng(seed)
    p = cn.init_params(L, rng).astype(np.float32)
    p += (0.02 * rng.standard_normal(p.size)).astype(np.float32)
    # a smooth-plus-noise source, like a residual field
    r = rng.standard_normal((B, S, S, S))
    r += 0.5 * np.roll(r, 1, axis=1) + 0.5 * np.roll(r, 1, axis=3)
    r = r.astype(np.float32)
    # targets correlated with the input, as potentials are with sources: the
    # output of another network.  (With targets independent of the input
    # the loss gradient is a small residue of cancelling terms and moves by
    # tens of percent under BF16 storage alone.)
    teacher = cn.init_params(L, np.random.default_rng(seed + 1000))
    t = cn.guess(teacher, r.astype(np.float64), L, periodic, 0.5)
    return p, r, t.astype(np.float32)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# shapes: several 128-voxel tiles with ragged tails (20^3 = 62.5 tiles,
# 10^3 = 7.8), the deepest network, both boundary kinds
CASES = [(2, 8, 2, False), (3, 20, 1, False), (3, 20, 1, True), (4, 16, 1, True),
         (4, 24, 2, False)]


@pytest.mark.parametrize("L,S,B,periodic", CASES)
def test_forward_matches_oracle(L, S, B, periodic):
    p, r, _ = _inputs(L, S, B, 100 + S, periodic)
    net = _net(L, p, 0.5)
    got = net.forward(torch.from_numpy(r).cuda(), periodic).cpu().numpy().astype(np.float64)
    ref = cn.guess(p.astype(np.float64), r.astype(np.float64), L, periodic, 0.5, quant=True)
    # BF16 storage on both sides; FP32 vs FP64 accumulation flips a few
    # BF16 roundings (2^-9 relative each)
    assert _rel(got, ref) < 1e-2
    np.testing.assert_allclose(got, ref, rtol=0, atol=3e-2 * np.abs(ref).max())
    net.close()


@pytest.mark.parametrize("L,S,B,periodic", CASES)
@pytest.mark.parametrize("kind", [0, 1])
def test_loss_and_gradient_match_oracle(L, S, B, periodic, kind):
    p, r, t = _inputs(L, S, B, 200 + S + kind, periodic)
    net = _net(L, p, 0.5)
    loss = net.loss_grad(torch.from_numpy(r).cuda(), torch.from_numpy(t).cuda(), periodic,
                         kind)
    g = net.grad().astype(np.float64)
    args = (p.astype(np.float64), r.astype(np.float64), t.astype(np.float64), L, periodic,
            kind, 0.5)
    rl, rg, sc = cn.loss_grad(*args, quant=True, want_scale=True)
    _, rg64 = cn.loss_grad(*args)
    assert abs(loss - rl) <= 1e-2 * abs(rl)
    o = 0
    for ci, co, _ in cn.layers(L):
        nw = 27 * ci * co
        for a, b in ((slice(o, o + nw), "w"), (slice(o + nw, o + nw + co), "b")):
            # against the oracle with the same BF16 storage: relative to the
            # gradient or, where its terms cancel (the output bias under the
            # periodic residual loss sums a Laplacian: zero), to the sum of
            # the terms' magnitudes
            err = np.linalg.norm(g[a] - rg[a])
            assert err < 1.5e-2 * np.linalg.norm(rg[a]) or err < 1e-2 * np.linalg.norm(sc[a]), \
                (ci, co, b, _rel(g[a], rg[a]), err / np.linalg.norm(sc[a]))
            # and against the FP64 network: the whole effect of BF16 storage
            err64 = np.linalg.norm(g[a] - rg64[a])
            assert err64 < 8e-2 * np.linalg.norm(rg64[a]) or err64 < 1e-2 * np.linalg.norm(sc[a])
        o += nw + co
    net.close()


def test_adam_step_matches_definition():
    L, S = 2, 8
    p, r, t = _inputs(L, S, 1, 7)
    net = _net(L, p, 1.0)
    net.loss_grad(torch.from_numpy(r).cuda(), torch.from_numpy(t).cuda(), False, 1)
    g = net.grad().astype(np.float64)
    lr = 1e-3
    net.adam(lr)
    got = net.params().astype(np.float64)
    # first Adam step: m = (1-b1) g, v = (1-b2) g^2, bias corrections 1-b1, 1-b2
    m = 0.1 * g / 0.1
    v = 0.001 * g * g / 0.001
    ref = p.astype(np.float64) - lr * m / (np.sqrt(v) + 1e-8)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-6)
    net.close()


def test_training_reduces_the_residual_loss():
    L, S = 3, 16
    p, r, _ = _inputs(L, S, 2, 11)
    # target: the exact correction A^-1 r (periodic, zero mean)
    k = np.fft.fftfreq(S) * 2 * np.pi
    lam = sum(np.meshgrid(*(2 * np.cos(k) - 2,) * 3, indexing="ij"))
    lam[0, 0, 0] = 1.0
    rr = r - r.mean(axis=(1, 2, 3), keepdims=True)
    t = np.real(np.fft.ifftn(np.fft.fftn(rr, axes=(1, 2, 3)) / lam, axes=(1, 2, 3)))
    rd = torch.from_numpy(rr.astype(np.float32)).cuda()
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    net = _net(L, p, 1.0)
    first = net.loss_grad(rd, td, True, 1)
    for _ in range(60):
        net.loss_grad(rd, td, True, 1)
        net.adam(2e-3)
    last = net.loss_grad(rd, td, True, 1)
    assert last < 0.5 * first, (first, last)
    net.close()


def _sim(n, box, a0, steps, guess, seed=5, rtol=1e-7):
    from paper_1709_04703_gb300.sim import Sim
    pos, mom, ids = ics.zeldovich(n, -1.5, 0.5, seed, a0)
    return Sim(pos, mom, ids, n, box, a0, 1.0, steps, rtol=rtol, guess=guess)


def test_solver_with_network_reaches_the_same_solution():
    """The network only changes the start: every solve still iterates to
    rtol, and the run agrees with the warm-start run."""
    n, box, a0, steps = 32, 4000.0, 0.3, 6
    warm = _sim(n, box, a0, steps, "warm")
    warm.step(steps)
    pw, mw, iw = warm.particles()
    sw = warm.stats()
    learned = _sim(n, box, a0, steps, "learned")
    net = _net(4, cn.init_params(4, np.random.default_rng(3)).astype(np.float32), 0.05)
    learned.set_guess(net)
    for _ in range(steps):
        learned.step(1)
        st = learned.stats()
        assert st["resid_last"] <= 1e-7
        fits = st["cube_side"] >= 16 and st["cube_side"] % 8 == 0
        assert st["guess_used_last"] == int(fits)
    pl, ml, il = learned.particles()
    assert learned.stats()["n_active"] == sw["n_active"]
    np.testing.assert_array_equal(il, iw)
    np.testing.assert_allclose(pl, pw, rtol=0, atol=1e-3)
    np.testing.assert_allclose(ml, mw, rtol=1e-3, atol=1e-3 * np.abs(mw).max())
    assert learned.stats()["guess_used_total"] >= 1
    learned.close()
    warm.close()
    net.close()


def test_learned_mode_needs_a_network():
    from paper_1709_04703_gb300 import _lib as L
    sim = _sim(16, 1000.0, 0.5, 2, "learned")
    with pytest.raises(L.PmError):
        sim.step(1)
    sim.close()


@pytest.mark.parametrize("a0,periodic", [(0.05, True), (0.75, False)])
def test_captured_pairs_solve_the_correction_equation(a0, periodic):
    """Captured (r, e): r is the residual of the start, e the correction the
    solve added, so A e = r - r_final with |r_final| <= rtol |f|."""
    n = 64
    sim = _sim(n, 3000.0, a0, 8, "warm")
    r = torch.zeros(n ** 3, device="cuda")
    e = torch.zeros(n ** 3, device="cuda")
    sim.capture(r, e)
    for _ in range(2):
        sim.step(1)
    st = sim.stats()
    s = st["cube_side"]
    assert bool(st["periodic"]) == periodic
    rr = r[:s ** 3].cpu().numpy().astype(np.float64).reshape(1, s, s, s)
    ee = e[:s ** 3].cpu().numpy().astype(np.float64).reshape(1, s, s, s)
    assert np.linalg.norm(rr) > 0
    resid = cn.laplacian(ee, periodic) - rr
    assert np.linalg.norm(resid) <= 1e-3 * np.linalg.norm(rr)
    sim.capture(None, None)
    sim.close()


def test_trained_network_shrinks_the_start_residual():
    """What the trained network gains over the method without it: on the
    128^3 workload (not trained on), its correction shrinks the residual of
    the warm start several-fold, and the solves need no more V-cycles."""
    from paper_1709_04703_gb300 import train_guess as tg
    cfg = dict(ics.WORKLOADS["pm128"])
    steps = 30
    warm = tg.evaluate(cfg, None, guess="warm", steps=steps)
    net = tg.load(tg.DEFAULT_WEIGHTS)
    lrn = tg.evaluate(cfg, net, guess="learned", steps=steps)
    net.close()
    assert lrn["guess_used"] == steps            # 128 is a multiple of 8
    ratio = np.array(lrn["resid_guess"]) / np.array(lrn["resid_start"])
    assert np.median(ratio) < 0.5, ratio
    assert lrn["vcycles_total"] <= warm["vcycles_total"]
    assert max(lrn["resid_start"][1:]) < 1.0     # warm starts in both runs
