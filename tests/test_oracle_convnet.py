"""Pins of the FP64 network oracle (oracle/convnet.py) against definitions
that do not go through its own code paths: loop-by-loop sums, the 7-point
operator of oracle/pm.py (Eq. 3 in cell units), adjoint identities, and
central finite differences of the loss."""
import numpy as np
import pytest

from oracle import convnet as cn
from oracle import pm


def _conv_loops(x, w, b, periodic):
    B, D, H, W, C = x.shape
    O = w.shape[0]
    out = np.zeros((B, D, H, W, O))
    for bb in range(B):
        for z in range(D):
            for y in range(H):
                for xx in range(W):
                    for o in range(O):
                        acc = b[o]
                        for t, (dz, dy, dx) in enumerate(cn.TAPS):
                            zz, yy, x2 = z + dz, y + dy, xx + dx
                            if periodic:
                                zz, yy, x2 = zz % D, yy % H, x2 % W
                            elif not (0 <= zz < D and 0 <= yy < H and 0 <= x2 < W):
                                continue
                            for c in range(C):
                                acc += x[bb, zz, yy, x2, c] * w[o, t, c]
                        out[bb, z, y, xx, o] = acc
    return out


@pytest.mark.parametrize("periodic", [False, True])
def test_conv_matches_loop_definition(periodic):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 2, 4, 2))
    w = rng.standard_normal((3, 27, 2))
    b = rng.standard_normal(3)
    np.testing.assert_allclose(cn.conv(x, w, b, periodic), _conv_loops(x, w, b, periodic),
                               rtol=1e-12, atol=1e-12)


def test_tap_order():
    """Tap t reads the neighbour at (dz, dy, dx) = (t//9 - 1, (t//3)%3 - 1, t%3 - 1)."""
    x = np.zeros((1, 3, 3, 3, 1))
    x[0, 2, 1, 0, 0] = 1.0             # z = 2, y = 1, x = 0
    w = np.zeros((1, 27, 1))
    w[0, 2 * 9 + 1 * 3 + 0, 0] = 1.0   # dz = +1, dy = 0, dx = -1
    out = cn.conv(x, w, np.zeros(1), False)
    assert out[0, 1, 1, 1, 0] == 1.0 and np.count_nonzero(out) == 1


@pytest.mark.parametrize("periodic", [False, True])
def test_laplacian_weights_reproduce_the_7_point_operator(periodic):
    rng = np.random.default_rng(2)
    f = rng.standard_normal((5, 6, 7)) if not periodic else rng.standard_normal((6, 6, 6))
    w = np.zeros((1, 27, 1))
    for t, (dz, dy, dx) in enumerate(cn.TAPS):
        m = abs(dz) + abs(dy) + abs(dx)
        w[0, t, 0] = -6.0 if m == 0 else (1.0 if m == 1 else 0.0)
    got = cn.conv(f[None, ..., None], w, np.zeros(1), periodic)[0, ..., 0]
    ref = (pm.apply_laplacian_periodic(f) if periodic
           else pm.apply_laplacian_padded(np.pad(f, 1)))
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)
    np.testing.assert_allclose(cn.laplacian(f[None], periodic)[0], ref, rtol=0, atol=1e-12)


def test_pool_and_upsample_definitions():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 4, 6, 2, 3))
    p = cn.pool2(x)
    assert p.shape == (2, 2, 3, 1, 3)
    assert np.isclose(p[1, 1, 2, 0, 2], x[1, 2:4, 4:6, 0:2, 2].mean())
    u = cn.up2(p)
    assert u.shape == x.shape and u[1, 3, 5, 1, 2] == p[1, 1, 2, 0, 2]
    np.testing.assert_allclose(cn.pool2(cn.up2(p)), p, rtol=1e-15)
    # adjoints: <up2 a, b> = <a, up2_backward b>, <pool2 a, b> = <a, pool2_backward b>
    b = rng.standard_normal(x.shape)
    assert np.isclose((u * b).sum(), (p * cn.up2_backward(b)).sum())
    c = rng.standard_normal(p.shape)
    assert np.isclose((p * c).sum(), (x * cn.pool2_backward(c)).sum())


def test_bf16_rounding():
    v = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -2.5, 3.0e38, 1e-40])
    got = cn.bf16(v)
    assert got[0] == 1.0
    assert got[1] == 1.0                   # tie to even
    assert got[2] == 1 + 2.0 ** -6         # tie to even (upwards)
    assert got[3] == -2.5
    assert np.isfinite(got[4])
    # BF16 subnormals are multiples of 2^-133: nearest one
    assert abs(got[5] - 1e-40) <= 2.0 ** -134 and (got[5] / 2.0 ** -133) % 1 == 0


def test_guess_is_homogeneous():
    """The network sees r / rms(r) and rescales: guess(c r) = c guess(r)."""
    rng = np.random.default_rng(4)
    L = 2
    p = cn.init_params(L, rng)
    r = rng.standard_normal((1, 4, 4, 4))
    g1 = cn.guess(p, r, L, False, out_scale=0.3)
    g2 = cn.guess(p, 7.0 * r, L, False, out_scale=0.3)
    np.testing.assert_allclose(g2, 7.0 * g1, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("L,S,B,periodic,kind", [
    (1, 4, 2, False, 0), (2, 4, 2, False, 0), (2, 4, 2, True, 1), (2, 4, 1, False, 1),
    (3, 8, 1, True, 0), (3, 8, 1, False, 1)])
def test_gradient_matches_finite_differences(L, S, B, periodic, kind):
    rng = np.random.default_rng(10 + L + 2 * S + kind)
    p = cn.init_params(L, rng)
    p += 0.05 * rng.standard_normal(p.size)      # nonzero biases, too
    r = rng.standard_normal((B, S, S, S))
    t = rng.standard_normal((B, S, S, S))
    loss, g = cn.loss_grad(p, r, t, L, periodic, kind, out_scale=0.5)
    assert g.shape == (cn.num_params(L),)
    # coordinates from every convolution, weights and biases
    idx, o = [], 0
    for ci, co, _ in cn.layers(L):
        nw = 27 * ci * co
        idx += list(o + rng.choice(nw, 3, replace=False)) + [o + nw + rng.integers(co)]
        o += nw + co
    h = 1e-6
    for i in idx:
        pp, pm_ = p.copy(), p.copy()
        pp[i] += h
        pm_[i] -= h
        fd = (cn.loss_grad(pp, r, t, L, periodic, kind, 0.5)[0]
              - cn.loss_grad(pm_, r, t, L, periodic, kind, 0.5)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-7 * abs(loss), (i, fd, g[i])


def test_quantised_forward_stays_close():
    """BF16 storage changes the output by about the BF16 unit roundoff."""
    rng = np.random.default_rng(5)
    L = 2
    p = cn.init_params(L, rng)
    r = rng.standard_normal((1, 8, 8, 8))
    a = cn.guess(p, r, L, False)
    b = cn.guess(p, r, L, False, quant=True)
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 3e-2
