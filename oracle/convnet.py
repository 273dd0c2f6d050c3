"""The learned initial guess network in FP64 (oracle; test infrastructure only).

Not in the paper: a small U-shaped 3-D convolutional network that maps the
residual r of a start potential to a correction e ~ A^-1 r, A being the
7-point operator of Sec. 2.1 (Eq. 3 in cell units).  This module is the plain
definition of that network, its losses and its parameter gradient, used to
check the tensor-core kernels.  Pins (tests/test_oracle_convnet.py): the
convolution against a loop-by-loop evaluation of its defining sum and, with
Laplacian weights, against the 7-point operator of oracle/pm.py; pooling and
upsampling against their definitions; the parameter gradient of both losses
and both boundary kinds against central finite differences of the loss.

Layout and parameterisation (shared with the CUDA library by definition,
not by code):
* activations channels-last [B, D, H, W, C], fields [B, z, y, x];
* levels L in 1..4, channels c_l = 8 * 2^l;
* input x = [r * s, 1, 0 x 6] with s = 1 / rms(r) per sample;
* e_0 = relu(conv(x)), e_l = relu(conv(pool(e_{l-1}))); d_{L-1} = e_{L-1},
  d_l = relu(conv(concat(up(d_{l+1}), e_l))); y = conv(d_0) (8 channels,
  linear); guess = y[..., 0] * rms(r) * out_scale;
* parameters, per convolution in the order enc_0..enc_{L-1},
  dec_{L-2}..dec_0, out: weights [cout][27 cin] (column tap * cin + ci, tap =
  (dz+1)*9 + (dy+1)*3 + (dx+1)) then biases [cout];
* convolutions are 3x3x3 "same": zero outside each sample, or periodic.
With quant=True every tensor the kernels store in BF16 (inputs, weights,
activations, gradients of activations) is rounded to BF16 here as well, so
that the comparison with the kernels measures accumulation order only.
"""
import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def bf16(x):
    """Round to the nearest BF16 value (ties to even), via FP32."""
    a = np.ascontiguousarray(np.asarray(x, np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(a.shape)


def layers(L):
    """(cin, cout, relu) of every convolution in parameter order."""
    out = [((8 if l == 0 else 8 << (l - 1)), 8 << l, True) for l in range(L)]
    out += [((8 << (l + 1)) + (8 << l), 8 << l, True) for l in range(L - 2, -1, -1)]
    out.append((8, 8, False))
    return out


def num_params(L):
    return sum(27 * ci * co + co for ci, co, _ in layers(L))


def unpack(params, L):
    """[(W[cout, 27, cin], b[cout])] from the flat parameter vector."""
    out, o = [], 0
    for ci, co, _ in layers(L):
        w = np.asarray(params[o:o + 27 * ci * co], np.float64).reshape(co, 27, ci)
        o += 27 * ci * co
        b = np.asarray(params[o:o + co], np.float64)
        o += co
        out.append((w, b))
    return out


def init_params(L, rng):
    """He-normal weights, zero biases (the output convolution scaled down)."""
    p = []
    for k, (ci, co, relu) in enumerate(layers(L)):
        std = np.sqrt(2.0 / (27 * ci)) * (1.0 if relu else 0.1)
        p.append(rng.standard_normal(27 * ci * co) * std)
        p.append(np.zeros(co))
    return np.concatenate(p)


def shift(x, dz, dy, dx, periodic):
    """out[b, z, y, x] = x[b, z+dz, y+dy, x+dx] (zero outside, or wrapped)."""
    if periodic:
        return np.roll(x, (-dz, -dy, -dx), axis=(1, 2, 3))
    out = np.zeros_like(x)
    D, H, W = x.shape[1:4]

    def sl(d, n):
        return slice(max(0, -d), n - max(0, d)), slice(max(0, d), n - max(0, -d))
    (tz, sz), (ty, sy), (tx, sx) = sl(dz, D), sl(dy, H), sl(dx, W)
    out[:, tz, ty, tx] = x[:, sz, sy, sx]
    return out


def conv(x, w, b, periodic):
    """out[v, o] = b[o] + sum_tap sum_c x[v + tap, c] w[o, tap, c]."""
    out = np.broadcast_to(b, x.shape[:4] + (w.shape[0],)).copy()
    for t, (dz, dy, dx) in enumerate(TAPS):
        out += shift(x, dz, dy, dx, periodic) @ w[:, t, :].T
    return out


def conv_backward(x, w, g, periodic, need_dx=True):
    """(dW, db, dx) of conv for the output gradient g."""
    dw = np.zeros_like(w)
    dx = np.zeros_like(x) if need_dx else None
    for t, (dz, dy, dx_) in enumerate(TAPS):
        xs = shift(x, dz, dy, dx_, periodic)
        dw[:, t, :] = np.einsum('bzyxo,bzyxc->oc', g, xs)
        if need_dx:
            dx += shift(g @ w[:, t, :], -dz, -dy, -dx_, periodic)
    db = g.sum(axis=(0, 1, 2, 3))
    return dw, db, dx


def conv_backward_abs(x, g, periodic):
    """Sums of |terms| of dW and db (sum_v |x(v + tap)| |g(v)| and
    sum_v |g(v)|): the scale of the rounding error of those sums."""
    ax, ag = np.abs(x), np.abs(g)
    dw = np.zeros((g.shape[-1], 27, x.shape[-1]))
    for t, (dz, dy, dx) in enumerate(TAPS):
        dw[:, t, :] = np.einsum('bzyxo,bzyxc->oc', ag, shift(ax, dz, dy, dx, periodic))
    return dw, ag.sum(axis=(0, 1, 2, 3))


def pool2(x):
    B, D, H, W, C = x.shape
    return x.reshape(B, D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4, 6))


def pool2_backward(g):
    return up2(g) / 8.0


def up2(x):
    return x.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)


def up2_backward(g):
    B, D, H, W, C = g.shape
    return g.reshape(B, D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4, 6))


def laplacian(d, periodic):
    """7-point operator sum_nb d - 6 d on fields [B, z, y, x] (zero outside
    each sample, or periodic)."""
    x = d[..., None]
    acc = -6.0 * x
    for e in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
        acc = acc + shift(x, *e, periodic)
    return acc[..., 0]


def rms_scales(r, out_scale):
    """Per-sample s_in = 1/rms(r), s_out = rms(r) out_scale, t_scale = 1/s_out."""
    B = r.shape[0]
    rms = np.sqrt((r.reshape(B, -1) ** 2).mean(axis=1))
    s_in = np.where(rms > 0, 1.0 / np.where(rms > 0, rms, 1.0), 0.0)
    s_out = rms * out_scale
    t_scale = np.where(s_out > 0, 1.0 / np.where(s_out > 0, s_out, 1.0), 0.0)
    return s_in, s_out, t_scale


def forward(params, r, L, periodic, out_scale=1.0, quant=False):
    """Network output y [B, S, S, S, 8] and the intermediate tensors."""
    q = bf16 if quant else (lambda a: a)
    P = unpack(params, L)
    if quant:
        P = [(bf16(w), b) for w, b in P]
    s_in, s_out, t_scale = rms_scales(r, out_scale)
    if quant:
        s_in = np.float32(s_in).astype(np.float64)
    B = r.shape[0]
    x = np.zeros(r.shape + (8,))
    x[..., 0] = q(r * s_in.reshape(B, 1, 1, 1))
    x[..., 1] = 1.0
    c = dict(x=x, P=P, s_out=s_out, t_scale=t_scale)
    k = 0
    e, p = [], [None]
    for l in range(L):
        inp = x if l == 0 else q(pool2(e[-1]))
        if l > 0:
            p.append(inp)
        w, b = P[k]
        k += 1
        e.append(q(np.maximum(conv(inp, w, b, periodic), 0.0)))
    d = [None] * L
    d[L - 1] = e[L - 1]
    cat = [None] * L
    for l in range(L - 2, -1, -1):
        cat[l] = np.concatenate([up2(d[l + 1]), e[l]], axis=-1)
        w, b = P[k]
        k += 1
        d[l] = q(np.maximum(conv(cat[l], w, b, periodic), 0.0))
    w, b = P[k]
    y = conv(d[0], w, b, periodic)
    c.update(e=e, p=p, d=d, cat=cat, y=y)
    return y, c


def guess(params, r, L, periodic, out_scale=1.0, quant=False):
    """The correction field e ~ A^-1 r the network proposes, [B, S, S, S]."""
    y, c = forward(params, r, L, periodic, out_scale, quant)
    return y[..., 0] * c['s_out'].reshape(-1, 1, 1, 1)


def loss_grad(params, r, target, L, periodic, loss_kind, out_scale=1.0, quant=False,
              want_scale=False):
    """Loss and its gradient with respect to the flat parameter vector.
    t = target * t_scale (per sample); loss_kind 0: mean (y0 - t)^2;
    1: mean (A (y0 - t))^2 with A the 7-point operator.  want_scale adds a
    third result: per parameter, the sum of the absolute values of the terms
    its gradient sums (where the terms cancel, the rounding error of the
    gradient is measured against this)."""
    q = bf16 if quant else (lambda a: a)
    y, c = forward(params, r, L, periodic, out_scale, quant)
    B = r.shape[0]
    n = r.size
    dlt = y[..., 0] - target * c['t_scale'].reshape(B, 1, 1, 1)
    gy = np.zeros_like(y)
    if loss_kind == 0:
        loss = float((dlt ** 2).mean())
        gy[..., 0] = q(2.0 * dlt / n)
    else:
        a = laplacian(dlt, periodic)
        loss = float((a ** 2).mean())
        gy[..., 0] = q(2.0 * laplacian(a, periodic) / n)
    P = c['P']
    grads = [None] * len(P)
    scales = [None] * len(P)
    k = len(P) - 1
    w, _ = P[k]
    dw, db, g = conv_backward(c['d'][0], w, gy, periodic)
    grads[k] = (dw, db)
    if want_scale:
        scales[k] = conv_backward_abs(c['d'][0], gy, periodic)
    g = q(g)
    k -= 1
    skip = [None] * L
    for l in range(0, L - 1):
        g = g * (c['d'][l] > 0)
        w, _ = P[k]
        dw, db, gcat = conv_backward(c['cat'][l], w, g, periodic)
        grads[k] = (dw, db)
        if want_scale:
            scales[k] = conv_backward_abs(c['cat'][l], g, periodic)
        k -= 1
        gcat = q(gcat)
        cu = 8 << (l + 1)
        g = q(up2_backward(gcat[..., :cu]))
        skip[l] = gcat[..., cu:]
    for l in range(L - 1, -1, -1):
        if l < L - 1:
            g = q(g + skip[l])
        g = g * (c['e'][l] > 0)
        w, _ = P[k]
        inp = c['x'] if l == 0 else c['p'][l]
        dw, db, gin = conv_backward(inp, w, g, periodic, need_dx=l > 0)
        grads[k] = (dw, db)
        if want_scale:
            scales[k] = conv_backward_abs(inp, g, periodic)
        k -= 1
        if l > 0:
            g = q(pool2_backward(q(gin)))
    flat = np.concatenate([np.concatenate([dw.reshape(-1), db]) for dw, db in grads])
    if want_scale:
        sc = np.concatenate([np.concatenate([dw.reshape(-1), db]) for dw, db in scales])
        return loss, flat, sc
    return loss, flat
