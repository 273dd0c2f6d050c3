"""Learned initial guess of the Poisson solve (not in the paper): Python
front end of the pm_guess_* calls of libpmshrink.  The network, its
forward and backward passes and Adam all run in the library's kernels; this
module marshals arguments only.

Network (levels L, channels 8 * 2^l): 3x3x3 convolutions + ReLU, 2x average
pooling down, nearest 2x upsampling + skip concatenation up, a final linear
convolution; input the residual r of a start potential scaled to unit RMS
(plus a constant domain-mask channel), output a correction e ~ A^-1 r.
Parameters: FP32 masters, per convolution W[cout][27 cin] then b[cout].
"""
import ctypes as C

import numpy as np
import torch

from . import _lib as L


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def init_params(levels, seed=0):
    """He-normal weights, zero biases, the output convolution scaled down."""
    rng = np.random.default_rng(seed)
    out = []
    chans = [((8 if l == 0 else 8 << (l - 1)), 8 << l, True) for l in range(levels)]
    chans += [((8 << (l + 1)) + (8 << l), 8 << l, True) for l in range(levels - 2, -1, -1)]
    chans.append((8, 8, False))
    for ci, co, relu in chans:
        std = np.sqrt(2.0 / (27 * ci)) * (1.0 if relu else 0.1)
        out.append(rng.standard_normal(27 * ci * co) * std)
        out.append(np.zeros(co))
    return np.concatenate(out).astype(np.float32)


class GuessNet:
    """One network instance on its own CUDA stream."""

    def __init__(self, levels=4, params=None, out_scale=1.0, seed=0):
        self._lib = L.load()
        self.levels = int(levels)
        self.stream = torch.cuda.Stream()
        self._g = C.c_void_p()
        code = self._lib.pm_guess_create(self.levels, C.c_void_p(self.stream.cuda_stream),
                                         C.byref(self._g))
        if code != L.PM_OK:
            raise L.PmError(code, "pm_guess_create failed")
        self.n_params = int(self._lib.pm_guess_num_params(self._g))
        self.set_params(init_params(self.levels, seed) if params is None else params, out_scale)

    def _check(self, code):
        if code != L.PM_OK:
            raise L.PmError(code, self._lib.pm_guess_last_error(self._g).decode())

    def close(self):
        if getattr(self, "_g", None):
            self._lib.pm_guess_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params, out_scale=None):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {p.size}")
        if out_scale is not None:
            self.out_scale = float(out_scale)
        torch.cuda.synchronize()
        self._check(self._lib.pm_guess_set_params(self._g, p.ctypes.data,
                                                  C.c_float(self.out_scale)))

    def params(self):
        p = np.zeros(self.n_params, np.float32)
        self._check(self._lib.pm_guess_get_params(self._g, p.ctypes.data, None))
        return p

    def grad(self):
        g = np.zeros(self.n_params, np.float32)
        self._check(self._lib.pm_guess_get_params(self._g, None, g.ctypes.data))
        return g

    @staticmethod
    def _field(t):
        if t.dtype != torch.float32 or not t.is_cuda or t.dim() != 4:
            raise ValueError("fields: CUDA float32 tensors [B, S, S, S]")
        return t.contiguous()

    def forward(self, r, periodic=False):
        """Correction e for residuals r [B, S, S, S] (CUDA float32)."""
        r = self._field(r)
        out = torch.empty_like(r)
        self.stream.wait_stream(torch.cuda.current_stream())
        self._check(self._lib.pm_guess_forward(self._g, _ptr(r), r.shape[0], r.shape[1],
                                               1 if periodic else 0, _ptr(out)))
        return out

    def loss_grad(self, r, target, periodic=False, loss_kind=1):
        """Loss of the network on (r, target) and its parameter gradient
        (kept on the device for adam() / grad())."""
        r, target = self._field(r), self._field(target)
        loss = C.c_double()
        self.stream.wait_stream(torch.cuda.current_stream())
        self._check(self._lib.pm_guess_loss_grad(self._g, _ptr(r), _ptr(target), r.shape[0],
                                                 r.shape[1], 1 if periodic else 0,
                                                 int(loss_kind), C.byref(loss)))
        return loss.value

    def adam(self, lr):
        self._check(self._lib.pm_guess_adam(self._g, C.c_float(lr)))
        torch.cuda.current_stream().wait_stream(self.stream)
