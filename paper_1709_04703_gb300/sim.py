"""Python front end of libpmshrink: torch supplies device memory and the
stream, the C library does the work (see include/pmshrink.h)."""
import ctypes as C

import numpy as np
import torch

from . import _lib as L

_PREC = {"mixed": L.PM_MIXED, "fp32": L.PM_FP32_PLAIN, "fp64": L.PM_FP64_PLAIN,
         "mixed64": L.PM_MIXED_FP64}
_GUESS = {"warm": L.PM_GUESS_WARM, "zero": L.PM_GUESS_ZERO, "learned": L.PM_GUESS_LEARNED}
_BC = {"paper": L.PM_BC_PAPER, "open": L.PM_BC_OPEN, "periodic": L.PM_BC_PERIODIC}
_GRAVITY = {"poisson": L.PM_GRAVITY_POISSON, "diffusion": L.PM_GRAVITY_DIFFUSION,
            "diffusion_ade": L.PM_GRAVITY_DIFFUSION_ADE}
# shrink: True / "on" drops leavers into the lightcone; False / "off" keeps
# everything; "record" keeps everything and records lightcone crossings
_SHRINK = {False: L.PM_SHRINK_OFF, True: L.PM_SHRINK_ON, "off": L.PM_SHRINK_OFF,
           "on": L.PM_SHRINK_ON, "record": L.PM_SHRINK_RECORD}


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class _On:
    """Order work on `stream` after the caller's current stream, and the
    caller's stream after it (device tensors cross between the two)."""

    def __init__(self, stream):
        self.stream = stream

    def __enter__(self):
        self.stream.wait_stream(torch.cuda.current_stream())

    def __exit__(self, *a):
        torch.cuda.current_stream().wait_stream(self.stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def pack(pos, mom, ids=None, extra=None):
    """(N,3) float32 positions/momenta (+ int32 ids) -> two (N,4) float32
    arrays: pos4 = (x, y, z, id bits), mom4 = (px, py, pz, extra)."""
    pos = np.asarray(pos, dtype=np.float32)
    mom = np.asarray(mom, dtype=np.float32)
    n = len(pos)
    p4 = np.zeros((n, 4), np.float32)
    m4 = np.zeros((n, 4), np.float32)
    p4[:, :3] = pos
    m4[:, :3] = mom
    ids = np.arange(n, dtype=np.int32) if ids is None else np.asarray(ids, np.int32)
    p4[:, 3] = ids.view(np.float32)
    if extra is not None:
        m4[:, 3] = extra
    return p4, m4


def unpack(p4, m4):
    p4 = np.asarray(p4, np.float32)
    m4 = np.asarray(m4, np.float32)
    ids = np.ascontiguousarray(p4[:, 3]).view(np.int32).copy()
    return p4[:, :3].copy(), m4[:, :3].copy(), ids, m4[:, 3].copy()


def _config(n_mesh, n_particles, box, a_init, a_final, n_steps, rtol=1e-7, precision="mixed",
            guess="warm", bc="paper", shrink=True, buffer_cells=1.0, max_vcycles=50,
            store_forces=False, omega_m=0.3, omega_l=0.7):
    lib = L.load()
    cfg = L.PmConfig()
    lib.pm_config_default(C.byref(cfg))
    cfg.n_mesh = int(n_mesh)
    cfg.n_particles = int(n_particles)
    cfg.box_mpch = float(box)
    cfg.omega_m, cfg.omega_l = float(omega_m), float(omega_l)
    cfg.a_init, cfg.a_final, cfg.n_steps = float(a_init), float(a_final), int(n_steps)
    cfg.rtol, cfg.max_vcycles = float(rtol), int(max_vcycles)
    cfg.precision = _PREC[precision]
    cfg.guess = _GUESS[guess]
    cfg.bc = _BC[bc]
    cfg.shrink = _SHRINK[shrink]
    cfg.buffer_cells = float(buffer_cells)
    cfg.store_forces = 1 if store_forces else 0
    return cfg


class Batch:
    """Many independent realisations advancing together (pm_batch_*):
    one kernel launch per phase over all of them."""

    def __init__(self, realisations, a_init, a_final, n_steps, rtol=1e-7, max_vcycles=50,
                 buffer_cells=1.0, store_forces=False, inner_vcycles=1):
        """realisations: list of dicts with pos, mom, ids, n_mesh, box."""
        lib = L.load()
        R = len(realisations)
        cfgs = (L.PmConfig * R)()
        self.stream = torch.cuda.Stream()
        self._sp = C.c_void_p(self.stream.cuda_stream)
        self.caps = []
        keep = []
        pp = (C.c_void_p * R)()
        mp = (C.c_void_p * R)()
        for r, re in enumerate(realisations):
            cfgs[r] = _config(re["n_mesh"], len(re["pos"]), re["box"], a_init, a_final,
                              n_steps, rtol=rtol, max_vcycles=max_vcycles,
                              buffer_cells=buffer_cells, store_forces=store_forces)
            cfgs[r].inner_vcycles = int(inner_vcycles)
            p4, m4 = pack(re["pos"], re["mom"], re["ids"])
            dp, dm = torch.from_numpy(p4).cuda(), torch.from_numpy(m4).cuda()
            keep += [dp, dm]
            pp[r] = dp.data_ptr()
            mp[r] = dm.data_ptr()
            self.caps.append(len(re["pos"]))
        self._b = C.c_void_p()
        with _On(self.stream):
            code = lib.pm_batch_init(R, cfgs, pp, mp, 0, self._sp, C.byref(self._b))
        if code != L.PM_OK:
            raise L.PmError(code, lib.pm_batch_last_error(None).decode())
        self._lib = lib
        self.R = R

    def _check(self, code):
        if code != L.PM_OK:
            raise L.PmError(code, self._lib.pm_batch_last_error(self._b).decode())

    def step(self, k=1):
        self._check(self._lib.pm_batch_step(self._b, int(k)))

    def set_solve(self, persistent=True, wait_seconds=2.0, extra_arrivals=0):
        """persistent: one cooperative launch per solve, decided on the
        device (else a V-cycle graph with host decisions); wait_seconds: the
        longest wait at one of its grid barriers; extra_arrivals > 0 only to
        test that limit (every barrier then runs out: PM_ETIMEOUT)."""
        self._check(self._lib.pm_batch_set_solve(self._b, int(bool(persistent)),
                                                 float(wait_seconds), int(extra_arrivals)))

    def stats(self, r):
        s = L.PmStats()
        self._check(self._lib.pm_batch_stats(self._b, int(r), C.byref(s)))
        return {f: getattr(s, f) for f, _ in L.PmStats._fields_}

    def particles(self, r):
        n = C.c_int64()
        cap = self.caps[r]
        p4 = np.zeros((cap, 4), np.float32)
        m4 = np.zeros((cap, 4), np.float32)
        self._check(self._lib.pm_batch_get_particles(self._b, int(r), p4.ctypes.data,
                                                     m4.ctypes.data, 1, C.byref(n)))
        pos, mom, ids, _ = unpack(p4[:n.value], m4[:n.value])
        return pos, mom, ids

    def forces(self, r):
        """grad(Phi) at realisation r's particles in its last step, (N, 3)."""
        n = C.c_int64()
        f4 = np.zeros((self.caps[r], 4), np.float32)
        self._check(self._lib.pm_batch_get_forces(self._b, int(r), f4.ctypes.data, 1,
                                                  C.byref(n)))
        return f4[:n.value, :3].copy()

    def lightcone(self, r):
        n = C.c_int64()
        cap = self.caps[r]
        p4 = np.zeros((cap, 4), np.float32)
        m4 = np.zeros((cap, 4), np.float32)
        self._check(self._lib.pm_batch_get_lightcone(self._b, int(r), p4.ctypes.data,
                                                     m4.ctypes.data, 1, C.byref(n)))
        return unpack(p4[:n.value], m4[:n.value])

    def close(self):
        if getattr(self, "_b", None):
            self._lib.pm_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Sim:
    """One shrinking-domain PM run (one context of the C library)."""

    def __init__(self, pos, mom, ids, n_mesh, box, a_init, a_final, n_steps,
                 rtol=1e-7, precision="mixed", guess="warm", bc="paper",
                 shrink=True, buffer_cells=1.0, max_vcycles=50, store_forces=False,
                 omega_m=0.3, omega_l=0.7, host_init=False, gravity="poisson",
                 c_eff_factor=0.019, assignment="cic", domain="cube", sort_every=0,
                 inner_vcycles=1):
        lib = L.load()
        cfg = L.PmConfig()
        lib.pm_config_default(C.byref(cfg))
        cfg.n_mesh = int(n_mesh)
        cfg.n_particles = int(len(pos))
        cfg.box_mpch = float(box)
        cfg.omega_m, cfg.omega_l = float(omega_m), float(omega_l)
        cfg.a_init, cfg.a_final, cfg.n_steps = float(a_init), float(a_final), int(n_steps)
        cfg.rtol, cfg.max_vcycles = float(rtol), int(max_vcycles)
        cfg.precision = _PREC[precision]
        cfg.guess = _GUESS[guess]
        cfg.bc = _BC[bc]
        cfg.shrink = _SHRINK[shrink]
        cfg.buffer_cells = float(buffer_cells)
        cfg.store_forces = 1 if store_forces else 0
        cfg.gravity = _GRAVITY[gravity]
        cfg.c_eff_factor = float(c_eff_factor)
        cfg.assignment = {"cic": L.PM_ASSIGN_CIC, "tsc": L.PM_ASSIGN_TSC}[assignment]
        cfg.domain = {"cube": L.PM_DOMAIN_CUBE, "sphere": L.PM_DOMAIN_SPHERE,
                      "ball": L.PM_DOMAIN_BALL}[domain]
        cfg.sort_every = int(sort_every)
        cfg.inner_vcycles = int(inner_vcycles)
        self.cfg = cfg
        self.n_particles = int(len(pos))
        # the context runs on its own stream so that its V-cycle can be
        # captured as a CUDA graph
        self.stream = torch.cuda.Stream()
        self._sp = C.c_void_p(self.stream.cuda_stream)
        p4, m4 = pack(pos, mom, ids)
        self._ctx = C.c_void_p()
        with _On(self.stream):
            if host_init:
                code = lib.pm_init(C.byref(cfg), p4.ctypes.data, m4.ctypes.data, 1,
                                   self._sp, C.byref(self._ctx))
            else:
                dp = torch.from_numpy(p4).cuda()
                dm = torch.from_numpy(m4).cuda()
                code = lib.pm_init(C.byref(cfg), _ptr(dp), _ptr(dm), 0, self._sp,
                                   C.byref(self._ctx))
        L.check(code, None)
        self._lib = lib

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.pm_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, code):
        L.check(code, self._ctx)

    # -- stepping ----------------------------------------------------------
    def step(self, k=1):
        self._check(self._lib.pm_step(self._ctx, int(k)))

    def shrink(self, a):
        n = C.c_int64()
        self._check(self._lib.pm_shrink(self._ctx, float(a), C.byref(n)))
        return n.value

    def stats(self):
        s = L.PmStats()
        self._check(self._lib.pm_stats(self._ctx, C.byref(s)))
        return {f: getattr(s, f) for f, _ in L.PmStats._fields_}

    def smoother_tiles(self):
        """The fused smoother's launch shape per level side, as pm_init
        picked it: {side: (tile height, planes per CTA)}."""
        cnt = C.c_int32(0)
        self._check(self._lib.pm_smoother_tiles(self._ctx, None, None, None, 0, C.byref(cnt)))
        m = cnt.value
        sides, ty, zc = (C.c_int32 * max(m, 1))(), (C.c_int32 * max(m, 1))(), \
            (C.c_int32 * max(m, 1))()
        self._check(self._lib.pm_smoother_tiles(self._ctx, sides, ty, zc, m, C.byref(cnt)))
        return {sides[i]: (ty[i], zc[i]) for i in range(m)}

    def save(self, path):
        """Checkpoint the run at the current step boundary (pm_save)."""
        self._check(self._lib.pm_save(self._ctx, str(path).encode()))

    def load(self, path):
        """Resume from a checkpoint of a run with the same configuration."""
        self._check(self._lib.pm_load(self._ctx, str(path).encode()))

    def schedule(self):
        m = self.cfg.n_steps + 1
        out = {k: np.zeros(m) for k in ("a", "dtau", "a_half", "chi")}
        self._check(self._lib.pm_schedule(self._ctx, *[out[k].ctypes.data for k in
                                                       ("a", "dtau", "a_half", "chi")]))
        return out

    # -- state -------------------------------------------------------------
    def particles(self):
        """(pos, mom, ids) of the active particles as numpy arrays."""
        n = C.c_int64()
        cap = self.n_particles
        p4 = np.zeros((cap, 4), np.float32)
        m4 = np.zeros((cap, 4), np.float32)
        self._check(self._lib.pm_get_particles(self._ctx, p4.ctypes.data, m4.ctypes.data, 1,
                                               C.byref(n)))
        pos, mom, ids, _ = unpack(p4[:n.value], m4[:n.value])
        return pos, mom, ids

    def particles_device(self, pos4, mom4):
        """Copy active particles into device float4 tensors (N_cap, 4)."""
        n = C.c_int64()
        with _On(self.stream):
            self._check(self._lib.pm_get_particles(self._ctx, _ptr(pos4), _ptr(mom4), 0,
                                                   C.byref(n)))
        return n.value

    def set_particles(self, pos4, mom4, n, host=False):
        if host:
            self._check(self._lib.pm_set_particles(self._ctx, C.c_void_p(pos4.ctypes.data),
                                                   C.c_void_p(mom4.ctypes.data), int(n), 1))
        else:
            with _On(self.stream):
                self._check(self._lib.pm_set_particles(self._ctx, _ptr(pos4), _ptr(mom4),
                                                       int(n), 0))

    def get_particles_host(self, pos4, mom4):
        """Copy active particles into caller-owned host float4 buffers."""
        n = C.c_int64()
        self._check(self._lib.pm_get_particles(
            self._ctx, C.c_void_p(pos4.data_ptr() if torch.is_tensor(pos4) else pos4.ctypes.data),
            C.c_void_p(mom4.data_ptr() if torch.is_tensor(mom4) else mom4.ctypes.data), 1,
            C.byref(n)))
        return n.value

    def lightcone(self):
        """(pos, mom, ids, a_cross) of the lightcone records."""
        n = C.c_int64()
        cap = self.n_particles
        p4 = np.zeros((cap, 4), np.float32)
        m4 = np.zeros((cap, 4), np.float32)
        self._check(self._lib.pm_get_lightcone(self._ctx, p4.ctypes.data, m4.ctypes.data, 1,
                                               C.byref(n)))
        return unpack(p4[:n.value], m4[:n.value])

    def forces(self):
        n = C.c_int64()
        f4 = np.zeros((self.n_particles, 4), np.float32)
        self._check(self._lib.pm_get_forces(self._ctx, f4.ctypes.data, 1, C.byref(n)))
        return f4[:n.value, :3].copy()

    def potential(self):
        """(phi (side+2)^3 float64 incl. ghost layer, lo, side) of the last solve."""
        n = self.cfg.n_mesh
        buf = np.zeros((n + 2) ** 3)
        lo, side = C.c_int32(), C.c_int32()
        self._check(self._lib.pm_get_potential(self._ctx, buf.ctypes.data, C.byref(lo),
                                               C.byref(side)))
        s = side.value
        return buf[:(s + 2) ** 3].reshape(s + 2, s + 2, s + 2), lo.value, s

    def solve_potential(self, delta, a, bc="open", want64=True):
        """Solve sum_nb(Phi) - 6 Phi = S(a) delta on the whole mesh.
        delta: (n,n,n) float64 (numpy or cuda tensor).  Returns
        (phi32 cuda tensor, phi64 cuda tensor or None, vcycles, resid)."""
        n = self.cfg.n_mesh
        d = delta if torch.is_tensor(delta) else torch.from_numpy(np.ascontiguousarray(delta))
        d = d.to(device="cuda", dtype=torch.float64).contiguous()
        phi = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
        phi64 = torch.empty((n, n, n), dtype=torch.float64, device="cuda") if want64 else None
        vc, res = C.c_int32(), C.c_double()
        with _On(self.stream):
            self._check(self._lib.pm_potential(self._ctx, _ptr(d), float(a), _BC[bc],
                                               _ptr(phi), _ptr(phi64), C.byref(vc),
                                               C.byref(res)))
        return phi, phi64, vc.value, res.value

    # -- learned initial guess ---------------------------------------------
    def set_guess(self, net):
        """Attach a GuessNet (or None) for guess="learned"."""
        self._net = net
        self._check(self._lib.pm_set_guess(self._ctx, net._g if net is not None else None))

    def capture(self, r, e):
        """Arm (device float32 tensors of n_mesh^3 elements) or disarm (None,
        None) the capture of (residual of the start, correction) pairs."""
        if r is not None:
            n3 = self.cfg.n_mesh ** 3
            for t in (r, e):
                if t.dtype != torch.float32 or not t.is_cuda or t.numel() < n3:
                    raise ValueError("capture buffers: CUDA float32 of n_mesh^3 elements")
        self._cap = (r, e)
        torch.cuda.synchronize()
        self._check(self._lib.pm_capture(self._ctx, _ptr(r), _ptr(e)))

    def profile(self, enable=True):
        self._check(self._lib.pm_profile(self._ctx, 1 if enable else 0))

    def profile_read(self):
        """{class: {"ms", "groups", "bytes"}} of the per-kernel-class timers."""
        out = {}
        for c, name in enumerate(L.PROF_CLASSES):
            t, g, b = C.c_double(), C.c_int64(), C.c_double()
            self._check(self._lib.pm_profile_read(self._ctx, c, C.byref(t), C.byref(g),
                                                  C.byref(b)))
            out[name] = {"ms": t.value, "groups": g.value, "bytes": b.value}
        return out


def sort_particles(pos4_dev, mom4_dev, n_mesh):
    """(pos4, mom4) reordered by the mesh cell of the CIC base node (stable);
    mom4_dev may be None."""
    import torch
    lib = L.load()
    n = pos4_dev.shape[0]
    po = torch.empty_like(pos4_dev)
    mo = torch.empty_like(mom4_dev) if mom4_dev is not None else None
    code = lib.pm_sort_particles(_ptr(pos4_dev), _ptr(mom4_dev), n, int(n_mesh), _ptr(po),
                                 _ptr(mo), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    L.check(code, None)
    return po, mo


def power_spectrum(pos4_dev, box, n_mesh, n_bins, subtract_shot=True):
    """P(k) of device float4 particles (positions in cells of n_mesh)."""
    lib = L.load()
    k = np.zeros(n_bins)
    p = np.zeros(n_bins)
    m = np.zeros(n_bins)
    L.check(lib.pm_power_spectrum(_ptr(pos4_dev), int(pos4_dev.shape[0]), float(box),
                                  int(n_mesh), int(n_bins), 1 if subtract_shot else 0,
                                  k.ctypes.data, p.ctypes.data, m.ctypes.data, _stream()))
    return k, p, m


def deposit(pos4_dev, n_mesh, lo=0, side=None, periodic=True, mom4_dev=None,
            drift_coef=0.0, rho=None, assignment="cic"):
    """Fixed-point CIC (or TSC) deposit; returns (rho int64 cuda tensor
    [z,y,x], escaped).  With mom4_dev the positions are drifted in place first."""
    lib = L.load()
    side = n_mesh if side is None else side
    if rho is None:
        rho = torch.zeros((n_mesh, n_mesh, n_mesh), dtype=torch.int64, device="cuda")
    esc = C.c_int64()
    fn = lib.pm_deposit_tsc if assignment == "tsc" else lib.pm_deposit
    L.check(fn(_ptr(pos4_dev), _ptr(mom4_dev), int(pos4_dev.shape[0]),
                           float(drift_coef), int(n_mesh), int(lo), int(side),
                           1 if periodic else 0, _ptr(rho), C.byref(esc), _stream()))
    return rho, esc.value


def power_spectrum_jing(pos4_dev, box, n_mesh, n_bins, subtract_shot=True, alias_range=3,
                        max_iter=30, tol=1e-6):
    """P(k) with the full alias correction (pm_power_spectrum_jing):
    (k, P, modes, slopes, passes)."""
    lib = L.load()
    k = np.zeros(n_bins)
    p = np.zeros(n_bins)
    m = np.zeros(n_bins)
    nu = np.zeros(n_bins)
    passes = C.c_int32()
    L.check(lib.pm_power_spectrum_jing(_ptr(pos4_dev), int(pos4_dev.shape[0]), float(box),
                                       int(n_mesh), int(n_bins), 1 if subtract_shot else 0,
                                       int(alias_range), int(max_iter), float(tol),
                                       k.ctypes.data, p.ctypes.data, m.ctypes.data,
                                       nu.ctypes.data, C.byref(passes), _stream()))
    return k, p, m, nu, passes.value
