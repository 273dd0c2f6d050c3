"""ctypes binding of libpmshrink.so (argument marshalling only).

Every function here forwards to the C ABI declared in include/pmshrink.h;
all arithmetic of the PM step runs in the library's CUDA kernels.  Loading
fails loudly when the library has not been built: there is no CPU fallback.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpmshrink.so")

PM_OK, PM_EINVAL, PM_ENOMEM, PM_ECUDA, PM_ENOCONV, PM_EOVERFLOW, PM_ETIMEOUT, PM_EIO = range(8)
PM_MIXED, PM_FP32_PLAIN, PM_FP64_PLAIN, PM_MIXED_FP64 = 0, 1, 2, 3
PM_GUESS_WARM, PM_GUESS_ZERO, PM_GUESS_LEARNED = 0, 1, 2
PM_GRAVITY_POISSON, PM_GRAVITY_DIFFUSION, PM_GRAVITY_DIFFUSION_ADE = 0, 1, 2
PM_BC_PAPER, PM_BC_OPEN, PM_BC_PERIODIC = 0, 1, 2
PM_SHRINK_OFF, PM_SHRINK_ON, PM_SHRINK_RECORD = 0, 1, 2
PM_ASSIGN_CIC, PM_ASSIGN_TSC = 0, 1
PM_DOMAIN_CUBE, PM_DOMAIN_SPHERE, PM_DOMAIN_BALL = 0, 1, 2
PM_SHRINK_STATIC_MAX_PARTICLES = 1 << 22
PM_MG_OMEGA = 1.25  # the multigrid smoother's SOR factor (include/pmshrink.h)

STATUS_NAMES = {0: "PM_OK", 1: "PM_EINVAL", 2: "PM_ENOMEM", 3: "PM_ECUDA",
                4: "PM_ENOCONV", 5: "PM_EOVERFLOW", 6: "PM_ETIMEOUT", 7: "PM_EIO"}

# every entry point declared in include/pmshrink.h
EXPORTED = [
    "pm_config_default", "pm_init", "pm_step", "pm_shrink", "pm_potential",
    "pm_power_spectrum", "pm_power_spectrum_jing", "pm_deposit", "pm_deposit_tsc", "pm_sort_particles", "pm_stats", "pm_schedule", "pm_save", "pm_load",
    "pm_get_particles", "pm_set_particles", "pm_get_lightcone", "pm_get_forces",
    "pm_get_potential", "pm_profile", "pm_profile_read", "pm_launch_count", "pm_last_error",
    "pm_destroy", "pm_shrink_static", "pm_shrink_static_error",
    "pm_batch_init", "pm_batch_step", "pm_batch_stats", "pm_batch_get_particles",
    "pm_batch_get_lightcone", "pm_batch_get_forces", "pm_batch_set_solve",
    "pm_batch_last_error", "pm_batch_destroy",
    "pm_mg_smooth", "pm_mg_restrict", "pm_mg_prolong", "pm_selftest_wait", "pm_nn_gemm_bf16", "pm_guess_create", "pm_guess_num_params", "pm_guess_set_params",
    "pm_guess_get_params", "pm_guess_forward", "pm_guess_loss_grad", "pm_guess_adam",
    "pm_guess_last_error", "pm_guess_destroy", "pm_set_guess", "pm_capture",
    "pm_mg_cluster_size", "pm_smoother_tiles",
]
PROF_CLASSES = ["deposit", "source", "boundary", "smooth0", "transfer0", "coarse",
                "defect", "correct", "gather", "compact", "guess", "ade", "sort"]


class PmConfig(C.Structure):
    _fields_ = [
        ("n_mesh", C.c_int32), ("n_particles", C.c_int64), ("box_mpch", C.c_double),
        ("omega_m", C.c_double), ("omega_l", C.c_double), ("a_init", C.c_double),
        ("a_final", C.c_double), ("n_steps", C.c_int32), ("rtol", C.c_double),
        ("max_vcycles", C.c_int32), ("precision", C.c_int32), ("guess", C.c_int32),
        ("bc", C.c_int32), ("shrink", C.c_int32), ("buffer_cells", C.c_double),
        ("store_forces", C.c_int32), ("gravity", C.c_int32), ("c_eff_factor", C.c_double),
        ("assignment", C.c_int32), ("domain", C.c_int32), ("sort_every", C.c_int32),
        ("inner_vcycles", C.c_int32),
    ]


class PmStats(C.Structure):
    _fields_ = [
        ("step", C.c_int32), ("a", C.c_double), ("n_active", C.c_int64),
        ("n_lightcone", C.c_int64), ("cube_lo", C.c_int32), ("cube_side", C.c_int32),
        ("periodic", C.c_int32), ("vcycles_last", C.c_int32),
        ("vcycles_total", C.c_int64), ("resid_last", C.c_double),
        ("escaped", C.c_int64), ("particle_steps", C.c_int64),
        ("guess_used_last", C.c_int32), ("guess_used_total", C.c_int64),
        ("resid_start", C.c_double), ("resid_guess", C.c_double),
    ]


class PmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load():
    """Load the shared library once; raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with "
            "`python -m paper_1709_04703_gb300.build` (nvcc, sm_103a)")
    lib = C.CDLL(LIB_PATH)
    P, I32, I64, D, F = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_float
    sig = {
        "pm_config_default": (None, [C.POINTER(PmConfig)]),
        "pm_init": (I32, [C.POINTER(PmConfig), P, P, I32, P, C.POINTER(P)]),
        "pm_step": (I32, [P, I32]),
        "pm_shrink": (I32, [P, D, C.POINTER(I64)]),
        "pm_potential": (I32, [P, P, D, I32, P, P, C.POINTER(I32), C.POINTER(D)]),
        "pm_power_spectrum": (I32, [P, I64, D, I32, I32, I32, P, P, P, P]),
        "pm_power_spectrum_jing": (I32, [P, I64, D, I32, I32, I32, I32, I32, D, P, P, P, P, P,
                                         P]),
        "pm_deposit": (I32, [P, P, I64, F, I32, I32, I32, I32, P, C.POINTER(I64), P]),
        "pm_deposit_tsc": (I32, [P, P, I64, F, I32, I32, I32, I32, P, C.POINTER(I64), P]),
        "pm_sort_particles": (I32, [P, P, I64, I32, P, P, P]),
        "pm_stats": (I32, [P, C.POINTER(PmStats)]),
        "pm_save": (I32, [P, C.c_char_p]),
        "pm_load": (I32, [P, C.c_char_p]),
        "pm_schedule": (I32, [P, P, P, P, P]),
        "pm_get_particles": (I32, [P, P, P, I32, C.POINTER(I64)]),
        "pm_set_particles": (I32, [P, P, P, I64, I32]),
        "pm_get_lightcone": (I32, [P, P, P, I32, C.POINTER(I64)]),
        "pm_get_forces": (I32, [P, P, I32, C.POINTER(I64)]),
        "pm_get_potential": (I32, [P, P, C.POINTER(I32), C.POINTER(I32)]),
        "pm_profile": (I32, [P, I32]),
        "pm_profile_read": (I32, [P, I32, C.POINTER(D), C.POINTER(I64), C.POINTER(D)]),
        "pm_launch_count": (I64, []),
        "pm_smoother_tiles": (I32, [P, P, P, P, I32, C.POINTER(I32)]),
        "pm_shrink_static": (I32, [P, P, I64, I32, D, D, D, D, D, P, P, P, P,
                                   C.POINTER(I64), P]),
        "pm_shrink_static_error": (C.c_char_p, []),
        "pm_batch_init": (I32, [I32, C.POINTER(PmConfig), C.POINTER(P), C.POINTER(P), I32, P,
                                C.POINTER(P)]),
        "pm_batch_step": (I32, [P, I32]),
        "pm_batch_stats": (I32, [P, I32, C.POINTER(PmStats)]),
        "pm_batch_get_particles": (I32, [P, I32, P, P, I32, C.POINTER(I64)]),
        "pm_batch_get_lightcone": (I32, [P, I32, P, P, I32, C.POINTER(I64)]),
        "pm_batch_get_forces": (I32, [P, I32, P, I32, C.POINTER(I64)]),
        "pm_batch_set_solve": (I32, [P, I32, C.c_double, I32]),
        "pm_mg_cluster_size": (I32, []),
        "pm_batch_last_error": (C.c_char_p, [P]),
        "pm_batch_destroy": (None, [P]),
        "pm_selftest_wait": (I32, [I32, I64, P]),
        "pm_mg_restrict": (I32, [P, P, I32, I32, F, F, P, P, P]),
        "pm_mg_prolong": (I32, [P, P, I32, I32, F, P]),
        "pm_nn_gemm_bf16": (I32, [P, P, P, I32, I32, I32, P]),
        "pm_mg_smooth": (I32, [P, P, P, I32, I32, C.c_float, C.c_float, I32, I32, I32, P]),
        "pm_guess_create": (I32, [I32, P, C.POINTER(P)]),
        "pm_guess_num_params": (I64, [P]),
        "pm_guess_set_params": (I32, [P, P, C.c_float]),
        "pm_guess_get_params": (I32, [P, P, P]),
        "pm_guess_forward": (I32, [P, P, I32, I32, I32, P]),
        "pm_guess_loss_grad": (I32, [P, P, P, I32, I32, I32, I32, C.POINTER(D)]),
        "pm_set_guess": (I32, [P, P]),
        "pm_capture": (I32, [P, P, P]),
        "pm_guess_adam": (I32, [P, C.c_float]),
        "pm_guess_last_error": (C.c_char_p, [P]),
        "pm_guess_destroy": (None, [P]),
        "pm_last_error": (C.c_char_p, [P]),
        "pm_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code, ctx=None):
    if code != PM_OK:
        msg = load().pm_last_error(ctx)
        raise PmError(code, msg.decode() if msg else "")
