"""ctypes view of libnufftjac.so: the C ABI declared in include/nufftjac.h, same names.

Argument marshalling only; every computation runs in the library's CUDA kernels.
Loading fails loudly when the library has not been built.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnufftjac.so")

NUFFT_OK = 0
NUFFT_ERR_INVALID_ARG = -1
NUFFT_ERR_UNSUPPORTED = -2
NUFFT_ERR_OOM = -3
NUFFT_ERR_CUDA = -4
NUFFT_ERR_TIMEOUT = -5

NUFFT_SPREAD_AUTO, NUFFT_SPREAD_STRIPS, NUFFT_SPREAD_TILES, NUFFT_SPREAD_GENERAL = 0, 1, 2, 3
SPREAD_VARIANTS = {"auto": 0, "strips": 1, "tiles": 2, "general": 3}
NUFFT_KERNEL_DIRECT, NUFFT_KERNEL_TABLE = 0, 1
KERNEL_MODES = {"direct": 0, "table": 1}
GATHER_VARIANTS = {"auto": 0, "pairs": 1, "quads": 2}

EXPORTED = (
    "nufft_default_opts", "nufft_plan", "nufft_set_points", "nufft_sort_points", "nufft_forward", "nufft_adjoint",
    "nufft_jvp_omega", "nufft_vjp_omega_x", "nufft_workspace_bytes", "nufft_get_info", "nufft_destroy",
    "nufft_status_string", "nufft_last_error", "nufft_launch_count", "nufft_profile_enable",
    "nufft_profile_read", "nufft_forward_noalloc",
)

NUFFT_NOALLOC_SCRATCH_BYTES = 32 << 20
NUFFT_MAX_COILS = 128


class nufft_opts(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("sigma", ctypes.c_double),
                ("J", ctypes.c_int), ("beta", ctypes.c_double), ("max_coils", ctypes.c_int),
                ("bin_size", ctypes.c_int * 3), ("deterministic", ctypes.c_int), ("spread_variant", ctypes.c_int),
                ("strip_part", ctypes.c_int), ("kernel_mode", ctypes.c_int),
                ("table_density", ctypes.c_int), ("gather_variant", ctypes.c_int)]


class nufft_plan_info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("k", ctypes.c_int64 * 3),
                ("J", ctypes.c_int), ("sigma", ctypes.c_double), ("beta", ctypes.c_double),
                ("m", ctypes.c_int64), ("bin_size", ctypes.c_int * 3), ("nbins", ctypes.c_int),
                ("max_coils", ctypes.c_int), ("workspace_bytes", ctypes.c_size_t)]


class NufftError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__("%s failed: %s (%d): %s" % (where, status_string(status), status, msg))
        self.status = status


_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libnufftjac.so is not built (run __graft_entry__.build()); "
                               "there is no fallback path")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        L.nufft_default_opts.argtypes = [ctypes.POINTER(nufft_opts), i32, ctypes.POINTER(ctypes.c_int64)]
        L.nufft_default_opts.restype = None
        L.nufft_plan.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(nufft_opts), i64, vp, vp]
        L.nufft_set_points.argtypes = [vp, i64, vp, vp]
        L.nufft_sort_points.argtypes = [vp, vp]
        L.nufft_forward.argtypes = [vp, i32, vp, vp, vp, vp]
        L.nufft_adjoint.argtypes = [vp, i32, vp, vp, vp, vp]
        L.nufft_jvp_omega.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp]
        L.nufft_vjp_omega_x.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp]
        L.nufft_forward_noalloc.argtypes = [ctypes.POINTER(nufft_opts), i64, vp, i32, vp, vp, vp, vp]
        L.nufft_forward_noalloc.restype = i32
        L.nufft_workspace_bytes.argtypes = [ctypes.POINTER(nufft_opts), i64, i32]
        L.nufft_workspace_bytes.restype = ctypes.c_size_t
        L.nufft_get_info.argtypes = [vp, ctypes.POINTER(nufft_plan_info)]
        L.nufft_destroy.argtypes = [vp]
        L.nufft_destroy.restype = None
        L.nufft_status_string.argtypes = [i32]
        L.nufft_status_string.restype = ctypes.c_char_p
        L.nufft_last_error.argtypes = []
        L.nufft_last_error.restype = ctypes.c_char_p
        L.nufft_launch_count.argtypes = []
        L.nufft_launch_count.restype = i64
        L.nufft_profile_enable.argtypes = [vp, i32]
        L.nufft_profile_read.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
        for name in ("nufft_plan", "nufft_set_points", "nufft_sort_points", "nufft_forward", "nufft_adjoint", "nufft_jvp_omega",
                     "nufft_vjp_omega_x", "nufft_get_info", "nufft_profile_enable", "nufft_profile_read"):
            getattr(L, name).restype = i32
        _lib = L
    return _lib


def status_string(status):
    return lib().nufft_status_string(int(status)).decode()


def _check(status, where):
    if status != NUFFT_OK:
        raise NufftError(status, where, lib().nufft_last_error().decode())


# ---- same-name wrappers (raw pointers as Python ints; raise NufftError on failure)

def nufft_default_opts(dim, n):
    o = nufft_opts()
    arr = (ctypes.c_int64 * 3)(*([int(v) for v in n] + [1] * (3 - len(n))))
    lib().nufft_default_opts(ctypes.byref(o), int(dim), arr)
    return o


def nufft_plan(opts, m, omega_ptr, stream=0):
    h = ctypes.c_void_p()
    _check(lib().nufft_plan(ctypes.byref(h), ctypes.byref(opts), int(m), omega_ptr, stream), "nufft_plan")
    return h.value


def nufft_set_points(plan, m, omega_ptr, stream=0):
    _check(lib().nufft_set_points(plan, int(m), omega_ptr, stream), "nufft_set_points")


def nufft_sort_points(plan, stream=0):
    _check(lib().nufft_sort_points(plan, stream), "nufft_sort_points")


def nufft_forward(plan, C, x, smaps, y, stream=0):
    _check(lib().nufft_forward(plan, int(C), x, smaps, y, stream), "nufft_forward")


def nufft_adjoint(plan, C, y, smaps, x, stream=0):
    _check(lib().nufft_adjoint(plan, int(C), y, smaps, x, stream), "nufft_adjoint")


def nufft_jvp_omega(plan, C, x, smaps, domega, dy, y_or_null, stream=0):
    _check(lib().nufft_jvp_omega(plan, int(C), x, smaps, domega, dy, y_or_null, stream), "nufft_jvp_omega")


def nufft_vjp_omega_x(plan, C, x, smaps, v, grad_omega, grad_x, stream=0):
    _check(lib().nufft_vjp_omega_x(plan, int(C), x, smaps, v, grad_omega, grad_x, stream), "nufft_vjp_omega_x")


def nufft_workspace_bytes(opts, m, C=0):
    return int(lib().nufft_workspace_bytes(ctypes.byref(opts), int(m), int(C)))


def nufft_get_info(plan):
    info = nufft_plan_info()
    _check(lib().nufft_get_info(plan, ctypes.byref(info)), "nufft_get_info")
    return info


def nufft_destroy(plan):
    lib().nufft_destroy(plan)


def nufft_launch_count():
    return int(lib().nufft_launch_count())


def nufft_profile_enable(plan, enable):
    _check(lib().nufft_profile_enable(plan, int(bool(enable))), "nufft_profile_enable")


def nufft_profile_read(plan, max_kinds=32):
    names = (ctypes.c_char_p * max_kinds)()
    launches = (ctypes.c_int * max_kinds)()
    ms = (ctypes.c_double * max_kinds)()
    n = ctypes.c_int()
    _check(lib().nufft_profile_read(plan, max_kinds, names, launches, ms, ctypes.byref(n)), "nufft_profile_read")
    return {names[i].decode(): (launches[i], ms[i]) for i in range(min(n.value, max_kinds))}


def nufft_forward_noalloc(opts, m, omega_ptr, C, x, smaps, y, stream=0):
    _check(lib().nufft_forward_noalloc(ctypes.byref(opts), int(m), omega_ptr, int(C), x, smaps, y, stream),
           "nufft_forward_noalloc")
