"""ctypes binding of liblbm.so (declared in ``include/lbm.h``).

Argument marshalling only: every function here forwards to the C entry
point of the same name and raises :class:`LBMError` on a non-zero status.
Nothing computes on the host. Loading fails loudly if the library has not
been built (``python -m paper_1309_1983_gb300.build``); there is no fallback.
``LBM_LIBRARY`` (environment) names another build of the same library to
load instead, e.g. the checked debug build ``liblbm_check.so``.
"""

from __future__ import annotations

import ctypes
import os
import re

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("LBM_LIBRARY") or os.path.join(_PKG, "liblbm.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "lbm.h")

LBM_OK = 0
LBM_EINVAL = -1
LBM_ENOMEM = -2
LBM_ECUDA = -3
LBM_ETIMEOUT = -4
LBM_ENONFINITE = -5
LBM_EUNBOUND = -6
LBM_ERANGE = -7
LBM_ENOTSUP = -8

LBM_WALL_X = 0x01
LBM_WALL_Y = 0x02
LBM_WALL_Z = 0x04
LBM_LID = 0x08
LBM_STORE_F32 = 0x00
LBM_STORE_F16 = 0x10
LBM_STORE_BF16 = 0x20
LBM_FORCE = 0x40
LBM_ADJOINT = 0x80
LBM_WALLS_ONSITE = 0x100
LBM_BUF_F, LBM_BUF_FORCE, LBM_BUF_RHO, LBM_BUF_U, LBM_BUF_LAMBDA, LBM_BUF_GRADF = range(6)
LBM_CAVITY = LBM_WALL_X | LBM_WALL_Y | LBM_WALL_Z | LBM_LID
LBM_WALLS_AUTO = 0
LBM_WALLS_BRANCH = 1
LBM_WALLS_SELECT = 2
LBM_STREAM_PULL = 0
LBM_STREAM_PUSH = 1
LBM_STREAM_COPY = 2
LBM_STREAM_PULL_L2 = 3
LBM_KERNEL_NODE = 0
LBM_KERNEL_PAIR = 1
LBM_KERNEL_BULK = 2
LBM_KERNEL_BULK1 = 3
LBM_KERNEL_X2 = 4
LBM_KERNEL_X4 = 5
LBM_KERNEL_TMA = 6


class LBMError(RuntimeError):
    def __init__(self, code: int, call: str, detail: str = ""):
        self.code = code
        super().__init__(f"{call}: {strerror(code)}" + (f" ({detail})" if detail else ""))


class Layout(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("pitch", ctypes.c_int), ("elem_bytes", ctypes.c_int),
        ("plane", ctypes.c_size_t), ("f_bytes", ctypes.c_size_t),
        ("lambda_bytes", ctypes.c_size_t), ("cells", ctypes.c_size_t),
    ]


_vp = ctypes.c_void_p
_i = ctypes.c_int
_f = ctypes.c_float
_u32 = ctypes.c_uint32
_dp = ctypes.POINTER(ctypes.c_double)

# name -> argtypes (every function returns int unless listed in _RESTYPE)
_SIGNATURES = {
    "lbm_strerror": [_i],
    "lbm_last_error": [],
    "lbm_create": [_i, _i, _i, _f, _u32, ctypes.POINTER(_vp)],
    "lbm_destroy": [_vp],
    "lbm_get_layout": [_vp, ctypes.POINTER(Layout)],
    "lbm_buffer_bytes": [_vp, _i, ctypes.POINTER(ctypes.c_size_t)],
    "lbm_bind": [_vp, _vp, _vp, _vp, _vp],
    "lbm_set_lid": [_vp, _f, _f, _f],
    "lbm_set_tau": [_vp, _f],
    "lbm_set_block": [_vp, _i, _i],
    "lbm_set_kernel": [_vp, _i],
    "lbm_set_pair_block": [_vp, _i, _i],
    "lbm_set_wall_mode": [_vp, _i],
    "lbm_set_graph_steps": [_vp, _i],
    "lbm_autotune": [_vp, ctypes.c_char_p, _i, _vp, _vp, _vp],
    "lbm_current": [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp)],
    "lbm_init_equilibrium": [_vp, _vp, _vp],
    "lbm_step": [_vp, _i],
    "lbm_step_moments": [_vp, _i, _vp, _vp],
    "lbm_step_to": [_vp, _vp, _vp],
    "lbm_step_to_moments": [_vp, _vp, _vp, _vp, _vp],
    "lbm_step_push": [_vp, _vp, _vp],
    "lbm_stream": [_vp, _vp, _vp, _i],
    "lbm_moments": [_vp, _vp, _vp, _dp],
    "lbm_moments_noalloc": [_vp, _i, _i, _i, _u32, _vp, _vp, _vp, _vp, _vp],
    "lbm_sync": [_vp],
    "lbm_get_f": [_vp, _vp],
    "lbm_get_buffer": [_vp, _vp, _vp],
    "lbm_set_f": [_vp, _vp],
    "lbm_run_host": [_vp, _vp, _i, _vp, _vp],
    "lbm_adjoint_seed": [_vp, _vp, _vp, _vp, _vp, _vp],
    "lbm_adjoint_step": [_vp, _vp, _vp, _vp, _vp],
    "lbm_adjoint_step_moments": [_vp, _vp, _vp, _vp, _vp, _vp],
    "lbm_adjoint_u0": [_vp, _vp, _vp, _vp],
    "lbm_batch_create": [_i, _vp, _vp, _vp, _u32, ctypes.POINTER(_vp)],
    "lbm_batch_destroy": [_vp],
    "lbm_batch_layout": [_vp, _vp, _vp, _vp, _vp],
    "lbm_batch_bind": [_vp, _vp, _vp, _vp],
    "lbm_batch_set_tiling": [_vp, _i, _i],
    "lbm_batch_autotune": [_vp, ctypes.c_char_p, _i, _vp, _vp, _vp],
    "lbm_batch_set_timeout": [_vp, ctypes.c_double],
    "lbm_batch_inject_barrier_fault": [_vp, _i],
    "lbm_batch_use_graph": [_vp, _i],
    "lbm_batch_info": [_vp, _vp, _vp, _vp, _vp],
    "lbm_batch_current": [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp)],
    "lbm_batch_init_rest": [_vp],
    "lbm_batch_step": [_vp, _i],
    "lbm_batch_step_launches": [_vp, _i],
    "lbm_batch_moments": [_vp, _vp, _vp],
    "lbm_batch_get_f": [_vp, _i, _vp],
    "lbm_batch_set_f": [_vp, _i, _vp],
    "lbm_batch_init_equilibrium": [_vp, _vp],
    "lbm_batch_step_to": [_vp, _vp, _vp],
    "lbm_batch_step_to_moments": [_vp, _vp, _vp, _vp, _vp],
    "lbm_batch_adjoint_seed": [_vp, _vp, _vp, _vp, _vp, _vp],
    "lbm_batch_adjoint_step": [_vp, _vp, _vp, _vp, _vp],
    "lbm_batch_adjoint_step_moments": [_vp, _vp, _vp, _vp, _vp, _vp],
    "lbm_batch_adjoint_u0": [_vp, _vp, _vp, _vp],
    "lbm_batch_run": [_vp, _i, _vp, _vp, _vp, _vp],
    "lbm_batch_adjoint_run": [_vp, _i, _vp, _vp, _vp, _vp, _vp],
    "lbm_check_status": [_vp, _vp, _vp, _vp],
    "lbm_check_reset": [],
    "lbm_check_narrow": [ctypes.c_size_t],
}
_RESTYPE = {"lbm_strerror": ctypes.c_char_p, "lbm_last_error": ctypes.c_char_p}

_lib = None


def header_symbols(path: str = HEADER):
    """Names of the functions declared in include/lbm.h."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)))


def load(path: str = LIB_PATH):
    """Load liblbm.so and attach the signatures. Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"library not found at {path}: build it with "
            "`python -m paper_1309_1983_gb300.build` (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, args in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = _RESTYPE.get(name, ctypes.c_int)
    _lib = lib
    return lib


def strerror(code: int) -> str:
    try:
        return load().lbm_strerror(code).decode()
    except Exception:  # library missing: still give a readable message
        return f"status {code}"


def last_error() -> str:
    return load().lbm_last_error().decode()


def check(code: int, call: str) -> None:
    if code != LBM_OK:
        raise LBMError(code, call, last_error())


def call(name: str, *args) -> None:
    """Call ``name`` and raise LBMError on failure."""
    check(getattr(load(), name)(*args), name)


def create(nx, ny, nz, tau, flags) -> int:
    h = _vp()
    call("lbm_create", nx, ny, nz, float(tau), flags, ctypes.byref(h))
    return h.value


def layout(h) -> Layout:
    out = Layout()
    call("lbm_get_layout", h, ctypes.byref(out))
    return out


def current(h):
    a, b = _vp(), _vp()
    call("lbm_current", h, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def moments(h, rho_ptr, u_ptr, want_mass: bool):
    m = ctypes.c_double()
    call("lbm_moments", h, rho_ptr, u_ptr, ctypes.byref(m) if want_mass else None)
    return m.value if want_mass else None


def check_status():
    """The LBM_CHECK build's record: (refused, first_addr, first_bytes,
    first_kind); raises LBMError(LBM_ENOTSUP) in the normal build."""
    n, a = ctypes.c_ulonglong(), ctypes.c_ulonglong()
    b, k = ctypes.c_uint(), ctypes.c_uint()
    call("lbm_check_status", ctypes.byref(n), ctypes.byref(a), ctypes.byref(b), ctypes.byref(k))
    return n.value, a.value, b.value, k.value
