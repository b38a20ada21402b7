"""ctypes binding of ``libglmsur.so`` (the C ABI declared in include/glm_sur.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  The functions keep the C names; pointers are passed as ints
(``tensor.data_ptr()``) and streams as ``torch.cuda.Stream.cuda_stream``.
Importing this module never loads the library; the first call does, and it
raises if the library has not been built (there is no fallback).
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libglmsur.so")

GLM_SUR_OK = 0
GLM_SUR_INVALID_ARG = 1
GLM_SUR_RANK_DEFICIENT = 2
GLM_SUR_BREAKDOWN = 3
GLM_SUR_STAGNATED = 4
GLM_SUR_NOT_CONVERGED = 5
GLM_SUR_TIMEOUT = 6
GLM_SUR_NONFINITE = 7
GLM_SUR_OOM = 8
GLM_SUR_CUDA_ERROR = 9
STATUS_NAMES = {0: "ok", 1: "invalid_arg", 2: "rank_deficient", 3: "breakdown", 4: "stagnated",
                5: "not_converged", 6: "timeout", 7: "nonfinite", 8: "oom", 9: "cuda_error"}

GLM_SUR_PREC_FP64 = 0
GLM_SUR_PREC_FP32_REFINE = 1

GLM_SUR_STEP_AUTO = 0
GLM_SUR_STEP_SIMT = 1

GLM_SUR_PRECOND_IDENTITY = 0
GLM_SUR_PRECOND_SCALED = 1
GLM_SUR_PRECOND_DIAG = 2

GLM_SUR_ALG_GLMPCG2 = 0
GLM_SUR_ALG_GLMPCG3 = 1


class GlmSurOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("stagnation_window", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("max_refine", ctypes.c_int), ("chunk", ctypes.c_int), ("inner_shift", ctypes.c_double),
                ("reduce_rows", ctypes.c_int), ("step_kernels", ctypes.c_int), ("precond", ctypes.c_int),
                ("algorithm", ctypes.c_int)]


# (name, restype, argtypes) of every exported entry point
_VP, _I, _I64, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
SIGNATURES = {
    "glm_sur_default_opts": (None, [ctypes.POINTER(GlmSurOpts)]),
    "glm_sur_setup": (_I, [ctypes.POINTER(_VP), _I, _I64, ctypes.POINTER(_I), _VP, _I64, _VP,
                           ctypes.POINTER(GlmSurOpts), _VP]),
    "glm_sur_get_setup_status": (_I, [_VP]),
    "glm_sur_set_omega": (_I, [_VP, _VP, _VP]),
    "glm_sur_set_opts": (_I, [_VP, ctypes.POINTER(GlmSurOpts)]),
    "glm_sur_solve": (_I, [_VP, _VP, _I64, _I, _VP, _I64, _VP, _VP, _VP]),
    "glm_sur_get_status": (_I, [_VP, ctypes.POINTER(_I), _I]),
    "glm_sur_set_restrictions": (_I, [_VP, _VP, _I64, _I, _VP]),
    "glm_sur_solve_restricted": (_I, [_VP, _VP, _I64, _VP, _I64, _I, _VP, _I64, _VP, _VP, _VP]),
    "glm_sur_solve_ne": (_I, [_VP, _VP, _I64, _I, _VP, _I64, _VP, _VP, _VP]),
    "glm_sur_mvrglm_setup": (_I, [_VP, _I, _I64, _I, _VP, _I64, _VP, _VP, _VP, _I64, _VP, _VP]),
    "glm_sur_backward": (_I, [_VP, _VP, _I64, _I, _VP, _I64, _VP, _I64, _VP, _VP, _VP]),
    "glm_sur_get_w": (_I, [_VP, _VP, _I64, _VP]),
    "glm_sur_get_factors": (_I, [_VP, _VP, _I64, _VP, _VP]),
    "glm_sur_destroy": (None, [_VP]),
    "glm_sur_launch_count": (ctypes.c_int64, [_VP]),
    "glm_sur_step_path": (_I, [_VP]),
    "glm_sur_ols_static": (_I, [_VP, _VP, _I64, _I, _VP, _I64, _VP]),
    "glm_sur_profile_steps": (_I, [_VP, _I, ctypes.POINTER(_D), _VP]),
    "glm_sur_batch_setup": (_I, [ctypes.POINTER(_VP), _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                 ctypes.POINTER(_I), _VP, _VP, ctypes.POINTER(GlmSurOpts), _VP]),
    "glm_sur_batch_get_setup_status": (_I, [_VP]),
    "glm_sur_batch_solve": (_I, [_VP, _VP, _I, _VP, _VP, _VP, _VP]),
    "glm_sur_batch_get_status": (_I, [_VP, ctypes.POINTER(_I)]),
    "glm_sur_batch_get_work": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_longlong)]),
    "glm_sur_batch_tile": (_I, [_VP, ctypes.POINTER(ctypes.c_float)]),
    "glm_sur_batch_grid": (_I, [_VP]),
    "glm_sur_batch_launch_count": (ctypes.c_int64, [_VP]),
    "glm_sur_batch_destroy": (None, [_VP]),
    "glm_sur_status_string": (ctypes.c_char_p, [_I]),
    "glm_sur_version": (ctypes.c_char_p, []),
}

_lib = None


class GlmSurError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().glm_sur_status_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)} ({msg})")
        self.code = code


def lib() -> ctypes.CDLL:
    """Load the in-tree library (raises when it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2510_14471_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(code: int, where: str) -> None:
    if code != GLM_SUR_OK:
        raise GlmSurError(code, where)


def default_opts() -> GlmSurOpts:
    o = GlmSurOpts()
    lib().glm_sur_default_opts(ctypes.byref(o))
    return o


def glm_sur_setup(G: int, M: int, n_i, X_ptr: int, ldx: int, Omega_ptr: int, opts: GlmSurOpts | None,
                  stream: int) -> int:
    h = ctypes.c_void_p()
    arr = (ctypes.c_int * G)(*[int(v) for v in n_i])
    rc = lib().glm_sur_setup(ctypes.byref(h), G, M, arr, X_ptr, ldx, Omega_ptr,
                             ctypes.byref(opts) if opts is not None else None, stream)
    check(rc, "glm_sur_setup")
    return h.value


def glm_sur_mvrglm_setup(G: int, M: int, N: int, Z0_ptr: int, ldz: int, Omega0_ptr: int, k_i, C_ptr: int,
                         ldc: int, opts: GlmSurOpts | None, stream: int) -> int:
    h = ctypes.c_void_p()
    arr = (ctypes.c_int * G)(*[int(v) for v in k_i])
    rc = lib().glm_sur_mvrglm_setup(ctypes.byref(h), G, M, N, Z0_ptr, ldz, Omega0_ptr, arr, C_ptr, ldc,
                                    ctypes.byref(opts) if opts is not None else None, stream)
    check(rc, "glm_sur_mvrglm_setup")
    return h.value


def glm_sur_get_setup_status(h: int) -> int:
    return lib().glm_sur_get_setup_status(h)


def glm_sur_set_omega(h: int, Omega_ptr: int, stream: int) -> None:
    check(lib().glm_sur_set_omega(h, Omega_ptr, stream), "glm_sur_set_omega")


def glm_sur_set_opts(h: int, opts: GlmSurOpts) -> None:
    check(lib().glm_sur_set_opts(h, ctypes.byref(opts)), "glm_sur_set_opts")


def glm_sur_solve(h: int, Y_ptr: int, ldy: int, k: int, b_ptr: int, ldb: int, iters_ptr: int,
                  relres_ptr: int, stream: int) -> None:
    check(lib().glm_sur_solve(h, Y_ptr, ldy, k, b_ptr, ldb, iters_ptr, relres_ptr, stream), "glm_sur_solve")


def glm_sur_set_restrictions(h: int, C_ptr: int, ldc: int, kc: int, stream: int) -> None:
    check(lib().glm_sur_set_restrictions(h, C_ptr, ldc, kc, stream), "glm_sur_set_restrictions")


def glm_sur_solve_ne(h: int, Y_ptr: int, ldy: int, k: int, b_ptr: int, ldb: int, iters_ptr: int,
                     relres_ptr: int, stream: int = 0) -> None:
    check(lib().glm_sur_solve_ne(h, Y_ptr, ldy, k, b_ptr, ldb, iters_ptr, relres_ptr, stream), "glm_sur_solve_ne")


def glm_sur_solve_restricted(h: int, Y_ptr: int, ldy: int, d_ptr: int, ldd: int, k: int, b_ptr: int, ldb: int,
                             iters_ptr: int, relres_ptr: int, stream: int) -> None:
    check(lib().glm_sur_solve_restricted(h, Y_ptr, ldy, d_ptr, ldd, k, b_ptr, ldb, iters_ptr, relres_ptr, stream),
          "glm_sur_solve_restricted")


def glm_sur_backward(h: int, g_ptr: int, ldg: int, k: int, dy_ptr: int, ldy: int, dom_ptr: int, ldo: int,
                     iters_ptr: int, relres_ptr: int, stream: int) -> None:
    check(lib().glm_sur_backward(h, g_ptr, ldg, k, dy_ptr, ldy, dom_ptr, ldo, iters_ptr, relres_ptr, stream),
          "glm_sur_backward")


def glm_sur_get_status(h: int, k: int):
    arr = (ctypes.c_int * k)()
    rc = lib().glm_sur_get_status(h, arr, k)
    if rc in (GLM_SUR_INVALID_ARG, GLM_SUR_CUDA_ERROR):
        check(rc, "glm_sur_get_status")
    return [int(v) for v in arr]


def glm_sur_get_w(h: int, w_ptr: int, ldw: int, stream: int) -> None:
    check(lib().glm_sur_get_w(h, w_ptr, ldw, stream), "glm_sur_get_w")


def glm_sur_get_factors(h: int, Q_ptr: int, ldq: int, R_ptr: int, stream: int) -> None:
    check(lib().glm_sur_get_factors(h, Q_ptr, ldq, R_ptr, stream), "glm_sur_get_factors")


def glm_sur_launch_count(h: int) -> int:
    return int(lib().glm_sur_launch_count(h))


def glm_sur_step_path(h: int) -> int:
    return int(lib().glm_sur_step_path(h))


def glm_sur_profile_steps(h: int, reps: int, stream: int):
    ms = (ctypes.c_double * 5)()
    check(lib().glm_sur_profile_steps(h, reps, ms, stream), "glm_sur_profile_steps")
    return [float(v) for v in ms]


def glm_sur_ols_static(h: int, Y_ptr: int, ldy: int, k: int, b_ptr: int, ldb: int, stream: int) -> int:
    """Per-block least squares from the handle's factors without allocating
    device memory; returns the status code (GLM_SUR_INVALID_ARG when the
    request exceeds the library's fixed scratch array)."""
    return int(lib().glm_sur_ols_static(h, Y_ptr, ldy, k, b_ptr, ldb, stream))


def glm_sur_destroy(h: int) -> None:
    lib().glm_sur_destroy(h)


def glm_sur_batch_setup(count: int, G, M, n_i, X_ptr: int, Omega_ptr: int, opts, stream: int) -> int:
    h = ctypes.c_void_p()
    ga = (ctypes.c_int * count)(*[int(v) for v in G])
    ma = (ctypes.c_int * count)(*[int(v) for v in M])
    na = (ctypes.c_int * len(n_i))(*[int(v) for v in n_i])
    rc = lib().glm_sur_batch_setup(ctypes.byref(h), count, ga, ma, na, X_ptr, Omega_ptr,
                                   ctypes.byref(opts) if opts is not None else None, stream)
    check(rc, "glm_sur_batch_setup")
    return h.value


def glm_sur_batch_get_setup_status(h: int) -> int:
    return int(lib().glm_sur_batch_get_setup_status(h))


def glm_sur_batch_solve(h: int, Y_ptr: int, k: int, b_ptr: int, iters_ptr: int, relres_ptr: int,
                        stream: int) -> None:
    check(lib().glm_sur_batch_solve(h, Y_ptr, k, b_ptr, iters_ptr, relres_ptr, stream), "glm_sur_batch_solve")


def glm_sur_batch_get_status(h: int, n: int):
    arr = (ctypes.c_int * n)()
    rc = lib().glm_sur_batch_get_status(h, arr)
    if rc in (GLM_SUR_INVALID_ARG, GLM_SUR_CUDA_ERROR):
        check(rc, "glm_sur_batch_get_status")
    return [int(v) for v in arr]


def glm_sur_batch_get_work(h: int, count: int):
    steps = (_I * count)()
    cycles = (ctypes.c_longlong * count)()
    check(lib().glm_sur_batch_get_work(h, steps, cycles), "glm_sur_batch_get_work")
    return [int(v) for v in steps], [int(v) for v in cycles]


def glm_sur_batch_grid(h: int) -> int:
    return int(lib().glm_sur_batch_grid(h))


def glm_sur_batch_tile(h: int):
    ms = (ctypes.c_float * 3)()
    t = int(lib().glm_sur_batch_tile(h, ms))
    return t, [float(v) for v in ms]


def glm_sur_batch_launch_count(h: int) -> int:
    return int(lib().glm_sur_batch_launch_count(h))


def glm_sur_batch_destroy(h: int) -> None:
    lib().glm_sur_batch_destroy(h)


def glm_sur_version() -> str:
    return lib().glm_sur_version().decode()
