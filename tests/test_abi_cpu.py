"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (no device calls: runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(glm_sur_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2510_14471_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("glm_sur_setup", "glm_sur_solve", "glm_sur_destroy", "glm_sur_get_status",
                 "glm_sur_set_omega", "glm_sur_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header(libpath):
    from paper_2510_14471_gb300 import _lib
    assert set(declared_functions()) == set(_lib.SIGNATURES)


def test_host_only_calls(libpath):
    from paper_2510_14471_gb300 import _lib
    L = _lib.lib()
    o = _lib.default_opts()
    assert o.precision == 0 and o.chunk % 2 == 0 and o.tol > 0 and o.reduce_rows == 0
    assert L.glm_sur_status_string(2).decode().startswith("rank")
    assert "sm_103a" in _lib.glm_sur_version()
    # argument validation happens before any device work
    h = ctypes.c_void_p()
    n_i = (ctypes.c_int * 2)(3, 4)
    assert L.glm_sur_setup(ctypes.byref(h), 0, 10, n_i, 1, 10, 1, None, None) == _lib.GLM_SUR_INVALID_ARG
    assert L.glm_sur_setup(ctypes.byref(h), 2, 2, n_i, 1, 2, 1, None, None) == _lib.GLM_SUR_INVALID_ARG
    assert L.glm_sur_solve(None, 1, 1, 1, 1, 1, None, None, None) == _lib.GLM_SUR_INVALID_ARG
    # adjoint, restricted and batched entry points reject null handles / bad sizes on the host
    assert L.glm_sur_backward(None, 1, 1, 1, 1, 1, 1, 1, None, None, None) == _lib.GLM_SUR_INVALID_ARG
    assert L.glm_sur_solve_restricted(None, 1, 1, None, 1, 1, 1, 1, None, None, None) == _lib.GLM_SUR_INVALID_ARG
    assert L.glm_sur_set_restrictions(None, 1, 1, 1, None) == _lib.GLM_SUR_INVALID_ARG
    assert L.glm_sur_solve_ne(None, 1, 1, 1, 1, 1, None, None, None) == _lib.GLM_SUR_INVALID_ARG
    k_i = (ctypes.c_int * 2)(1, 70)    # more restrictions than regressors in equation 2
    assert L.glm_sur_mvrglm_setup(ctypes.byref(h), 2, 100, 60, 1, 100, 1, k_i, 1, 71, None, None) == \
        _lib.GLM_SUR_INVALID_ARG
    assert L.glm_sur_mvrglm_setup(None, 2, 100, 60, 1, 100, 1, k_i, 1, 71, None, None) == _lib.GLM_SUR_INVALID_ARG
    bh = ctypes.c_void_p()
    g1 = (ctypes.c_int * 1)(2)
    m1 = (ctypes.c_int * 1)(100)
    nb = (ctypes.c_int * 2)(3, 4)
    assert L.glm_sur_batch_setup(ctypes.byref(bh), 0, g1, m1, nb, 1, 1, None, None) == _lib.GLM_SUR_INVALID_ARG
    g_big = (ctypes.c_int * 1)(33)    # more equations than a batched instance may have
    assert L.glm_sur_batch_setup(ctypes.byref(bh), 1, g_big, m1, nb, 1, 1, None, None) == _lib.GLM_SUR_INVALID_ARG
    assert L.glm_sur_batch_solve(None, 1, 8, 1, None, None, None) == _lib.GLM_SUR_INVALID_ARG
    steps = (ctypes.c_int * 1)()
    assert L.glm_sur_batch_get_work(None, steps, None) == _lib.GLM_SUR_INVALID_ARG
    assert L.glm_sur_batch_tile(None, None) <= 0
    assert L.glm_sur_batch_grid(None) == -1


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2510_14471_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True):
        src = open(path).read()
        assert "oracle" not in re.findall(r"^\s*(?:from|import)\s+(\w+)", src, flags=re.M), path
