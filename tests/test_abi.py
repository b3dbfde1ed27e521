"""The C-ABI library: builds, loads, exports every entry point of include/ibf.h,
and rejects bad arguments on the host before touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2609_19130_gb300 import _native as N
from paper_2609_19130_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return N.lib()


def header_functions():
    src = open(os.path.join(ROOT, "include", "ibf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ibf_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    declared = header_functions()
    assert len(declared) >= 10
    assert sorted(N.EXPORTS) == declared
    for name in declared:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for s in range(0, 9):
        assert N.status_string(s) and N.status_string(s) != "unknown status"
    assert N.status_string(99) == "unknown status"


def _plan(grid_kw, opts_kw=None, n=1):
    g = dict(nx=16, ny=16, nz=8, lx=1.0, ly=1.0, lz=1.0, zf=None, beta=0.0,
             bc_x=0, bc_y=0, bc_zlo=1, bc_zhi=1)
    g.update(grid_kw)
    arr = (N.ibf_grid * n)()
    for i in range(n):
        arr[i] = N.ibf_grid(**g)
    o = dict(precision=1, refine_steps=1, autotune=0, pressure=0, inv_re=0.0)
    o.update(opts_kw or {})
    h = C.c_void_p()
    st = N.lib().ibf_projection_plan(C.byref(h), arr, n, C.byref(N.ibf_opts(**o)), 0)
    return st, h


@pytest.mark.parametrize("kw,expect", [
    (dict(nx=0), N.IBF_ERR_INVALID_ARG),
    (dict(nz=0), N.IBF_ERR_INVALID_ARG),
    (dict(lx=-1.0), N.IBF_ERR_INVALID_ARG),
    (dict(lz=float("nan")), N.IBF_ERR_INVALID_ARG),
    (dict(nx=5), N.IBF_ERR_UNSUPPORTED_SIZE),       # prime 5
    (dict(ny=2048), N.IBF_ERR_UNSUPPORTED_SIZE),    # > 32*32
    (dict(nx=27), N.IBF_ERR_UNSUPPORTED_SIZE),      # 27 = 3*9, 9 not a register size
    (dict(bc_x=2), N.IBF_ERR_UNSUPPORTED_BC),       # Dirichlet x
    (dict(bc_y=2), N.IBF_ERR_UNSUPPORTED_BC),       # Dirichlet y
    (dict(bc_x=1, nx=5), N.IBF_ERR_UNSUPPORTED_SIZE),  # wall-bounded x: same FFT sizes
    (dict(bc_zlo=2), N.IBF_ERR_UNSUPPORTED_BC),      # Dirichlet bottom
    (dict(bc_zhi=0), N.IBF_ERR_UNSUPPORTED_BC),      # periodic z
    (dict(bc_zlo=7), N.IBF_ERR_INVALID_ARG),
    (dict(beta=-1.0), N.IBF_ERR_INVALID_ARG),
])
def test_grid_validation_on_host(lib, kw, expect):
    st, h = _plan(kw)
    assert st == expect
    assert not h.value


def test_explicit_faces_validation(lib):
    bad = np.array([0.0, 0.5, 0.4, 1.0])      # not ascending
    st, h = _plan(dict(nz=3, zf=bad.ctypes.data_as(C.POINTER(C.c_double))))
    assert st == N.IBF_ERR_INVALID_ARG
    bad2 = np.array([0.0, 0.3, 0.6, 0.9])     # does not end at lz
    st, h = _plan(dict(nz=3, zf=bad2.ctypes.data_as(C.POINTER(C.c_double))))
    assert st == N.IBF_ERR_INVALID_ARG


@pytest.mark.parametrize("okw", [dict(precision=3), dict(refine_steps=-1), dict(refine_steps=9),
                                 dict(precision=0, refine_steps=1), dict(pressure=3),
                                 dict(pressure=2, inv_re=-1.0), dict(inv_re=float('nan'))])
def test_opts_validation(lib, okw):
    st, h = _plan({}, okw)
    assert st == N.IBF_ERR_INVALID_ARG


def test_null_arguments(lib):
    L = N.lib()
    assert L.ibf_projection_plan(None, None, 1, None, 0) == N.IBF_ERR_INVALID_ARG
    assert L.ibf_project(None, None, None, 1e-3, 1.0, None, None) == N.IBF_ERR_INVALID_ARG
    assert L.ibf_project_backward(None, None, None, 1e-3, 1.0, None) == N.IBF_ERR_INVALID_ARG
    assert L.ibf_plan_sync_status(None) == N.IBF_ERR_INVALID_ARG
    assert L.ibf_plan_destroy(None) == N.IBF_OK
    assert L.ibf_plan_get_info(None, None) == N.IBF_ERR_INVALID_ARG
    assert L.ibf_profile_read(None, None, None, None, 0) == 0


def test_valid_plan_without_gpu_reports_cuda_error(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, h = _plan({})
    assert st == N.IBF_ERR_CUDA
    assert not h.value
    assert N.last_error()


@pytest.mark.parametrize("bad,beta", [(dict(rows=3), 0.0), (dict(yz_kernel=5), 0.0),
                                      (dict(yz_kernel=4), 1.5)])  # spectral z needs a uniform z
def test_tuning_validation_on_host(lib, bad, beta):
    """Forced launch shapes are checked on the host before the device is touched."""
    g = (N.ibf_grid * 1)()
    g[0] = N.ibf_grid(16, 16, 8, 1.0, 1.0, 1.0, None, beta, 0, 0, 1, 1)
    t = (N.ibf_tuning * 1)()
    t[0] = N.ibf_tuning(*(bad.get(f, 0) for f in N.TUNING_FIELDS))
    h = C.c_void_p()
    o = N.ibf_opts(1, 1, 0, 0, 0.0)
    assert N.lib().ibf_projection_plan_tuned(C.byref(h), g, 1, C.byref(o), 0, t) == N.IBF_ERR_INVALID_ARG
    assert not h.value


@pytest.mark.parametrize("kw,okw,expect", [
    (dict(lx=float("inf")), {}, N.IBF_ERR_INVALID_ARG),      # rdx would be 0
    (dict(lz=float("nan")), {}, N.IBF_ERR_INVALID_ARG),
    (dict(nx=5), {}, N.IBF_ERR_UNSUPPORTED_SIZE),
    (dict(nx=1 << 10, ny=1 << 10, nz=1 << 15), {}, N.IBF_ERR_UNSUPPORTED_SIZE),  # above 2^34 cells
    (dict(bc_x=1), {}, N.IBF_ERR_UNSUPPORTED_BC),            # walls in x: not on this entry point
    (dict(bc_zhi=2), {}, N.IBF_ERR_UNSUPPORTED_BC),          # outlet: not on this entry point
    (dict(beta=float("inf")), {}, N.IBF_ERR_INVALID_ARG),
    ({}, dict(pressure=1), N.IBF_ERR_INVALID_ARG),
    ({}, dict(precision=0, refine_steps=1), N.IBF_ERR_INVALID_ARG),
])
def test_noalloc_validation_on_host(lib, kw, okw, expect):
    """ibf_project_noalloc applies the plan's grid checks and its own restrictions on the
    host, before any CUDA call (the device pointers below are never dereferenced)."""
    g = dict(nx=16, ny=16, nz=8, lx=1.0, ly=1.0, lz=1.0, zf=None, beta=0.0,
             bc_x=0, bc_y=0, bc_zlo=1, bc_zhi=1)
    g.update(kw)
    o = dict(precision=1, refine_steps=1, autotune=0, pressure=0, inv_re=0.0)
    o.update(okw)
    fake = C.c_void_p(0x1000)
    f = N.ibf_fields(fake, fake, fake, fake)
    st = N.lib().ibf_project_noalloc(C.byref(N.ibf_grid(**g)), C.byref(N.ibf_opts(**o)), C.byref(f),
                                     C.byref(f), 1e-3, 1.0, None)
    assert st == expect
