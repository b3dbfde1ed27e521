"""ibf_project_noalloc: the projection for callers that may not allocate device memory.

It takes its workspace from one fixed device array instead of allocating it; its
results must match the allocating entry point (ibf_project through a plan) on two
calls in a row, with a different grid and precision on the second call, within the
tolerances the parity tests use, and the FP64 oracle on one grid in both precisions.
This file is collected last on purpose."""
import ctypes as C
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2609_19130_gb300 import FP64, MIXED, Grid, Plan, synth  # noqa: E402
from paper_2609_19130_gb300 import _native as N  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2609_19130_gb300 import build
    build.build()


def noalloc(grid, precision, refine, u, v, w):
    cg = N.ibf_grid(grid.nx, grid.ny, grid.nz, grid.lx, grid.ly, grid.lz, None, grid.beta,
                    grid.bc_x, grid.bc_y, grid.bc_zlo, grid.bc_zhi)
    opts = N.ibf_opts(N.IBF_MIXED if precision == MIXED else N.IBF_FP64, refine, 0, 0)
    outs = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(w),
            torch.empty((grid.nz, grid.ny, grid.nx), dtype=torch.float64, device="cuda"))
    fin = N.ibf_fields(u.data_ptr(), v.data_ptr(), w.data_ptr(), None)
    fout = N.ibf_fields(*(t.data_ptr() for t in outs))
    st = N.lib().ibf_project_noalloc(C.byref(cg), C.byref(opts), C.byref(fin), C.byref(fout), 1e-3, 1.0,
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, outs


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_noalloc_matches_allocating_entry_point_twice():
    cases = [(Grid(64, 48, 40, 2 * math.pi, 2 * math.pi, 2.0, beta=2.0), MIXED, 1, 1e-9, 3),
             (Grid(32, 96, 24, 1.0, 1.5, 1.0, beta=1.0), FP64, 0, 1e-12, 4)]
    for grid, prec, refine, tol, seed in cases:          # two calls in a row
        u, v, w = synth.uniform_velocity_torch(seed, grid.nx, grid.ny, grid.nz, "cuda")
        st, got = noalloc(grid, prec, refine, u, v, w)
        assert st == N.IBF_OK, N.status_string(st)
        plan = Plan([grid], precision=prec, refine_steps=refine)
        ref = plan.project(u, v, w, 1e-3)
        torch.cuda.synchronize()
        for a, b in zip(got, ref):
            assert rel(a, b) <= tol
        plan.close()


def test_noalloc_rejects_grids_beyond_its_array():
    grid = Grid(256, 256, 128, 1.0, 1.0, 1.0)               # 8.4e6 cells: workspace > 64 MiB
    u = v = torch.zeros(1, dtype=torch.float64, device="cuda")
    w = torch.zeros(1, dtype=torch.float64, device="cuda")
    st, _ = noalloc(grid, MIXED, 1, u, v, w)
    assert st == N.IBF_ERR_UNSUPPORTED_SIZE


@pytest.mark.parametrize("prec,refine,tol,utol", [(MIXED, 1, 1e-9, 1e-9), (FP64, 0, 1e-12, 1e-11)])
def test_noalloc_matches_oracle(prec, refine, tol, utol):
    """One stretched grid (96 = 12 x 8 along x, 48 = 8 x 6 along y, 36 levels) against the
    FP64 oracle, with the parity tests' tolerances: phi in relative L2, the velocity in
    max error relative to max|u*|."""
    nx, ny, nz = 96, 48, 36
    grid = Grid(nx, ny, nz, 2 * math.pi, 1.3, 2.0, beta=2.5)
    hu, hv, hw = synth.uniform_velocity_np(41, nx, ny, nz)
    u, v, w = (torch.from_numpy(a).cuda() for a in (hu, hv, hw))
    st, got = noalloc(grid, prec, refine, u, v, w)
    assert st == N.IBF_OK, N.status_string(st)
    torch.cuda.synchronize()
    og = O.Grid(nx, ny, nz, lx=grid.lx, ly=grid.ly, lz=2.0, beta=2.5)
    phi, uo, vo, wo, _ = O.project(og, hu, hv, hw, dt=1e-3)
    gp = got[3].cpu().numpy()
    assert np.linalg.norm(gp - phi) / np.linalg.norm(phi) <= tol
    umax = max(np.abs(a).max() for a in (hu, hv, hw))
    for a, b in zip(got[:3], (uo, vo, wo)):
        assert np.abs(a.cpu().numpy() - b).max() <= utol * umax
