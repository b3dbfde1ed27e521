"""GB300-native pressure projection of the IB-Flows fractional-step solver.

Python binding over libibf.so (include/ibf.h).  PyTorch provides device memory
and streams; every step of the projection runs in the library's CUDA kernels.

    plan = Plan([Grid(nx, ny, nz, lx, ly, lz, beta=2.0)], precision="mixed", refine_steps=1)
    u, v, w, p = plan.project(u_star, v_star, w_star, dt=1e-3)
    u, v, w, p = Projection.apply(plan, 1e-3, 1.0, u_star, v_star, w_star)   # differentiable
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _native as N

__all__ = ["Grid", "Plan", "Projection", "IBFError", "FP64", "MIXED"]

FP64, MIXED = "fp64", "mixed"
IBFError = N.IBFError


@dataclass
class Grid:
    """One staggered grid (cells nx x ny x nz on [0,lx] x [0,ly] x [0,lz]).

    z faces: explicit ascending `zf` (nz+1 values, zf[0]=0, zf[nz]=lz), or the tanh
    map with clustering factor `beta` (0: uniform).  x and y are periodic by default;
    bc_x / bc_y = IBF_BC_NEUMANN makes that direction wall-bounded (DCT-II transform)."""
    nx: int
    ny: int
    nz: int
    lx: float = 1.0
    ly: float = 1.0
    lz: float = 1.0
    beta: float = 0.0
    zf: np.ndarray | None = None
    bc_x: int = N.IBF_BC_PERIODIC
    bc_y: int = N.IBF_BC_PERIODIC
    bc_zlo: int = N.IBF_BC_NEUMANN
    bc_zhi: int = N.IBF_BC_NEUMANN

    @property
    def shapes(self):
        """(u, v, w) shapes; a wall-bounded x (y) direction adds the far wall face to u (v)."""
        nxu = self.nx + (self.bc_x == N.IBF_BC_NEUMANN)
        nyv = self.ny + (self.bc_y == N.IBF_BC_NEUMANN)
        return ((self.nz, self.ny, nxu), (self.nz, nyv, self.nx), (self.nz + 1, self.ny, self.nx))

    @property
    def cells(self):
        return self.nx * self.ny * self.nz


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(int(getattr(stream, "cuda_stream", stream) or 0))


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _check_field(t, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous with shape {tuple(shape)}, got {tuple(t.shape)}")


class Plan:
    """A projection plan for a batch of grids on one device (owns its workspace)."""

    def __init__(self, grids, precision: str = MIXED, refine_steps: int = 1, device: int | None = None,
                 autotune: bool = False, tuning=None, pressure: int = N.IBF_P_PHI, inv_re: float = 0.0):
        """tuning: None, or one dict per grid with any of the ibf_tuning fields (rows,
        x_n1, y_n1, yz_kernel, mb, tri) to force; the rest default (or are autotuned).
        pressure: IBF_P_PHI (p output = phi), IBF_P_EXPLICIT (p_n + phi) or IBF_P_IMPLICIT
        (p_n + phi - alpha dt/(2 Re) lap phi, inv_re = 1/Re); p_n is the 4th input field."""
        if isinstance(grids, Grid):
            grids = [grids]
        self.grids = list(grids)
        if device is None:
            import torch
            device = torch.cuda.current_device() if torch.cuda.is_available() else 0
        self.device = int(device)
        self.precision = precision
        self.refine_steps = int(refine_steps) if precision == MIXED else 0
        arr = (N.ibf_grid * len(self.grids))()
        self._zf_keep = []
        for i, g in enumerate(self.grids):
            zf = None
            if g.zf is not None:
                z = np.ascontiguousarray(g.zf, dtype=np.float64)
                self._zf_keep.append(z)
                zf = z.ctypes.data_as(C.POINTER(C.c_double))
            arr[i] = N.ibf_grid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, zf, g.beta, g.bc_x, g.bc_y, g.bc_zlo, g.bc_zhi)
        self.pressure = int(pressure)
        opts = N.ibf_opts(N.IBF_MIXED if precision == MIXED else N.IBF_FP64, self.refine_steps, int(autotune),
                          self.pressure, float(inv_re))
        h = C.c_void_p()
        tun = None
        if tuning is not None:
            if len(tuning) != len(self.grids):
                raise ValueError("one tuning dict per grid")
            tun = (N.ibf_tuning * len(self.grids))()
            for i, t in enumerate(tuning):
                unknown = set(t or {}) - set(N.TUNING_FIELDS)
                if unknown:
                    raise ValueError(f"unknown tuning fields {sorted(unknown)}")
                tun[i] = N.ibf_tuning(*(int((t or {}).get(f, 0)) for f in N.TUNING_FIELDS))
        st = N.lib().ibf_projection_plan_tuned(C.byref(h), arr, len(self.grids), C.byref(opts), self.device, tun)
        N.check(st, "ibf_projection_plan")
        self._h = h

    # ------------------------------------------------------------ raw calls
    @property
    def handle(self):
        return self._h

    def project_into(self, ins, outs, dt, alpha=1.0, stats=None, stream=None):
        """ins: per grid (u, v, w[, p_n[, q]]) CUDA float64 tensors (p_n for a pressure-update
        plan, q a cell-centred mass source of Eq. elliptic; either may be None); outs:
        per grid (u, v, w, p)."""
        n = len(self.grids)
        fin = (N.ibf_fields * n)()
        fout = (N.ibf_fields * n)()
        for g in range(n):
            u, v, w = ins[g][:3]
            pn = ins[g][3] if len(ins[g]) > 3 else None
            qs = ins[g][4] if len(ins[g]) > 4 else None
            if self.pressure != N.IBF_P_PHI and pn is None:
                raise ValueError("this plan updates the pressure: pass (u, v, w, p_n) per grid")
            uo, vo, wo, po = outs[g]
            fin[g] = N.ibf_fields(u.data_ptr(), v.data_ptr(), w.data_ptr(), pn.data_ptr() if pn is not None else None,
                                  qs.data_ptr() if qs is not None else None)
            fout[g] = N.ibf_fields(uo.data_ptr(), vo.data_ptr(), wo.data_ptr(), po.data_ptr())
        st_ptr = None
        if stats is not None:
            md, mdi, cp = stats
            st_ptr = C.byref(N.ibf_stats(_ptr(md), _ptr(mdi), _ptr(cp)))
        s = N.lib().ibf_project(self._h, fin, fout, float(dt), float(alpha), st_ptr, _stream_handle(stream))
        N.check(s, "ibf_project")

    def backward_into(self, gouts, gins, dt, alpha=1.0, stream=None):
        n = len(self.grids)
        fo = (N.ibf_fields * n)()
        fi = (N.ibf_fields * n)()
        for g in range(n):
            gu, gv, gw, gp = gouts[g]
            fo[g] = N.ibf_fields(gu.data_ptr(), gv.data_ptr(), gw.data_ptr(), gp.data_ptr() if gp is not None else None)
            a, b, c = gins[g][:3]
            fi[g] = N.ibf_fields(a.data_ptr(), b.data_ptr(), c.data_ptr(), None)
        s = N.lib().ibf_project_backward(self._h, fo, fi, float(dt), float(alpha), _stream_handle(stream))
        N.check(s, "ibf_project_backward")

    def viscous_solve_into(self, ins, outs, beta, stream=None):
        """Factored implicit viscous solve (ibf_viscous_solve): ins / outs per grid
        (u, v, w) CUDA float64 tensors in the velocity layouts; outs may alias ins."""
        n = len(self.grids)
        fin = (N.ibf_fields * n)()
        fout = (N.ibf_fields * n)()
        for g in range(n):
            u, v, w = ins[g][:3]
            uo, vo, wo = outs[g][:3]
            fin[g] = N.ibf_fields(u.data_ptr(), v.data_ptr(), w.data_ptr(), None)
            fout[g] = N.ibf_fields(uo.data_ptr(), vo.data_ptr(), wo.data_ptr(), None)
        s = N.lib().ibf_viscous_solve(self._h, fin, fout, float(beta), _stream_handle(stream))
        N.check(s, "ibf_viscous_solve")

    def viscous_solve(self, fields, beta, out=None, stream=None):
        """(I - beta Lz)^-1 (I - beta Ly)^-1 (I - beta Lx)^-1 of each component of each
        grid; fields: per grid (u, v, w).  Returns per grid (u, v, w), new tensors unless
        `out` is given."""
        import torch
        if len(fields) != len(self.grids):
            raise ValueError("one (u, v, w) per grid")
        outs = []
        for g, (grid, f) in enumerate(zip(self.grids, fields)):
            for t, sh, nm in zip(f[:3], grid.shapes, ("u", "v", "w")):
                _check_field(t, sh, nm)
            outs.append(out[g] if out is not None else tuple(torch.empty_like(t) for t in f[:3]))
        self.viscous_solve_into(fields, outs, beta, stream=stream)
        return outs

    # ------------------------------------------------------------ conveniences
    def project(self, u, v, w, dt, alpha=1.0, out=None, stats=False, stream=None, p=None, q=None):
        """Single-grid convenience: returns (u, v, w, p) (new tensors unless `out` is given);
        `p` is p_n for plans with a pressure update, `q` an optional mass source."""
        import torch
        if len(self.grids) != 1:
            raise ValueError("project() is for single-grid plans; use project_batch()")
        res = self.project_batch([(u, v, w, p, q)], dt, alpha,
                                 out=[out] if out is not None else None, stats=stats, stream=stream)
        return res[0] if not stats else (res[0][0], res[1])

    def project_batch(self, fields, dt, alpha=1.0, out=None, stats=False, stream=None):
        import torch
        if len(fields) != len(self.grids):
            raise ValueError("one (u, v, w) per grid")
        outs = []
        for g, (grid, f) in enumerate(zip(self.grids, fields)):
            su, sv, sw = grid.shapes
            for t, sh, nm in zip(f[:3], (su, sv, sw), ("u", "v", "w")):
                _check_field(t, sh, nm)
            for extra, nm in zip(f[3:5], ("p", "q")):
                if extra is not None:
                    _check_field(extra, (grid.nz, grid.ny, grid.nx), nm)
            if out is not None:
                o = out[g]
            else:
                o = (torch.empty_like(f[0]), torch.empty_like(f[1]), torch.empty_like(f[2]),
                     torch.empty((grid.nz, grid.ny, grid.nx), dtype=torch.float64, device=f[0].device))
            outs.append(o)
        st = None
        if stats:
            dev = fields[0][0].device
            st = tuple(torch.zeros(len(self.grids), dtype=torch.float64, device=dev) for _ in range(3))
        self.project_into(fields, outs, dt, alpha, st, stream)
        if stats:
            return outs, {"max_div": st[0], "max_div_in": st[1], "compat": st[2]}
        return outs

    def tuning(self, g=0):
        """Launch shape grid g uses (dict of the ibf_tuning fields)."""
        t = N.ibf_tuning()
        N.check(N.lib().ibf_plan_get_tuning(self._h, int(g), C.byref(t)), "ibf_plan_get_tuning")
        return {f: getattr(t, f) for f in N.TUNING_FIELDS}

    def sync_status(self):
        return N.lib().ibf_plan_sync_status(self._h)

    def info(self):
        i = N.ibf_plan_info()
        N.check(N.lib().ibf_plan_get_info(self._h, C.byref(i)), "ibf_plan_get_info")
        return {"workspace_bytes": i.workspace_bytes, "ngrids": i.ngrids, "precision": i.precision,
                "refine_steps": i.refine_steps, "total_cells": i.total_cells}

    def profile(self, enable=True):
        N.check(N.lib().ibf_profile_enable(self._h, int(enable)), "ibf_profile_enable")

    def profile_read(self, reset=False):
        cap = 64
        names = (C.c_char_p * cap)()
        cnt = (C.c_longlong * cap)()
        ms = (C.c_double * cap)()
        n = N.lib().ibf_profile_read(self._h, names, cnt, ms, cap)
        out = {names[i].decode(): (int(cnt[i]), float(ms[i])) for i in range(n)}
        if reset:
            N.lib().ibf_profile_reset(self._h)
        return out

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            N.lib().ibf_plan_destroy(h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _projection_function():
    import torch

    class Projection(torch.autograd.Function):
        """(u*, v*, w*) -> (u, v, w, phi) through a plan, with ibf_project_backward as
        its vector-Jacobian product.  Unbatched tensors for a one-grid plan, or tensors
        with a leading batch dimension B for a plan of B grids of identical shape."""

        @staticmethod
        def forward(ctx, plan, dt, alpha, u, v, w):
            ctx.plan, ctx.dt, ctx.alpha = plan, dt, alpha
            u, v, w = u.contiguous(), v.contiguous(), w.contiguous()
            batched = u.dim() == 4
            ctx.batched = batched
            n = len(plan.grids)
            if not batched:
                uo, vo, wo, po = plan.project(u, v, w, dt, alpha)
                return uo, vo, wo, po
            if u.shape[0] != n:
                raise ValueError("leading dimension must equal the number of grids of the plan")
            g = plan.grids[0]
            uo, vo, wo = torch.empty_like(u), torch.empty_like(v), torch.empty_like(w)
            po = torch.empty((n, g.nz, g.ny, g.nx), dtype=torch.float64, device=u.device)
            plan.project_into([(u[b], v[b], w[b]) for b in range(n)],
                              [(uo[b], vo[b], wo[b], po[b]) for b in range(n)], dt, alpha)
            return uo, vo, wo, po

        @staticmethod
        def backward(ctx, gu, gv, gw, gp):
            plan = ctx.plan
            n = len(plan.grids)
            su, sv, sw = plan.grids[0].shapes
            pre = (n,) if ctx.batched else ()
            dev = next(t.device for t in (gu, gv, gw, gp) if t is not None)
            z = lambda sh: torch.zeros(pre + tuple(sh), dtype=torch.float64, device=dev)
            gu = gu.contiguous() if gu is not None else z(su)
            gv = gv.contiguous() if gv is not None else z(sv)
            gw = gw.contiguous() if gw is not None else z(sw)
            gp = gp.contiguous() if gp is not None else None
            a, b, c = torch.empty_like(gu), torch.empty_like(gv), torch.empty_like(gw)
            if ctx.batched:
                plan.backward_into([(gu[i], gv[i], gw[i], gp[i] if gp is not None else None) for i in range(n)],
                                   [(a[i], b[i], c[i]) for i in range(n)], ctx.dt, ctx.alpha)
            else:
                plan.backward_into([(gu, gv, gw, gp)], [(a, b, c)], ctx.dt, ctx.alpha)
            return None, None, None, a, b, c

    return Projection


class _LazyProjection:
    _fn = None

    def __getattr__(self, name):
        if _LazyProjection._fn is None:
            _LazyProjection._fn = _projection_function()
        return getattr(_LazyProjection._fn, name)


Projection = _LazyProjection()
