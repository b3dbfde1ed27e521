"""Pressure update of Eq. (pressure) on the GPU against the oracle.

out.p = p_n + phi (explicit viscous terms) or p_n + phi - alpha dt/(2 Re) lap(phi)
(Crank-Nicolson viscous terms).  The GPU takes lap(phi) as the right-hand side the
solve satisfies (b - <b>); the oracle applies its discrete Laplacian to its own phi.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2609_19130_gb300 import FP64, MIXED, Grid, Plan, synth  # noqa: E402
from paper_2609_19130_gb300 import _native as N  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {FP64: 1e-11, MIXED: 1e-8}
NEU = N.IBF_BC_NEUMANN


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2609_19130_gb300 import build
    build.build()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.mark.parametrize("prec", [FP64, MIXED])
@pytest.mark.parametrize("pmode", [N.IBF_P_EXPLICIT, N.IBF_P_IMPLICIT])
@pytest.mark.parametrize("walls", [(False, False), (True, True)])
def test_pressure_update_matches_oracle(prec, pmode, walls):
    nx, ny, nz = 24, 16, 12
    wx, wy = walls
    g = Grid(nx, ny, nz, 2 * math.pi, 1.5, 2.0, beta=2.0, bc_x=NEU if wx else 0, bc_y=NEU if wy else 0)
    og = O.Grid(nx, ny, nz, lx=g.lx, ly=g.ly, lz=g.lz, beta=g.beta, wall_x=wx, wall_y=wy)
    u, v, w = synth.uniform_velocity_np(51, nx, ny, nz, wall_x=wx, wall_y=wy)
    p_n = synth.normal_np(52, 1, (nz, ny, nx))
    dt, alpha, inv_re = 2e-3, 8.0 / 15.0, 1.0 / 50.0
    phi_o, u_o, v_o, w_o, _ = O.project(og, u, v, w, dt=dt, alpha=alpha)
    want = O.pressure_update(og, p_n, phi_o, dt, alpha, inv_re if pmode == N.IBF_P_IMPLICIT else 0.0)
    plan = Plan([g], precision=prec, refine_steps=1 if prec == MIXED else 0, pressure=pmode, inv_re=inv_re)
    pd = cuda(p_n)
    uo, vo, wo, po = plan.project(cuda(u), cuda(v), cuda(w), dt, alpha, p=pd)
    torch.cuda.synchronize()
    assert plan.sync_status() in (0, 7)
    assert rel_l2(po.cpu().numpy(), want) <= TOL[prec], rel_l2(po.cpu().numpy(), want)
    assert np.abs(uo.cpu().numpy() - u_o).max() <= 10 * TOL[prec]
    assert np.array_equal(pd.cpu().numpy(), p_n)          # p_n not modified
    # in place: p_{n+1} overwrites p_n
    ui, vi, wi = cuda(u), cuda(v), cuda(w)
    plan.project_into([(ui, vi, wi, pd)], [(ui, vi, wi, pd)], dt, alpha)
    torch.cuda.synchronize()
    assert rel_l2(pd.cpu().numpy(), want) <= TOL[prec]
    plan.close()


def test_pressure_update_needs_p_n():
    g = Grid(16, 16, 8, 1.0, 1.0, 1.0, beta=1.0)
    plan = Plan([g], precision=MIXED, pressure=N.IBF_P_EXPLICIT)
    u, v, w = (cuda(a) for a in synth.uniform_velocity_np(3, 16, 16, 8))
    with pytest.raises(ValueError):
        plan.project(u, v, w, 1e-3)
    plan.close()
