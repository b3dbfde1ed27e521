"""Spectral z (ibf_tuning.yz_kernel = 4): DCT-II along z instead of the tridiagonal
sweep, for uniform z with Neumann walls at both ends.  On such a grid the cell-centred
z Laplacian is diagonalised by the DCT-II, so the projection equals the oracle's
Thomas solve (Section "Fluid domain", projection paragraph) up to rounding: the same
tolerances as every other launch shape."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2609_19130_gb300 import FP64, MIXED, Grid, Plan, synth  # noqa: E402
from paper_2609_19130_gb300 import _native as N  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {FP64: 1e-12, MIXED: 1e-9}
NEU = N.IBF_BC_NEUMANN


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2609_19130_gb300 import build
    build.build()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


GRIDS = [  # (nx, ny, nz, wall_x, wall_y): several z FFT factorisations, odd and tiny nz, walls
    (32, 24, 16, False, False), (24, 16, 12, False, False), (16, 12, 9, False, False),
    (12, 8, 1, False, False), (16, 12, 2, False, False), (24, 16, 32, True, False),
    (16, 24, 8, False, True), (48, 32, 24, False, False),
]


@pytest.mark.parametrize("gdesc", GRIDS, ids=lambda d: "{}x{}x{}{}{}".format(*d[:3], "_wx" if d[3] else "",
                                                                            "_wy" if d[4] else ""))
@pytest.mark.parametrize("prec", [FP64, MIXED])
@pytest.mark.parametrize("mb", [1, 3])
def test_spectral_z_matches_oracle(gdesc, prec, mb):
    nx, ny, nz, wx, wy = gdesc
    g = Grid(nx, ny, nz, 2 * math.pi, 1.3, 2.0, beta=0.0, bc_x=NEU if wx else 0, bc_y=NEU if wy else 0)
    og = O.Grid(nx, ny, nz, lx=g.lx, ly=g.ly, lz=g.lz, beta=0.0, wall_x=wx, wall_y=wy)
    u, v, w = synth.uniform_velocity_np(57, nx, ny, nz, wall_x=wx, wall_y=wy)
    phi_o, u_o, v_o, w_o, st_o = O.project(og, u, v, w, dt=2e-3, alpha=0.5)
    plan = Plan([g], precision=prec, refine_steps=1 if prec == MIXED else 0, tuning=[dict(yz_kernel=4, mb=mb)])
    assert plan.tuning(0)["yz_kernel"] == 4
    (uo, vo, wo, po), st = plan.project(cuda(u), cuda(v), cuda(w), 2e-3, 0.5, stats=True)
    torch.cuda.synchronize()
    assert plan.sync_status() in (0, N.IBF_WARN_INCOMPATIBLE_RHS)
    plan.close()
    umax = max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max())
    assert rel_l2(po.cpu().numpy(), phi_o) <= TOL[prec], rel_l2(po.cpu().numpy(), phi_o)
    for a, b in ((uo, u_o), (vo, v_o), (wo, w_o)):
        assert np.abs(a.cpu().numpy() - b).max() <= 10 * TOL[prec] * umax
    assert float(st["max_div"][0]) <= 10 * TOL[prec] * st_o[1]


def test_spectral_z_batch_with_other_shapes():
    """A plan mixing the spectral-z path with the streaming and split paths."""
    specs = [((32, 24, 16, 0.0), dict(yz_kernel=4)), ((24, 16, 12, 2.0), dict(yz_kernel=1, mb=1)),
             ((16, 16, 8, 0.0), dict(yz_kernel=3, mb=2)), ((16, 12, 6, 0.0), dict(yz_kernel=4, mb=2))]
    grids = [Grid(nx, ny, nz, 2 * math.pi, 2 * math.pi, 2.0, beta=b) for (nx, ny, nz, b), _ in specs]
    fields = [synth.uniform_velocity_np(60 + i, gr.nx, gr.ny, gr.nz) for i, gr in enumerate(grids)]
    for prec in (FP64, MIXED):
        plan = Plan(grids, precision=prec, refine_steps=1 if prec == MIXED else 0, tuning=[t for _, t in specs])
        outs = plan.project_batch([tuple(cuda(a) for a in f) for f in fields], 1e-3)
        torch.cuda.synchronize()
        for gr, f, o in zip(grids, fields, outs):
            og = O.Grid(gr.nx, gr.ny, gr.nz, lx=gr.lx, ly=gr.ly, lz=gr.lz, beta=gr.beta)
            phi_o = O.project(og, *f)[0]
            assert rel_l2(o[3].cpu().numpy(), phi_o) <= TOL[prec]
        plan.close()


def test_spectral_z_rejected_where_it_does_not_apply():
    for g in (Grid(16, 12, 8, 2 * math.pi, 1.0, 2.0, beta=1.5),                          # stretched z
              Grid(16, 12, 8, 2 * math.pi, 1.0, 2.0, beta=0.0, bc_zhi=N.IBF_BC_DIRICHLET),  # outlet
              Grid(16, 12, 10, 2 * math.pi, 1.0, 2.0, beta=0.0)):                        # nz = 10: 5 no FFT size
        with pytest.raises(N.IBFError) as ei:
            Plan([g], precision=MIXED, tuning=[dict(yz_kernel=4)])
        assert ei.value.status in (N.IBF_ERR_INVALID_ARG, N.IBF_ERR_UNSUPPORTED_SIZE)


def test_autotune_on_uniform_z_matches_oracle():
    """The autotuner offers spectral z on a uniform grid; whatever it picks matches the oracle."""
    g = Grid(64, 48, 32, 2 * math.pi, 1.5, 2.0, beta=0.0)
    og = O.Grid(64, 48, 32, lx=g.lx, ly=g.ly, lz=g.lz, beta=0.0)
    u, v, w = synth.uniform_velocity_np(64, 64, 48, 32)
    phi_o = O.project(og, u, v, w, dt=2e-3, alpha=0.5)[0]
    plan = Plan([g], precision=MIXED, refine_steps=1, autotune=True)
    assert plan.tuning(0)["yz_kernel"] in (1, 2, 3, 4)
    (uo, vo, wo, po) = plan.project(cuda(u), cuda(v), cuda(w), 2e-3, 0.5)
    torch.cuda.synchronize()
    plan.close()
    assert rel_l2(po.cpu().numpy(), phi_o) <= TOL[MIXED]
