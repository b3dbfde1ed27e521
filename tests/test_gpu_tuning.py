"""Launch shapes (ibf_tuning) and the plan-time autotuner on the GPU.

Every forced variant of the y/z step (streaming kernels with several column-block
widths; resident-slab kernel with Thomas + pivot table, partial cyclic reduction and
full cyclic reduction), alternative FFT factorisations and x-kernel row blocks must
give the oracle's projection within the usual tolerances; the autotuner's choice
must be a complete, valid shape and give the same result as the defaults.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2609_19130_gb300 import FP64, MIXED, Grid, IBFError, Plan, synth  # noqa: E402
from paper_2609_19130_gb300 import _native as N  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {FP64: 1e-12, MIXED: 1e-9}
NEU = N.IBF_BC_NEUMANN


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2609_19130_gb300 import build
    build.build()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def project(g, prec, tuning, u, v, w, autotune=False):
    plan = Plan([g], precision=prec, refine_steps=1 if prec == MIXED else 0, tuning=tuning, autotune=autotune)
    (uo, vo, wo, po), st = plan.project(cuda(u), cuda(v), cuda(w), 2e-3, 0.5, stats=True)
    torch.cuda.synchronize()
    assert plan.sync_status() in (0, 7)
    used = plan.tuning(0)
    plan.close()
    return [x.cpu().numpy() for x in (uo, vo, wo, po)], {k: float(t.cpu()[0]) for k, t in st.items()}, used


def oracle(g, u, v, w):
    og = O.Grid(g.nx, g.ny, g.nz, lx=g.lx, ly=g.ly, lz=g.lz, beta=g.beta,
                wall_x=g.bc_x == NEU, wall_y=g.bc_y == NEU)
    return O.project(og, u, v, w, dt=2e-3, alpha=0.5)


GRIDS = [  # (nx, ny, nz, beta, wall_x, wall_y): power-of-two, odd and tiny nz; walls
    (48, 24, 16, 2.0, False, False), (32, 12, 17, 1.5, False, False), (24, 16, 5, 1.0, True, False),
    (16, 24, 9, 2.5, False, True), (12, 8, 1, 0.0, False, False),
    # two and three planes: the pipelined y/z kernels (mixed, one x-mode per block) fill
    # and drain their rings in fewer iterations than they hold
    (16, 12, 2, 1.0, False, False), (24, 12, 3, 1.5, True, False),
]
VARIANTS = [
    dict(yz_kernel=1, mb=1), dict(yz_kernel=1, mb=3), dict(yz_kernel=1, mb=8),
    dict(yz_kernel=2, mb=1, tri=1), dict(yz_kernel=2, mb=2, tri=1), dict(yz_kernel=2, mb=1, tri=2),
    dict(yz_kernel=2, mb=2, tri=3), dict(yz_kernel=2, mb=4, tri=0),   # tri 0: default (Thomas + table)
    dict(yz_kernel=2, mb=1, tri=99),                                   # replaced by full reduction below
    dict(rows=2), dict(rows=6), dict(x_n1=2, y_n1=2), dict(x_n1=4, y_n1=4),
    # rows divisible by 4 take the half-block forward x-FFT CTAs on the mixed path; 4 and
    # 12 give the narrow grids odd row chunks per warp (rows processed two at a time)
    dict(rows=4), dict(rows=12),
    dict(yz_kernel=3, mb=1), dict(yz_kernel=3, mb=4), dict(yz_kernel=3, mb=2, y_n1=2),
]


def _variant(v, nz):
    v = dict(v)
    if v.get("tri") == 99:
        v["tri"] = 1 + int(math.floor(math.log2(nz)))   # 1 + log2(nz): cyclic reduction to one equation
    return v


@pytest.mark.parametrize("gdesc", GRIDS, ids=lambda d: "{}x{}x{}{}{}".format(*d[:3], "_wx" if d[4] else "",
                                                                            "_wy" if d[5] else ""))
@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_forced_variants_match_oracle(gdesc, prec):
    nx, ny, nz, beta, wx, wy = gdesc
    g = Grid(nx, ny, nz, 2 * math.pi, 1.7, 2.0, beta=beta, bc_x=NEU if wx else 0, bc_y=NEU if wy else 0)
    u, v, w = synth.uniform_velocity_np(41, nx, ny, nz, wall_x=wx, wall_y=wy)
    phi_o, u_o, v_o, w_o, st_o = oracle(g, u, v, w)
    umax = max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max())
    tried = 0
    for var in VARIANTS:
        var = _variant(var, nz)
        if var.get("x_n1") and nx % var["x_n1"]:
            continue
        if var.get("y_n1") and ny % var["y_n1"]:
            continue
        if var.get("rows") and var["rows"] > ny + (ny & 1):
            continue
        if var.get("tri", 0) > 1 + int(math.floor(math.log2(nz))):
            continue
        (ug, vg, wg, pg), st, used = project(g, prec, [var], u, v, w)
        for k, val in var.items():
            if val > 0:
                want = {"mb": min(val, nx // 2 + 1 if not wx else nx)}.get(k, val)
                assert used[k] == want, (k, used)
        assert rel_l2(pg, phi_o) <= TOL[prec], (var, rel_l2(pg, phi_o))
        for a, b in ((ug, u_o), (vg, v_o), (wg, w_o)):
            assert np.abs(a - b).max() <= 10 * TOL[prec] * umax, (var, np.abs(a - b).max())
        tried += 1
    assert tried >= 9


def test_invalid_tunings_rejected():
    g = Grid(24, 16, 8, 1.0, 1.0, 1.0, beta=1.0)
    for bad, status in ((dict(x_n1=5), N.IBF_ERR_UNSUPPORTED_SIZE),     # 5 does not divide 24
                        (dict(tri=9), N.IBF_ERR_INVALID_ARG),           # > 1 + log2(8)
                        (dict(yz_kernel=4), N.IBF_ERR_INVALID_ARG),     # spectral z on a stretched z
                        (dict(yz_kernel=5), N.IBF_ERR_INVALID_ARG),
                        (dict(rows=3), N.IBF_ERR_INVALID_ARG)):         # rows must be even
        with pytest.raises(IBFError) as ei:
            Plan([g], precision=MIXED, tuning=[bad])
        assert ei.value.status == status, (bad, ei.value.status)
    big = Grid(192, 192, 256, 1.0, 1.0, 1.0, beta=1.0)                   # slab of 192x256 complex: too big
    with pytest.raises(IBFError) as ei:
        Plan([big], precision=FP64, tuning=[dict(yz_kernel=2, mb=1)])
    assert ei.value.status == N.IBF_ERR_UNSUPPORTED_SIZE


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_autotune_matches_defaults_and_oracle(prec):
    nx, ny, nz = 64, 48, 32
    g = Grid(nx, ny, nz, 2 * math.pi, 2 * math.pi, 2.0, beta=2.0)
    u, v, w = synth.uniform_velocity_np(43, nx, ny, nz)
    phi_o, *_ = oracle(g, u, v, w)
    (_, _, _, p_def), _, used_def = project(g, prec, None, u, v, w)
    (_, _, _, p_tun), _, used = project(g, prec, None, u, v, w, autotune=True)
    assert all(val > 0 for val in used.values()), used
    assert used["yz_kernel"] in (1, 2) and 1 <= used["tri"] <= 1 + int(math.log2(nz))
    assert rel_l2(p_tun, phi_o) <= TOL[prec] and rel_l2(p_def, phi_o) <= TOL[prec]
    # forced fields survive the autotuner
    (_, _, _, p_f), _, used_f = project(g, prec, [dict(yz_kernel=1, mb=2)], u, v, w, autotune=True)
    assert used_f["yz_kernel"] == 1 and used_f["mb"] == 2
    assert rel_l2(p_f, phi_o) <= TOL[prec]
