"""Mass source q of Eq. (elliptic) on the GPU: lap(phi) = (D u* - q)/(alpha dt), so the
projected velocity satisfies D u = q; compared with the oracle's composition of its
pinned divergence, solve and gradient."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2609_19130_gb300 import FP64, MIXED, Grid, Plan, synth  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {FP64: dict(phi=1e-12, u=1e-11, div=1e-11), MIXED: dict(phi=1e-9, u=1e-9, div=1e-9)}


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2609_19130_gb300 import build
    build.build()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.mark.parametrize("prec", [FP64, MIXED])
@pytest.mark.parametrize("shape", [(32, 24, 16), (12, 6, 5), (96, 64, 9)])
def test_mass_source_matches_oracle(prec, shape):
    nx, ny, nz = shape
    g = Grid(nx, ny, nz, 2 * math.pi, 1.2, 2.0, beta=2.0)
    og = O.Grid(nx, ny, nz, lx=g.lx, ly=g.ly, lz=g.lz, beta=g.beta)
    u, v, w = synth.uniform_velocity_np(91, nx, ny, nz)
    q = synth.uniform_np(92, 1, (nz, ny, nx), -50.0, 50.0)
    q -= np.sum(q * og.hz[:, None, None]) / (np.sum(og.hz) * nx * ny)   # compatible source
    phi_o, u_o, v_o, w_o, compat = O.project_q(og, u, v, w, q, dt=2e-3, alpha=0.5)
    plan = Plan([g], precision=prec, refine_steps=1 if prec == MIXED else 0)
    (uo, vo, wo, po), st = plan.project(cuda(u), cuda(v), cuda(w), 2e-3, 0.5, stats=True, q=cuda(q))
    torch.cuda.synchronize()
    assert plan.sync_status() in (0, 7)
    t = TOL[prec]
    umax = max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max())
    assert rel_l2(po.cpu().numpy(), phi_o) <= t["phi"], rel_l2(po.cpu().numpy(), phi_o)
    for a, b in ((uo, u_o), (vo, v_o), (wo, w_o)):
        assert np.abs(a.cpu().numpy() - b).max() <= t["u"] * umax
    # the constraint D u = q holds; the statistics measure its defect
    du = O.divergence(og, uo.cpu().numpy(), vo.cpu().numpy(), wo.cpu().numpy())
    din = np.abs(O.divergence(og, u, v, w) - q).max()
    assert np.abs(du - q).max() <= t["div"] * din
    assert float(st["max_div"][0]) <= t["div"] * din
    assert abs(float(st["max_div_in"][0]) - din) <= 1e-6 * din
    plan.close()


def test_repeated_projections_captured_in_one_graph():
    """The outer loop of repeated projections with a mass source (Section "Fluid
    Mechanics": q updated between projections; here a fixed q and each projection's
    output fed to the next) captured once into a CUDA graph and replayed: bit-identical
    to the eager loop, and each pass leaves D u = q."""
    nx, ny, nz = 48, 32, 16
    g = Grid(nx, ny, nz, 2 * math.pi, 1.5, 2.0, beta=1.5)
    og = O.Grid(nx, ny, nz, lx=g.lx, ly=g.ly, lz=g.lz, beta=g.beta)
    un, vn, wn = synth.uniform_velocity_np(93, nx, ny, nz)
    qn = synth.uniform_np(94, 1, (nz, ny, nx), -5.0, 5.0)
    # compatible source: the volume-weighted mean of q - D u* removed (walls in z)
    vol = np.diff(og.zf)[:, None, None] * np.ones((nz, ny, nx))
    qn = qn - float(np.sum(vol * (qn - O.divergence(og, un, vn, wn))) / np.sum(vol))
    u, v, w = (cuda(a) for a in (un, vn, wn))
    q = cuda(qn)
    plan = Plan([g], precision=MIXED, refine_steps=1)
    bufs = [tuple(torch.empty_like(t) for t in (u, v, w)) for _ in range(3)]
    p = torch.empty((nz, ny, nx), dtype=torch.float64, device="cuda")

    def loop(stream):
        src = (u, v, w)
        for b in bufs:
            plan.project_into([src + (None, q)], [b + (p,)], 1e-3, 1.0, stream=stream)
            src = b

    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        loop(s)
    torch.cuda.synchronize()
    eager = [tuple(t.clone() for t in b) for b in bufs]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        loop(s)
    for b in bufs:
        for t in b:
            t.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for b, e in zip(bufs, eager):
        for x, y in zip(b, e):
            assert torch.equal(x, y)
    # the first pass: D u = q to the mixed tolerance, relative to max|D u* - q|
    d_in = O.divergence(og, un, vn, wn) - qn
    d_out = O.divergence(og, *(t.cpu().numpy() for t in bufs[0])) - qn
    assert np.abs(d_out).max() <= 1e-9 * np.abs(d_in).max()
    plan.close()
