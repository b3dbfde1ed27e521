"""Config 3 (batched uneven grids in one CUDA graph) and config 5 (differentiable
projection) on the GPU, through the C ABI."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2609_19130_gb300 import FP64, MIXED, Grid, Plan, Projection, synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2609_19130_gb300 import build
    build.build()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def config3_grids():
    return [Grid(nx, ny, nz, 2 * math.pi, 2 * math.pi, 2.0, beta=beta) for nx, ny, nz, beta in
            synth.batch_grid_draws(1, 64)]


def test_config3_graph_replay_matches_eager_and_oracle():
    """64 uneven grids, mixed precision with refinement, launch shapes autotuned per
    grid shape (tridiagonal variant, column blocks, FFT factors, row blocks)."""
    grids = config3_grids()
    plan = Plan(grids, precision=MIXED, refine_steps=1, autotune=True)
    tunings = [plan.tuning(g) for g in range(len(grids))]
    assert all(all(v > 0 for v in t.values()) for t in tunings)
    ins, outs, outs_g = [], [], []
    for i, g in enumerate(grids):
        u, v, w = synth.uniform_velocity_torch(1000 + i, g.nx, g.ny, g.nz, "cuda")
        ins.append((u, v, w))
        mk = lambda: (torch.empty_like(u), torch.empty_like(v), torch.empty_like(w),
                      torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64, device="cuda"))
        outs.append(mk())
        outs_g.append(mk())
    st = tuple(torch.zeros(len(grids), dtype=torch.float64, device="cuda") for _ in range(3))
    plan.project_into(ins, outs, 1e-3, 1.0, stats=st)
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    # capture one ibf_project of all 64 grids into a CUDA graph, replay twice
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.project_into(ins, outs_g, 1e-3, 1.0, stream=s)   # warm the stream once
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.project_into(ins, outs_g, 1e-3, 1.0)
    for _ in range(2):
        for o in outs_g:
            for t in o:
                t.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for a, b in zip(outs, outs_g):
            for x, y in zip(a, b):
                assert torch.equal(x, y)
    # every grid divergence-free to the mixed tolerance
    md, mdi = st[0].cpu().numpy(), st[1].cpu().numpy()
    assert np.all(md <= 1e-9 * mdi), (md / mdi).max()
    # element-wise parity of every grid with the oracle (mixed tolerances: phi relative
    # L2 1e-9, velocity 1e-9 max|u*|)
    for i, g in enumerate(grids):
        og = O.Grid(g.nx, g.ny, g.nz, lx=g.lx, ly=g.ly, lz=g.lz, beta=g.beta)
        host = [t.cpu().numpy() for t in ins[i]]
        phi, uo, vo, wo, _ = O.project(og, *host, dt=1e-3)
        assert rel_l2(outs[i][3].cpu().numpy(), phi) <= 1e-9, (i, g)
        umax = max(np.abs(a).max() for a in host)
        for a, b in zip(outs[i][:3], (uo, vo, wo)):
            assert np.abs(a.cpu().numpy() - b).max() <= 1e-9 * umax, (i, g)
    plan.close()
    # the default launch shapes give the same projection (to the mixed tolerance)
    plan_d = Plan(grids, precision=MIXED, refine_steps=1)
    outs_d = [tuple(torch.empty_like(t) for t in o) for o in outs]
    plan_d.project_into(ins, outs_d, 1e-3, 1.0)
    torch.cuda.synchronize()
    for a, b in zip(outs, outs_d):
        assert float(torch.linalg.norm(a[3] - b[3]) / torch.linalg.norm(b[3])) <= 2e-9
    plan_d.close()


def test_config5_finite_differences_batch8_256cube():
    """loss = sum(w . P(u*)) over a batch of 8 256^3 grids (mixed, 1 refinement); the
    autograd gradient against central differences (eps = 1e-3) on 32 random entries,
    the two perturbed projections differenced element-wise in fp64 before summing."""
    n, B, eps = 256, 8, 1e-3
    grids = [Grid(n, n, n, 2 * math.pi, 2 * math.pi, 2.0, beta=2.0) for _ in range(B)]
    plan = Plan(grids, precision=MIXED, refine_steps=1)
    su, sv, sw = grids[0].shapes
    u = torch.stack([synth.uniform_torch(5, 1 + b, su, device="cuda") for b in range(B)])
    v = torch.stack([synth.uniform_torch(5, 17 + b, sv, device="cuda") for b in range(B)])
    w = torch.stack([synth.uniform_torch(5, 33 + b, sw, device="cuda") for b in range(B)])
    w[:, 0].zero_()
    w[:, -1].zero_()
    wts = [torch.stack([synth.normal_torch(6, 50 + 4 * b + c, sh, device="cuda") for b in range(B)])
           for c, sh in enumerate((su, sv, sw, (n, n, n)))]
    x = [t.clone().requires_grad_(True) for t in (u, v, w)]
    outs = Projection.apply(plan, 1e-3, 1.0, *x)
    loss = sum((o * wt).sum() for o, wt in zip(outs, wts))
    loss.backward()
    grads = [t.grad for t in x]
    rng = np.random.default_rng(5)
    gmax = max(float(g.abs().max()) for g in grads)
    worst = 0.0
    with torch.no_grad():
        for _ in range(32):
            comp = int(rng.integers(0, 3))
            flat = int(rng.integers(0, x[comp].numel()))
            base = [t.detach().clone() for t in (u, v, w)]
            plus = [t.clone() for t in base]
            minus = [t.clone() for t in base]
            plus[comp].view(-1)[flat] += eps
            minus[comp].view(-1)[flat] -= eps
            op = Projection.apply(plan, 1e-3, 1.0, *plus)
            om = Projection.apply(plan, 1e-3, 1.0, *minus)
            fd = sum(float(((a - b) * wt).sum()) for a, b, wt in zip(op, om, wts)) / (2 * eps)
            ad = float(grads[comp].view(-1)[flat])
            worst = max(worst, abs(fd - ad) / gmax)
    assert worst <= 1e-3, worst
    plan.close()


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-10), (MIXED, 1e-8)])
def test_config5_dense_adjoint_16cube(prec, tol):
    """The GPU adjoint on a 16^3 copy of the config-5 setup against the oracle's dense P^T."""
    n = 16
    g = Grid(n, n, n, 2 * math.pi, 2 * math.pi, 2.0, beta=2.0)
    og = O.Grid(n, n, n, lx=g.lx, ly=g.ly, lz=2.0, beta=2.0)
    dp = dense.DenseProjection(n, n, n, g.lx, g.ly, og.zf)
    su, sv, sw = g.shapes
    gu, gv, gw = (synth.normal_np(6, i + 1, s) for i, s in enumerate((su, sv, sw)))
    gp = synth.normal_np(6, 4, (n, n, n))
    ref = dp.project_T(gu, gv, gw, gp, dt=1e-3, alpha=1.0)
    plan = Plan([g], precision=prec, refine_steps=1 if prec == MIXED else 0)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    a, b, c = (torch.empty(s, dtype=torch.float64, device="cuda") for s in (su, sv, sw))
    plan.backward_into([(cu(gu), cu(gv), cu(gw), cu(gp))], [(a, b, c)], 1e-3, 1.0)
    torch.cuda.synchronize()
    for x_, y_ in zip((a, b, c), ref):
        assert rel_l2(x_.cpu().numpy(), y_) <= tol
    plan.close()
