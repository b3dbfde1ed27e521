"""Factored implicit viscous solve (ibf_viscous_solve) on the GPU vs the oracle.

Section "Fluid Mechanics", Eq. (nstime_discr) with Crank-Nicolson viscous terms, and
Section "Fluid domain", provisional-step paragraph: one tridiagonal solve per
direction, Sherman-Morrison on the periodic lines.  The oracle (oracle/viscous.py)
runs exactly those algorithms in fp64; the library inverts the periodic operators
in Fourier space (the same inverse) and solves z by Thomas.

Tolerances (max |out - oracle| / max |oracle|): fp64 1e-12 (rounding of two FFT round
trips and a Thomas sweep, ~1e-15 per operation, with the factors below 1);
mixed 2e-6: fp32 transforms (round trip error ~ log2(N) 2^-24 relative to the
field's norm) and an fp32 Thomas sweep on a diagonally dominant system (error a few
2^-24), referred to the largest value.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from oracle import viscous as V  # noqa: E402
from paper_2609_19130_gb300 import FP64, MIXED, Grid, Plan, synth  # noqa: E402
from paper_2609_19130_gb300 import _native as N  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {FP64: 1e-12, MIXED: 2e-6}


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2609_19130_gb300 import build
    build.build()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def rel_max(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def oracle_solve(g, u, v, w, beta):
    zf = O.zfaces_tanh(g.nz, g.lz, g.beta)
    return V.viscous_solve(g.nx, g.ny, g.nz, g.lx, g.ly, zf, u, v, w, beta)


CASES = [(32, 24, 16, 2.0), (12, 6, 5, 1.0), (96, 64, 17, 2.5), (1, 1, 12, 2.0), (16, 16, 1, 0.0),
         (24, 18, 7, 1.5), (2, 3, 4, 1.0)]
BETAS = [0.0, 1e-4, 0.02, 1e-4]  # the tables follow beta back and forth


@pytest.mark.parametrize("case", CASES, ids=lambda c: "{}x{}x{}".format(*c[:3]))
@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_viscous_matches_oracle(case, prec):
    nx, ny, nz, bmap = case
    g = Grid(nx, ny, nz, 2 * math.pi, 1.3, 2.0, beta=bmap)
    u, v, w = synth.uniform_velocity_np(81, nx, ny, nz)
    w[0] = synth.uniform_np(82, 1, w[0].shape, -1.0, 1.0)  # wall faces of the input are ignored
    plan = Plan([g], precision=prec, refine_steps=0)
    for beta in BETAS:
        ref = oracle_solve(g, u, v, w, beta)
        (uo, vo, wo), = plan.viscous_solve([(cuda(u), cuda(v), cuda(w))], beta)
        torch.cuda.synchronize()
        for got, r, nm in zip((uo, vo, wo), ref, "uvw"):
            e = rel_max(got.cpu().numpy(), r)
            assert e <= TOL[prec], (nm, beta, e)
        wn = wo.cpu().numpy()
        assert not wn[0].any() and not wn[nz].any()
    plan.close()


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_viscous_batch_launch_shapes_and_alias(prec):
    """Several grids in one plan (one per launch shape of the y/z path), results written
    over the inputs."""
    specs = [((48, 24, 20, 2.0), None), ((24, 32, 9, 1.0), dict(yz_kernel=2, mb=2)),
             ((32, 16, 12, 1.5), dict(yz_kernel=3, mb=4))]
    grids = [Grid(nx, ny, nz, 2 * math.pi, 2 * math.pi, 2.0, beta=b) for (nx, ny, nz, b), _ in specs]
    tun = [t for _, t in specs]
    plan = Plan(grids, precision=prec, refine_steps=0, tuning=tun)
    beta = 0.01
    fields = [synth.uniform_velocity_np(90 + i, gr.nx, gr.ny, gr.nz) for i, gr in enumerate(grids)]
    dev = [tuple(cuda(a) for a in f) for f in fields]
    plan.viscous_solve(dev, beta, out=dev)  # in place
    torch.cuda.synchronize()
    for gr, f, d in zip(grids, fields, dev):
        ref = oracle_solve(gr, *f, beta)
        for got, r in zip(d, ref):
            assert rel_max(got.cpu().numpy(), r) <= TOL[prec]
    plan.close()


def test_viscous_rejects_walls_and_bad_beta():
    g = Grid(16, 12, 8, 2 * math.pi, 1.0, 2.0, beta=1.0, bc_x=N.IBF_BC_NEUMANN)
    plan = Plan([g], precision=MIXED, refine_steps=1)
    u, v, w = (torch.zeros(s, dtype=torch.float64, device="cuda") for s in g.shapes)
    with pytest.raises(N.IBFError) as ei:
        plan.viscous_solve([(u, v, w)], 0.1)
    assert ei.value.status == N.IBF_ERR_UNSUPPORTED_BC
    plan.close()
    g = Grid(16, 12, 8, 2 * math.pi, 1.0, 2.0, beta=1.0)
    plan = Plan([g], precision=FP64)
    u, v, w = (torch.zeros(s, dtype=torch.float64, device="cuda") for s in g.shapes)
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(N.IBFError) as ei:
            plan.viscous_solve([(u, v, w)], bad)
        assert ei.value.status == N.IBF_ERR_INVALID_ARG
    plan.close()


def test_viscous_graph_capture_replays():
    """No allocation or host synchronisation inside: capturable into a CUDA graph."""
    g = Grid(64, 48, 24, 2 * math.pi, 2 * math.pi, 2.0, beta=2.0)
    plan = Plan([g], precision=MIXED, refine_steps=1)
    u, v, w = (cuda(a) for a in synth.uniform_velocity_np(95, g.nx, g.ny, g.nz))
    out = tuple(torch.empty_like(t) for t in (u, v, w))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.viscous_solve([(u, v, w)], 0.01, out=[out], stream=s)  # warm-up on the capture stream
    torch.cuda.synchronize()
    eager = tuple(t.clone() for t in out)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        plan.viscous_solve([(u, v, w)], 0.01, out=[out], stream=s)
    for t in out:
        t.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for a, b in zip(out, eager):
        assert torch.equal(a, b)
    plan.close()
