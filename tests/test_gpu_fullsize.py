"""The bench's workload in the bench's launch configuration (1024x1024x512, 2 pi x 2 pi x
[0, 2], tanh clustering 2.5, k^-5/3 velocity of seed 4, dt = 1e-3) against the FP64
oracle's projection of the same workload, stored at sampled cells in
tests/golden/fullsize_1024x1024x512_oracle.txt (written by make_fullsize_golden.py with
the oracle alone, about 20 minutes on 8 host cores, so it is not re-run here).

The velocity is generated on the GPU here and on the host for the stored run; the two
differ by a few 1e-15 (torch's FFTs), which moves phi by ~4e-16 relative: far below the
bounds.

On this grid the z systems of the low horizontal modes are ill-conditioned (faces 2.7e-4
apart at the walls): two FP64 solvers of the same discrete system agree to a few 1e-12
of phi, and the FP64 oracle itself is ~4e-12 from the exact discrete solution (shown on
64 x 64 planes of the same z by tests/test_gpu_divergence_floor.py with the refined
oracle).  The bounds here are therefore, relative to max|phi| and max|u*| at the sampled
cells: FP64 1e-11 for phi and the velocity, mixed 1e-9 (the stated mixed tolerance); the
divergence of the FP64 path must not exceed the oracle's own (1.09e-9 of max|D u*|), the
mixed path's (two sweeps, the benchmark's count) the stated 1e-9.
"""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2609_19130_gb300 import FP64, MIXED, Grid, Plan, synth  # noqa: E402

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize_1024x1024x512_oracle.txt")


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2609_19130_gb300 import build
    build.build()


def load_golden():
    head, psum, samples = {}, {}, []
    for line in open(GOLDEN):
        t = line.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "s":
            samples.append((int(t[1]), int(t[2]), int(t[3]), *map(float, t[4:8])))
        elif t[0] == "psum":
            psum[int(t[1])] = float(t[2])
        else:
            head[t[0]] = [float(x) for x in t[1:]]
    return head, psum, samples


def divergence(g, u, v, w, zf):
    dx, dy = g.lx / g.nx, g.ly / g.ny
    hz = (zf[1:] - zf[:-1]).view(-1, 1, 1)
    return (torch.roll(u, -1, 2) - u) / dx + (torch.roll(v, -1, 1) - v) / dy + (w[1:] - w[:-1]) / hz


@pytest.fixture(scope="module")
def workload():
    if torch.cuda.get_device_properties(0).total_memory < 120e9:
        pytest.skip("needs the GB300's memory")
    head, psum, samples = load_golden()
    nx, ny, nz = (int(x) for x in head["grid"][:3])
    beta = head["grid"][3]
    g = Grid(nx, ny, nz, 2 * math.pi, 2 * math.pi, 2.0, beta=beta)
    dev = torch.device("cuda", 0)
    u, v, w = synth.kolmogorov_velocity_torch(int(head["grid"][4]), nx, ny, nz, dev)
    k = torch.arange(nz + 1, dtype=torch.float64, device=dev)
    zf = 1.0 + torch.tanh(beta * (2 * k / nz - 1)) / math.tanh(beta)
    zf[0], zf[-1] = 0.0, 2.0
    return g, (u, v, w), zf, head, psum, samples


@pytest.mark.parametrize("prec,refine", [(FP64, 0), (MIXED, 2)])
def test_bench_workload_against_stored_oracle(workload, prec, refine):
    g, (u, v, w), zf, head, psum, samples = workload
    din = divergence(g, u, v, w, zf).abs().max().item()
    oracle_div = head["stats"][0] / head["stats"][1]
    assert abs(din - head["stats"][1]) <= 1e-12 * din
    plan = Plan([g], precision=prec, refine_steps=refine)
    t = plan.tuning(0)
    assert (t["x_n1"], t["y_n1"], t["yz_kernel"]) == (32, 32, 1)
    (uo, vo, wo, po), st = plan.project(u, v, w, 1e-3, stats=True)
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    plan.close()
    rel_div = divergence(g, uo, vo, wo, zf).abs().max().item() / din
    # the library's own statistic agrees with this independent evaluation
    assert abs(float(st["max_div"][0]) / float(st["max_div_in"][0]) - rel_div) <= 0.05 * rel_div
    assert torch.equal(wo[0], w[0]) and torch.equal(wo[-1], w[-1])
    ks, js, is_ = (torch.tensor([s[c] for s in samples], device=uo.device) for c in range(3))
    got = torch.stack([po[ks, js, is_], uo[ks, js, is_], vo[ks, js, is_], wo[ks, js, is_]], 1).cpu().numpy()
    ref = np.array([s[3:] for s in samples])
    phimax, umax = head["phimax"][0], head["umax"][0]
    tol = 1e-11 if prec == FP64 else 1e-9
    e_phi = np.abs(got[:, 0] - ref[:, 0]).max() / phimax
    e_vel = np.abs(got[:, 1:] - ref[:, 1:]).max() / umax
    assert e_phi <= tol, e_phi
    assert e_vel <= tol, e_vel
    # the plane sums of phi carry the (0,0) mode of the solve
    ps = po.sum(dim=(1, 2)).cpu().numpy()
    pref = np.array([psum[k] for k in range(g.nz)])
    assert np.abs(ps - pref).max() <= 10 * tol * np.abs(pref).max()
    if prec == FP64:
        assert rel_div <= oracle_div, (rel_div, oracle_div)
    else:
        assert rel_div <= 1e-9, rel_div


def test_bench_workload_one_sweep_phi(workload):
    """One refinement sweep: phi within the stated 1e-9 of the oracle's."""
    g, (u, v, w), zf, head, psum, samples = workload
    plan = Plan([g], precision=MIXED, refine_steps=1)
    _, _, _, po = plan.project(u, v, w, 1e-3)
    torch.cuda.synchronize()
    plan.close()
    ks, js, is_ = (torch.tensor([s[c] for s in samples], device=po.device) for c in range(3))
    got = po[ks, js, is_].cpu().numpy()
    ref = np.array([s[3] for s in samples])
    assert np.abs(got - ref).max() <= 1e-9 * head["phimax"][0]
