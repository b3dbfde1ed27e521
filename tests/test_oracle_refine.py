"""Pins of oracle/refine.py (extended-precision refinement of the oracle's solve), on the
host.  The exact discrete solution is known when b is formed from a chosen phi by the
discrete Laplacian in extended precision: the refined solve must return that phi to
within FP64 rounding, while the plain FP64 oracle, on the strongly stretched z of the
benchmark, is off by about 1e-12 (the conditioning of the low modes' z systems)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from oracle import refine as RF
from paper_2609_19130_gb300 import synth


def _field(nx, ny, nz, g, seed):
    """A smooth phi dominated by low modes (cos x cos y cos(pi z / 2) shapes) plus noise,
    with zero volume-weighted mean."""
    x = (np.arange(nx) + 0.5) * g.lx / nx
    y = (np.arange(ny) + 0.5) * g.ly / ny
    zc = 0.5 * (g.zf[1:] + g.zf[:-1])
    p = 1000.0 * np.cos(math.pi * zc / 2)[:, None, None] * (np.cos(x)[None, None, :] + np.cos(y)[None, :, None])
    p = p + 300.0 * np.cos(math.pi * zc)[:, None, None] + synth.uniform_np(seed, 9, (nz, ny, nx))
    V = np.diff(g.zf)[:, None, None]
    return p - np.sum(V * p) / (np.sum(V) * nx * ny)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_laplacian_ld_matches_oracle_laplacian():
    for top in (False, True):
        g = O.Grid(12, 8, 40, lx=2.0, ly=1.5, lz=2.0, beta=2.5, dirichlet_top=top)
        p = synth.uniform_np(3, 1, (40, 8, 12))
        a = np.asarray(RF.laplacian_ld(g, p), dtype=np.float64)
        b = O.laplacian(g, p)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_refinement_recovers_known_phi_on_the_benchmark_z():
    """16 x 16 planes on the benchmark's z (tanh 2.5, 512 levels, [0, 2])."""
    nx, ny, nz = 16, 16, 512
    g = O.Grid(nx, ny, nz, lx=2 * math.pi, ly=2 * math.pi, lz=2.0, beta=2.5)
    phi = _field(nx, ny, nz, g, 5)
    b = RF.laplacian_ld(g, phi)                       # exact to longdouble rounding
    raw, _ = O.poisson(g, np.asarray(b, dtype=np.float64))
    ref, res = RF.refined_poisson(g, b, sweeps=2)
    e_raw, e_ref = rel(raw, phi), rel(ref, phi)
    assert e_ref <= 1e-15, (e_raw, e_ref)
    assert e_raw > 10 * e_ref                          # the plain FP64 solve is visibly off here
    assert res[1] < res[0]


def test_refinement_changes_nothing_where_fp64_suffices():
    nx, ny, nz = 8, 12, 16
    g = O.Grid(nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, beta=0.0)
    phi = _field(nx, ny, nz, g, 6)
    b = RF.laplacian_ld(g, phi)
    raw, _ = O.poisson(g, np.asarray(b, dtype=np.float64))
    ref, _ = RF.refined_poisson(g, b)
    assert rel(raw, phi) <= 1e-13 and rel(ref, phi) <= 1e-15


def test_refinement_with_dirichlet_outlet():
    nx, ny, nz = 8, 8, 64
    g = O.Grid(nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, beta=2.0, dirichlet_top=True)
    phi = 100.0 * synth.uniform_np(7, 2, (nz, ny, nx))
    b = RF.laplacian_ld(g, phi)
    ref, _ = RF.refined_poisson(g, b)
    assert rel(ref, phi) <= 1e-14
