"""Failure detection on the GPU without faulting it: non-finite input reported through the
device error word, an injected allocation failure (host-side hook) reported as OOM with
nothing leaked, and the error word cleared by the reading call."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2609_19130_gb300 import FP64, MIXED, Grid, Plan, synth  # noqa: E402
from paper_2609_19130_gb300 import _native as N  # noqa: E402

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2609_19130_gb300 import build
    build.build()


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_nonfinite_input_reported_then_cleared(prec):
    g = Grid(16, 12, 8, 1.0, 1.0, 1.0, beta=1.0)
    plan = Plan([g], precision=prec, refine_steps=1 if prec == MIXED else 0)
    u, v, w = (torch.from_numpy(a).cuda() for a in synth.uniform_velocity_np(5, 16, 12, 8))
    bad = u.clone()
    bad[3, 4, 5] = float("nan")
    plan.project(bad, v, w, 1e-3)
    torch.cuda.synchronize()
    assert plan.sync_status() == N.IBF_ERR_NONFINITE
    plan.project(u, v, w, 1e-3)                    # clean input: the word was cleared
    torch.cuda.synchronize()
    assert plan.sync_status() == N.IBF_OK
    plan.close()


def test_injected_allocation_failure():
    """IBF_FAULT_OOM_AT=n makes the n-th device allocation of the process fail: the plan
    call returns IBF_ERR_OOM and frees what it had allocated; later plans succeed."""
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import torch\n"
        "from paper_2609_19130_gb300 import Grid, Plan, IBFError, _native as N\n"
        "g = Grid(16, 16, 8, 1.0, 1.0, 1.0)\n"
        "torch.cuda.init(); free0 = torch.cuda.mem_get_info()[0]\n"
        "try:\n"
        "    Plan([g]); print('no error'); sys.exit(1)\n"
        "except IBFError as e:\n"
        "    assert e.status == N.IBF_ERR_OOM, e.status\n"
        "torch.cuda.synchronize(); free1 = torch.cuda.mem_get_info()[0]\n"
        "assert abs(free0 - free1) < (4 << 20), (free0, free1)\n"
        "p = Plan([g]); p.close(); print('ok')\n" % ROOT)
    env = dict(os.environ, IBF_FAULT_OOM_AT="5")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr


def test_lost_copy_reported_as_timeout():
    """IBF_FAULT_LOSE_COPY makes the round-based forward y/z kernel skip one of its bulk
    plane copies: the wait for it gives up after its poll limit (no hang, no fault), the
    column blocks stop, and ibf_plan_sync_status reports IBF_ERR_TIMEOUT; a plan built
    without the hook in the same process then projects normally."""
    code = (
        "import sys, os; sys.path.insert(0, %r)\n"
        "import torch\n"
        "from paper_2609_19130_gb300 import Grid, Plan, MIXED, synth, _native as N\n"
        "g = Grid(64, 32, 12, 1.0, 1.0, 1.0, beta=1.5)\n"
        "tun = [dict(yz_kernel=1, mb=1)]\n"
        "u, v, w = (torch.from_numpy(a).cuda() for a in synth.uniform_velocity_np(3, 64, 32, 12))\n"
        "p = Plan([g], precision=MIXED, refine_steps=1, tuning=tun)\n"
        "p.project(u, v, w, 1e-3); torch.cuda.synchronize()\n"
        "st = p.sync_status(); p.close()\n"
        "assert st == N.IBF_ERR_TIMEOUT, st\n"
        "os.environ.pop('IBF_FAULT_LOSE_COPY')\n"
        "q = Plan([g], precision=MIXED, refine_steps=1, tuning=tun)\n"
        "q.project(u, v, w, 1e-3); torch.cuda.synchronize()\n"
        "assert q.sync_status() == N.IBF_OK\n"
        "q.close(); print('ok')\n" % ROOT)
    env = dict(os.environ, IBF_FAULT_LOSE_COPY="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
