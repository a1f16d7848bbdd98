"""NVTX ranges per pass (FS_NVTX=1): with the ranges on and no tool attached,
a solve and a batch still run and match the run without them (the flag is
read once per process, so the traced run is a subprocess)."""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, %r)
from paper_2412_12308_gb300 import fsolve as fs
fs.load()
n = 512
f = torch.tensor(np.random.default_rng(1).standard_normal((n, n)), dtype=torch.float32, device="cuda")
p = fs.fs_plan_create(n, n, 1.0, 1.0, 0)
u = torch.empty_like(f)
fs.fs_poisson_solve(p, f, u)
st = fs.fs_state_create(p, f)
o = torch.empty_like(f)
fs.fs_batch_wait(fs.fs_batch_submit([fs.fs_request(fs.FS_OP_DIFFUSION_ADVANCE, state=st, out_u=o, D=0.01, t=0.1)]))
torch.cuda.synchronize()
print(float(u.double().sum()), float(o.double().sum()))
"""


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "-c", SCRIPT % ROOT], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout.strip().splitlines()[-1]


def test_nvtx_ranges_do_not_change_results(gpu_lib):
    assert _run({"FS_NVTX": "1"}) == _run({"FS_NVTX": "0"})
