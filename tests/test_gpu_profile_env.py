"""SDMM_PROFILE=1 makes the entry points print their GPU time (a child
process, since the variable is read once per process)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch
from paper_2111_13094_gb300 import api
from paper_2111_13094_gb300 import synthetic as syn
K, dims = 4, (2, 2, 2)
pi, mu_x, mu_w, L = syn.random_mixtures(1, dims, K)
cfg = api.config(K)
st = api.MixtureState(8, K)
st.set_params(torch.from_numpy(pi), torch.from_numpy(mu_x), torch.from_numpy(mu_w), torch.from_numpy(L))
api.prepare(cfg, st)
qx = torch.from_numpy(syn.query_points(2, 1000)).cuda()
api.sample(cfg, st, qx, grid=api.Grid((0, 0, 0), (1, 1, 1), dims), seed=3)
torch.cuda.synchronize()
"""


def test_profile_environment_prints_call_times():
    env = dict(os.environ, SDMM_PROFILE="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stderr.splitlines() if x.startswith("sdmm: ")]
    names = [x.split()[1] for x in lines]
    assert "prepare" in names and "sample" in names, r.stderr[-2000:]
    assert all(float(x.split()[2]) >= 0.0 and x.endswith(" ms") for x in lines)
