"""Input validation on the GPU: counts of non-unit directions, bad weights and
non-finite positions against a brute-force count of planted faults."""
import numpy as np
import pytest
import torch

from paper_2111_13094_gb300 import api
from paper_2111_13094_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def test_validate_counts_planted_faults():
    b = syn.single_region(seed=3, N=100_000, K=4)
    s = np.ascontiguousarray(b.samples.copy())
    s[3:6, 10] *= 1.001                      # |w| off by 1e-3
    s[3:6, 20] = [0.0, 0.0, 0.0]
    s[4, 30] = np.nan
    s[6, 40] = -1.0
    s[6, 50] = np.inf
    s[6, 60] = np.nan
    s[0, 70] = np.inf
    s[2, 80] = np.nan
    s[3:6, 90] *= 1.000001                   # within 1e-5
    n2 = (s[3:6].astype(np.float64) ** 2).sum(0)
    want = [int((~(np.abs(n2 - 1.0) <= 2e-5)).sum()),
            int((~((s[6] >= 0) & np.isfinite(s[6]))).sum()),
            int((~np.isfinite(s[:3]).all(0)).sum())]
    assert want == [3, 3, 2]
    batch = api.SampleBatch(torch.from_numpy(s).cuda(), torch.from_numpy(b.offsets).cuda())
    got = api.validate_samples(batch, unit_tol=1e-5).cpu().tolist()
    assert got == want
    clean = api.SampleBatch(torch.from_numpy(np.ascontiguousarray(b.samples)).cuda(),
                            torch.from_numpy(b.offsets).cuda())
    assert api.validate_samples(clean, unit_tol=1e-5).cpu().tolist() == [0, 0, 0]
