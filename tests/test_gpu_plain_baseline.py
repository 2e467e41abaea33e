"""The plain one-patch-at-a-time GPU solver used as the benchmark's comparison arm solves the
same problem: its tau matches the oracle's."""
import numpy as np
import pytest

from oracle import tilt_oracle as O
from paper_1205_5351_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_plain_gpu_solver_matches_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from baseline.plain_gpu import tilt_plain
    for p in synth.mixed_affine_batch(2, first=3):
        tau, _ = tilt_plain(torch.from_numpy(p.img).cuda(), p.tau0, p.ttype, p.m, p.n, max_outer=2)
        ref = O.tilt(p.img.astype(np.float64), p.tau0, p.ttype, p.m, p.n, O.Params(max_outer=2))
        assert O.tau_error(tau, ref.tau) <= 1e-3
