"""The Sec. 6.2 sweeps on the GPU: a sample of the range-of-convergence grid and of the
corruption levels solved as one grouped submission through the C ABI, against the FP64
oracle (tau within 1e-3, same rectification verdict)."""
import numpy as np
import pytest

from oracle import tilt_oracle as O
from paper_1205_5351_gb300 import sweeps, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_sweep_sample_matches_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1205_5351_gb300 import build, tilt
    build.build()
    grid = synth.convergence_grid()
    pick = [grid[i * 21 + j] for i in (0, 2, 5) for j in (0, 4)]              # theta 0, 6, 15 deg; skew 0, 0.2
    corr = synth.corruption_sweep(textures=1)
    pick += [corr[lv] for lv in (0, 4, 10)]                                        # 0, 20, 50 % corrupted
    prm = tilt.default_params(max_outer=6)
    with tilt.Context(0) as ctx:
        res = sweeps.solve(ctx, pick, prm)
    for p, r in zip(pick, res):
        ref = O.tilt(p.img.astype(np.float64), p.tau0, p.ttype, p.m, p.n, O.Params(max_outer=6))
        assert O.tau_error(r["tau"], ref.tau) <= 1e-3, (p.meta, r["tau"], ref.tau)
        assert sweeps.rectified(r["tau"], p.tau_true) == sweeps.rectified(ref.tau, p.tau_true)
