"""Host-side scoring of the Sec. 6.2 sweeps (no GPU): the rectification test and the grids."""
import math

import numpy as np

from paper_1205_5351_gb300 import sweeps, synth


def _tau(L, c=(50.0, 40.0)):
    return np.array([L[0, 0], L[0, 1], c[0], L[1, 0], L[1, 1], c[1]])


def test_rectified_accepts_scalings_swaps_and_flips_only():
    LG = synth.linear_part(17.0, 0.3)
    tau_true = _tau(LG)
    for S in (np.diag([1.0, 1.0]), np.diag([1.3, 0.7]), np.diag([-1.0, 2.0]), np.array([[0.0, 1.2], [0.9, 0.0]])):
        assert sweeps.rectified(_tau(LG @ S), tau_true)
    # translation does not matter
    assert sweeps.rectified(_tau(LG, c=(3.0, -7.0)), tau_true)
    # a residual rotation of 5 degrees, or a skew of 0.1, is not rectified; 1 degree is
    for S, ok in ((synth.linear_part(5.0, 0.0), False), (synth.linear_part(0.0, 0.1), False),
                  (synth.linear_part(1.0, 0.0), True)):
        assert sweeps.rectified(_tau(LG @ S), tau_true) == ok
    assert abs(sweeps.misalignment(_tau(LG @ synth.linear_part(2.0, 0.0)), tau_true) - math.tan(math.radians(2.0))) < 1e-12


def test_sweep_grids_match_the_paper():
    g = synth.convergence_grid()
    assert len(g) == 11 * 21
    assert {p.meta["theta_deg"] for p in g} == {3.0 * i for i in range(11)}          # 0 .. pi/6, step pi/60
    assert {p.meta["skew"] for p in g} == {round(0.05 * j, 2) for j in range(21)}    # 0 .. 1, step 0.05
    assert all(p.meta["kind"] == "checker" for p in g)
    c = synth.corruption_sweep(textures=2)
    assert len(c) == 2 * 21 and sorted({p.meta["corruption"] for p in c}) == list(synth.CORRUPTION_LEVELS)
    # nested corruption: a texture's corrupted pixels at one level are corrupted at the next
    a, b = c[3].img, c[4].img
    clean = c[0].img
    assert np.all((a != clean) <= (b != clean))
    # scoring: a perfect solve rectifies everything
    res = [{"status": 0, "tau": p.tau_true} for p in g]
    m = sweeps.convergence_map(g, res)
    assert m["rate"] == 1.0 and len(m["rectified"]) == 11 and len(m["rectified"][0]) == 21
    r = sweeps.corruption_rates(c, [{"status": 0, "tau": p.tau0} for p in c])
    assert r["textures"] == 2 and r["success_rate"] == [0.0] * 21                   # identity start: 10 deg off
