"""The seeded input generators: determinism, the size and kind mix of each workload, and the
rank of the rendered textures (a rank-r texture on an axis-aligned grid has rank <= r + 1,
a checkerboard rank 2), so that the inputs are what the workload descriptions say."""
import numpy as np

from paper_1205_5351_gb300 import synth


def _rank(X, rel=1e-6):
    s = np.linalg.svd(np.asarray(X, np.float64), compute_uv=False)
    return int((s > rel * s[0]).sum())


def test_batches_are_deterministic_and_indexed_by_seed():
    a = synth.mixed_affine_batch(6)
    b = synth.mixed_affine_batch(6)
    c = synth.mixed_affine_batch(2, first=4)
    for p, q in zip(a, b):
        np.testing.assert_array_equal(p.img, q.img)
        np.testing.assert_array_equal(p.tau0, q.tau0)
    np.testing.assert_array_equal(a[4].img, c[0].img)
    np.testing.assert_array_equal(a[5].tau_true, c[1].tau_true)


def test_affine_batch_sizes_and_mix():
    ps = synth.mixed_affine_batch(256)
    m = np.array([p.m for p in ps])
    n = np.array([p.n for p in ps])
    assert m.min() >= 40 and m.max() <= 120 and n.min() >= 40 and n.max() <= 120
    assert (m != n).mean() > 0.9                      # independent sides
    checker = np.mean([p.meta["kind"] == "checker" for p in ps])
    assert 0.4 < checker < 0.6
    assert all(p.ttype == 6 and abs(p.meta["theta_deg"]) <= 30 and abs(p.meta["skew"]) <= 0.2 for p in ps)
    assert all(0.0 <= p.meta["corruption"] <= 0.1 for p in ps)


def test_textures_have_the_stated_rank_on_an_aligned_grid():
    rng = np.random.default_rng(1)
    for r in (1, 3, 5):
        p = synth.make_patch(rng, 48, 40, kind="lowrank", rank=r)
        assert _rank(p.img) <= r + 1
    p = synth.make_patch(rng, 48, 40, kind="checker", period=8)
    assert _rank(p.img) == 2
    # rotated, the same texture is no longer low rank on the canvas grid (what TILT undoes)
    q = synth.make_patch(np.random.default_rng(1), 48, 40, kind="lowrank", rank=1, theta_deg=17.0)
    assert _rank(q.img, 1e-3) > 4


def test_projective_and_multistart_workloads():
    ps = synth.projective_batch(4)
    assert all(p.m == p.n == 200 and p.ttype == 8 for p in ps)
    assert all(abs(p.tau_true[6]) <= 1e-3 and abs(p.tau_true[7]) <= 1e-3 for p in ps)
    ms = synth.multistart_batch(1, side=64)
    assert len(ms) == len(synth.MULTISTART_ANGLES) == 9
    np.testing.assert_array_equal(ms[0].img, ms[8].img)          # one window, nine starts
    assert len({round(float(np.arctan2(p.tau0[3], p.tau0[0])), 6) for p in ms}) == 9


def test_served_stream_rate_and_mix():
    times, ps = synth.served_stream(400)
    t = np.asarray(times)
    assert np.all(np.diff(t) >= 0)
    assert abs(np.mean(np.diff(t)) - 1 / 2000.0) < 0.15 / 2000.0  # Poisson at 2000/s
    sides = np.array([[p.m, p.n] for p in ps])
    assert sides.min() >= 32 and sides.max() <= 256
    proj = np.mean([p.ttype == 8 for p in ps])
    assert 0.4 < proj < 0.6
