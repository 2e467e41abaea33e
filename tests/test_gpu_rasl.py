"""RASL image sets (Sec. 1: TILT's model with one image per column) on the GPU, through the
C ABI, against the oracle: one step, one inner loop and the outer loop element by element on
small sets, and properties that hold at any size on a batch."""
import math

import numpy as np
import pytest

from oracle import tilt_oracle as O
from paper_1205_5351_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1205_5351_gb300 import build, tilt
    build.build()
    return tilt


@pytest.fixture(scope="module")
def ctx(T):
    with T.Context(0) as c:
        yield c


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a, np.float64) - b) / (nb if nb > 0 else 1.0)


def _sets(count, nimg, m, n, ttype, seed0, **kw):
    return [synth.rasl_set(np.random.default_rng(10_000 + seed0 + i), nimg, m, n, ttype=ttype, **kw)
            for i in range(count)]


def _run(T, ctx, sets, prm, planes=True):
    imgs = np.stack([s.imgs for s in sets])
    tau0 = np.stack([s.tau0 for s in sets])
    s0 = sets[0]
    return ctx.rasl(imgs, s0.m, s0.n, tau0, s0.ttype, prm, planes=planes)


# (nimg, m, n, ttype): small windows (the SVT through the QR factorisation of M, whose
# buffers fit in shared memory); 33 images (three columns for some warps); 40 images of
# 48 x 48 (R = 2304: M too large for shared memory, so the one-sided Jacobi on M itself with
# B in device memory and staged sweeps)
CASES = [(6, 12, 14, 6), (9, 16, 11, 8), (33, 20, 20, 6), (40, 48, 48, 6)]
QR_PATH = {(6, 12, 14): 1, (9, 16, 11): 1, (33, 20, 20): 1, (40, 48, 48): 0}


@pytest.mark.parametrize("nimg,m,n,ttype", CASES)
def test_rasl_one_iteration_parity(T, ctx, nimg, m, n, ttype):
    # warp + normalise per column, the Gram blocks, the Woodbury form of W^T W, one LADMAP
    # iteration and dtau per image: every output at the per-kernel bound, relative Frobenius
    # error <= 1e-5
    sets = _sets(2, nimg, m, n, ttype, nimg)
    out = _run(T, ctx, sets, T.default_params(max_outer=1, max_inner=1))
    errs = []
    for k, s in enumerate(sets):
        ref = O.rasl(s.imgs.astype(np.float64), s.tau0, ttype, m, n, O.Params(max_outer=1, max_inner=1))
        r = out["results"][k]
        assert (r["status"], r["outer_iters"], r["inner_iters"]) == (2, 1, 1), r
        assert r["svt_qr"] == QR_PATH[(nimg, m, n)], r
        # the step in image space, J dtau (J the stacked Jacobian at tau0): independent of how
        # the transform is parametrised
        Jb = O.rasl_stacked_jacobian(O.rasl_warp(s.imgs.astype(np.float64), s.tau0, ttype, m, n)[1])
        dt_g, dt_r = (out["tau"][k] - s.tau0).ravel(), (ref.tau - s.tau0).ravel()
        e = dict(D=rel(out["Dhat"][k], ref.Dhat), A=rel(out["A"][k], ref.A), E=rel(out["E"][k], ref.E),
                 E_abs=np.linalg.norm(out["E"][k] - ref.E) / np.linalg.norm(ref.Dhat),
                 dtau=rel(dt_g, dt_r), dG=rel(Jb @ dt_g, Jb @ dt_r))
        errs.append(e)
    print("one-iteration errors", errs)
    for e in errs:
        assert e["D"] <= 1e-5 and e["A"] <= 1e-5 and e["dG"] <= 1e-5, e
        # E = T(N) with T 1-Lipschitz: its error is that of N, FP32 rounding at the scale of
        # D_hat, while E's entries sit just above the threshold (relative to ||E|| the same
        # error reads up to 3e-5, measured)
        assert e["E_abs"] <= 1e-5, e
        # the parameters themselves: dtau_c = (G^-1 J^T r)_c amplifies the rounding of r by up
        # to cond(G), 2e3-3e4 for the affine sets and 3e5-8e5 for the projective ones (whose
        # perspective entries multiply pixel coordinates); measured 1e-6-3e-6 affine, 1e-5
        # projective
        assert e["dtau"] <= (1e-5 if ttype == 6 else 1e-4), e


@pytest.mark.parametrize("nimg,m,n,ttype", CASES)
def test_rasl_inner_loop_parity(T, ctx, nimg, m, n, ttype):
    # one outer step with the inner loop run to Cond1/Cond2: the FP32 rounding of every
    # iteration carries into the next, so A, E and dtau at 1e-4 relative (as for TILT's inner
    # loop), the iteration counts within one, equal numerical rank
    sets = _sets(2, nimg, m, n, ttype, 100 + nimg)
    out = _run(T, ctx, sets, T.default_params(max_outer=1))
    errs = []
    for k, s in enumerate(sets):
        ref = O.rasl(s.imgs.astype(np.float64), s.tau0, ttype, m, n, O.Params(max_outer=1))
        r = out["results"][k]
        errs.append(dict(iters=(r["inner_iters"], ref.inner_iters), A=rel(out["A"][k], ref.A),
                         E=rel(out["E"][k], ref.E), dtau=rel(out["tau"][k] - s.tau0, ref.tau - s.tau0),
                         rank=(r["rank"], ref.rank), obj=abs(r["objective"] - ref.objective) / ref.objective))
    print("inner-loop errors", errs)
    for e in errs:
        assert abs(e["iters"][0] - e["iters"][1]) <= 1, e
        assert e["A"] <= 1e-4 and e["E"] <= 1e-4 and e["dtau"] <= 1e-4, e
        assert e["rank"][0] == e["rank"][1] and e["obj"] <= 1e-5, e


@pytest.mark.parametrize("eps_svd", [0.0, 0.05])
@pytest.mark.parametrize("nimg,m,n,ttype", [CASES[0], CASES[3]])
def test_rasl_inner_loop_with_the_warm_start_gate(T, ctx, nimg, m, n, ttype, eps_svd):
    # the gate of Algorithm 2 on the Jacobi warm start (||M_k - M_k-1|| < eps_svd ||M_k||): with
    # eps_svd = 0 no SVD is warm-started, with 0.05 those after the first few iterations are;
    # the SVT is exact either way, so the result is the oracle's at the inner loop's bounds,
    # E's error measured at the scale of the data (E = T(N) is 1-Lipschitz in N, whose rounding
    # is at the scale of D_hat; relative to the small ||E|| the cold 48 x 48 sets read 1.1e-4)
    sets = _sets(1, nimg, m, n, ttype, 300 + nimg)
    s = sets[0]
    out = _run(T, ctx, sets, T.default_params(max_outer=1, eps_svd=eps_svd))
    off = _run(T, ctx, sets, T.default_params(max_outer=1))
    ref = O.rasl(s.imgs.astype(np.float64), s.tau0, ttype, m, n, O.Params(max_outer=1))
    r, r_off = out["results"][0], off["results"][0]
    assert r_off["svd_warm"] == r_off["inner_iters"] - 1, r_off
    if eps_svd == 0.0:
        assert r["svd_warm"] == 0, r
    else:
        assert 0 < r["svd_warm"] <= r["inner_iters"] - 1, r
    e = dict(iters=(r["inner_iters"], ref.inner_iters), A=rel(out["A"][0], ref.A), E=rel(out["E"][0], ref.E),
             E_abs=np.linalg.norm(out["E"][0] - ref.E) / np.linalg.norm(ref.Dhat),
             dtau=rel(out["tau"][0] - s.tau0, ref.tau - s.tau0), rank=(r["rank"], ref.rank))
    print("gated inner loop", eps_svd, e, r["svd_warm"], r["svd_sweeps"], r_off["svd_sweeps"])
    assert abs(e["iters"][0] - e["iters"][1]) <= 1, e
    assert e["A"] <= 1e-4 and e["E_abs"] <= 1e-4 and e["dtau"] <= 1e-4, e
    assert e["rank"][0] == e["rank"][1], e


def test_rasl_outer_loop_parity(T, ctx):
    # three outer steps: tau within 1e-3 relative of the oracle's (the benchmark spec's bound for
    # transforms), equal rank and outer iterations.  (The displacement tau - tau0 alone, held to
    # 1e-5 after one iteration and 1e-4 after one inner loop above, drifts further from one
    # outer step to the next: measured 7e-5 to 1.3e-3 after three.)
    nimg, m, n, ttype = 12, 20, 24, 6
    sets = _sets(3, nimg, m, n, ttype, 500)
    prm = T.default_params(max_outer=3)
    out = _run(T, ctx, sets, prm, planes=False)
    errs = []
    for k, s in enumerate(sets):
        ref = O.rasl(s.imgs.astype(np.float64), s.tau0, ttype, m, n, O.Params(max_outer=3))
        r = out["results"][k]
        errs.append(dict(outer=(r["outer_iters"], ref.outer_iters), tau=O.tau_error(out["tau"][k].ravel(), ref.tau.ravel()),
                         dtau=rel(out["tau"][k] - s.tau0, ref.tau - s.tau0), rank=(r["rank"], ref.rank)))
    print("outer-loop errors", errs)
    for e in errs:
        assert e["outer"][0] == e["outer"][1] and e["rank"][0] == e["rank"][1], e
        assert e["tau"] <= 1e-3, e


def _corner_spread(taus, st):
    U, V = O.corner_uv(st.m, st.n)
    pts = []
    for t, tt in zip(taus, st.tau_true):
        x, y, _, _ = O.map_points(t, st.ttype, U, V)
        H = np.array([[tt[0], tt[1], tt[2]], [tt[3], tt[4], tt[5]], [0.0, 0.0, 1.0]])
        q = np.linalg.solve(H, np.vstack([x, y, np.ones(4)]))
        pts.append((q[:2] / q[2]).T)
    pts = np.array(pts)
    return float(np.max(np.linalg.norm(pts - pts.mean(axis=0), axis=2)))


def test_rasl_batch_properties(T, ctx):
    # a batch in the benchmark's launch configuration (one launch, all sets), full default
    # parameters: every set finishes with a valid status, keeps its mean transform (the
    # constraint rows), and ends nearly as low-rank as the rendering transforms make it
    # (nuclear norm of its data matrix, evaluated by the oracle's warp)
    sets = synth.rasl_batch(24, first=0, nimg=16, side=24)
    out = _run(T, ctx, sets, None, planes=False)
    for k, s in enumerate(sets):
        r = out["results"][k]
        assert r["status"] in (0, 1, 2), r
        tau = out["tau"][k]
        assert np.all(np.isfinite(tau))
        np.testing.assert_allclose(tau.mean(axis=0), s.tau0.mean(axis=0), atol=5e-3)
        imgs = s.imgs.astype(np.float64)
        nuc = {}
        for name, tt in (("gpu", tau), ("true", s.tau_true), ("tau0", s.tau0)):
            D = O.rasl_warp(imgs, tt, s.ttype, s.m, s.n)[0]
            nuc[name] = float(np.linalg.svd(D, compute_uv=False).sum())
        # within 15 % of the way from the rendering transforms' value back to tau0's (the
        # oracle on this batch: 9.3 % at worst, below the rendering value on 14 of 24 sets)
        gap = (nuc["gpu"] - nuc["true"]) / (nuc["tau0"] - nuc["true"])
        assert gap <= 0.15, (k, nuc)
        # and the corners closer together than at the start (the largest distance over the
        # images: an image whose last steps alternate between two transforms can keep it high)
        assert _corner_spread(tau, s) < _corner_spread(s.tau0, s), k
    # sampled sets of the same launch configuration against the oracle, both stopped after
    # three outer steps (most sets never meet the outer stopping rule: their last steps
    # alternate between two transforms, a period-2 cycle that both sides follow but whose
    # phase rounding shifts, so full solves agree only to a few 1e-3)
    out3 = _run(T, ctx, sets, T.default_params(max_outer=3), planes=False)
    for k in (0, 5, 11, 23):
        s = sets[k]
        ref = O.rasl(s.imgs.astype(np.float64), s.tau0, s.ttype, s.m, s.n, O.Params(max_outer=3))
        assert out3["results"][k]["rank"] == ref.rank
        assert O.tau_error(out3["tau"][k].ravel(), ref.tau.ravel()) <= 1e-3


def test_rasl_host_and_device_images_agree(T, ctx):
    sets = _sets(3, 8, 14, 14, 6, 900)
    imgs = np.stack([s.imgs for s in sets])
    tau0 = np.stack([s.tau0 for s in sets])
    a = ctx.rasl(imgs, 14, 14, tau0, 6, T.default_params(max_outer=2))
    b = ctx.rasl(torch.from_numpy(imgs).cuda(), 14, 14, tau0, 6, T.default_params(max_outer=2))
    np.testing.assert_array_equal(a["tau"], b["tau"])
    assert a["kernel_ms"] > 0


def test_rasl_edge_cases(T, ctx):
    sets = _sets(4, 6, 10, 10, 6, 950, corruption=0.0)
    imgs = np.stack([s.imgs for s in sets])
    tau0 = np.stack([s.tau0 for s in sets])
    imgs[1, 2, 5, 5:9] = np.nan           # a non-finite sample under image 2's window
    imgs[2, 3] = 0.5                      # a constant image: its Gram block is singular
    imgs[3, :] = 0.0                      # an all-zero set: a column of norm zero
    out = ctx.rasl(imgs, 10, 10, tau0, 6, T.default_params(max_outer=2))
    st = [r["status"] for r in out["results"]]
    assert st[0] in (0, 1, 2) and st[1:] == [-1, -2, -3], st
    # the failed sets keep their starting transforms
    np.testing.assert_array_equal(out["tau"][3], tau0[3])
    # argument checks (nothing is launched)
    with pytest.raises(T.TiltError):
        ctx.rasl(np.zeros((1, 129, 12, 12), np.float32), 10, 10, np.zeros((1, 129, 6)), 6)
    with pytest.raises(T.TiltError):
        ctx.rasl(np.zeros((1, 30, 12, 12), np.float32), 5, 5, np.zeros((1, 30, 6)), 6)
    bad = tau0.copy()
    bad[0, 0, 0] = np.inf
    with pytest.raises(T.TiltError):
        ctx.rasl(imgs, 10, 10, bad, 6)
    empty = ctx.rasl(np.zeros((0, 6, 12, 12), np.float32), 10, 10, np.zeros((0, 6, 6)), 6)
    assert empty["tau"].shape == (0, 6, 6) and empty["results"] == []
