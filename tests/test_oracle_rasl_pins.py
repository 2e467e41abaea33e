"""Pins for the oracle's RASL variant (Sec. 1: TILT's model with one image per column of the
data matrix).  Each checks it against finite differences, a closed form, the optimality
conditions of the inner problem, or the known alignment of a rendered image set."""
import math

import numpy as np
import pytest

from oracle import tilt_oracle as O
from paper_1205_5351_gb300 import synth


def _kink_free_set(nimg, m, n, ttype, seed=3):
    """A rendered set and transforms near tau0 at which no window sample lies within 1e-4 px
    of a bilinear cell boundary (the interpolant has kinks there)."""
    st = synth.rasl_set(np.random.default_rng(seed), nimg, m, n, ttype=ttype, corruption=0.0)
    U, V = O.window_uv(m, n)
    rng = np.random.default_rng(seed + 100)
    taus = []
    for i in range(nimg):
        for _ in range(200):
            t = st.tau0[i] + np.r_[rng.uniform(-0.03, 0.03, 2), rng.uniform(-0.4, 0.4),
                                   rng.uniform(-0.03, 0.03, 2), rng.uniform(-0.4, 0.4),
                                   rng.uniform(-2e-4, 2e-4, ttype - 6)]
            x, y, _, _ = O.map_points(t, ttype, U, V)
            if np.minimum(np.abs(x - np.round(x)), np.abs(y - np.round(y))).min() > 1e-4:
                break
        else:
            raise AssertionError("no kink-free tau found")
        taus.append(t)
    return st.imgs.astype(np.float64), np.array(taus)


@pytest.mark.parametrize("ttype", [O.AFFINE, O.PROJECTIVE])
def test_stacked_jacobian_matches_central_differences(ttype):
    # the block of image i in the stacked Jacobian is d vec(D_hat) / d tau_i (R18): central
    # differences of the whole data matrix, which also show that tau_i moves column i only
    nimg, m, n = 4, 9, 11
    imgs, taus = _kink_free_set(nimg, m, n, ttype)
    D, Js, norms, _ = O.rasl_warp(imgs, taus, ttype, m, n)
    Jb = O.rasl_stacked_jacobian(Js)
    p = ttype
    assert Jb.shape == (m * n * nimg, nimg * p)
    for i in range(nimg):
        for k in range(p):
            h = 1e-7 if k < 6 else 1e-10
            tp, tm = taus.copy(), taus.copy()
            tp[i, k] += h
            tm[i, k] -= h
            Dp = O.rasl_warp(imgs, tp, ttype, m, n)[0]
            Dm = O.rasl_warp(imgs, tm, ttype, m, n)[0]
            fd = ((Dp - Dm) / (2 * h)).ravel()
            col = Jb[:, i * p + k]
            assert np.linalg.norm(fd - col) <= 1e-6 * np.linalg.norm(col), (i, k)
            others = np.delete(Dp - Dm, i, axis=1)
            assert np.abs(others).max() == 0.0
    # every column has unit norm and its block is orthogonal to it (the norm is constant)
    np.testing.assert_allclose(np.linalg.norm(D, axis=0), 1.0, rtol=1e-14)
    for i, J in enumerate(Js):
        assert np.abs(D[:, i] @ J).max() < 1e-12 * np.abs(J).max() * m * n
    assert np.all(norms > 0)


def test_constraint_rows_fix_the_mean_transform():
    # Q = [I ... I]: Q dtau is the sum of the increments; the stacked least-squares system
    # [J; Q] dtau = [r; 0] (Eq. two_linear_constraint) solved by LAPACK matches the operator's
    rng = np.random.default_rng(5)
    nimg, mn, p = 5, 30, 6
    Js = [rng.standard_normal((mn, p)) for _ in range(nimg)]
    Q = O.rasl_constraint_rows(nimg, p)
    dt = rng.standard_normal(nimg * p)
    np.testing.assert_allclose(Q @ dt, dt.reshape(nimg, p).sum(axis=0), rtol=1e-14)
    X = rng.standard_normal((mn, nimg))
    op = O.rasl_operator(Js)
    Jb = O.rasl_stacked_jacobian(Js)
    ref = np.linalg.lstsq(np.vstack([Jb, Q]), np.r_[X.ravel(), np.zeros(p)], rcond=None)[0]
    np.testing.assert_allclose(op.coeffs(X), ref, rtol=1e-10, atol=1e-12)
    # W r = 0 exactly for r = J dtau with Q dtau = 0 (Proposition 1, Sec. 4.3)
    null = np.linalg.svd(Q)[2][p:].T
    r = (Jb @ (null @ rng.standard_normal(nimg * p - p))).reshape(mn, nimg)
    assert np.abs(op(r)).max() < 1e-10 * np.abs(r).max()


def test_rasl_inner_loop_kkt():
    # the inner problem of one outer step, solved tightly: the KKT conditions of
    # min ||A||_* + lam ||E||_1 s.t. D_hat + J dtau = A + E, Q dtau = 0
    st = synth.rasl_set(np.random.default_rng(11), 6, 12, 12, corruption=0.05)
    imgs = st.imgs.astype(np.float64)
    D, Js, _, _ = O.rasl_warp(imgs, st.tau0, st.ttype, st.m, st.n)
    op = O.rasl_operator(Js)
    lam = 1 / math.sqrt(D.shape[0])
    prm = O.Params(eps1=1e-10, eps2=1e-4, max_inner=20000)
    res = O.inner_ladmap(D, None, None, lam, D, np.zeros_like(D), np.zeros_like(D), prm, op=op)
    assert res.converged
    # Cond2 bounds the dual residual by eps2 d0 (Frobenius), d0 = ||W^T W D_hat||_F
    tol = prm.eps2 * float(np.linalg.norm(op(D)))
    Yt = res.Yt
    U, s, Vt = np.linalg.svd(res.A, full_matrices=False)
    r = int(np.sum(s > 1e-6 * s[0]))
    assert np.linalg.norm(Yt, 2) <= 1 + tol
    np.testing.assert_allclose(U[:, :r].T @ (-Yt) @ Vt[:r].T, np.eye(r), atol=tol)
    supp = np.abs(res.E) > 1e-9
    assert supp.sum() > 0
    np.testing.assert_allclose(-Yt[supp], lam * np.sign(res.E[supp]), atol=tol)
    assert np.abs(Yt[~supp]).max() <= lam + tol
    dt = op.coeffs(res.A + res.E - D)
    Jb = O.rasl_stacked_jacobian(Js)
    assert np.linalg.norm(D.ravel() + Jb @ dt - (res.A + res.E).ravel()) < 1e-7
    assert np.abs(dt.reshape(6, -1).sum(axis=0)).max() < 1e-7 * max(1.0, np.abs(dt).max())


def _corner_spread(taus, st):
    """Largest distance of a window corner, mapped into texture coordinates through
    tau_true_i^-1 o tau_i, from the mean over the images: 0 when the set is aligned."""
    U, V = O.corner_uv(st.m, st.n)
    pts = []
    for t, tt in zip(taus, st.tau_true):
        x, y, _, _ = O.map_points(t, st.ttype, U, V)
        H = np.array([[tt[0], tt[1], tt[2]], [tt[3], tt[4], tt[5]], [0.0, 0.0, 1.0]])
        q = np.linalg.solve(H, np.vstack([x, y, np.ones(4)]))
        pts.append((q[:2] / q[2]).T)
    pts = np.array(pts)
    return float(np.max(np.linalg.norm(pts - pts.mean(axis=0), axis=2)))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_rasl_aligns_a_rendered_set(seed):
    # ten views of one rank-2 texture, each under its own similarity: RASL must bring the
    # windows into register at least as well as the rendering transforms themselves do
    # (nuclear norm of the aligned data matrix no larger than at tau_true) and shrink the
    # misalignment of the window corners several-fold
    st = synth.rasl_set(np.random.default_rng(synth.seed_for(9, seed)), 10, 20, 20, corruption=0.0)
    imgs = st.imgs.astype(np.float64)
    res = O.rasl(imgs, st.tau0, st.ttype, st.m, st.n, O.Params(max_outer=15))
    nuc = {}
    for name, T in (("tau0", st.tau0), ("true", st.tau_true), ("rasl", res.tau)):
        D = O.rasl_warp(imgs, T, st.ttype, st.m, st.n)[0]
        nuc[name] = float(np.linalg.svd(D, compute_uv=False).sum())
    assert nuc["rasl"] <= nuc["true"] * (1 + 1e-3), nuc
    assert nuc["tau0"] - nuc["true"] > 0.2
    before, after = _corner_spread(st.tau0, st), _corner_spread(res.tau, st)
    assert after < before / 3, (before, after)
    # the increments sum to zero at every step, so the mean transform stays where it started
    np.testing.assert_allclose(res.tau.mean(axis=0), st.tau0.mean(axis=0), atol=5e-3)
