"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, step by step and end
to end.  Tolerances: per-step relative Frobenius error <= 1e-5 (the FP32 kernels against
FP64 on identical FP32 inputs); end to end ||tau_gpu - tau_oracle|| / ||tau_oracle|| <= 1e-3
and identical numerical rank of A at 1e-3 sigma_max."""
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
    c = T.Context(0)
    yield c
    c.close()


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a, np.float64) - b) / (nb if nb > 0 else 1.0)


def _patch(seed, m, n, ttype, theta=12.0):
    rng = np.random.default_rng(seed)
    p = synth.make_patch(rng, m, n, kind="lowrank" if seed % 2 else "checker", rank=3, period=7,
                         theta_deg=theta, skew=0.1, persp=(4e-4, -3e-4), ttype=ttype, corruption=0.05)
    jitter = rng.uniform(-0.05, 0.05, ttype) * np.r_[1, 1, 10, 1, 1, 10, 1e-3, 1e-3][:ttype]
    return p, p.tau0 + jitter


WARP_CASES = [(1, 50, 50, 6), (2, 37, 53, 6), (3, 64, 40, 8), (4, 120, 97, 6), (5, 9, 130, 8), (6, 200, 200, 8),
              (7, 2, 2, 6), (8, 512, 300, 8)]


@pytest.mark.parametrize("seed,m,n,ttype", WARP_CASES)
def test_warp_jacobian_parity(T, ctx, seed, m, n, ttype):
    p, tau = _patch(seed, m, n, ttype)
    img = torch.from_numpy(p.img).cuda()
    Dh_d, J_d, norm, oob = ctx.warp_jacobian(img, m, n, tau, ttype)
    Dh = T.from_long_layout(Dh_d.cpu().numpy(), m, n)
    J = T.jacobian_to_rows(J_d.cpu().numpy(), m, n, ttype)
    Dref, Jref, sref, oref = O.warp_normalise_jacobian(p.img.astype(np.float64), tau, ttype, m, n)
    assert oob == oref
    assert abs(norm - sref) <= 1e-6 * sref
    assert rel(Dh, Dref) <= 1e-5
    assert rel(J, Jref) <= 1e-5


@pytest.mark.parametrize("seed,m,n,ttype", [(11, 40, 56, 6), (12, 97, 64, 8), (13, 200, 200, 8)])
def test_gram_parity(T, ctx, seed, m, n, ttype):
    p, tau = _patch(seed, m, n, ttype)
    _, J_d, _, _ = ctx.warp_jacobian(torch.from_numpy(p.img).cuda(), m, n, tau, ttype)
    Q, G, Gi = ctx.gram(J_d, m, n, tau, ttype)
    J = T.jacobian_to_rows(J_d.cpu().numpy(), m, n, ttype).astype(np.float64)
    Qref = O.constraint_rows(tau, ttype, m, n)
    op = O.WtW(J, Qref)
    assert rel(Q, Qref) <= 1e-12
    assert rel(G, op.G) <= 1e-9
    assert rel(Gi, op.Ginv) <= 1e-7


SVT_CASES = [(21, 50, 50), (22, 64, 40), (23, 40, 64), (24, 120, 97), (25, 3, 2), (26, 2, 7), (27, 128, 128),
             (28, 200, 200), (29, 256, 130), (30, 512, 512), (31, 37, 1), (32, 1, 5)]


@pytest.mark.parametrize("seed,m,n", SVT_CASES)
def test_svt_parity(T, ctx, seed, m, n):
    rng = np.random.default_rng(seed)
    r = max(1, min(m, n) // 4)
    M = (rng.standard_normal((m, r)) @ rng.standard_normal((r, n)) / math.sqrt(n)
         + 0.02 * rng.standard_normal((m, n))).astype(np.float32)
    s = np.linalg.svd(M.astype(np.float64), compute_uv=False)
    eps = float(s[min(len(s) - 1, r)] * 1.5)
    A_d, sig, sweeps = ctx.svt(torch.from_numpy(T.to_long_layout(M)).cuda(), m, n, eps)
    A = T.from_long_layout(A_d.cpu().numpy(), m, n)
    Aref = O.svt(M.astype(np.float64), eps)[0]
    assert rel(A, Aref) <= 1e-5, (rel(A, Aref), sweeps)
    assert rel(np.sort(sig)[::-1], s) <= 1e-5
    assert sweeps < 40


def test_svt_edge_cases(T, ctx):
    # zero matrix, threshold above every singular value, threshold zero (A = M)
    m, n = 33, 21
    Z = np.zeros((m, n), np.float32)
    A_d, sig, _ = ctx.svt(torch.from_numpy(T.to_long_layout(Z)).cuda(), m, n, 0.1)
    assert np.all(A_d.cpu().numpy() == 0) and np.all(sig == 0)
    rng = np.random.default_rng(0)
    M = rng.standard_normal((m, n)).astype(np.float32)
    A_d, _, _ = ctx.svt(torch.from_numpy(T.to_long_layout(M)).cuda(), m, n, 1e3)
    assert np.all(A_d.cpu().numpy() == 0)
    A_d, _, _ = ctx.svt(torch.from_numpy(T.to_long_layout(M)).cuda(), m, n, 0.0)
    assert rel(T.from_long_layout(A_d.cpu().numpy(), m, n), M.astype(np.float64)) <= 1e-5


def _inner_inputs(T, ctx, seed, m, n, ttype):
    p, tau = _patch(seed, m, n, ttype, theta=4.0)
    Dh_d, J_d, _, _ = ctx.warp_jacobian(torch.from_numpy(p.img).cuda(), m, n, tau, ttype)
    Dh = T.from_long_layout(Dh_d.cpu().numpy(), m, n).astype(np.float64)
    J = T.jacobian_to_rows(J_d.cpu().numpy(), m, n, ttype).astype(np.float64)
    return tau, Dh_d, J_d, Dh, J


@pytest.mark.parametrize("seed,m,n,ttype", [(41, 50, 50, 6), (42, 37, 61, 8), (43, 120, 97, 6), (44, 200, 160, 8)])
def test_one_inner_iteration_parity(T, ctx, seed, m, n, ttype):
    # one LADMAP iteration from the cold start A = D_hat, E = Y = 0 (K2 + K3 + K4)
    tau, Dh_d, J_d, Dh, J = _inner_inputs(T, ctx, seed, m, n, ttype)
    mu0 = O.default_mu0(Dh)
    prm = T.default_params(max_inner=1)
    A_d = Dh_d.clone()
    E_d = torch.zeros_like(Dh_d)
    Y_d = torch.zeros_like(Dh_d)
    out = ctx.inner(Dh_d, J_d, m, n, tau, ttype, prm, mu0, A_d, E_d, Y_d)
    Q = O.constraint_rows(tau, ttype, m, n)
    lam = 1 / math.sqrt(max(m, n))
    ref = O.inner_ladmap(Dh, J, Q, lam, Dh, 0 * Dh, 0 * Dh, O.Params(max_inner=1), mu0=mu0)
    assert out["iters"] == 1
    # every result of one iteration at the per-kernel bound: relative Frobenius error <= 1e-5
    # (measured on these cases: A <= 4.1e-7, E exact, Y <= 1.1e-7, dtau <= 1.7e-6,
    # c1 and c2 <= 5e-8)
    for name, dev, want in (("A", A_d, ref.A), ("E", E_d, ref.E), ("Y", Y_d, ref.Yt)):
        got = T.from_long_layout(dev.cpu().numpy(), m, n)
        assert rel(got, want) <= 1e-5, (name, rel(got, want))
    dt_ref = O.delta_tau(O.WtW(J, Q), ref.A, ref.E, Dh)
    assert rel(out["dtau"], dt_ref) <= 1e-5, rel(out["dtau"], dt_ref)
    assert abs(out["c1"] - ref.c1) <= 1e-5 * ref.c1 and abs(out["c2"] - ref.c2) <= 1e-5 * ref.c2


@pytest.mark.parametrize("seed,m,n,ttype", [(51, 50, 50, 6), (52, 64, 45, 8), (53, 120, 110, 6),
                                            (54, 200, 170, 8)])
def test_inner_loop_parity(T, ctx, seed, m, n, ttype):
    # The 200 x 170 window runs its dense products (warm start, SVT coefficients and
    # reconstruction) on the tensor cores in 3xTF32, whose error per product (~1e-6 relative,
    # the probe of the product engine measured 5e-7 to 1.4e-6) is about ten times that of the
    # FP32 SIMT products of the smaller windows; carried through the loop it left E at 1.7e-4
    # and dtau at 1.1e-4 relative (measured), so those two are held to 1e-3 there, everything
    # else as below.
    # the whole inner loop to convergence: the FP32 rounding of every iteration (about
    # 1e-7 relative, see the one-iteration test) carries into the next over 56-73
    # iterations, so the converged A, E and dtau are compared at 1e-4 relative (measured:
    # A <= 2.9e-6, E <= 2.2e-5 relative to ||E|| -- E's small entries sit at the threshold
    # lam/mu --, dtau <= 1.5e-5), and the iteration counts agree to one (a stopping test that
    # lands within rounding of its threshold may flip)
    tau, Dh_d, J_d, Dh, J = _inner_inputs(T, ctx, seed, m, n, ttype)
    mu0 = O.default_mu0(Dh)
    A_d, E_d, Y_d = Dh_d.clone(), torch.zeros_like(Dh_d), torch.zeros_like(Dh_d)
    out = ctx.inner(Dh_d, J_d, m, n, tau, ttype, T.default_params(), mu0, A_d, E_d, Y_d)
    Q = O.constraint_rows(tau, ttype, m, n)
    lam = 1 / math.sqrt(max(m, n))
    ref = O.inner_ladmap(Dh, J, Q, lam, Dh, 0 * Dh, 0 * Dh, O.Params(), mu0=mu0)
    assert ref.converged
    A = T.from_long_layout(A_d.cpu().numpy(), m, n)
    E = T.from_long_layout(E_d.cpu().numpy(), m, n)
    tc_window = min(m, n) >= 160
    assert rel(A, ref.A) <= 1e-4, rel(A, ref.A)
    assert rel(E, ref.E) <= (1e-3 if tc_window else 1e-4), rel(E, ref.E)
    dt_ref = O.delta_tau(O.WtW(J, Q), ref.A, ref.E, Dh)
    assert rel(out["dtau"], dt_ref) <= (1e-3 if tc_window else 1e-4), rel(out["dtau"], dt_ref)
    assert abs(out["iters"] - ref.iters) <= 1, (out["iters"], ref.iters)
    assert O.numerical_rank(A) == O.numerical_rank(ref.A)


def _solve(ctx, T, patches, params=None, on_device=True):
    items = [(torch.from_numpy(p.img).cuda() if on_device else p.img, p.m, p.n, p.tau0, p.ttype) for p in patches]
    tickets = ctx.submit_batch(items, params, on_device=on_device)
    return [ctx.wait(t, 600000, with_planes=True, m=p.m, n=p.n) for t, p in zip(tickets, patches)]


def test_end_to_end_small_affine(T, ctx):
    # the 50 x 50 FP64 case: rank-3 texture, 20 deg, skew 0.15, 5 % corruption, inner tol 1e-7
    p = synth.small_affine()
    prm = T.default_params(eps1=1e-7)
    r = _solve(ctx, T, [p], prm)[0]   # the 50 x 50 case states an inner tolerance of 1e-7
    ref = O.tilt(p.img.astype(np.float64), p.tau0, p.ttype, p.m, p.n, O.Params(eps1=1e-7))
    assert r["status"] in (0, 1, 2)
    assert O.tau_error(r["tau"], ref.tau) <= 1e-3
    assert r["rank"] == ref.rank
    assert r["outer_iters"] == ref.outer_iters


@pytest.mark.parametrize("first", [0, 7])
def test_end_to_end_mixed_batch_sample(T, ctx, first):
    patches = synth.mixed_affine_batch(4, first=first)
    res = _solve(ctx, T, patches)
    for p, r in zip(patches, res):
        ref = O.tilt(p.img.astype(np.float64), p.tau0, p.ttype, p.m, p.n, O.Params())
        assert O.tau_error(r["tau"], ref.tau) <= 1e-3, (p.m, p.n, r["tau"], ref.tau)
        assert r["rank"] == ref.rank


@pytest.mark.parametrize("seed,m,n", [(61, 64, 50), (62, 200, 160)])
def test_warm_svt_reorthonormalises_a_drifted_v(T, ctx, seed, m, n):
    # the solver's warm start (Sec. 5) from the right singular vectors of a nearby matrix: an
    # orthonormal V is used as it is; a V whose column norms drifted past 1e-4 is first
    # re-orthonormalised in FP64; either way the SVT matches the oracle's and V comes back
    # orthonormal.  (200 x 160 runs the warm-start product on the tensor cores.)
    rng = np.random.default_rng(seed)
    r = max(2, n // 8)
    M0 = rng.standard_normal((m, r)) @ rng.standard_normal((r, n)) / math.sqrt(n) + 0.02 * rng.standard_normal((m, n))
    M = (M0 + 0.01 * rng.standard_normal((m, n))).astype(np.float32)
    V0 = np.linalg.svd(M0)[2].T                      # n x n (m >= n: X = M)
    s = np.linalg.svd(M.astype(np.float64), compute_uv=False)
    eps = float(s[r] * 1.5)
    Aref = O.svt(M.astype(np.float64), eps)[0]
    M_t = torch.from_numpy(T.to_long_layout(M)).cuda()
    _, _, cold_sweeps = ctx.svt(M_t, m, n, eps)
    for drift, want_reorth in ((0.0, 0), (3e-3, 1)):
        V = V0 @ (np.eye(n) + drift * rng.standard_normal((n, n)))
        V_t = torch.from_numpy(np.ascontiguousarray(V.T).astype(np.float32).reshape(-1)).cuda()   # column-major
        A_d, sig, sweeps, reorth = ctx.svt_warm(M_t, m, n, eps, V_t)
        assert reorth == want_reorth
        assert rel(T.from_long_layout(A_d.cpu().numpy(), m, n), Aref) <= 1e-5
        assert rel(np.sort(sig)[::-1], s) <= 1e-5
        Vn = V_t.cpu().numpy().reshape(n, n).T.astype(np.float64)
        assert np.abs(Vn.T @ Vn - np.eye(n)).max() <= 1e-5
        assert sweeps < cold_sweeps


@pytest.mark.parametrize("seed,m,n", [(71, 9, 6), (72, 64, 48), (73, 120, 100), (74, 40, 70)])
def test_cayley_warm_start_step_parity(T, ctx, seed, m, n):
    # one step of Algorithm 2 (Sec. 5, Appendix A) from the exact factors of a nearby matrix:
    # f'(0), f''(0), t and the curve point U(t), Sigma(t), V(t) against the oracle's.  The
    # step works on X (M, or M^T when m < n: U and V exchange roles)
    rng = np.random.default_rng(seed)
    M0 = rng.standard_normal((m, n))
    M = (M0 + 0.03 * rng.standard_normal((m, n))).astype(np.float32)
    X0 = M0 if m >= n else M0.T
    X = M.astype(np.float64) if m >= n else M.T.astype(np.float64)
    U0, s0, Vt0 = np.linalg.svd(X0, full_matrices=False)
    U0, s0, V0 = U0.astype(np.float32).astype(np.float64), s0.astype(np.float32).astype(np.float64), \
        Vt0.T.astype(np.float32).astype(np.float64)
    _, _, _, f1, f2 = O.svdws_derivatives(X, U0, s0, V0)
    ws = O.svd_warm_start(X, U0, s0, V0)
    R, C = X.shape
    U_t = torch.from_numpy(np.ascontiguousarray(U0.T).astype(np.float32).reshape(-1)).cuda()
    S_t = torch.from_numpy(s0.astype(np.float32)).cuda()
    V_t = torch.from_numpy(np.ascontiguousarray(V0.T).astype(np.float32).reshape(-1)).cuda()
    out = ctx.svd_cayley(torch.from_numpy(T.to_long_layout(M)).cuda(), m, n, U_t, S_t, V_t)
    assert abs(out["f1"] - f1) <= 1e-4 * abs(f1) and abs(out["f2"] - f2) <= 1e-4 * abs(f2), (out, f1, f2)
    assert abs(out["t"] - (-f1 / f2)) <= 1e-4 * abs(f1 / f2)
    assert out["accepted"] == (ws is not None)
    Ut = U_t.cpu().numpy().reshape(C, R).T.astype(np.float64)
    St = S_t.cpu().numpy().astype(np.float64)
    Vt = V_t.cpu().numpy().reshape(C, C).T.astype(np.float64)
    for got, want in ((Ut, ws[0]), (St, ws[1]), (Vt, ws[2]), ((Ut * St) @ Vt.T, (ws[0] * ws[1]) @ ws[2].T)):
        assert rel(got, want) <= 1e-5, rel(got, want)
    # the curve keeps the factors orthonormal (Sec. 5.1, property 2)
    assert np.abs(Ut.T @ Ut - np.eye(C)).max() <= 1e-5 and np.abs(Vt.T @ Vt - np.eye(C)).max() <= 1e-5


@pytest.mark.parametrize("seed,m,n,ttype", [(51, 50, 50, 6), (52, 64, 45, 8)])
def test_inner_loop_with_the_papers_svd_warm_start(T, ctx, seed, m, n, ttype):
    # the inner loop with Algorithm 2 (svd_ws = 1, gate eps_svd = 0.05) against the oracle's
    # inner loop with the same warm start: the approximate SVDs change the trajectory (the
    # oracle needs 129 / 135 iterations here against 60 / 56 with exact SVDs), and FP32 can
    # flip a gate or acceptance decision that FP64 takes the other way, so iteration and
    # step counts are compared to 10 % and A, E at 1e-3 relative
    tau, Dh_d, J_d, Dh, J = _inner_inputs(T, ctx, seed, m, n, ttype)
    mu0 = O.default_mu0(Dh)
    A_d, E_d, Y_d = Dh_d.clone(), torch.zeros_like(Dh_d), torch.zeros_like(Dh_d)
    out = ctx.inner(Dh_d, J_d, m, n, tau, ttype, T.default_params(svd_ws=1, eps_svd=0.05), mu0, A_d, E_d, Y_d)
    Q = O.constraint_rows(tau, ttype, m, n)
    lam = 1 / math.sqrt(max(m, n))
    ref = O.inner_ladmap(Dh, J, Q, lam, Dh, 0 * Dh, 0 * Dh, O.Params(svd_warm=True, eps_svd=0.05), mu0=mu0)
    assert ref.converged and ref.svd_warm_used > 0
    assert abs(out["iters"] - ref.iters) <= max(3, ref.iters // 10), (out["iters"], ref.iters)
    assert abs(out["cayley_steps"] - ref.svd_warm_used) <= max(3, ref.svd_warm_used // 10), \
        (out["cayley_steps"], ref.svd_warm_used)
    A = T.from_long_layout(A_d.cpu().numpy(), m, n)
    E = T.from_long_layout(E_d.cpu().numpy(), m, n)
    assert rel(A, ref.A) <= 1e-3 and rel(E, ref.E) <= 1e-3, (rel(A, ref.A), rel(E, ref.E))
