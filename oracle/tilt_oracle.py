"""FP64 CPU oracle for TILT solved by LADMAP with warm starts (Ren & Lin, arXiv 1205.5351).

TEST INFRASTRUCTURE ONLY.  Only tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module.  It shares no code with the CUDA path and
never imports it.  Plain NumPy in float64; library primitives used as steps: matrix
products, ``numpy.linalg.svd`` (LAPACK), ``numpy.linalg.inv`` / ``solve``.

What it computes (paper section / equation named on every function):

* Step 1 of Algorithm 1 -- warp D o tau, normalise, Jacobian of the normalised warp.
* The reformulated inner problem (Eq. TILT_LADMAP) with the additional constraints
  Q dtau = 0 (Sec. 4.3, Eq. add_constraints, W, WTW_property), solved by LADMAP
  (Eqs. A, E, Y, mu, rho) in the form of Eq. newvars2 with the Y-in-span trick (Sec. 4.2),
  the variable warm start (Eq. warm_start, Eq. Y_new_warmstart) and the stopping rules
  (Eqs. Cond1, Cond2).
* Singular value thresholding (Eqs. A_1, S_operator) by an exact LAPACK SVD; optionally
  the SVD warm start of Algorithm 2 (Sec. 5, Appendix A).
* Steps 3-4 of Algorithm 1: dtau (Eq. Delta_tau, stacked with Q as in
  Eq. two_linear_constraint) and tau <- tau + dtau.
* The comparison method of Sec. 2.2: the ADM of Zhang et al. for the inner loop
  (Eq. TILT_3), with the three blocks A, E, dtau updated in turn and mu <- rho mu.
* RASL (Sec. 1): the same model with one image per column of the data matrix, so the
  Jacobian of vec(D_hat) is block-diagonal (one block of p columns per image); the same
  W^T W (with constraint rows that fix the set's mean transform), LADMAP inner loop and
  outer loop.

Readings of points where the paper is silent or inconsistent (each is listed in the
design notes of the repository):

* R1  Y update uses +mu (Eq. Y), not the minus sign printed inside Algorithm 1.
* R2  N_k is centred at E_k (Eq. E / Sec. 4.2), not at A_{k+1} as printed in Sec. 4.3.
* R3  eta = 1 for both blocks (Sec. 3.2 uses ||J_perp|| = 1).
* R4  Pixel (i, j) of an m x n window has centred coordinates u = j - (n-1)/2,
      v = i - (m-1)/2; affine tau = [a11 a12 a13 a21 a22 a23] maps to
      x = a11 u + a12 v + a13, y = a21 u + a22 v + a23; projective tau = [h1..h8] maps to
      x = (h1 u + h2 v + h3)/(h7 u + h8 v + 1), y = (h4 u + h5 v + h6)/(same).
      x indexes image columns, y image rows.
* R5  D o tau is the bilinear interpolant of the image; its gradient is the exact
      gradient of that interpolant on the cell floor(x), floor(y) (the last cell for
      x = W-1 or y = H-1).  Outside the image the coordinate is clamped to the edge and
      the derivative along a clamped axis is zero; such pixels are counted.
* R6  Q has l = 3 rows: the derivatives w.r.t. tau of the centroid (x, y) of the four
      window corners mapped by tau and of the signed area of the mapped quadrilateral,
      the area row divided by (m-1)(n-1).
* R7  mu_0 = 1.25 / ||D_hat||_2, reset at every outer step (Algorithm 1 lists mu_0 among
      the initial conditions of each inner loop); mu_max = 1e10; rho_0 = 1.5 and
      eps_2 = 0.1 (the rho rule of Eq. rho only lets mu grow while c2 < eps_2, so a small
      eps_2 freezes mu); eps_1 = 1e-5; the Cond1 denominator and numerator use W^T W (the
      operator the iteration carries) in place of J_perp.
* R8  The outer loop stops when dtau moves no corner of the window by more than
      outer_tol pixels, or after max_outer steps.
* R9  A_0 is the normalised D o tau^0.
* R10 The SVD runs on the m x n matrix as given; singular values are non-negative.
* R16 ADM (Sec. 2.2) parameters, not printed: mu_0 = 1.25/||D||_2, rho = 1.25, stop when
      ||D + J dtau - A - E||_F / ||D||_F < 1e-7 (the usual inexact-ALM settings of the cited
      line of work).
* R18 RASL (Sec. 1 states only that it shares TILT's model with one image per column):
      column i of D_hat is image i warped by tau_i over the m x n window (pixels in row-major
      order) divided by its own Frobenius norm, J_i the Jacobian of that normalised column
      (the quotient rule of Step 1, per column); the Jacobian of vec(D_hat) in the stacked
      parameters is block-diagonal; additional constraints Q = [I_p ... I_p], i.e. the
      increments dtau_i sum to zero: the low-rank objective cannot see a transform applied to
      every image at once, and without these rows that common part of dtau swings by about a
      pixel from one outer step to the next (TILT's Q fixes the window's position and size for
      the same reason); W^T W and dtau as in Sec. 4.3 with these J and Q;
      lambda = 1/sqrt(max(mn, N)); LADMAP parameters, warm starts and mu_0 as for TILT (R7,
      R9); the outer loop stops when no window corner of any image moves by outer_tol pixels
      (R8 per image).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

AFFINE = 6
PROJECTIVE = 8


# ============================================================================ parameters
@dataclasses.dataclass
class Params:
    """Solver parameters (Algorithm 1 inputs; values the paper leaves open are readings)."""

    lam: float = -1.0            # <= 0 -> 1/sqrt(max(m, n))
    eps1: float = 1e-5           # Cond1 threshold
    eps2: float = 0.1            # Cond2 / rho threshold
    rho0: float = 1.5
    mu0: float = -1.0            # <= 0 -> 1.25/||D_hat||_2
    mu_max: float = 1e10
    max_inner: int = 500
    max_outer: int = 10
    outer_tol: float = 1e-2      # pixels of corner displacement (R8)
    svd_warm: bool = False       # Algorithm 2 (Cayley-curve warm start) on/off
    eps_svd: float = 0.05        # relative gate ||M_k - M_{k-1}||_F < eps_svd * ||M_k||_F
    use_q: bool = True           # additional constraints Q dtau = 0 (Sec. 4.3)


# ============================================================================ warp (Step 1)
def window_uv(m: int, n: int):
    """Centred window coordinates (R4): arrays U (column offset) and V (row offset), m x n."""
    u = np.arange(n, dtype=np.float64) - (n - 1) / 2.0
    v = np.arange(m, dtype=np.float64) - (m - 1) / 2.0
    U, V = np.meshgrid(u, v)
    return U, V


def map_points(tau: np.ndarray, ttype: int, U: np.ndarray, V: np.ndarray):
    """tau(u, v) -> (x, y) and the derivatives dx/dtau, dy/dtau (R4), shape (..., p)."""
    t = np.asarray(tau, dtype=np.float64)
    if ttype == AFFINE:
        x = t[0] * U + t[1] * V + t[2]
        y = t[3] * U + t[4] * V + t[5]
        one = np.ones_like(U)
        zero = np.zeros_like(U)
        dx = np.stack([U, V, one, zero, zero, zero], axis=-1)
        dy = np.stack([zero, zero, zero, U, V, one], axis=-1)
        return x, y, dx, dy
    if ttype == PROJECTIVE:
        nx = t[0] * U + t[1] * V + t[2]
        ny = t[3] * U + t[4] * V + t[5]
        den = t[6] * U + t[7] * V + 1.0
        x = nx / den
        y = ny / den
        zero = np.zeros_like(U)
        dx = np.stack([U / den, V / den, 1.0 / den, zero, zero, zero, -x * U / den, -x * V / den], axis=-1)
        dy = np.stack([zero, zero, zero, U / den, V / den, 1.0 / den, -y * U / den, -y * V / den], axis=-1)
        return x, y, dx, dy
    raise ValueError("ttype must be 6 (affine) or 8 (projective)")


def bilinear(img: np.ndarray, x: np.ndarray, y: np.ndarray):
    """Bilinear interpolant of ``img`` at (x, y) with its exact gradient (R5).

    Returns value, d/dx, d/dy and the out-of-bounds mask."""
    img = np.asarray(img, dtype=np.float64)
    H, W = img.shape
    inx = (x >= 0.0) & (x <= W - 1.0)
    iny = (y >= 0.0) & (y <= H - 1.0)
    xc = np.clip(x, 0.0, W - 1.0)
    yc = np.clip(y, 0.0, H - 1.0)
    x0 = np.minimum(np.floor(xc), W - 2.0)
    y0 = np.minimum(np.floor(yc), H - 2.0)
    fx = xc - x0
    fy = yc - y0
    xi = x0.astype(np.int64)
    yi = y0.astype(np.int64)
    I00 = img[yi, xi]
    I01 = img[yi, xi + 1]
    I10 = img[yi + 1, xi]
    I11 = img[yi + 1, xi + 1]
    val = (1.0 - fy) * ((1.0 - fx) * I00 + fx * I01) + fy * ((1.0 - fx) * I10 + fx * I11)
    gx = ((1.0 - fy) * (I01 - I00) + fy * (I11 - I10)) * inx
    gy = ((1.0 - fx) * (I10 - I00) + fx * (I11 - I01)) * iny
    return val, gx, gy, ~(inx & iny)


def warp(img, tau, ttype, m, n):
    """D o tau (m x n) and the raw Jacobian d(D o tau)/dtau (mn x p, row-major pixels)."""
    U, V = window_uv(m, n)
    x, y, dx, dy = map_points(tau, ttype, U, V)
    val, gx, gy, oob = bilinear(img, x, y)
    Jraw = gx[..., None] * dx + gy[..., None] * dy
    return val, Jraw.reshape(m * n, -1), int(oob.sum())


def normalise_jacobian(Dtau: np.ndarray, Jraw: np.ndarray):
    """Algorithm 1, Step 1: D_hat = D o tau / ||D o tau||_F and the Jacobian of the
    normalised warp, J = (Jraw - D_hat (D_hat^T Jraw)) / ||D o tau||_F (quotient rule)."""
    s = float(np.linalg.norm(Dtau))
    Dhat = Dtau / s
    d = Dhat.reshape(-1)
    J = (Jraw - np.outer(d, d @ Jraw)) / s
    return Dhat, J, s


def warp_normalise_jacobian(img, tau, ttype, m, n):
    """Step 1 of Algorithm 1 at tau: (D_hat, J, ||D o tau||_F, out-of-bounds count)."""
    Dtau, Jraw, oob = warp(img, tau, ttype, m, n)
    Dhat, J, s = normalise_jacobian(Dtau, Jraw)
    return Dhat, J, s, oob


# ============================================================================ constraints Q (Sec. 4.3)
def corner_uv(m: int, n: int):
    a = (n - 1) / 2.0
    b = (m - 1) / 2.0
    U = np.array([-a, a, a, -a])
    V = np.array([-b, -b, b, b])
    return U, V


def constraint_rows(tau, ttype, m, n) -> np.ndarray:
    """Q (3 x p) of Eq. add_constraints under reading R6: linearised centroid and area of
    the window quadrilateral mapped by tau."""
    U, V = corner_uv(m, n)
    x, y, dx, dy = map_points(tau, ttype, U, V)
    qx = dx.mean(axis=0)
    qy = dy.mean(axis=0)
    xn, yn = np.roll(x, -1), np.roll(y, -1)
    dxn, dyn = np.roll(dx, -1, axis=0), np.roll(dy, -1, axis=0)
    darea = 0.5 * (dx * yn[:, None] + x[:, None] * dyn - dxn * y[:, None] - xn[:, None] * dy).sum(axis=0)
    return np.stack([qx, qy, darea / ((m - 1) * (n - 1))])


def corner_shift(tau, dtau, ttype, m, n) -> float:
    """Largest displacement, in pixels, of a window corner when tau becomes tau + dtau (R8)."""
    U, V = corner_uv(m, n)
    x0, y0, _, _ = map_points(tau, ttype, U, V)
    x1, y1, _, _ = map_points(np.asarray(tau) + np.asarray(dtau), ttype, U, V)
    return float(np.max(np.hypot(x1 - x0, y1 - y0)))


def polygon_area(x, y) -> float:
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


# ============================================================================ W^T W (Sec. 4.1, 4.3)
class WtW:
    """The operator W^T W = I - J (J^T J + Q^T Q)^{-1} J^T (Eq. WTW_property), applied to a
    vectorised matrix without forming it (Eq. Jperpv).  Q = None gives J_perp."""

    def __init__(self, J: np.ndarray, Q: np.ndarray | None):
        self.J = np.asarray(J, dtype=np.float64)
        G = self.J.T @ self.J
        if Q is not None:
            G = G + Q.T @ Q
        self.G = G
        self.Ginv = np.linalg.inv(G)

    def __call__(self, X: np.ndarray) -> np.ndarray:
        x = X.reshape(-1)
        return (x - self.J @ (self.Ginv @ (self.J.T @ x))).reshape(X.shape)

    def coeffs(self, X: np.ndarray) -> np.ndarray:
        """G^{-1} J^T vec(X): the dtau that the stacked system of Eq. two_linear_constraint
        assigns to a residual X (Eq. Delta_tau)."""
        return self.Ginv @ (self.J.T @ X.reshape(-1))


# ============================================================================ shrinkage operators
def soft_threshold(X: np.ndarray, eps: float) -> np.ndarray:
    """T_eps(x) = sgn(x) max(|x| - eps, 0), entrywise (Sec. 3.2)."""
    return np.sign(X) * np.maximum(np.abs(X) - eps, 0.0)


def svt(M: np.ndarray, eps: float, svd=None):
    """S_eps(M) = U T_eps(Sigma) V^T (Eqs. A_1, S_operator).  Returns (A, U, s, Vt) where
    (U, s, Vt) is the SVD used (exact LAPACK unless ``svd`` supplies one)."""
    if svd is None:
        U, s, Vt = np.linalg.svd(M, full_matrices=False)
    else:
        U, s, Vt = svd
        # a warm-started factorisation may carry negative diagonal entries (Sec. 5: the
        # sign of Sigma is free); fold the sign into U before thresholding.
        sg = np.where(s < 0, -1.0, 1.0)
        U = U * sg
        s = np.abs(s)
    A = (U * np.maximum(s - eps, 0.0)) @ Vt
    return A, U, s, Vt


# ============================================================================ SVD warm start (Alg. 2, App. A)
def svdws_derivatives(M, U, S, V):
    """Appendix A: projected gradients P_U, P_Sigma, P_V (Eqs. projected_gradient1-3) and
    f'(0), f''(0) of f(t) = 1/2 ||M - U(t) Sigma(t) V(t)^T||_F^2 along the curve of
    Eq. curve_to_search.  S is the (signed) diagonal as a vector."""
    X = (U * S) @ V.T                         # U Sigma V^T
    PU = X @ M.T - M @ X.T                    # m x m, antisymmetric
    PV = X.T @ M - M.T @ X                    # n x n, antisymmetric
    PS = S - np.einsum("ij,ij->j", U, M @ V)  # diag(Sigma - U^T M V)
    h0 = M - X
    UPSVt = (U * PS) @ V.T
    h1 = PU @ X + UPSVt - X @ PV
    Z = h1 + UPSVt
    h2 = -PU @ Z + Z @ PV
    f1 = float(np.sum(h0 * h1))
    f2 = float(np.sum(h1 * h1) + np.sum(h0 * h2))
    return PU, PS, PV, f1, f2


def cayley(P: np.ndarray, X: np.ndarray, t: float) -> np.ndarray:
    """X(t) = (I + t/2 P)^{-1} (I - t/2 P) X (Sec. 5.1, Wen-Yin curve)."""
    I = np.eye(P.shape[0])
    return np.linalg.solve(I + 0.5 * t * P, (I - 0.5 * t * P) @ X)


def curve_point(M, U, S, V, PU, PS, PV, t):
    """(U(t), Sigma(t), V(t)) of Eq. curve_to_search."""
    return cayley(PU, U, t), S - t * PS, cayley(PV, V, t)


def curve_objective(M, U, S, V) -> float:
    return 0.5 * float(np.sum((M - (U * S) @ V.T) ** 2))


def svd_warm_start(M, U, S, V):
    """One step of Algorithm 2 from the factors of M_{k-1}.  Returns (U, S, V) or None when
    the quadratic model has no minimiser or the step does not decrease f (reading: fall
    back to a full SVD)."""
    PU, PS, PV, f1, f2 = svdws_derivatives(M, U, S, V)
    if not (f2 > 0.0):
        return None
    t = -f1 / f2
    Ut, St, Vt_ = curve_point(M, U, S, V, PU, PS, PV, t)
    if curve_objective(M, Ut, St, Vt_) > curve_objective(M, U, S, V):
        return None
    return Ut, St, Vt_


# ============================================================================ inner loop (Sec. 3-5)
@dataclasses.dataclass
class InnerResult:
    A: np.ndarray
    E: np.ndarray
    Yt: np.ndarray
    iters: int
    converged: bool
    mu_trace: list
    c1: float
    c2: float
    sigma: np.ndarray            # singular values of the last M_k
    svd_warm_used: int = 0


def default_mu0(Dhat: np.ndarray) -> float:
    return 1.25 / float(np.linalg.norm(Dhat, 2))


def inner_ladmap(Dhat, J, Q, lam, A0, E0, Yt0, prm: Params, mu0: float | None = None,
                 trace: list | None = None, op=None) -> InnerResult:
    """LADMAP for min ||A||_* + lam ||E||_1 s.t. W^T W (A + E) = W^T W D_hat
    (Eq. reformulated_TILT2), in the form of Eq. newvars2 with readings R1-R3, R7.

    One iteration k:
        M_k   = A_k - Yt_k/mu_k - P_k,          P_k = W^T W (A_k + E_k - D_hat)
        A_k+1 = S_{1/mu_k}(M_k)
        N_k   = E_k - Yt_k/mu_k - W^T W (A_k+1 + E_k - D_hat)
        E_k+1 = T_{lam/mu_k}(N_k)
        P_k+1 = W^T W (A_k+1 + E_k+1 - D_hat);  Yt_k+1 = Yt_k + mu_k P_k+1
        c1 = ||P_k+1||_F / d0,  c2 = mu_k max(||A_k+1 - A_k||_F, ||E_k+1 - E_k||_F) / d0,
        d0 = ||W^T W D_hat||_F; rho = rho0 if c2 < eps2 else 1; mu_k+1 = min(mu_max, rho mu_k)
    and the loop stops when c1 < eps1 and c2 < eps2 (Eqs. Cond1, Cond2).
    ``op`` replaces WtW(J, Q) by a prepared operator (RASL: rasl_operator).
    """
    op = WtW(J, Q) if op is None else op
    A = np.array(A0, dtype=np.float64)
    E = np.array(E0, dtype=np.float64)
    Yt = op(np.asarray(Yt0, dtype=np.float64))           # Eq. Y_new_warmstart
    d0 = float(np.linalg.norm(op(Dhat)))
    mu = default_mu0(Dhat) if mu0 is None else float(mu0)
    P = op(A + E - Dhat)
    mus = []
    svd_prev = None
    M_prev = None
    warm_used = 0
    c1 = c2 = math.inf
    converged = False
    k = 0
    s = None
    for k in range(1, prm.max_inner + 1):
        mus.append(mu)
        M = A - Yt / mu - P
        svd = None
        if prm.svd_warm and svd_prev is not None and M_prev is not None:
            if np.linalg.norm(M - M_prev) < prm.eps_svd * np.linalg.norm(M):
                ws = svd_warm_start(M, *svd_prev)
                if ws is not None:
                    svd = (ws[0], ws[1], ws[2].T)
                    warm_used += 1
        A1, Uf, s, Vtf = svt(M, 1.0 / mu, svd)
        if prm.svd_warm:
            svd_prev = (Uf, s, Vtf.T)
            M_prev = M
        P1 = op(A1 + E - Dhat)
        N = E - Yt / mu - P1
        E1 = soft_threshold(N, lam / mu)
        P2 = op(A1 + E1 - Dhat)
        Yt = Yt + mu * P2
        c1 = float(np.linalg.norm(P2)) / d0
        c2 = mu * max(float(np.linalg.norm(A1 - A)), float(np.linalg.norm(E1 - E))) / d0
        rho = prm.rho0 if c2 < prm.eps2 else 1.0
        if trace is not None:
            trace.append(dict(k=k, mu=mu, c1=c1, c2=c2, rank=int(np.sum(s > 1.0 / mu))))
        A, E, P = A1, E1, P2
        if c1 < prm.eps1 and c2 < prm.eps2:
            converged = True
            break
        mu = min(prm.mu_max, rho * mu)
    return InnerResult(A, E, Yt, k, converged, mus, c1, c2, s, warm_used)


def delta_tau(op: WtW, A, E, Dhat) -> np.ndarray:
    """Step 3 of Algorithm 1: dtau = (J^T J + Q^T Q)^{-1} J^T (A + E - D_hat), the
    solution of the stacked system of Eq. two_linear_constraint (Eq. Delta_tau when Q is
    absent)."""
    return op.coeffs(A + E - Dhat)


# ============================================================================ ADM baseline (Sec. 2.2)
@dataclasses.dataclass
class AdmParams:
    """Parameters of the ADM of Zhang et al. for the inner loop (values the paper leaves open
    are readings: R16)."""

    lam: float = -1.0            # <= 0 -> 1/sqrt(max(m, n))
    tol: float = 1e-7            # stop when ||D + J dtau - A - E||_F / ||D||_F < tol
    rho: float = 1.25            # mu <- rho mu
    mu0: float = -1.0            # <= 0 -> 1.25/||D||_2
    max_iter: int = 1000


@dataclasses.dataclass
class AdmResult:
    A: np.ndarray
    E: np.ndarray
    Y: np.ndarray
    dtau: np.ndarray
    iters: int
    converged: bool
    residual: float


def adm_inner(D, J, lam, prm: AdmParams) -> AdmResult:
    """The ADM of Zhang et al. as Sec. 2.2 states it: minimise the augmented Lagrangian of
    Eq. TILT_3, L = ||A||_* + lam||E||_1 + <Y, D + J dtau - A - E> + mu/2 ||D + J dtau - A - E||^2,
    over A, E and dtau in turn (Gauss-Seidel), then update Y and mu:
        A_k+1    = S_{1/mu}(D + J dtau_k - E_k + Y_k/mu)        (minimiser over A, Eq. A_1)
        E_k+1    = T_{lam/mu}(D + J dtau_k - A_k+1 + Y_k/mu)    (minimiser over E, Eq. E_1)
        dtau_k+1 = (J^T J)^{-1} J^T (A_k+1 + E_k+1 - D - Y_k/mu)  (least squares in dtau)
        Y_k+1    = Y_k + mu (D + J dtau_k+1 - A_k+1 - E_k+1),   mu_k+1 = rho mu_k
    from A_0 = D, E_0 = 0, dtau_0 = 0, Y_0 = 0 (Sec. 6.1).  D is an m x n array, J is
    (m n) x p with rows in row-major pixel order."""
    D = np.asarray(D, dtype=np.float64)
    J = np.asarray(J, dtype=np.float64)
    shape = D.shape
    d = D.reshape(-1)
    G = J.T @ J
    mu = 1.25 / float(np.linalg.norm(D, 2)) if prm.mu0 <= 0 else float(prm.mu0)
    A = D.copy()
    E = np.zeros(shape)
    Y = np.zeros(shape)
    dtau = np.zeros(J.shape[1])
    nD = float(np.linalg.norm(D))
    res = math.inf
    converged = False
    k = 0
    for k in range(1, prm.max_iter + 1):
        Jd = (J @ dtau).reshape(shape)
        A = svt(D + Jd - E + Y / mu, 1.0 / mu)[0]
        E = soft_threshold(D + Jd - A + Y / mu, lam / mu)
        dtau = np.linalg.solve(G, J.T @ (A + E - D - Y / mu).reshape(-1)) if J.shape[1] else dtau
        R = D + (J @ dtau).reshape(shape) - A - E
        Y = Y + mu * R
        res = float(np.linalg.norm(R)) / nD
        if res < prm.tol:
            converged = True
            break
        mu = prm.rho * mu
    return AdmResult(A, E, Y, dtau, k, converged, res)


# ============================================================================ Algorithm 1
@dataclasses.dataclass
class TiltResult:
    tau: np.ndarray
    A: np.ndarray
    E: np.ndarray
    Dhat: np.ndarray
    objective: float
    rank: int
    outer_iters: int
    inner_iters: int
    converged: bool
    oob: int
    inner_per_outer: list


def nuclear_norm(A) -> float:
    return float(np.linalg.svd(A, compute_uv=False).sum())


def numerical_rank(A, rel: float = 1e-3) -> int:
    s = np.linalg.svd(A, compute_uv=False)
    if s.size == 0 or s[0] <= 0:
        return 0
    return int(np.sum(s > rel * s[0]))


def resolve_lambda(prm: Params, m: int, n: int) -> float:
    return prm.lam if prm.lam > 0 else 1.0 / math.sqrt(max(m, n))


def tilt(img, tau0, ttype, m, n, prm: Params | None = None, trace: list | None = None) -> TiltResult:
    """Algorithm 1 (TILT via LADMAP + VWS), optionally with Algorithm 2 for the SVDs."""
    prm = prm or Params()
    lam = resolve_lambda(prm, m, n)
    tau = np.array(tau0, dtype=np.float64)
    Dhat, J, _, oob = warp_normalise_jacobian(img, tau, ttype, m, n)
    A = Dhat.copy()                                   # R9
    E = np.zeros((m, n))
    Yt = np.zeros((m, n))
    inner_total = 0
    per_outer = []
    converged = False
    i = 0
    for i in range(1, prm.max_outer + 1):
        if i > 1:
            Dhat, J, _, oob = warp_normalise_jacobian(img, tau, ttype, m, n)
        Q = constraint_rows(tau, ttype, m, n) if prm.use_q else None
        res = inner_ladmap(Dhat, J, Q, lam, A, E, Yt, prm, trace=trace)
        A, E, Yt = res.A, res.E, res.Yt
        inner_total += res.iters
        per_outer.append(res.iters)
        dtau = delta_tau(WtW(J, Q), A, E, Dhat)
        shift = corner_shift(tau, dtau, ttype, m, n)
        tau = tau + dtau
        if shift < prm.outer_tol:
            converged = True
            break
    obj = nuclear_norm(A) + lam * float(np.abs(E).sum())
    return TiltResult(tau, A, E, Dhat, obj, numerical_rank(A), i, inner_total, converged, oob, per_outer)


def objective(A, E, lam) -> float:
    """||A||_* + lam ||E||_1 (Eq. TILT_2)."""
    return nuclear_norm(A) + lam * float(np.abs(E).sum())


def tau_error(tau, tau_ref) -> float:
    return float(np.linalg.norm(np.asarray(tau) - np.asarray(tau_ref)) / np.linalg.norm(tau_ref))


# ============================================================================ RASL (Sec. 1)
def rasl_warp(imgs, taus, ttype, m, n):
    """Step 1 of Algorithm 1 for an image set (R18): D_hat (mn x N, column i = image i
    warped by tau_i, normalised), the per-column Jacobians J_i (mn x p each), the norms
    ||I_i o tau_i||_F and the total out-of-bounds count."""
    cols, Js, norms = [], [], []
    oob = 0
    for img, tau in zip(imgs, taus):
        Dhat_i, J_i, s_i, o_i = warp_normalise_jacobian(img, tau, ttype, m, n)
        cols.append(Dhat_i.reshape(-1))
        Js.append(J_i)
        norms.append(s_i)
        oob += o_i
    return np.stack(cols, axis=1), Js, np.array(norms), oob


def rasl_stacked_jacobian(Js) -> np.ndarray:
    """The Jacobian of vec(D_hat) (row-major, entry r N + i for pixel r of image i) with
    respect to the stacked parameters [tau_1; ...; tau_N] (entry i p + k): block-diagonal,
    image i's block J_i (R18)."""
    N = len(Js)
    mn, p = Js[0].shape
    Jb = np.zeros((mn * N, N * p))
    for i, J in enumerate(Js):
        Jb[i::N, i * p:(i + 1) * p] = J
    return Jb


def rasl_constraint_rows(N: int, p: int) -> np.ndarray:
    """Q = [I_p ... I_p] (p x Np): the increments of the set's transforms sum to zero (R18)."""
    return np.tile(np.eye(p), (1, N))


def rasl_operator(Js) -> WtW:
    """W^T W = I - J (J^T J + Q^T Q)^{-1} J^T (Eq. WTW_property) for the stacked,
    block-diagonal Jacobian and the constraint rows of R18."""
    N = len(Js)
    p = Js[0].shape[1]
    return WtW(rasl_stacked_jacobian(Js), rasl_constraint_rows(N, p))


@dataclasses.dataclass
class RaslResult:
    tau: np.ndarray              # (N, p)
    A: np.ndarray                # (mn, N)
    E: np.ndarray
    Dhat: np.ndarray             # D_hat at the last outer step's tau (before its update)
    objective: float
    rank: int
    outer_iters: int
    inner_iters: int
    converged: bool
    oob: int
    inner_per_outer: list


def rasl(imgs, taus0, ttype, m, n, prm: Params | None = None) -> RaslResult:
    """Algorithm 1 for an image set (RASL, R18): warp every image by its tau_i, the LADMAP
    inner loop with the column-wise W^T W and warm starts, dtau_i per image, until no
    window corner moves by outer_tol pixels."""
    prm = prm or Params()
    taus = np.array(taus0, dtype=np.float64)
    N = taus.shape[0]
    lam = prm.lam if prm.lam > 0 else 1.0 / math.sqrt(max(m * n, N))
    Dhat, Js, _, oob = rasl_warp(imgs, taus, ttype, m, n)
    A = Dhat.copy()                                   # R9
    E = np.zeros_like(Dhat)
    Yt = np.zeros_like(Dhat)
    inner_total = 0
    per_outer = []
    converged = False
    i = 0
    for i in range(1, prm.max_outer + 1):
        if i > 1:
            Dhat, Js, _, oob = rasl_warp(imgs, taus, ttype, m, n)
        op = rasl_operator(Js)
        res = inner_ladmap(Dhat, None, None, lam, A, E, Yt, prm, op=op)
        A, E, Yt = res.A, res.E, res.Yt
        inner_total += res.iters
        per_outer.append(res.iters)
        dtaus = op.coeffs(A + E - Dhat).reshape(N, -1)
        shift = max(corner_shift(taus[k], dtaus[k], ttype, m, n) for k in range(N))
        taus = taus + dtaus
        if shift < prm.outer_tol:
            converged = True
            break
    obj = nuclear_norm(A) + lam * float(np.abs(E).sum())
    return RaslResult(taus, A, E, Dhat, obj, numerical_rank(A), i, inner_total, converged, oob, per_outer)
