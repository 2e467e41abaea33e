// Inner LADMAP loop (Sec. 3.2 with the reorganisations of Sec. 4.2-4.3) and the outer
// loop of Algorithm 1, executed by one CTA per problem.
#pragma once

#include "tilt_cayley.cuh"
#include "tilt_device.cuh"

namespace tilt {

// Float scalars of one inner iteration, computed once by thread 0 in FP64 and read by all
// threads from shared memory (Scratch::fs).
enum { FS_IMU = 0, FS_THR = 1, FS_MU = 2, FS_IMUN = 3, FS_QRN = 4, FS_CC = 8 };
// Loop control word (Scratch::iscal[5]) set by thread 0 at the end of an iteration.
enum { LOOP_GO = 0, LOOP_CONVERGED = 1, LOOP_BAD = 2, LOOP_CANCELLED = 3 };

struct InnerOut {
    int iters, sweeps, warm, reorth, cayley, rank;
    bool converged, bad, cancelled, tc_timeout;
    double c1, c2, mu_last, nuc, l1;
};

struct SvdBufs {
    float* B;
    float* V;
    float* T;
    float* Z;              // C x Cp SVT coefficients (shared memory where they fit, else global)
    unsigned char* stage;  // stage buffers of the tensor-core products (shared memory)
    int nbuf;              // 1 or 2 stage buffers
    bool tc;               // products on the tensor cores (else register-tiled FP32 SIMT)
};

__device__ inline unsigned long long clk() { return clock64(); }

// Soft threshold T_eps(x) = sgn(x) max(|x| - eps, 0) (Sec. 3.2).
__device__ inline float soft(float x, float eps) {
    const float a = fabsf(x) - eps;
    return a > 0.f ? copysignf(a, x) : 0.f;
}

struct SvtStepOut {
    int sweeps;
    bool warm, tc_timeout, reorth;
    bool cayley;                    // the SVD came from an accepted step of Algorithm 2
    unsigned long long t_svd_end;   // clock at the end of the SVD (start of the reconstruction)
};

// Kept singular values after a step of Algorithm 2: the signs of Sigma folded into U (so
// Sigma >= 0), sigma_k = Sigma_k, w_k = (sigma_k - eps)_+, and the kept list, nuclear norm and
// rank as svt_weights gives them.  All threads.
static __device__ void svt_select_factors(const Dims& d, CayBufs cb, float eps, float* sigma, float* w, int* kept,
                                          Scratch* sc) {
    const int C = d.C, R = d.R, ldb = d.ldb;
    for (int e = threadIdx.x; e < R * C; e += NT) {
        const int k = e / R, r = e % R;
        if (cb.S[k] < 0.f) cb.U[(size_t)k * ldb + r] = -cb.U[(size_t)k * ldb + r];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < C; k += NT) {
        const float s = fabsf(cb.S[k]);
        cb.S[k] = s;
        sigma[k] = s;
        w[k] = s > eps ? s - eps : 0.f;
    }
    __syncthreads();
    svt_select(C, eps, sigma, w, kept, sc);
}

// Singular value thresholding of a tall M (in buf.T, tall_qr_ok) through its QR factorisation:
//   M = Q R_c by Householder reflectors H_j = I - beta_j v_j v_j^T, in place: R_c on and above
//   the diagonal of T's top C x C block, v_j below it (v_j's head in vhead); then the
//   one-sided Jacobi of the C x C matrix B_c = R_c V (warm from V, else B_c = R_c, V = I),
//   whose columns then hold U_c Sigma.  With B = Q B_c the left-factor SVT of svt_into becomes
//   S_eps(M) = Q [X_c; 0],   X_c = sum_kept (w_k / sigma_k^2) b_k (R_c^T b_k)^T   (b_k: B_c's),
//   and Q = H_0 ... H_{C-1} = I - Vh Th Vh^T in the compact WY form (Schreiber and Van Loan,
//   1989: Th upper triangular, Th_jj = beta_j, Th[0:j, j] = -beta_j Th[0:j, 0:j] Vh[:, 0:j]^T v_j),
//   so A' = [X_c; 0] - Vh (Th (Vh_top^T X_c)) is one R x C x C product whose epilogue stores
//   A (||A' - A||^2 in scal[7], J^T A' in ja[] when d.p > 0).  The sweeps' dot products run over
//   C rows instead of R.  Buffers: B_c in buf.Z (C x C, stride Cp); buf.B holds
//   tall_small_floats(d).  T is overwritten.  All threads.
template <int NCH>
static __device__ SvtStepOut svt_tall_qr(const Dims& d, SvdBufs& buf, const SmemLayout& L, bool& haveV, bool gate_ok,
                                         float eps, float* __restrict__ A, const float* __restrict__ J) {
    Scratch* sc = L.sc;
    const int p = d.p, S = d.S, R = d.R, C = d.C, ldb = d.ldb, ldv = d.ldv, Cp = d.Cp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* T = buf.T;
    float* Bc = buf.Z;                        // C x C at stride Cp
    float* S0 = buf.B;                        // the SVT coefficients, then W1 = Vh_top^T X_c
    float* Xc = S0 + (size_t)C * Cp;
    float* S2 = Xc + (size_t)C * Cp;          // Vh^T Vh, then W2 = Th W1 (row-major: S2[a Cp + c])
    float* Th = S2 + (size_t)C * Cp;
    float* vhead = Th + (size_t)C * Cp;
    float* beta = vhead + Cp;
    SvtStepOut so;
    so.sweeps = 0;
    so.warm = false;
    so.tc_timeout = false;
    so.reorth = false;
    so.cayley = false;
    const bool warm = haveV && gate_ok;
    if (warm && v_drift(buf.V, ldv, C, sc) > 1e-4f) {
        v_reorth_fp64(buf.V, ldv, C, sc);
        so.reorth = true;
    }
    // ---- Householder QR of T: H_j maps x = T[j .., j] to alpha e_1, alpha = -sign(x_0) ||x||,
    // with v = (x_0 - alpha, x_1, ...) and beta = 1 / (||x||^2 + |x_0| ||x||)
    float* n2s = &sc->fs[FS_QRN];             // ||T[j .., j]||^2 of the next column
    if (warp == 0) {
        float s2 = 0.f;
        for (int i = lane; i < R; i += 32) s2 = fmaf(T[i], T[i], s2);
        s2 = warp_sum(s2);
        if (lane == 0) *n2s = s2;
    }
    __syncthreads();
    for (int j = 0; j < C; ++j) {
        float* tj = T + (size_t)j * ldb;
        if (threadIdx.x == 0) {
            const float x0 = tj[j], nrm2 = *n2s, nrm = sqrtf(nrm2);
            const float alpha = nrm > 0.f ? (x0 >= 0.f ? -nrm : nrm) : 0.f;
            vhead[j] = x0 - alpha;
            beta[j] = nrm > 0.f ? 1.f / (nrm2 + fabsf(x0) * nrm) : 0.f;
            tj[j] = alpha;
        }
        __syncthreads();
        const float v0 = vhead[j], bj = beta[j];
        for (int k = j + 1 + warp; k < C; k += NW) {
            float* tk = T + (size_t)k * ldb;
            const float tkj = tk[j];              // read by every lane before lane 0 rewrites it
            float w = 0.f, w1 = 0.f;
            int i = j + 1 + lane;
#pragma unroll 2
            for (; i + 32 < R; i += 64) {
                w = fmaf(tj[i], tk[i], w);
                w1 = fmaf(tj[i + 32], tk[i + 32], w1);
            }
            if (i < R) w = fmaf(tj[i], tk[i], w);
            w = warp_sum(w + w1) + v0 * tkj;
            const float f = bj * w;
            if (lane == 0) tk[j] = tkj - f * v0;
            float s2 = 0.f;
#pragma unroll 4
            for (int i2 = j + 1 + lane; i2 < R; i2 += 32) {
                const float t = fmaf(-f, tj[i2], tk[i2]);
                tk[i2] = t;
                s2 = fmaf(t, t, s2);
            }
            if (k == j + 1) {
                s2 = warp_sum(s2);
                if (lane == 0) *n2s = s2;
            }
        }
        __syncthreads();
    }
    // ---- B_c = R_c V (warm) or R_c (cold, V = I); the SVD of B_c
    for (int e = threadIdx.x; e < C * Cp; e += NT) {
        const int c = e / Cp, i = e - c * Cp;
        float v = 0.f;
        if (i < C) {
            if (warm) {
                for (int k = i; k < C; ++k) v = fmaf(T[(size_t)k * ldb + i], buf.V[(size_t)c * ldv + k], v);
            } else {
                v = i <= c ? T[(size_t)c * ldb + i] : 0.f;
            }
        }
        Bc[e] = v;
    }
    if (!warm) set_identity(buf.V, ldv, Cp);
    __syncthreads();
    so.warm = warm;
    const int js = default_schedule(C, C);
    so.sweeps = k2_jacobi<NCH, false>(Bc, Cp, buf.V, ldv, C, C, jacobi_tol(C), warm ? 30 : 40, sc->flag,
                                      jsched_width(js), jsched_order(js), nullptr);
    haveV = true;
    svt_weights(Bc, Cp, C, C, eps, L.sigma, L.w, L.kept, sc);
    so.t_svd_end = clk();
    // ---- X_c = sum_kept (w_k / sigma_k^2) b_k (R_c^T b_k)^T and the compact WY form.  The
    // small products run with consecutive threads on consecutive columns of row-major operands
    // (R_c^T, X_c, W1, W2 are stored by rows), so that no shared-memory access of a warp strides
    // across one bank
    const int nk = sc->iscal[1];
    float* Rt = Th;                            // R_c by rows until Th is formed
    for (int e = threadIdx.x; e < C * C; e += NT) {
        const int i = e / C, c = e - i * C;
        Rt[(size_t)i * Cp + c] = i <= c ? T[(size_t)c * ldb + i] : 0.f;
    }
    // Vh^T Vh by 4 x 4 tiles (upper block triangle), one warp per tile, lanes on consecutive rows
    // (Vh[i, a] = T[i, a] below the diagonal, vhead[a] on it, 0 above)
    {
        const int ntc = Cp >> 2;
        for (int t = warp; t < ntc * ntc; t += NW) {
            const int ta = t / ntc, tb = t - ta * ntc;
            if (ta > tb) continue;
            const int a0 = 4 * ta, b0 = 4 * tb;
            float g[4][4];
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) g[x][y] = 0.f;
            for (int i = a0 + lane; i < R; i += 32) {
                float va[4], vb[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int a = a0 + u, b = b0 + u;
                    va[u] = a < C ? (i > a ? T[(size_t)a * ldb + i] : (i == a ? vhead[a] : 0.f)) : 0.f;
                    vb[u] = b < C ? (i > b ? T[(size_t)b * ldb + i] : (i == b ? vhead[b] : 0.f)) : 0.f;
                }
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) g[x][y] = fmaf(va[x], vb[y], g[x][y]);
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) g[x][y] = warp_sum(g[x][y]);
            if (lane == 0)
                for (int x = 0; x < 4; ++x)
                    for (int y = 0; y < 4; ++y) {
                        const int a = a0 + x, b = b0 + y;
                        if (a < b && b < C) S2[(size_t)b * Cp + a] = g[x][y];
                    }
        }
    }
    __syncthreads();
    // the coefficients Z (nk x C, by rows): (w_k / sigma_k^2) (R_c^T b_k)^T
    for (int e = threadIdx.x; e < nk * C; e += NT) {
        const int q = e / C, c = e - q * C;
        const int k = L.kept[q];
        const float* bk = Bc + (size_t)k * Cp;
        float z = 0.f;
        for (int i = 0; i <= c; ++i) z = fmaf(bk[i], Rt[(size_t)i * Cp + c], z);
        const float sg = L.sigma[k];
        S0[(size_t)q * Cp + c] = z * (L.w[k] / (sg * sg));
    }
    __syncthreads();
    // X_c = B_c,K Z (by rows)
    for (int e = threadIdx.x; e < C * C; e += NT) {
        const int i = e / C, c = e - i * C;
        float x = 0.f;
        for (int q = 0; q < nk; ++q) x = fmaf(Bc[(size_t)L.kept[q] * Cp + i], S0[(size_t)q * Cp + c], x);
        Xc[(size_t)i * Cp + c] = x;
    }
    // Th by its column recurrence (one warp; R_c^T is no longer needed)
    if (warp == 0) {
        for (int j = 0; j < C; ++j) {
            for (int i = lane; i < j; i += 32) {
                float t = 0.f;
                for (int k = i; k < j; ++k) t = fmaf(Th[(size_t)k * Cp + i], S2[(size_t)j * Cp + k], t);
                Th[(size_t)j * Cp + i] = -beta[j] * t;
            }
            if (lane == 0) Th[(size_t)j * Cp + j] = beta[j];
            __syncwarp();
        }
    }
    __syncthreads();
    // W1 = Vh_top^T X_c (into S0, by rows), then W2 = Th W1 (into S2, by rows)
    for (int e = threadIdx.x; e < C * C; e += NT) {
        const int a = e / C, c = e - a * C;
        const float* ta = T + (size_t)a * ldb;
        float w = vhead[a] * Xc[(size_t)a * Cp + c];
        for (int i = a + 1; i < C; ++i) w = fmaf(ta[i], Xc[(size_t)i * Cp + c], w);
        S0[(size_t)a * Cp + c] = w;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < C * Cp; e += NT) {
        const int a = e / Cp, c = e - a * Cp;
        float w = 0.f;
        if (c < C)
            for (int k = a; k < C; ++k) w = fmaf(Th[(size_t)k * Cp + a], S0[(size_t)k * Cp + c], w);
        S2[(size_t)a * Cp + c] = w;
    }
    __syncthreads();
    // ---- A' = [X_c; 0] - Vh W2: one row of four columns per item, consecutive threads on
    // consecutive rows (coalesced accesses of A; W2's rows are broadcast float4 reads).  A
    // thread takes its items four at a time and loads their old values of A before any of
    // their stores, so the loads of a batch are in flight together (a load of A that follows
    // a store to A cannot be moved ahead of it)
    float acc[1 + PMAX];
#pragma unroll
    for (int k2 = 0; k2 < 1 + PMAX; ++k2) acc[k2] = 0.f;
    const int nc4 = Cp >> 2;
    const int items = R * nc4;
    constexpr int NB = 4;
    for (int base = threadIdx.x; base < items; base += NB * NT) {
        float aold[NB][4];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int idx = base + b * NT;
            const int c4 = idx / R, i = idx - c4 * R;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = 4 * c4 + u;
                aold[b][u] = (idx < items && c < C) ? A[(size_t)c * R + i] : 0.f;
            }
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int idx = base + b * NT;
            if (idx >= items) break;
            const int c4 = idx / R, i = idx - c4 * R;
            const int c0 = 4 * c4;
            float4 sv = make_float4(0.f, 0.f, 0.f, 0.f);
            const int amax = min(i, C - 1);
            for (int a = 0; a <= amax; ++a) {
                const float vh = a == i ? vhead[a] : T[(size_t)a * ldb + i];
                const float4 w2 = *reinterpret_cast<const float4*>(S2 + (size_t)a * Cp + c0);
                sv.x = fmaf(vh, w2.x, sv.x);
                sv.y = fmaf(vh, w2.y, sv.y);
                sv.z = fmaf(vh, w2.z, sv.z);
                sv.w = fmaf(vh, w2.w, sv.w);
            }
            const float su[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = c0 + u;
                if (c < C) {
                    const float sa = (i < C ? Xc[(size_t)i * Cp + c] : 0.f) - su[u];
                    const int e = c * R + i;
                    const float da = sa - aold[b][u];
                    acc[0] = fmaf(da, da, acc[0]);
                    A[e] = sa;
#pragma unroll
                    for (int k2 = 0; k2 < PMAX; ++k2)
                        if (k2 < p) acc[1 + k2] = fmaf(J[(size_t)k2 * S + e], sa, acc[1 + k2]);
                }
            }
        }
    }
    block_sum_f<1 + PMAX>(acc, sc->red);
    if (threadIdx.x == 0) {
        sc->scal[7] = block_total(sc->red, 0);
        for (int k2 = 0; k2 < p; ++k2) sc->ja[k2] = block_total(sc->red, 1 + k2);
    }
    __syncthreads();
    return so;
}

// Singular value thresholding of the iteration's M (in buf.T): the one-sided Jacobi SVD,
// warm-started from V when one exists, the gate allows and V has not drifted (a6), then
// A' = S_eps(M) by the left-factor reconstruction (a7), stored into A with ||A' - A||^2 in
// scal[7] and J^T A' in ja[] (FP64 totals of FP32 partials).  All threads.
//
// Algorithm 2 (cay != nullptr, a workspace of cayley_floats()): when the previous factors
// exist (haveUS) and the gate allows, one Cayley step from them (cayley_step); if it is
// accepted, A' = U(t) (Sigma(t) - eps)_+ V(t)^T directly and the Jacobi SVD is skipped;
// otherwise, and on the first iteration, the full SVD runs and its factors are kept for the
// next step.
template <int NCH, bool TCP>
static __device__ __forceinline__ SvtStepOut svt_into(const Dims& d, SvdBufs& buf, const SmemLayout& L, bool& haveV, bool gate_ok,
                                      float eps, float* __restrict__ A, const float* __restrict__ J, int jsched,
                                      float* cay = nullptr, bool* haveUS = nullptr, bool tall = false) {
    Scratch* sc = L.sc;
    const int p = d.p, S = d.S, R = d.R, C = d.C, ldb = d.ldb, ldv = d.ldv, Cp = d.Cp;
    SvtStepOut so;
    so.sweeps = 0;
    so.warm = false;
    so.tc_timeout = false;
    so.reorth = false;
    so.cayley = false;
    if (TCP && cay && *haveUS && gate_ok) {
        CayBufs cb = carve_cayley(cay, d);
        const CayleyOut co = cayley_step(d, buf.T, cb, buf.V, sc);
        if (co.accepted) {
            svt_select_factors(d, cb, eps, L.sigma, L.w, L.kept, sc);
            so.cayley = true;
            so.warm = true;
            so.t_svd_end = clk();
            const int nk = sc->iscal[1];
            float acc[1 + PMAX];
#pragma unroll
            for (int k2 = 0; k2 < 1 + PMAX; ++k2) acc[k2] = 0.f;
            auto upd = [&](int r, int c, float sa) {
                const int e = c * R + r;
                const float da = sa - A[e];
                acc[0] = fmaf(da, da, acc[0]);
                A[e] = sa;
#pragma unroll
                for (int k2 = 0; k2 < PMAX; ++k2)
                    if (k2 < p) acc[1 + k2] = fmaf(J[(size_t)k2 * S + e], sa, acc[1 + k2]);
            };
            if (nk > 0) {
                const float* Uc = cb.U;
                const float* Vc = buf.V;
                const float* wk = L.w;
                const int* kept = L.kept;
                gemm_simt<4, 4>(R, C, nk, [=](int r, int q) { return Uc[(size_t)kept[q] * ldb + r] * wk[kept[q]]; },
                                [=](int q, int c) { return Vc[(size_t)kept[q] * ldv + c]; }, upd);
            } else {
                for (int e = threadIdx.x; e < S; e += NT) upd(e % R, e / R, 0.f);
            }
            block_sum_f<1 + PMAX>(acc, sc->red);
            if (threadIdx.x == 0) {
                sc->scal[7] = block_total(sc->red, 0);
                for (int k2 = 0; k2 < p; ++k2) sc->ja[k2] = block_total(sc->red, 1 + k2);
            }
            __syncthreads();
            return so;
        }
    }
    if (tall && tall_qr_ok(d)) return svt_tall_qr<NCH>(d, buf, L, haveV, gate_ok, eps, A, J);
    const bool warm = haveV && gate_ok;
    // FP32 rotations let V drift from orthogonal over many warm starts; past 1e-4 in a column
    // norm it is re-orthonormalised in FP64 and the warm start goes ahead
    if (warm && v_drift(buf.V, ldv, C, sc) > 1e-4f) {
        v_reorth_fp64(buf.V, ldv, C, sc);
        so.reorth = true;
    }
    if (warm) {
        if (TCP && buf.tc) {
            if (!warm_start_tc(buf.T, ldb, buf.V, ldv, buf.B, C, buf.stage, buf.nbuf, &sc->tc)) {
                so.tc_timeout = true;
                so.t_svd_end = clk();
                return so;
            }
        } else {
            gemm_TV<NCH >= 4 ? 8 : 4>(buf.T, ldb, buf.V, ldv, buf.B, Cp, C);
        }
    } else {
        for (int e = threadIdx.x; e < ldb * Cp; e += NT) buf.B[e] = buf.T[e];
        set_identity(buf.V, ldv, Cp);
    }
    so.warm = warm;
    if (TCP && jsched_order(jsched) == 2) {
        so.sweeps = k2_jacobi_staged<NCH>(buf.B, ldb, buf.V, ldv, R, C, jacobi_tol(R), warm ? 30 : 40, sc->flag,
                                          jsched_width(jsched), reinterpret_cast<float*>(buf.stage), &sc->tc, L.w);
        if (so.sweeps < 0) {
            so.sweeps = 0;
            so.tc_timeout = true;
            so.t_svd_end = clk();
            return so;
        }
    } else {
        so.sweeps = k2_jacobi<NCH>(buf.B, ldb, buf.V, ldv, R, C, jacobi_tol(R), warm ? 30 : 40, sc->flag,
                                   jsched_width(jsched), jsched_order(jsched), L.w);
    }
    haveV = true;
    svt_weights(buf.B, ldb, R, C, eps, L.sigma, L.w, L.kept, sc);
    if (TCP && cay) {
        // the factors of this exact SVD, for the next step of Algorithm 2: U = B / sigma
        CayBufs cb = carve_cayley(cay, d);
        for (int e = threadIdx.x; e < ldb * C; e += NT) {
            const int k = e / ldb, r = e % ldb;
            const float sg = L.sigma[k];
            cb.U[e] = (r < R && sg > 0.f) ? buf.B[(size_t)k * ldb + r] / sg : 0.f;
        }
        for (int k = threadIdx.x; k < C; k += NT) cb.S[k] = L.sigma[k];
        __syncthreads();
        *haveUS = true;
    }
    so.t_svd_end = clk();
    // A' = sum_kept w_k b_k v_k^T
    const int nk = sc->iscal[1];
    bool tc_ok = true;
    if (TCP && buf.tc)
        tc_ok = svt_coeffs_tc(buf.T, ldb, buf.B, ldb, R, C, L.sigma, L.w, L.kept, nk, buf.Z, Cp, buf.stage,
                              buf.nbuf, &sc->tc);
    else
        svt_coeffs_tiled(buf.T, ldb, buf.B, ldb, R, C, L.sigma, L.w, L.kept, nk, buf.Z, Cp);
    float acc[1 + PMAX];
#pragma unroll
    for (int k2 = 0; k2 < 1 + PMAX; ++k2) acc[k2] = 0.f;
    // A' = B_K Z (R x nk times nk x C); the epilogue stores A', accumulates ||A' - A||^2
    // and J^T A' (consecutive lanes or threads take consecutive rows: the A and J
    // accesses are coalesced)
    auto upd = [&](int r, int c, float sa) {
        const int e = c * R + r;
        const float da = sa - A[e];
        acc[0] = fmaf(da, da, acc[0]);
        A[e] = sa;
#pragma unroll
        for (int k2 = 0; k2 < PMAX; ++k2)
            if (k2 < p) acc[1 + k2] = fmaf(J[(size_t)k2 * S + e], sa, acc[1 + k2]);
    };
    if (TCP && nk > 0 && buf.tc && tc_ok) {
        const float* Bb = buf.B;
        const float* Zb = buf.Z;
        const int* kept = L.kept;
        auto la = [=](int r, int q) { return Bb[(size_t)kept[q] * ldb + r]; };
        auto lb = [=](int q, int c) { return Zb[(size_t)q * Cp + c]; };
        tc_ok = tc_gemm<NT, false, false>(R, C, nk, la, lb, upd, buf.stage, TC_KC, buf.nbuf, &sc->tc);
    } else if (nk > 0 && !(TCP && buf.tc)) {
        // one row of four columns per thread: a float4 of Z (rows at stride Cp, a
        // broadcast) feeds four FMAs
        const int nc4 = Cp >> 2;
        for (int idx = threadIdx.x; idx < R * nc4; idx += NT) {
            const int c4 = idx / R, r = idx - c4 * R;
            const int c0 = 4 * c4;
            float4 sv = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int q = 0; q < nk; ++q) {
                const float bq = buf.B[(size_t)L.kept[q] * ldb + r];
                const float4 z = *reinterpret_cast<const float4*>(buf.Z + (size_t)q * Cp + c0);
                sv.x = fmaf(bq, z.x, sv.x);
                sv.y = fmaf(bq, z.y, sv.y);
                sv.z = fmaf(bq, z.z, sv.z);
                sv.w = fmaf(bq, z.w, sv.w);
            }
            const float su[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (c0 + u < C) upd(r, c0 + u, su[u]);
        }
    } else if (nk == 0) {
        for (int e = threadIdx.x; e < S; e += NT) upd(e % R, e / R, 0.f);
    }
    if (!tc_ok) {
        so.tc_timeout = true;
        return so;
    }
    block_sum_f<1 + PMAX>(acc, sc->red);
    if (threadIdx.x == 0) {
        sc->scal[7] = block_total(sc->red, 0);
        for (int k2 = 0; k2 < p; ++k2) sc->ja[k2] = block_total(sc->red, 1 + k2);
    }
    __syncthreads();
    return so;
}

// The inner loop.  Entry: A, E, Y hold the warm start (Eq. warm_start), sc->G/Gi/jd/scal[1]
// hold J^T J + Q^T Q, its inverse, J^T D_hat and d0 = ||W^T W D_hat||_F (k5_gram).
// Exit: A, E, Y the result; sc->cvec = G^-1 J^T (A + E - D_hat), i.e. dtau (Eq. Delta_tau).
//
// Iteration k (Eq. newvars2 with readings: +mu in the Y update, N centred at E_k, eta = 1):
//   M = A - Y/mu - P                          (P = W^T W (A + E - D_hat) from iteration k-1)
//   A' = S_{1/mu}(M)                          (K2 Jacobi SVD, warm from V, + reconstruction)
//   P' = W^T W (A' + E - D_hat);  E' = T_{lam/mu}(E - Y/mu - P')
//   P'' = W^T W (A' + E' - D_hat);  Y' = Y + mu P''
//   c1 = ||P''|| / d0;  c2 = mu max(||A'-A||, ||E'-E||) / d0;  rho = rho0 if c2 < eps2 else 1
//   stop when c1 < eps1 and c2 < eps2; mu <- min(mu_max, rho mu)
// W^T W v = v - J (G^-1 (J^T v)); the J^T products of A' and E' are accumulated while
// those planes are produced, so every W^T W costs one extra pass only.
// TCP: the kernel carries the tensor-core path (the 2-CTA kernel, whose windows are all below
// the tensor-core size, leaves it out to save registers).
template <int NCH, bool TCP = true>
static __device__ InnerOut k_inner(const Dims& d, const Params& prm, double lam, double mu0, const float* __restrict__ Dhat,
                            const float* __restrict__ J, float* __restrict__ A, float* __restrict__ E,
                            float* __restrict__ Y, float* __restrict__ Mp, SvdBufs buf,
                            bool& haveV, const SmemLayout& L, Result* cyc, int jsched, const int* cancel,
                            float* cay = nullptr) {
    Scratch* sc = L.sc;
    const int p = d.p, S = d.S, R = d.R, ldb = d.ldb;
    // the gate of Algorithm 2 compares M with the previous iteration's M (kept in Mp); with the
    // gate off (eps_svd < 0) the previous M is neither read nor kept
    const bool gate = prm.eps_svd >= 0.0;
    // pixel e = c R + r of a thread's next element: e + NT
    const int stepr = NT % R, stepc = NT / R;
    bool haveUS = false;              // factors of a previous SVD of this inner loop (Algorithm 2)
    float* cay_ws = (TCP && prm.svd_ws == 1) ? cay : nullptr;
    InnerOut out;
    out.iters = 0; out.sweeps = 0; out.warm = 0; out.reorth = 0; out.cayley = 0; out.rank = 0;
    out.cancelled = false;
    out.converged = false; out.bad = false; out.tc_timeout = false;
    out.c1 = out.c2 = 0.0; out.mu_last = mu0; out.nuc = 0.0; out.l1 = 0.0;
    unsigned long long t0 = clk();

    // ---- prologue: J^T A, J^T E, J^T Y; project Y (Eq. Y_new_warmstart); P_0; M_0
    {
        float facc[3 * PMAX];
#pragma unroll
        for (int k = 0; k < 3 * PMAX; ++k) facc[k] = 0.f;
        for (int e = threadIdx.x; e < S; e += NT) {
            const float a = A[e], ee = E[e], y = Y[e];
#pragma unroll
            for (int k = 0; k < PMAX; ++k) {
                if (k < p) {
                    const float jk = J[(size_t)k * S + e];
                    facc[k] = fmaf(jk, a, facc[k]);
                    facc[PMAX + k] = fmaf(jk, ee, facc[PMAX + k]);
                    facc[2 * PMAX + k] = fmaf(jk, y, facc[2 * PMAX + k]);
                }
            }
        }
        double acc[3 * PMAX];
#pragma unroll
        for (int k = 0; k < 3 * PMAX; ++k) acc[k] = facc[k];
        block_sum64<3 * PMAX>(acc, sc->red);
        if (threadIdx.x == 0) {
            double v[PMAX];
            for (int k = 0; k < p; ++k) {
                sc->ja[k] = acc[k];
                sc->je[k] = acc[PMAX + k];
                v[k] = acc[k] + acc[PMAX + k] - sc->jd[k];
            }
            ginv_apply(sc, p, v, sc->cvec);                         // c_P
            for (int k = 0; k < p; ++k) v[k] = acc[2 * PMAX + k];
            ginv_apply(sc, p, v, sc->dtau);                         // c_Y (temporary)
        }
        __syncthreads();
        float cP[PMAX], cY[PMAX];
#pragma unroll
        for (int k = 0; k < PMAX; ++k) {
            cP[k] = k < p ? (float)sc->cvec[k] : 0.f;
            cY[k] = k < p ? (float)sc->dtau[k] : 0.f;
        }
        const float imu = (float)(1.0 / mu0);
        double g[2] = {0.0, 0.0};
        int r = threadIdx.x % R, c = threadIdx.x / R;
        for (int e = threadIdx.x; e < S; e += NT) {
            float jc = 0.f, jy = 0.f;
#pragma unroll
            for (int k = 0; k < PMAX; ++k) {
                if (k < p) {
                    const float jk = J[(size_t)k * S + e];
                    jc = fmaf(jk, cP[k], jc);
                    jy = fmaf(jk, cY[k], jy);
                }
            }
            const float a = A[e];
            const float y = Y[e] - jy;
            const float pp = (a + E[e] - Dhat[e]) - jc;
            Y[e] = y;
            const float mv = a - y * imu - pp;
            buf.T[(size_t)c * ldb + r] = mv;
            if (gate) {
                const float mo = Mp[e];
                g[0] += (double)((mv - mo) * (mv - mo));
                g[1] += (double)(mv * mv);
                Mp[e] = mv;
            }
            next_rc(r, c, R, stepr, stepc);
        }
        block_sum64<2>(g, sc->red);
        if (threadIdx.x == 0) { sc->scal[5] = g[0]; sc->scal[6] = g[1]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) cyc->cyc_elem += clk() - t0;

    const double d0 = sc->scal[1] > 0.0 ? sc->scal[1] : 1.0;
    // thread 0 keeps mu and every FP64 scalar; the others read floats from sc->fs
    if (threadIdx.x == 0) {
        sc->scal[12] = mu0;
        sc->fs[FS_IMU] = (float)(1.0 / mu0);
        sc->fs[FS_THR] = (float)(lam / mu0);
        sc->iscal[6] = prm.eps_svd < 0.0 || sc->scal[5] < prm.eps_svd * prm.eps_svd * sc->scal[6];
    }
    __syncthreads();
    for (int k = 1; k <= prm.max_inner; ++k) {
        out.iters = k;
        // ---- a6 + a7: SVD of M (in T), warm from V when the gate allows (Alg. 2 gate);
        // A' = S_{1/mu}(M); ||A' - A||^2 -> scal[7]; J^T A' -> ja
        t0 = clk();
        const SvtStepOut so = svt_into<NCH, TCP>(d, buf, L, haveV, sc->iscal[6] != 0, sc->fs[FS_IMU], A, J, jsched,
                                                 cay_ws, &haveUS);
        const unsigned long long t1 = so.t_svd_end;
        if (threadIdx.x == 0) cyc->cyc_svd += t1 - t0;
        if (so.warm) out.warm++;
        if (so.reorth) out.reorth++;
        if (so.cayley) out.cayley++;
        out.sweeps += so.sweeps;
        out.nuc = sc->scal[3];
        out.rank = sc->iscal[2];
        if (so.tc_timeout) {
            out.bad = out.tc_timeout = true;
            break;
        }
        if (threadIdx.x == 0) {
            double v[PMAX];
            for (int k2 = 0; k2 < p; ++k2) v[k2] = sc->ja[k2] + sc->je[k2] - sc->jd[k2];
            ginv_apply(sc, p, v, sc->cvec);                           // c'
            for (int k2 = 0; k2 < PMAX; ++k2) sc->fs[FS_CC + k2] = k2 < p ? (float)sc->cvec[k2] : 0.f;
        }
        __syncthreads();
        unsigned long long t2 = clk();
        if (threadIdx.x == 0) cyc->cyc_recon += t2 - t1;

        // ---- a8: E' = T_{lam/mu}(E - Y/mu - W^T W (A' + E - D_hat)); ||E' - E||^2; J^T E'; ||E'||_1
        const float imu = sc->fs[FS_IMU];
        const float thr = sc->fs[FS_THR];
        {
            float cc[PMAX];
#pragma unroll
            for (int k2 = 0; k2 < PMAX; ++k2) cc[k2] = sc->fs[FS_CC + k2];
            float acc[2 + PMAX];
#pragma unroll
            for (int k2 = 0; k2 < 2 + PMAX; ++k2) acc[k2] = 0.f;
            for (int e = threadIdx.x; e < S; e += NT) {
                float jv[PMAX];
                float jc = 0.f;
#pragma unroll
                for (int k2 = 0; k2 < PMAX; ++k2) {
                    jv[k2] = k2 < p ? J[(size_t)k2 * S + e] : 0.f;
                    jc = fmaf(jv[k2], cc[k2], jc);
                }
                const float ee = E[e];
                const float p1 = (A[e] + ee - Dhat[e]) - jc;
                const float nv = ee - Y[e] * imu - p1;
                const float en = soft(nv, thr);
                const float de = en - ee;
                acc[0] = fmaf(de, de, acc[0]);
                acc[1] += fabsf(en);
                E[e] = en;
#pragma unroll
                for (int k2 = 0; k2 < PMAX; ++k2) acc[2 + k2] = fmaf(jv[k2], en, acc[2 + k2]);
            }
            block_sum_f<2 + PMAX>(acc, sc->red);
            if (threadIdx.x == 0) {
                sc->scal[8] = block_total(sc->red, 0);
                sc->scal[9] = block_total(sc->red, 1);
                double v[PMAX];
                for (int k2 = 0; k2 < p; ++k2) {
                    sc->je[k2] = block_total(sc->red, 2 + k2);
                    v[k2] = sc->ja[k2] + sc->je[k2] - sc->jd[k2];
                }
                ginv_apply(sc, p, v, sc->cvec);                       // c'' (= dtau at exit)
                for (int k2 = 0; k2 < PMAX; ++k2) sc->fs[FS_CC + k2] = k2 < p ? (float)sc->cvec[k2] : 0.f;
                // Cond2 and the penalty update (Eqs. rho, mu)
                const double mu = sc->scal[12];
                const double dA = sqrt(sc->scal[7]), dE = sqrt(sc->scal[8]);
                const double c2 = mu * fmax(dA, dE) / d0;
                const double rho = (c2 < prm.eps2) ? prm.rho0 : 1.0;
                const double mu_next = fmin(prm.mu_max, rho * mu);
                sc->scal[13] = mu_next;
                sc->scal[14] = c2;
                sc->fs[FS_MU] = (float)mu;
                sc->fs[FS_IMUN] = (float)(1.0 / mu_next);
            }
            __syncthreads();
        }
        out.l1 = sc->scal[9];

        // ---- a9: P'' = W^T W (A' + E' - D_hat); Y' = Y + mu P''; next M = A' - Y'/mu_next - P''
        {
            float cc[PMAX];
#pragma unroll
            for (int k2 = 0; k2 < PMAX; ++k2) cc[k2] = sc->fs[FS_CC + k2];
            const float muf = sc->fs[FS_MU];
            const float imun = sc->fs[FS_IMUN];
            float acc[3] = {0.f, 0.f, 0.f};
            int r = threadIdx.x % R, c = threadIdx.x / R;
            for (int e = threadIdx.x; e < S; e += NT) {
                float jc = 0.f;
#pragma unroll
                for (int k2 = 0; k2 < PMAX; ++k2)
                    if (k2 < p) jc = fmaf(J[(size_t)k2 * S + e], cc[k2], jc);
                const float a = A[e];
                const float pp = (a + E[e] - Dhat[e]) - jc;
                const float y = fmaf(muf, pp, Y[e]);
                Y[e] = y;
                acc[0] = fmaf(pp, pp, acc[0]);
                const float mv = a - y * imun - pp;
                buf.T[(size_t)c * ldb + r] = mv;
                if (gate) {
                    const float mo = Mp[e];
                    acc[1] = fmaf(mv - mo, mv - mo, acc[1]);
                    acc[2] = fmaf(mv, mv, acc[2]);
                    Mp[e] = mv;
                }
                next_rc(r, c, R, stepr, stepc);
            }
            block_sum_f<3>(acc, sc->red);
            if (threadIdx.x == 0) {
                sc->scal[10] = block_total(sc->red, 0);
                sc->scal[5] = block_total(sc->red, 1);
                sc->scal[6] = block_total(sc->red, 2);
                // Cond1, the stopping decision, and the scalars of the next iteration
                const double c1 = sqrt(sc->scal[10]) / d0, c2 = sc->scal[14];
                const double mu_next = sc->scal[13];
                sc->scal[15] = c1;
                int ctl = LOOP_GO;
                if (!isfinite(c1) || !isfinite(c2)) ctl = LOOP_BAD;
                else if (cancel_requested(cancel)) ctl = LOOP_CANCELLED;   // the context is being destroyed
                else if (c1 < prm.eps1 && c2 < prm.eps2) ctl = LOOP_CONVERGED;
                sc->iscal[5] = ctl;
                sc->scal[16] = sc->scal[12];      // the mu of this iteration
                sc->scal[12] = mu_next;
                sc->fs[FS_IMU] = (float)(1.0 / mu_next);
                sc->fs[FS_THR] = (float)(lam / mu_next);
                sc->iscal[6] = prm.eps_svd < 0.0 || sc->scal[5] < prm.eps_svd * prm.eps_svd * sc->scal[6];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) cyc->cyc_elem += clk() - t2;
        const int ctl = sc->iscal[5];
        out.c1 = sc->scal[15];
        out.c2 = sc->scal[14];
        out.mu_last = sc->scal[16];
        if (ctl == LOOP_BAD) {
            out.bad = true;
            break;
        }
        if (ctl == LOOP_CANCELLED) {
            out.cancelled = true;
            break;
        }
        if (ctl == LOOP_CONVERGED) {
            out.converged = true;
            break;
        }
    }
    return out;
}

struct AdmOut {
    int iters, sweeps, warm;
    bool converged, bad, tc_timeout;
    double residual, mu_last;
};

// The ADM of Zhang et al. for the inner loop (Sec. 2.2, the comparison method): minimise the
// augmented Lagrangian of Eq. TILT_3 over A, E and dtau in turn, then update Y and mu:
//   A'    = S_{1/mu}(D + J dtau - E + Y/mu)
//   E'    = T_{lam/mu}(D + J dtau - A' + Y/mu)
//   dtau' = G^-1 J^T (A' + E' - D - Y/mu)            (G = J^T J, no constraint rows)
//   R = D + J dtau' - A' - E';  Y' = Y + mu R;  stop when ||R|| / ||D|| < tol;  mu <- rho mu
// from A = D, E = 0, dtau = 0, Y = 0.  Entry: sc->G/Gi/jd and scal[2] = ||D||^2 from
// k5_gram(use_q = false).  The SVT is the same one-sided Jacobi + left-factor reconstruction
// as LADMAP's (svt_into); J dtau is formed per pixel from the p planes.  Exit: A, E, Y,
// sc->dtau.
template <int NCH, bool TCP>
static __device__ AdmOut k_inner_adm(const Dims& d, double lam, double tol, double rho, double mu0, int max_iter,
                                     const float* __restrict__ D, const float* __restrict__ J, float* __restrict__ A,
                                     float* __restrict__ E, float* __restrict__ Y, SvdBufs buf, const SmemLayout& L,
                                     int jsched) {
    Scratch* sc = L.sc;
    const int p = d.p, S = d.S, R = d.R, ldb = d.ldb;
    AdmOut out;
    out.iters = out.sweeps = out.warm = 0;
    out.converged = out.bad = out.tc_timeout = false;
    out.residual = 0.0;
    out.mu_last = mu0;
    const double nD = sc->scal[2] > 0.0 ? sqrt(sc->scal[2]) : 1.0;
    // A_0 = D, E_0 = 0, Y_0 = 0, dtau_0 = 0; the first M = D
    for (int e = threadIdx.x; e < S; e += NT) {
        const float dv = D[e];
        A[e] = dv;
        E[e] = 0.f;
        Y[e] = 0.f;
        buf.T[(size_t)(e / R) * ldb + (e % R)] = dv;
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < PMAX; ++k) { sc->dtau[k] = 0.0; sc->jy[k] = 0.0; sc->fs[FS_CC + k] = 0.f; }
        sc->scal[12] = mu0;
        sc->fs[FS_IMU] = (float)(1.0 / mu0);
        sc->fs[FS_THR] = (float)(lam / mu0);
        sc->fs[FS_MU] = (float)mu0;
    }
    __syncthreads();
    bool haveV = false;
    for (int k = 1; k <= max_iter; ++k) {
        out.iters = k;
        // A' = S_{1/mu}(M), J^T A' -> ja
        const SvtStepOut so = svt_into<NCH, TCP>(d, buf, L, haveV, true, sc->fs[FS_IMU], A, J, jsched);
        if (so.warm) out.warm++;
        out.sweeps += so.sweeps;
        if (so.tc_timeout) {
            out.bad = out.tc_timeout = true;
            break;
        }
        const float imu = sc->fs[FS_IMU], thr = sc->fs[FS_THR], muf = sc->fs[FS_MU];
        // E' = T_{lam/mu}(D + J dtau - A' + Y/mu); J^T E'
        {
            float cc[PMAX];
#pragma unroll
            for (int k2 = 0; k2 < PMAX; ++k2) cc[k2] = sc->fs[FS_CC + k2];
            float acc[PMAX];
#pragma unroll
            for (int k2 = 0; k2 < PMAX; ++k2) acc[k2] = 0.f;
            for (int e = threadIdx.x; e < S; e += NT) {
                float jv[PMAX];
                float jd = 0.f;
#pragma unroll
                for (int k2 = 0; k2 < PMAX; ++k2) {
                    jv[k2] = k2 < p ? J[(size_t)k2 * S + e] : 0.f;
                    jd = fmaf(jv[k2], cc[k2], jd);
                }
                const float en = soft((D[e] + jd - A[e]) + Y[e] * imu, thr);
                E[e] = en;
#pragma unroll
                for (int k2 = 0; k2 < PMAX; ++k2) acc[k2] = fmaf(jv[k2], en, acc[k2]);
            }
            block_sum_f<PMAX>(acc, sc->red);
            if (threadIdx.x == 0) {
                // dtau' = G^-1 J^T (A' + E' - D - Y/mu)
                const double imu64 = 1.0 / sc->scal[12];
                double v[PMAX];
                for (int k2 = 0; k2 < p; ++k2) {
                    sc->je[k2] = block_total(sc->red, k2);
                    v[k2] = sc->ja[k2] + sc->je[k2] - sc->jd[k2] - sc->jy[k2] * imu64;
                }
                ginv_apply(sc, p, v, sc->dtau);
                for (int k2 = 0; k2 < PMAX; ++k2) sc->fs[FS_CC + k2] = k2 < p ? (float)sc->dtau[k2] : 0.f;
                const double mu_next = rho * sc->scal[12];
                sc->fs[FS_IMUN] = (float)(1.0 / mu_next);
            }
            __syncthreads();
        }
        // R = D + J dtau' - A' - E'; Y' = Y + mu R; ||R||^2; J^T Y'; next M = D + J dtau' - E' + Y'/(rho mu)
        {
            float cc[PMAX];
#pragma unroll
            for (int k2 = 0; k2 < PMAX; ++k2) cc[k2] = sc->fs[FS_CC + k2];
            const float imun = sc->fs[FS_IMUN];
            float acc[1 + PMAX];
#pragma unroll
            for (int k2 = 0; k2 < 1 + PMAX; ++k2) acc[k2] = 0.f;
            for (int e = threadIdx.x; e < S; e += NT) {
                float jv[PMAX];
                float jd = 0.f;
#pragma unroll
                for (int k2 = 0; k2 < PMAX; ++k2) {
                    jv[k2] = k2 < p ? J[(size_t)k2 * S + e] : 0.f;
                    jd = fmaf(jv[k2], cc[k2], jd);
                }
                const float dj = D[e] + jd;
                const float ee = E[e];
                const float r = (dj - A[e]) - ee;
                const float y = fmaf(muf, r, Y[e]);
                Y[e] = y;
                acc[0] = fmaf(r, r, acc[0]);
#pragma unroll
                for (int k2 = 0; k2 < PMAX; ++k2) acc[1 + k2] = fmaf(jv[k2], y, acc[1 + k2]);
                buf.T[(size_t)(e / R) * ldb + (e % R)] = (dj - ee) + y * imun;
            }
            block_sum_f<1 + PMAX>(acc, sc->red);
            if (threadIdx.x == 0) {
                const double res = sqrt(block_total(sc->red, 0)) / nD;
                sc->scal[15] = res;
                for (int k2 = 0; k2 < p; ++k2) sc->jy[k2] = block_total(sc->red, 1 + k2);
                int ctl = LOOP_GO;
                if (!isfinite(res)) ctl = LOOP_BAD;
                else if (res < tol) ctl = LOOP_CONVERGED;
                sc->iscal[5] = ctl;
                sc->scal[16] = sc->scal[12];
                if (ctl == LOOP_GO) {
                    const double mu_next = rho * sc->scal[12];
                    sc->scal[12] = mu_next;
                    sc->fs[FS_IMU] = (float)(1.0 / mu_next);
                    sc->fs[FS_THR] = (float)(lam / mu_next);
                    sc->fs[FS_MU] = (float)mu_next;
                }
            }
            __syncthreads();
        }
        const int ctl = sc->iscal[5];
        out.residual = sc->scal[15];
        out.mu_last = sc->scal[16];
        if (ctl == LOOP_BAD) { out.bad = true; break; }
        if (ctl == LOOP_CONVERGED) { out.converged = true; break; }
    }
    return out;
}

// Largest corner displacement (pixels) between tau and tau + dtau (outer stopping rule).
__device__ inline double corner_shift(const double* tau, const double* dtau, int ttype, int m, int n, int p) {
    const double a = 0.5 * (n - 1), b = 0.5 * (m - 1);
    const double cu[4] = {-a, a, a, -a}, cv[4] = {-b, -b, b, b};
    double t1[PMAX];
    for (int k = 0; k < PMAX; ++k) t1[k] = k < p ? tau[k] + dtau[k] : 0.0;
    double mx = 0.0;
    for (int c = 0; c < 4; ++c) {
        MapPt q0 = map_point(tau, ttype, cu[c], cv[c]);
        MapPt q1 = map_point(t1, ttype, cu[c], cv[c]);
        mx = fmax(mx, hypot(q1.x - q0.x, q1.y - q0.y));
    }
    return mx;
}

// Algorithm 1 for one problem.
template <int NCH, bool TCP = true>
static __device__ void solve_problem(const Problem& pr, const SmemLayout& L, Result& res) {
    Scratch* sc = L.sc;
    const Dims d = make_dims(pr.m, pr.n, pr.p);
    const Params& prm = pr.prm;
    const int S = d.S;
    SvdBufs buf;
    {
        float* sm = L.svd;
        const size_t nb = (size_t)d.ldb * d.Cp, nv = (size_t)d.ldv * d.Cp;
        if (pr.smem_svd & 1) { buf.B = sm; sm += nb; } else { buf.B = pr.pl.Bg; }
        if (pr.smem_svd & 2) { buf.V = sm; sm += nv; } else { buf.V = pr.pl.Vg; }
        if (pr.smem_svd & 4) { buf.T = sm; sm += nb; } else { buf.T = pr.pl.Tg; }
        if (pr.smem_svd & 8) { buf.Z = sm; sm += (size_t)d.C * d.Cp; } else { buf.Z = pr.pl.Zg; }
        buf.stage = reinterpret_cast<unsigned char*>(sm);  // after the buffers that live in shared memory
        buf.nbuf = pr.tc_nbuf;
        buf.tc = pr.tc_nbuf > 0;
    }
    // zero the SVD buffers (padding rows/columns are read by the tiled GEMM)
    {
        const size_t nb = (size_t)d.ldb * d.Cp, nv = (size_t)d.ldv * d.Cp;
        for (size_t e = threadIdx.x; e < nb; e += NT) { buf.B[e] = 0.f; buf.T[e] = 0.f; }
        for (size_t e = threadIdx.x; e < nv; e += NT) buf.V[e] = 0.f;
    }
    const double lam = prm.lam > 0.0 ? prm.lam : 1.0 / sqrt((double)max(pr.m, pr.n));
    if (threadIdx.x < PMAX) sc->tau[threadIdx.x] = threadIdx.x < pr.p ? pr.tau[threadIdx.x] : 0.0;
    res.cyc_warp = res.cyc_svd = res.cyc_recon = res.cyc_elem = res.cyc_other = 0;
    if (threadIdx.x == 0) {
        sc->iscal[7] = cancel_requested(pr.cancel);
        sc->iscal[0] = 0;
    }
    __syncthreads();

    int status = sc->iscal[7] ? -4 : 1;
    bool inner_maxed = false;
    int outer = 0, inner_total = 0, sweeps = 0, warm = 0, reorth = 0, cayley = 0, rank = 0;
    double c1 = 0.0, nuc = 0.0, l1 = 0.0;
    bool haveV = false;

    unsigned long long t0 = clk();
    if (status != -4) k1_warp_jacobian(pr.img, pr.ld, pr.H, pr.W, d, pr.ttype, sc->tau, pr.pl.Dhat, pr.pl.J, sc);
    if (threadIdx.x == 0) res.cyc_warp += clk() - t0;
    if (status == -4) {
        // cancelled before it started: tau stays tau0
    } else if (!isfinite(sc->scal[0])) {
        status = -1;                                   // a non-finite sample in the window
    } else if (!(sc->scal[0] > 0.0)) {
        status = -3;
    } else {
        for (int e = threadIdx.x; e < S; e += NT) {     // A_0 = D_hat (R9), E_0 = Y_0 = 0
            pr.pl.A[e] = pr.pl.Dhat[e];
            pr.pl.E[e] = 0.f;
            pr.pl.Y[e] = 0.f;
            pr.pl.Mp[e] = 0.f;
        }
        __syncthreads();
        for (outer = 1; outer <= prm.max_outer; ++outer) {
            t0 = clk();
            if (outer > 1) {
                k1_warp_jacobian(pr.img, pr.ld, pr.H, pr.W, d, pr.ttype, sc->tau, pr.pl.Dhat, pr.pl.J, sc);
                if (!isfinite(sc->scal[0])) { status = -1; break; }
                if (!(sc->scal[0] > 0.0)) { status = -3; break; }
            }
            unsigned long long t1 = clk();
            if (threadIdx.x == 0) res.cyc_warp += t1 - t0;
            if (!k5_gram(d, pr.ttype, sc->tau, pr.pl.Dhat, pr.pl.J, sc)) { status = -2; break; }
            double mu0 = prm.mu0;
            if (!(mu0 > 0.0)) mu0 = 1.25 / spectral_norm(pr.pl.Dhat, d, L.sigma, L.w, sc);
            if (threadIdx.x == 0) res.cyc_other += clk() - t1;
            InnerOut io = k_inner<NCH, TCP>(d, prm, lam, mu0, pr.pl.Dhat, pr.pl.J, pr.pl.A, pr.pl.E, pr.pl.Y,
                                  pr.pl.Mp, buf, haveV, L, &res, pr.jsched, pr.cancel, pr.pl.Cay);
            inner_total += io.iters;
            sweeps += io.sweeps;
            warm += io.warm;
            reorth += io.reorth;
            cayley += io.cayley;
            c1 = io.c1; nuc = io.nuc; l1 = io.l1; rank = io.rank;
            if (io.tc_timeout) { status = -5; break; }
            if (io.bad) { status = -1; break; }
            if (io.cancelled) { status = -4; break; }
            if (!io.converged) inner_maxed = true;
            // Steps 3-4: dtau = G^-1 J^T (A + E - D_hat) (= sc->cvec), tau <- tau + dtau
            if (threadIdx.x == 0) {
                double dt[PMAX];
                for (int k = 0; k < PMAX; ++k) dt[k] = k < pr.p ? sc->cvec[k] : 0.0;
                const double sh = corner_shift(sc->tau, dt, pr.ttype, pr.m, pr.n, pr.p);
                bool fin = isfinite(sh);
                for (int k = 0; k < pr.p; ++k) {
                    sc->tau[k] += dt[k];
                    fin = fin && isfinite(sc->tau[k]);
                }
                sc->scal[11] = fin ? sh : -1.0;
            }
            __syncthreads();
            const double sh = sc->scal[11];
            __syncthreads();
            if (sh < 0.0) { status = -1; break; }
            if (sh < prm.outer_tol) { status = 0; break; }
        }
        if (outer > prm.max_outer) outer = prm.max_outer;
    }
    if (status >= 0 && inner_maxed) status = 2;
    if (threadIdx.x == 0) {
        res.status = status;
        res.p = pr.p;
        for (int k = 0; k < 8; ++k) res.tau[k] = k < pr.p ? sc->tau[k] : 0.0;
        res.objective = nuc + lam * l1;
        res.lambda = lam;
        res.rank_A = rank;
        res.outer_iters = outer;
        res.inner_iters = inner_total;
        res.svd_sweeps = sweeps;
        res.svd_warm = warm;
        res.svd_reorth = reorth;
        res.svd_cayley = cayley;
        res.oob_pixels = sc->iscal[0];
        res.kkt_residual = c1;
    }
    __syncthreads();
}

// One CTA per problem: the whole of Algorithm 1.  The result record and the completion
// flag live in host-mapped memory, so the host sees every problem retire on its own.
// MINB CTAs per SM; NCH float4 chunks per lane keep a Jacobi column pair in registers
// (R <= 32 NCH), fewer for the 2-CTA variant so that it fits 64 registers per thread.
// TCP: the kernel carries the tensor-core path (only the launch class of large windows: the
// extra code costs the SIMT path registers).
template <int MINB, int NCH, bool TCP>
__global__ void __launch_bounds__(NT, MINB) solver_kernel(Problem* probs, const int* order) {
    extern __shared__ __align__(256) unsigned char smem_raw[];
    __shared__ Problem sp;
    __shared__ Result sres;
    SmemLayout L = carve_smem(smem_raw);
    if (TCP) tc_setup(&L.sc->tc, TC_TMEM_COLS);
    copy_to_shared(&sp, probs + order[blockIdx.x]);
    solve_problem<NCH, TCP>(sp, L, sres);
    if (threadIdx.x == 0) {
        *sp.res = sres;
        __threadfence_system();
        *sp.done = 1;
    }
    if (TCP) tc_teardown(&L.sc->tc, TC_TMEM_COLS);
}

}  // namespace tilt
