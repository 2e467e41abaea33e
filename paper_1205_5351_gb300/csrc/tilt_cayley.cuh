// The SVD warm start of Algorithm 2 (Sec. 5, Appendix A): one step along the Cayley curve of
// Eq. curve_to_search from the previous iteration's factors, accepted when it decreases
// f(t) = 1/2 ||M - U(t) Sigma(t) V(t)^T||_F^2.  Executed by all threads of the CTA that owns
// the problem, on X (the R x C long-side-contiguous form of M; the step commutes with
// transposition, P_U and P_V exchanging roles).  Dense products run as register-tiled SIMT
// GEMMs, the two linear systems of the Cayley transform by Gauss-Jordan elimination with
// partial pivoting; reductions (f'(0), f''(0), f(t)) are FP64 totals of FP32 partials.
#pragma once

#include "tilt_device.cuh"

namespace tilt {

// D (M x N) = A (M x K) B (K x N) on the SIMT pipes, TM x TN outputs per thread; la(m, k),
// lb(k, n) give operand elements, epi(m, n, v) receives each output once.  All threads.
template <int TM, int TN, class LA, class LB, class EPI>
__device__ __forceinline__ void gemm_simt(int M, int N, int K, LA la, LB lb, EPI epi) {
    const int mt = (M + TM - 1) / TM, nt = (N + TN - 1) / TN;
    for (int t = threadIdx.x; t < mt * nt; t += NT) {
        const int i0 = (t % mt) * TM, j0 = (t / mt) * TN;
        float acc[TM][TN];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
        for (int k = 0; k < K; ++k) {
            float a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = (i0 + i < M) ? la(i0 + i, k) : 0.f;
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = (j0 + j < N) ? lb(k, j0 + j) : 0.f;
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j)
                if (i0 + i < M && j0 + j < N) epi(i0 + i, j0 + j, acc[i][j]);
    }
    __syncthreads();
}

// Solve K Y = R in place (K: n x n, column-major stride ldk, destroyed; R: n x nr, stride ldr,
// overwritten by Y) by Gauss-Jordan elimination with partial pivoting.  false when a pivot is
// zero or not finite.  All threads.
static __device__ bool gj_solve(float* K, int ldk, int n, float* Rm, int ldr, int nr, Scratch* sc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* fr = reinterpret_cast<float*>(sc->red);          // staging of the pivot search
    int* ir = reinterpret_cast<int*>(fr + NW);
    for (int k = 0; k < n; ++k) {
        // pivot: largest |K[r][k]|, r >= k
        float best = -1.f;
        int bi = k;
        for (int r = k + threadIdx.x; r < n; r += NT) {
            const float v = fabsf(K[(size_t)k * ldk + r]);
            if (v > best) { best = v; bi = r; }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, off);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { fr[warp] = best; ir[warp] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            float b = fr[0];
            int i = ir[0];
            for (int w = 1; w < NW; ++w)
                if (fr[w] > b || (fr[w] == b && ir[w] < i)) { b = fr[w]; i = ir[w]; }
            sc->iscal[3] = i;
            sc->scal[19] = b;
        }
        __syncthreads();
        const int piv = sc->iscal[3];
        const float pv = (float)sc->scal[19];
        if (!(pv > 0.f) || !isfinite(pv)) return false;
        // swap rows k and piv of K and R
        if (piv != k) {
            for (int c = threadIdx.x; c < n + nr; c += NT) {
                float* a = c < n ? K + (size_t)c * ldk : Rm + (size_t)(c - n) * ldr;
                const float t = a[k];
                a[k] = a[piv];
                a[piv] = t;
            }
            __syncthreads();
        }
        // scale row k by 1 / K[k][k], then eliminate column k from every other row
        const float inv = 1.f / K[(size_t)k * ldk + k];
        __syncthreads();
        for (int c = k + threadIdx.x; c < n + nr; c += NT) {
            float* a = c < n ? K + (size_t)c * ldk : Rm + (size_t)(c - n) * ldr;
            a[k] *= inv;
        }
        __syncthreads();
        // column k of K before elimination: the multipliers
        const int cols = n + nr - k - 1;                     // columns k+1 .. n+nr-1
        for (int idx = threadIdx.x; idx < n * cols; idx += NT) {
            const int r = idx % n, c = k + 1 + idx / n;
            if (r == k) continue;
            float* a = c < n ? K + (size_t)c * ldk : Rm + (size_t)(c - n) * ldr;
            a[r] = fmaf(-K[(size_t)k * ldk + r], a[k], a[r]);
        }
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += NT) K[(size_t)k * ldk + r] = (r == k) ? 1.f : 0.f;
        __syncthreads();
    }
    return true;
}

// Workspace of the Cayley step (device memory): R x C planes at stride ldb, R x R at ldb,
// C x C at ldv.
struct CayBufs {
    float *U, *S;              // previous left factor (unit columns) and diagonal (C)
    float *X, *H0, *H1, *Z, *H2, *UPS, *MV;
    float *PU, *PV, *RV;       // R x R, C x C, C x C
};

__device__ inline CayBufs carve_cayley(float* base, const Dims& d) {
    CayBufs c;
    const size_t pl = (size_t)d.ldb * d.Cp;
    c.U = base;
    c.X = c.U + pl;
    c.H0 = c.X + pl;
    c.H1 = c.H0 + pl;
    c.Z = c.H1 + pl;
    c.H2 = c.Z + pl;
    c.UPS = c.H2 + pl;
    c.MV = c.UPS + pl;
    c.PU = c.MV + pl;
    c.PV = c.PU + (size_t)d.ldb * d.ldb;
    c.RV = c.PV + (size_t)d.ldv * d.Cp;
    c.S = c.RV + (size_t)d.ldv * d.Cp;
    return c;
}

struct CayleyOut {
    bool accepted;
    double f1, f2, t, f0, ft;
};

// One step of Algorithm 2 on Mx (R x C, stride ldb) from (cb.U, cb.S, V): Step 1 the projected
// gradients P_U = X M^T - M X^T, P_V = X^T M - M^T X, P_Sigma = Sigma - diag(U^T M V) with
// X = U Sigma V^T (Appendix A); Step 2 f'(0) = <h0, h1>, f''(0) = ||h1||^2 + <h0, h2> with
// h0 = M - X, h1 = P_U X + U P_Sigma V^T - X P_V, h2 = -P_U Z + Z P_V, Z = h1 + U P_Sigma V^T,
// and t = -f'(0) / f''(0); Step 3 the curve point U(t), Sigma(t), V(t) of Eq.
// curve_to_search.  Accepted (cb.U, cb.S, V overwritten) when f''(0) > 0 and f(t) <= f(0);
// otherwise nothing changes (the caller computes a full SVD).  All threads.
static __device__ CayleyOut cayley_step(const Dims& d, const float* __restrict__ Mx, CayBufs cb, float* V,
                                        Scratch* sc) {
    const int R = d.R, C = d.C, ldb = d.ldb, ldv = d.ldv;
    CayleyOut o;
    o.accepted = false;
    o.f1 = o.f2 = o.t = o.f0 = o.ft = 0.0;
    float* U = cb.U;
    const float* S = cb.S;
    // X = U Sigma V^T; h0 = M - X
    {
        float* X = cb.X;
        float* H0 = cb.H0;
        gemm_simt<4, 4>(R, C, C, [=](int r, int j) { return U[(size_t)j * ldb + r] * S[j]; },
                        [=](int j, int c) { return V[(size_t)j * ldv + c]; },
                        [=](int r, int c, float v) {
                            X[(size_t)c * ldb + r] = v;
                            H0[(size_t)c * ldb + r] = Mx[(size_t)c * ldb + r] - v;
                        });
    }
    // P_V = X^T M - M^T X (C x C): G = X^T M, then G - G^T
    {
        const float* X = cb.X;
        float* PV = cb.PV;
        gemm_simt<4, 4>(C, C, R, [=](int i, int r) { return X[(size_t)i * ldb + r]; },
                        [=](int r, int j) { return Mx[(size_t)j * ldb + r]; },
                        [=](int i, int j, float v) { PV[(size_t)j * ldv + i] = v; });
        for (int idx = threadIdx.x; idx < C * C; idx += NT) {
            const int i = idx % C, j = idx / C;
            if (i < j) {
                const float a = PV[(size_t)j * ldv + i], b = PV[(size_t)i * ldv + j];
                PV[(size_t)j * ldv + i] = a - b;
                PV[(size_t)i * ldv + j] = b - a;
            } else if (i == j) {
                PV[(size_t)j * ldv + i] = 0.f;
            }
        }
        __syncthreads();
    }
    // P_U = X M^T - M X^T (R x R)
    {
        const float* X = cb.X;
        float* PU = cb.PU;
        gemm_simt<4, 4>(R, R, C, [=](int r, int c) { return X[(size_t)c * ldb + r]; },
                        [=](int c, int s) { return Mx[(size_t)c * ldb + s]; },
                        [=](int r, int s, float v) { PU[(size_t)s * ldb + r] = v; });
        for (int idx = threadIdx.x; idx < R * R; idx += NT) {
            const int i = idx % R, j = idx / R;
            if (i < j) {
                const float a = PU[(size_t)j * ldb + i], b = PU[(size_t)i * ldb + j];
                PU[(size_t)j * ldb + i] = a - b;
                PU[(size_t)i * ldb + j] = b - a;
            } else if (i == j) {
                PU[(size_t)j * ldb + i] = 0.f;
            }
        }
        __syncthreads();
    }
    // P_Sigma_i = Sigma_i - u_i^T M v_i (MV = M V, then column dots in FP64), kept in the first
    // column of RV until the right-hand side of V(t) needs it, then in the first column of Z
    float* PS = cb.RV;
    {
        float* MV = cb.MV;
        gemm_simt<4, 4>(R, C, C, [=](int r, int j) { return Mx[(size_t)j * ldb + r]; },
                        [=](int j, int c) { return V[(size_t)c * ldv + j]; },
                        [=](int r, int c, float v) { MV[(size_t)c * ldb + r] = v; });
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int i = warp; i < C; i += NW) {
            double s = 0.0;
            for (int r = lane; r < R; r += 32) s += (double)U[(size_t)i * ldb + r] * (double)MV[(size_t)i * ldb + r];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) PS[i] = (float)((double)S[i] - s);
        }
        __syncthreads();
    }
    // UPS = U P_Sigma V^T; h1 = P_U X + UPS - X P_V; Z = h1 + UPS; h2 = -P_U Z + Z P_V
    {
        float* UPS = cb.UPS;
        gemm_simt<4, 4>(R, C, C, [=](int r, int j) { return U[(size_t)j * ldb + r] * PS[j]; },
                        [=](int j, int c) { return V[(size_t)j * ldv + c]; },
                        [=](int r, int c, float v) { UPS[(size_t)c * ldb + r] = v; });
        const float* PU = cb.PU;
        const float* PV = cb.PV;
        const float* X = cb.X;
        float* H1 = cb.H1;
        gemm_simt<4, 4>(R, C, R, [=](int r, int s) { return PU[(size_t)s * ldb + r]; },
                        [=](int s, int c) { return X[(size_t)c * ldb + s]; },
                        [=](int r, int c, float v) { H1[(size_t)c * ldb + r] = v + UPS[(size_t)c * ldb + r]; });
        float* Z = cb.Z;
        gemm_simt<4, 4>(R, C, C, [=](int r, int j) { return X[(size_t)j * ldb + r]; },
                        [=](int j, int c) { return PV[(size_t)c * ldv + j]; },
                        [=](int r, int c, float v) {
                            const size_t e = (size_t)c * ldb + r;
                            const float h = H1[e] - v;
                            H1[e] = h;
                            Z[e] = h + UPS[e];
                        });
        float* H2 = cb.H2;
        gemm_simt<4, 4>(R, C, R, [=](int r, int s) { return PU[(size_t)s * ldb + r]; },
                        [=](int s, int c) { return Z[(size_t)c * ldb + s]; },
                        [=](int r, int c, float v) { H2[(size_t)c * ldb + r] = -v; });
        gemm_simt<4, 4>(R, C, C, [=](int r, int j) { return Z[(size_t)j * ldb + r]; },
                        [=](int j, int c) { return PV[(size_t)c * ldv + j]; },
                        [=](int r, int c, float v) { H2[(size_t)c * ldb + r] += v; });
    }
    // f'(0), f''(0), f(0)
    {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int e = threadIdx.x; e < R * C; e += NT) {
            const size_t q = (size_t)(e / R) * ldb + (e % R);
            const float h0 = cb.H0[q], h1 = cb.H1[q], h2 = cb.H2[q];
            acc[0] = fmaf(h0, h1, acc[0]);
            acc[1] = fmaf(h1, h1, acc[1]);
            acc[2] = fmaf(h0, h2, acc[2]);
            acc[3] = fmaf(h0, h0, acc[3]);
        }
        block_sum_f<4>(acc, sc->red);
        o.f1 = block_total(sc->red, 0);
        o.f2 = block_total(sc->red, 1) + block_total(sc->red, 2);
        o.f0 = 0.5 * block_total(sc->red, 3);
        __syncthreads();
    }
    if (!(o.f2 > 0.0)) return o;
    o.t = -o.f1 / o.f2;
    const float a = (float)(0.5 * o.t);
    // U(t) = (I + a P_U)^-1 (I - a P_U) U: right-hand side into H2, system into P_U
    {
        const float* PU = cb.PU;
        float* RU = cb.H2;
        gemm_simt<4, 4>(R, C, R, [=](int r, int s) { return PU[(size_t)s * ldb + r]; },
                        [=](int s, int c) { return U[(size_t)c * ldb + s]; },
                        [=](int r, int c, float v) { RU[(size_t)c * ldb + r] = U[(size_t)c * ldb + r] - a * v; });
        float* K = cb.PU;
        for (int idx = threadIdx.x; idx < R * R; idx += NT) {
            const int i = idx % R, j = idx / R;
            const size_t q = (size_t)j * ldb + i;
            K[q] = (i == j ? 1.f : 0.f) + a * K[q];
        }
        __syncthreads();
        if (!gj_solve(K, ldb, R, RU, ldb, C, sc)) return o;
    }
    // V(t) = (I + a P_V)^-1 (I - a P_V) V: right-hand side into RV, system into P_V
    {
        for (int i = threadIdx.x; i < C; i += NT) cb.Z[i] = PS[i];      // Z is free after h2
        __syncthreads();
        const float* PV = cb.PV;
        float* RV = cb.RV;
        gemm_simt<4, 4>(C, C, C, [=](int i, int j) { return PV[(size_t)j * ldv + i]; },
                        [=](int j, int c) { return V[(size_t)c * ldv + j]; },
                        [=](int i, int c, float v) { RV[(size_t)c * ldv + i] = V[(size_t)c * ldv + i] - a * v; });
        float* K = cb.PV;
        for (int idx = threadIdx.x; idx < C * C; idx += NT) {
            const int i = idx % C, j = idx / C;
            const size_t q = (size_t)j * ldv + i;
            K[q] = (i == j ? 1.f : 0.f) + a * K[q];
        }
        __syncthreads();
        if (!gj_solve(K, ldv, C, RV, ldv, C, sc)) return o;
    }
    // Sigma(t) = Sigma - t P_Sigma (in X's first column: X is free after h1), and
    // f(t) = 1/2 ||M - U(t) Sigma(t) V(t)^T||^2
    {
        const float* RU = cb.H2;
        const float* RV = cb.RV;
        float* St = cb.X;
        const float tf = (float)o.t;
        const float* PSk = cb.Z;
        for (int i = threadIdx.x; i < C; i += NT) St[i] = S[i] - tf * PSk[i];
        __syncthreads();
        float acc[1] = {0.f};
        gemm_simt<4, 4>(R, C, C, [=](int r, int j) { return RU[(size_t)j * ldb + r] * St[j]; },
                        [=](int j, int c) { return RV[(size_t)j * ldv + c]; },
                        [&](int r, int c, float v) {
                            const float dv = Mx[(size_t)c * ldb + r] - v;
                            acc[0] = fmaf(dv, dv, acc[0]);
                        });
        block_sum_f<1>(acc, sc->red);
        o.ft = 0.5 * block_total(sc->red, 0);
        __syncthreads();
        if (!(o.ft <= o.f0)) return o;
        // accept: U <- U(t), Sigma <- Sigma(t), V <- V(t)
        for (int e = threadIdx.x; e < ldb * C; e += NT) U[e] = RU[e];
        for (int e = threadIdx.x; e < ldv * C; e += NT) V[e] = RV[e];
        float* Sw = cb.S;
        for (int i = threadIdx.x; i < C; i += NT) Sw[i] = St[i];
        __syncthreads();
    }
    o.accepted = true;
    return o;
}

}  // namespace tilt
