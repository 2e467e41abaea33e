// RASL (Sec. 1: TILT's model with one image per column of the data matrix) solved by the
// same LADMAP inner loop and outer loop as TILT, one CTA per image set.
//
// The Jacobian of vec(D_hat) in the stacked parameters [tau_1; ...; tau_N] is block-diagonal
// (block c: J_c, the derivative of column c by tau_c) and the constraint rows Q = [I_p ... I_p]
// keep the sum of the increments at zero, so
//   G = J^T J + Q^T Q = blockdiag(G_c) + (1 1^T) (x) I_p,         G_c = J_c^T J_c,
// and by the Sherman-Morrison-Woodbury identity, for v = J^T x (v_c = J_c^T x_c),
//   (G^-1 v)_c = b_c - G_c^-1 t,   b_c = G_c^-1 v_c,   t = K sum_c b_c,   K = (I_p + sum_c G_c^-1)^-1.
// W^T W x = x - J G^-1 J^T x (Eq. WTW_property) then acts on column c with its own
// coefficients c_c = (G^-1 v)_c.  A column pass is done by one warp per column (the column's
// coefficients are warp-uniform and its J^T products reduce with shuffles); the sum over the
// columns and t are formed by warp 0 between two CTA barriers.
#pragma once

#include "tilt_solver.cuh"

namespace tilt {

__device__ inline double* rasl_row(const RaslProblem& pr, int c) { return pr.col + (size_t)c * RASL_COLW; }

__device__ inline double warp_sum64(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Totals of p per-lane partials over the warp (every lane gets them).
__device__ inline void warp_sum_p(float (&v)[PMAX], int p) {
#pragma unroll
    for (int k = 0; k < PMAX; ++k)
        if (k < p) v[k] = warp_sum(v[k]);
}

// row[slot + k] = (G_c^-1 (v - sub))_k in FP64, by lanes k < p (v: warp totals; sub may be null).
__device__ inline void rasl_store_b(double* row, int slot, const float (&v)[PMAX], const double* sub, int p, int lane) {
    if (lane < p) {
        double b = 0.0;
#pragma unroll
        for (int j = 0; j < PMAX; ++j)
            if (j < p) b += row[RC_GI + lane * PMAX + j] * ((double)v[j] - (sub ? sub[j] : 0.0));
        row[slot + lane] = b;
    }
}

// t = K sum_c row_c[slot] into out[0 .. p) (K in sc->Gi).  Warp 0, between two CTA barriers
// (the b vectors are stored before, t is read after).  Fixed summation order.
__device__ inline void rasl_sum_t(const RaslProblem& pr, int slot, const Scratch* sc, double* out, int p, int lane) {
    double s[PMAX];
#pragma unroll
    for (int k = 0; k < PMAX; ++k) s[k] = 0.0;
    for (int c = lane; c < pr.nimg; c += 32) {
        const double* row = rasl_row(pr, c);
#pragma unroll
        for (int k = 0; k < PMAX; ++k)
            if (k < p) s[k] += row[slot + k];
    }
#pragma unroll
    for (int k = 0; k < PMAX; ++k)
        if (k < p) s[k] = warp_sum64(s[k]);
    if (lane < p) {
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < PMAX; ++j)
            if (j < p) t += sc->Gi[lane * PMAX + j] * s[j];
        out[lane] = t;
    }
}

// Coefficients c_c = b_c - G_c^-1 t of column c (b_c at row[slot]) as floats in every lane;
// keep: also as doubles in row[RC_CV].  All lanes of the warp.
__device__ inline void rasl_coeffs(double* row, int slot, const double* t, int p, int lane, float (&cf)[PMAX],
                                   bool keep) {
    double ck = 0.0;
    if (lane < p) {
        ck = row[slot + lane];
#pragma unroll
        for (int j = 0; j < PMAX; ++j)
            if (j < p) ck -= row[RC_GI + lane * PMAX + j] * t[j];
        if (keep) row[RC_CV + lane] = ck;
    }
#pragma unroll
    for (int k = 0; k < PMAX; ++k) {
        const double v = __shfl_sync(0xffffffffu, ck, k);
        cf[k] = k < p ? (float)v : 0.f;
    }
}

// W consecutive floats (W = 4: one 16-byte access; the column passes use it when R % 4 == 0,
// so every column of every plane starts on a 16-byte boundary).
template <int W>
__device__ __forceinline__ void ldw(const float* __restrict__ p, float (&v)[W]) {
    if constexpr (W == 4) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
#pragma unroll
        for (int u = 0; u < W; ++u) v[u] = p[u];
    }
}
template <int W>
__device__ __forceinline__ void stw(float* __restrict__ p, const float (&v)[W]) {
    if constexpr (W == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int u = 0; u < W; ++u) p[u] = v[u];
    }
}

// Column passes of the inner loop over rows [r0, r1) of one column, W rows per lane step
// (column pointers: A, E, D_hat, Y, Mp and T at the column's first row; Jc = J + c R, plane k
// at Jc + k S).
//   v += J_c^T (A + E - D_hat)
template <int W>
__device__ __forceinline__ void col_jt_residual(const float* __restrict__ A, const float* __restrict__ E,
                                                const float* __restrict__ D, const float* __restrict__ Jc, size_t S,
                                                int r0, int r1, int lane, int p, float (&v)[PMAX]) {
    for (int r = r0 + W * lane; r < r1; r += 32 * W) {
        float a[W], e[W], d[W], x[W];
        ldw<W>(A + r, a);
        ldw<W>(E + r, e);
        ldw<W>(D + r, d);
#pragma unroll
        for (int u = 0; u < W; ++u) x[u] = a[u] + e[u] - d[u];
#pragma unroll
        for (int k = 0; k < PMAX; ++k) {
            if (k < p) {
                float j[W];
                ldw<W>(Jc + (size_t)k * S + r, j);
#pragma unroll
                for (int u = 0; u < W; ++u) v[k] = fmaf(j[u], x[u], v[k]);
            }
        }
    }
}

//   E' = T_thr(E - Y imu - ((A + E - D_hat) - J_c cc)); acc += (||E' - E||^2, ||E'||_1);
//   w += J_c^T (A + E' - D_hat)
template <int W>
__device__ __forceinline__ void col_e_update(const float* __restrict__ A, float* __restrict__ E,
                                             const float* __restrict__ D, const float* __restrict__ Y,
                                             const float* __restrict__ Jc, size_t S, int r0, int r1, int lane, int p,
                                             const float (&cc)[PMAX], float imu, float thr, float (&acc)[2],
                                             float (&w)[PMAX]) {
    for (int r = r0 + W * lane; r < r1; r += 32 * W) {
        float a[W], e[W], d[W], y[W], jc[W], en[W];
        ldw<W>(A + r, a);
        ldw<W>(E + r, e);
        ldw<W>(D + r, d);
        ldw<W>(Y + r, y);
        float jv[PMAX][W];
#pragma unroll
        for (int u = 0; u < W; ++u) jc[u] = 0.f;
#pragma unroll
        for (int k = 0; k < PMAX; ++k) {
            if (k < p) {
                ldw<W>(Jc + (size_t)k * S + r, jv[k]);
            } else {
#pragma unroll
                for (int u = 0; u < W; ++u) jv[k][u] = 0.f;
            }
#pragma unroll
            for (int u = 0; u < W; ++u) jc[u] = fmaf(jv[k][u], cc[k], jc[u]);
        }
#pragma unroll
        for (int u = 0; u < W; ++u) {
            const float p1 = (a[u] + e[u] - d[u]) - jc[u];
            const float nv = e[u] - y[u] * imu - p1;
            en[u] = soft(nv, thr);
            const float de = en[u] - e[u];
            acc[0] = fmaf(de, de, acc[0]);
            acc[1] += fabsf(en[u]);
            const float x2 = a[u] + en[u] - d[u];
#pragma unroll
            for (int k = 0; k < PMAX; ++k) w[k] = fmaf(jv[k][u], x2, w[k]);
        }
        stw<W>(E + r, en);
    }
}

//   P'' = (A + E - D_hat) - J_c cc;  Y' = Y + mu P'';  M = A - Y' imun - P'' (into T, and into
//   Mp while the warm-start gate is on);  acc += (||P''||^2, ||M - M_prev||^2, ||M||^2), the
//   last two only while the gate is on
template <int W>
__device__ __forceinline__ void col_y_update(const float* __restrict__ A, const float* __restrict__ E,
                                             const float* __restrict__ D, float* __restrict__ Y, float* __restrict__ T,
                                             float* __restrict__ Mp, const float* __restrict__ Jc, size_t S, int r0,
                                             int r1, int lane, int p, const float (&cc)[PMAX], float muf, float imun,
                                             bool gate, float (&acc)[3]) {
    for (int r = r0 + W * lane; r < r1; r += 32 * W) {
        float a[W], e[W], d[W], y[W], mo[W], jc[W], mv[W];
        ldw<W>(A + r, a);
        ldw<W>(E + r, e);
        ldw<W>(D + r, d);
        ldw<W>(Y + r, y);
        if (gate) ldw<W>(Mp + r, mo);
#pragma unroll
        for (int u = 0; u < W; ++u) jc[u] = 0.f;
#pragma unroll
        for (int k = 0; k < PMAX; ++k) {
            if (k < p) {
                float j[W];
                ldw<W>(Jc + (size_t)k * S + r, j);
#pragma unroll
                for (int u = 0; u < W; ++u) jc[u] = fmaf(j[u], cc[k], jc[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < W; ++u) {
            const float pp = (a[u] + e[u] - d[u]) - jc[u];
            y[u] = fmaf(muf, pp, y[u]);
            acc[0] = fmaf(pp, pp, acc[0]);
            mv[u] = a[u] - y[u] * imun - pp;
            if (gate) {
                acc[1] = fmaf(mv[u] - mo[u], mv[u] - mo[u], acc[1]);
                acc[2] = fmaf(mv[u], mv[u], acc[2]);
            }
        }
        stw<W>(Y + r, y);
        stw<W>(T + r, mv);
        if (gate) stw<W>(Mp + r, mv);
    }
}

// s + c += x y without rounding error of the product and of the sum beyond FP32's own: the
// product's rounding error from an FMA and the sum's from Knuth's two-sum, carried in c (the
// compensated dot product of Ogita, Rump and Oishi, 2005).  The per-lane sums of the set's
// once-per-outer-step reductions run in FP32 this way, as accurate as FP64 sums of the same
// FP32 data and several times cheaper on this part (FP64 issues at 1/64 of the FP32 rate).
// (The _rn intrinsics keep the compiler from fusing a product into a neighbouring sum, which
// would break the error terms.)
__device__ __forceinline__ void dot2_add(float& s, float& c, float x, float y) {
    const float prod = __fmul_rn(x, y);
    const float perr = fmaf(x, y, -prod);
    const float t = __fadd_rn(s, prod);
    const float z = __fsub_rn(t, s);
    c = __fadd_rn(c, __fadd_rn(__fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(prod, z)), perr));
    s = t;
}

// Step 1 of Algorithm 1 for every image of the set: column c of D_hat is image c sampled at
// tau_c over the window (pixel r = i n + j), divided by its Frobenius norm; column c of J_k
// the derivative of that normalised column by tau_c[k] (the quotient rule, per column).  One
// warp per column, FP64 sums.  Leaves the smallest column norm in scal[0] (NaN when a sample
// is not finite) and the clamped-sample count in iscal[0].
static __device__ void rasl_warp(const RaslProblem& pr, const Dims& d, float* __restrict__ Dhat,
                                 float* __restrict__ J, Scratch* sc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = d.p, S = d.S, R = d.R, n = pr.n;
    const double hm = 0.5 * (pr.m - 1), hn = 0.5 * (pr.n - 1);
    if (threadIdx.x == 0) sc->iscal[0] = 0;
    __syncthreads();
    for (int c = warp; c < d.C; c += NW) {
        double* row = rasl_row(pr, c);
        double tau[PMAX];
#pragma unroll
        for (int k = 0; k < PMAX; ++k) tau[k] = k < p ? row[RC_TAU + k] : 0.0;
        const float* img = pr.imgs + (size_t)c * pr.img_stride;
        float* Dc = Dhat + (size_t)c * R;
        float* Jc = J + (size_t)c * R;
        float fs[1 + PMAX], fc[1 + PMAX];     // ||D||^2, D . Jraw_k (compensated FP32)
#pragma unroll
        for (int k = 0; k < 1 + PMAX; ++k) { fs[k] = 0.f; fc[k] = 0.f; }
        int nout = 0;
        for (int r = lane; r < R; r += 32) {
            const int i = r / n, j = r - i * n;
            const double u = (double)j - hn, v = (double)i - hm;
            float jr[PMAX];
            bool inside;
            const float val = warp_sample(img, pr.ld, pr.H, pr.W, pr.ttype, tau, u, v, jr, inside);
            Dc[r] = val;
            dot2_add(fs[0], fc[0], val, val);
            nout += inside ? 0 : 1;
#pragma unroll
            for (int k = 0; k < PMAX; ++k) {
                if (k < p) {
                    Jc[(size_t)k * S + r] = jr[k];
                    dot2_add(fs[1 + k], fc[1 + k], val, jr[k]);
                }
            }
        }
        double acc[2 + PMAX];
        acc[0] = warp_sum64((double)fs[0] + (double)fc[0]);
        acc[1] = warp_sum64((double)nout);
#pragma unroll
        for (int k = 0; k < PMAX; ++k) acc[2 + k] = warp_sum64((double)fs[1 + k] + (double)fc[1 + k]);
        const double s = sqrt(acc[0]);
        const float inv = (s > 0.0) ? (float)(1.0 / s) : 0.f;
        float a[PMAX];
#pragma unroll
        for (int k = 0; k < PMAX; ++k) a[k] = (s > 0.0 && k < p) ? (float)(acc[2 + k] / (s * s)) : 0.f;
        for (int r = lane; r < R; r += 32) {
            const float D = Dc[r];
            Dc[r] = D * inv;
#pragma unroll
            for (int k = 0; k < PMAX; ++k) {
                if (k < p) {
                    float* jp = Jc + (size_t)k * S + r;
                    *jp = (*jp - D * a[k]) * inv;
                }
            }
        }
        if (lane == 0) {
            row[RC_NORM] = s;
            atomicAdd(&sc->iscal[0], (int)acc[1]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double mn = INFINITY;
        bool fin = true;
        for (int c = 0; c < d.C; ++c) {
            const double s = rasl_row(pr, c)[RC_NORM];
            fin = fin && isfinite(s);
            mn = fmin(mn, s);
        }
        sc->scal[0] = fin ? mn : NAN;
    }
    __syncthreads();
}

// Per column: G_c = J_c^T J_c, its inverse, J_c^T D_hat_c and ||D_hat_c||^2 (FP64 sums in three
// passes of 15 products, one warp per column); then K = (I_p + sum_c G_c^-1)^-1 (sc->Gi) and
// d0 = ||W^T W D_hat||_F (scal[1]; ||D_hat_c - J_c c_c||^2 = ||D_hat_c||^2 - 2 jd_c . c_c +
// c_c^T G_c c_c per column).  Returns false when a G_c or I_p + sum_c G_c^-1 is singular.
static __device__ bool rasl_gram(const RaslProblem& pr, const Dims& d, const float* __restrict__ Dhat,
                                 const float* __restrict__ J, Scratch* sc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = d.p, S = d.S, R = d.R, C = d.C;
    constexpr int NPROD = 45, CH = 15;
    __shared__ int bad_s;
    if (threadIdx.x == 0) bad_s = 0;
    __syncthreads();
    for (int c = warp; c < C; c += NW) {
        double* row = rasl_row(pr, c);
        const float* Dc = Dhat + (size_t)c * R;
        const float* Jc = J + (size_t)c * R;
#pragma unroll 1
        for (int q0 = 0; q0 < NPROD; q0 += CH) {
            float fs[CH], fc[CH];
#pragma unroll
            for (int k = 0; k < CH; ++k) { fs[k] = 0.f; fc[k] = 0.f; }
            for (int r = lane; r < R; r += 32) {
                const float dh = Dc[r];
#pragma unroll
                for (int k = 0; k < CH; ++k) {
                    int a, b;
                    gram_index(q0 + k, a, b);
                    if (a >= p || b >= p) continue;
                    const float va = a < 0 ? dh : Jc[(size_t)a * S + r];
                    const float vb = b < 0 ? dh : Jc[(size_t)b * S + r];
                    dot2_add(fs[k], fc[k], va, vb);
                }
            }
            double acc[CH];
#pragma unroll
            for (int k = 0; k < CH; ++k) acc[k] = warp_sum64((double)fs[k] + (double)fc[k]);
            if (lane == 0)
                for (int k = 0; k < CH; ++k) row[RC_G + q0 + k] = acc[k];   // staging
        }
        __syncwarp();
        if (lane == 0) {
            double tot[NPROD];
            for (int q = 0; q < NPROD; ++q) tot[q] = row[RC_G + q];
            double G[PMAX * PMAX];
            for (int e = 0; e < PMAX * PMAX; ++e) G[e] = 0.0;
            for (int q = 0; q < 36; ++q) {
                int a, b;
                gram_index(q, a, b);
                if (a < p && b < p) { G[a * PMAX + b] = tot[q]; G[b * PMAX + a] = tot[q]; }
            }
            for (int a = 0; a < PMAX; ++a) row[RC_JD + a] = a < p ? tot[36 + a] : 0.0;
            row[RC_DD] = tot[44];
            for (int e = 0; e < PMAX * PMAX; ++e) row[RC_G + e] = G[e];
            if (!invert_pp(G, row + RC_GI, p)) atomicExch(&bad_s, 1);
        }
    }
    __syncthreads();
    if (bad_s) return false;
    if (threadIdx.x == 0) {
        double Ssum[PMAX * PMAX];
        for (int e = 0; e < PMAX * PMAX; ++e) Ssum[e] = 0.0;
        for (int c = 0; c < C; ++c) {
            const double* row = rasl_row(pr, c);
            for (int a = 0; a < p; ++a)
                for (int b = 0; b < p; ++b) Ssum[a * PMAX + b] += row[RC_GI + a * PMAX + b];
        }
        for (int a = 0; a < p; ++a) Ssum[a * PMAX + a] += 1.0;
        if (!invert_pp(Ssum, sc->Gi, p)) bad_s = 1;
    }
    __syncthreads();
    if (bad_s) return false;
    // d0: the coefficients of W^T W D_hat
    for (int c = threadIdx.x; c < C; c += NT) {
        double* row = rasl_row(pr, c);
        for (int a = 0; a < p; ++a) {
            double b = 0.0;
            for (int j = 0; j < p; ++j) b += row[RC_GI + a * PMAX + j] * row[RC_JD + j];
            row[RC_B + a] = b;
        }
    }
    __syncthreads();
    if (warp == 0) rasl_sum_t(pr, RC_B, sc, sc->cvec, p, lane);
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += NT) {
        double* row = rasl_row(pr, c);
        double cc[PMAX];
        for (int a = 0; a < p; ++a) {
            double v = row[RC_B + a];
            for (int j = 0; j < p; ++j) v -= row[RC_GI + a * PMAX + j] * sc->cvec[j];
            cc[a] = v;
        }
        double q2 = row[RC_DD];
        for (int a = 0; a < p; ++a) {
            q2 -= 2.0 * row[RC_JD + a] * cc[a];
            for (int b = 0; b < p; ++b) q2 += cc[a] * cc[b] * row[RC_G + a * PMAX + b];
        }
        row[RC_SHIFT + 1] = q2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double q2 = 0.0, dd = 0.0;
        for (int c = 0; c < C; ++c) {
            q2 += fmax(rasl_row(pr, c)[RC_SHIFT + 1], 0.0);
            dd += rasl_row(pr, c)[RC_DD];
        }
        sc->scal[1] = sqrt(q2);
        sc->scal[2] = dd;
    }
    __syncthreads();
    return true;
}

// The inner loop of one outer step, as k_inner (Eq. newvars2 with the same readings) with the
// W^T W of the image set.  Entry: A, E, Y the warm start; rasl_gram done.  Exit: A, E, Y the
// result; row[RC_CV] of column c = the c_c of W^T W (A + E - D_hat), i.e. dtau_c.
template <int NCH, bool TCP>
static __device__ InnerOut k_inner_rasl(const RaslProblem& pr, const Dims& d, const Params& prm, double lam, double mu0,
                                        const float* __restrict__ Dhat, const float* __restrict__ J,
                                        float* __restrict__ A, float* __restrict__ E, float* __restrict__ Y,
                                        float* __restrict__ Mp, SvdBufs buf, bool& haveV, const SmemLayout& L,
                                        RaslResult* cyc) {
    Scratch* sc = L.sc;
    const int p = d.p, S = d.S, R = d.R, C = d.C, ldb = d.ldb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Dims dsvt = d;
    dsvt.p = 0;                       // the SVT step accumulates no J^T products here
    const int R4 = (R % 4 == 0) ? R : 0;   // rows visited four at a time (16-byte accesses)
    // the previous M (Mp) is kept only for the gate of Algorithm 2 (off when eps_svd < 0)
    const bool gate = prm.eps_svd >= 0.0;
    InnerOut out;
    out.iters = 0; out.sweeps = 0; out.warm = 0; out.reorth = 0; out.cayley = 0; out.rank = 0;
    out.cancelled = false;
    out.converged = false; out.bad = false; out.tc_timeout = false;
    out.c1 = out.c2 = 0.0; out.mu_last = mu0; out.nuc = 0.0; out.l1 = 0.0;
    unsigned long long t0 = clk();

    // ---- prologue: Y <- W^T W Y (Eq. Y_new_warmstart); P = W^T W (A + E - D_hat); M_0
    for (int c = warp; c < C; c += NW) {
        double* row = rasl_row(pr, c);
        const float* Jc = J + (size_t)c * R;
        const size_t o = (size_t)c * R;
        float va[PMAX], vy[PMAX];
#pragma unroll
        for (int k = 0; k < PMAX; ++k) { va[k] = 0.f; vy[k] = 0.f; }
        for (int r = lane; r < R; r += 32) {
            const float ae = A[o + r] + E[o + r], y = Y[o + r];
#pragma unroll
            for (int k = 0; k < PMAX; ++k) {
                if (k < p) {
                    const float jk = Jc[(size_t)k * S + r];
                    va[k] = fmaf(jk, ae, va[k]);
                    vy[k] = fmaf(jk, y, vy[k]);
                }
            }
        }
        warp_sum_p(va, p);
        warp_sum_p(vy, p);
        rasl_store_b(row, RC_B, va, row + RC_JD, p, lane);
        rasl_store_b(row, RC_B2, vy, nullptr, p, lane);
    }
    __syncthreads();
    if (warp == 0) {
        rasl_sum_t(pr, RC_B, sc, sc->cvec, p, lane);
        rasl_sum_t(pr, RC_B2, sc, sc->dtau, p, lane);
    }
    __syncthreads();
    {
        const float imu = (float)(1.0 / mu0);
        float g[2] = {0.f, 0.f};
        for (int c = warp; c < C; c += NW) {
            double* row = rasl_row(pr, c);
            const float* Jc = J + (size_t)c * R;
            const size_t o = (size_t)c * R;
            float cP[PMAX], cY[PMAX];
            rasl_coeffs(row, RC_B, sc->cvec, p, lane, cP, false);
            rasl_coeffs(row, RC_B2, sc->dtau, p, lane, cY, false);
            for (int r = lane; r < R; r += 32) {
                float jc = 0.f, jy = 0.f;
#pragma unroll
                for (int k = 0; k < PMAX; ++k) {
                    if (k < p) {
                        const float jk = Jc[(size_t)k * S + r];
                        jc = fmaf(jk, cP[k], jc);
                        jy = fmaf(jk, cY[k], jy);
                    }
                }
                const float a = A[o + r];
                const float y = Y[o + r] - jy;
                const float pp = (a + E[o + r] - Dhat[o + r]) - jc;
                Y[o + r] = y;
                const float mv = a - y * imu - pp;
                buf.T[(size_t)c * ldb + r] = mv;
                if (gate) {
                    const float mo = Mp[o + r];
                    g[0] = fmaf(mv - mo, mv - mo, g[0]);
                    g[1] = fmaf(mv, mv, g[1]);
                    Mp[o + r] = mv;
                }
            }
        }
        block_sum_f<2>(g, sc->red);
        if (threadIdx.x == 0) { sc->scal[5] = block_total(sc->red, 0); sc->scal[6] = block_total(sc->red, 1); }
        __syncthreads();
    }
    if (threadIdx.x == 0) cyc->cyc_elem += clk() - t0;

    const double d0 = sc->scal[1] > 0.0 ? sc->scal[1] : 1.0;
    if (threadIdx.x == 0) {
        sc->scal[12] = mu0;
        sc->fs[FS_IMU] = (float)(1.0 / mu0);
        sc->fs[FS_THR] = (float)(lam / mu0);
        sc->iscal[6] = prm.eps_svd < 0.0 || sc->scal[5] < prm.eps_svd * prm.eps_svd * sc->scal[6];
    }
    __syncthreads();
    for (int k = 1; k <= prm.max_inner; ++k) {
        out.iters = k;
        // ---- a6 + a7: A' = S_{1/mu}(M), ||A' - A||^2 -> scal[7]
        t0 = clk();
        // tall data matrices (the set's shared-memory plan has room for T) take the QR path
        const SvtStepOut so = svt_into<NCH, TCP>(dsvt, buf, L, haveV, sc->iscal[6] != 0, sc->fs[FS_IMU], A, nullptr,
                                                 pr.jsched, nullptr, nullptr, pr.tall != 0);
        const unsigned long long t1 = so.t_svd_end;
        if (threadIdx.x == 0) cyc->cyc_svd += t1 - t0;
        if (so.warm) out.warm++;
        if (so.reorth) out.reorth++;
        out.sweeps += so.sweeps;
        out.nuc = sc->scal[3];
        out.rank = sc->iscal[2];
        if (so.tc_timeout) {
            out.bad = out.tc_timeout = true;
            break;
        }
        const unsigned long long t2 = clk();
        if (threadIdx.x == 0) cyc->cyc_recon += t2 - t1;

        // ---- a8: c' of W^T W (A' + E - D_hat), per column
        for (int c = warp; c < C; c += NW) {
            double* row = rasl_row(pr, c);
            const float* Jc = J + (size_t)c * R;
            const size_t o = (size_t)c * R;
            float v[PMAX];
#pragma unroll
            for (int k2 = 0; k2 < PMAX; ++k2) v[k2] = 0.f;
            col_jt_residual<4>(A + o, E + o, Dhat + o, Jc, S, 0, R4, lane, p, v);
            col_jt_residual<1>(A + o, E + o, Dhat + o, Jc, S, R4, R, lane, p, v);
            warp_sum_p(v, p);
            rasl_store_b(row, RC_B, v, nullptr, p, lane);
        }
        __syncthreads();
        if (warp == 0) rasl_sum_t(pr, RC_B, sc, sc->cvec, p, lane);
        __syncthreads();
        // E' = T_{lam/mu}(E - Y/mu - W^T W (A' + E - D_hat)); ||E' - E||^2; ||E'||_1; and the b of
        // W^T W (A' + E' - D_hat)
        const float imu = sc->fs[FS_IMU];
        const float thr = sc->fs[FS_THR];
        {
            float acc[2] = {0.f, 0.f};
            for (int c = warp; c < C; c += NW) {
                double* row = rasl_row(pr, c);
                const float* Jc = J + (size_t)c * R;
                const size_t o = (size_t)c * R;
                float cc[PMAX], w[PMAX];
                rasl_coeffs(row, RC_B, sc->cvec, p, lane, cc, false);
#pragma unroll
                for (int k2 = 0; k2 < PMAX; ++k2) w[k2] = 0.f;
                col_e_update<4>(A + o, E + o, Dhat + o, Y + o, Jc, S, 0, R4, lane, p, cc, imu, thr, acc, w);
                col_e_update<1>(A + o, E + o, Dhat + o, Y + o, Jc, S, R4, R, lane, p, cc, imu, thr, acc, w);
                warp_sum_p(w, p);
                rasl_store_b(row, RC_B2, w, nullptr, p, lane);
            }
            block_sum_f<2>(acc, sc->red);
            if (threadIdx.x == 0) {
                sc->scal[8] = block_total(sc->red, 0);
                sc->scal[9] = block_total(sc->red, 1);
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
            if (warp == 0) rasl_sum_t(pr, RC_B2, sc, sc->dtau, p, lane);
            __syncthreads();
        }
        out.l1 = sc->scal[9];

        // ---- a9: P'' = W^T W (A' + E' - D_hat); Y' = Y + mu P''; next M = A' - Y'/mu_next - P''
        {
            const float muf = sc->fs[FS_MU];
            const float imun = sc->fs[FS_IMUN];
            float acc[3] = {0.f, 0.f, 0.f};
            for (int c = warp; c < C; c += NW) {
                double* row = rasl_row(pr, c);
                const float* Jc = J + (size_t)c * R;
                const size_t o = (size_t)c * R;
                float cc[PMAX];
                rasl_coeffs(row, RC_B2, sc->dtau, p, lane, cc, true);
                float* Tc = buf.T + (size_t)c * ldb;
                col_y_update<4>(A + o, E + o, Dhat + o, Y + o, Tc, Mp + o, Jc, S, 0, R4, lane, p, cc, muf, imun, gate, acc);
                col_y_update<1>(A + o, E + o, Dhat + o, Y + o, Tc, Mp + o, Jc, S, R4, R, lane, p, cc, muf, imun, gate, acc);
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
                else if (c1 < prm.eps1 && c2 < prm.eps2) ctl = LOOP_CONVERGED;
                sc->iscal[5] = ctl;
                sc->scal[16] = sc->scal[12];
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
        if (ctl == LOOP_CONVERGED) {
            out.converged = true;
            break;
        }
    }
    return out;
}

// Algorithm 1 for one image set (RASL): warp every image by its tau_c, the inner loop with the
// set's W^T W and warm starts, dtau_c per image, until no window corner of any image moves by
// outer_tol pixels.  Statuses as solve_problem.
template <int NCH, bool TCP>
static __device__ void solve_rasl(const RaslProblem& pr, const SmemLayout& L, RaslResult& res) {
    Scratch* sc = L.sc;
    const int N = pr.nimg, p = pr.p;
    const Dims d = make_dims(pr.m * pr.n, N, p);
    const Params& prm = pr.prm;
    const int S = d.S;
    SvdBufs buf;
    const size_t nb = (size_t)d.ldb * d.Cp, nv = (size_t)d.ldv * d.Cp;
    // the QR path keeps V, T, B_c and its small buffers in shared memory (B is not formed)
    const size_t nbB = pr.tall ? tall_small_floats(d) : nb;
    {
        float* sm = L.svd;
        if (pr.tall) {
            buf.V = sm; sm += nv;
            buf.T = sm; sm += nb;
            buf.Z = sm; sm += (size_t)d.C * d.Cp;
            buf.B = sm; sm += nbB;
        } else {
            if (pr.smem_svd & 1) { buf.B = sm; sm += nb; } else { buf.B = pr.pl.Bg; }
            if (pr.smem_svd & 2) { buf.V = sm; sm += nv; } else { buf.V = pr.pl.Vg; }
            if (pr.smem_svd & 4) { buf.T = sm; sm += nb; } else { buf.T = pr.pl.Tg; }
            if (pr.smem_svd & 8) { buf.Z = sm; sm += (size_t)d.C * d.Cp; } else { buf.Z = pr.pl.Zg; }
        }
        buf.stage = reinterpret_cast<unsigned char*>(sm);
        buf.nbuf = 0;
        buf.tc = false;
    }
    {
        for (size_t e = threadIdx.x; e < nb; e += NT) buf.T[e] = 0.f;
        for (size_t e = threadIdx.x; e < nbB; e += NT) buf.B[e] = 0.f;
        for (size_t e = threadIdx.x; e < nv; e += NT) buf.V[e] = 0.f;
    }
    const double lam = prm.lam > 0.0 ? prm.lam : 1.0 / sqrt((double)max(pr.m * pr.n, N));
    for (int e = threadIdx.x; e < N * PMAX; e += NT) {
        const int c = e / PMAX, k = e - c * PMAX;
        rasl_row(pr, c)[RC_TAU + k] = k < p ? pr.tau[(size_t)c * p + k] : 0.0;
    }
    res.cyc_warp = res.cyc_svd = res.cyc_recon = res.cyc_elem = res.cyc_other = 0;
    __syncthreads();

    int status = 1;
    bool inner_maxed = false;
    int outer = 0, inner_total = 0, sweeps = 0, warm = 0, reorth = 0, rank = 0;
    double c1 = 0.0, nuc = 0.0, l1 = 0.0;
    bool haveV = false;

    unsigned long long t0 = clk();
    rasl_warp(pr, d, pr.pl.Dhat, pr.pl.J, sc);
    if (threadIdx.x == 0) res.cyc_warp += clk() - t0;
    if (!isfinite(sc->scal[0])) {
        status = -1;
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
                rasl_warp(pr, d, pr.pl.Dhat, pr.pl.J, sc);
                if (!isfinite(sc->scal[0])) { status = -1; break; }
                if (!(sc->scal[0] > 0.0)) { status = -3; break; }
            }
            const unsigned long long t1 = clk();
            if (threadIdx.x == 0) res.cyc_warp += t1 - t0;
            if (!rasl_gram(pr, d, pr.pl.Dhat, pr.pl.J, sc)) { status = -2; break; }
            double mu0 = prm.mu0;
            // the power iteration's R-vector lives in the P plane (free until the next inner loop)
            if (!(mu0 > 0.0)) mu0 = 1.25 / spectral_norm(pr.pl.Dhat, d, L.sigma, pr.pl.P, sc);
            if (threadIdx.x == 0) res.cyc_other += clk() - t1;
            InnerOut io = k_inner_rasl<NCH, TCP>(pr, d, prm, lam, mu0, pr.pl.Dhat, pr.pl.J, pr.pl.A, pr.pl.E, pr.pl.Y,
                                                 pr.pl.Mp, buf, haveV, L, &res);
            inner_total += io.iters;
            sweeps += io.sweeps;
            warm += io.warm;
            reorth += io.reorth;
            c1 = io.c1; nuc = io.nuc; l1 = io.l1; rank = io.rank;
            if (io.tc_timeout) { status = -5; break; }
            if (io.bad) { status = -1; break; }
            if (!io.converged) inner_maxed = true;
            // Steps 3-4 per image: dtau_c = row[RC_CV], tau_c <- tau_c + dtau_c
            for (int c = threadIdx.x; c < N; c += NT) {
                double* row = rasl_row(pr, c);
                double t[PMAX], dt[PMAX];
                for (int k = 0; k < PMAX; ++k) {
                    t[k] = k < p ? row[RC_TAU + k] : 0.0;
                    dt[k] = k < p ? row[RC_CV + k] : 0.0;
                }
                double sh = corner_shift(t, dt, pr.ttype, pr.m, pr.n, p);
                bool fin = isfinite(sh);
                for (int k = 0; k < p; ++k) {
                    row[RC_TAU + k] = t[k] + dt[k];
                    fin = fin && isfinite(row[RC_TAU + k]);
                }
                row[RC_SHIFT] = fin ? sh : -1.0;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double mx = 0.0;
                for (int c = 0; c < N; ++c) {
                    const double sh = rasl_row(pr, c)[RC_SHIFT];
                    mx = (sh < 0.0 || mx < 0.0) ? -1.0 : fmax(mx, sh);
                }
                sc->scal[11] = mx;
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
    for (int e = threadIdx.x; e < N * p; e += NT) {
        const int c = e / p, k = e - c * p;
        pr.tau[e] = rasl_row(pr, c)[RC_TAU + k];
    }
    if (threadIdx.x == 0) {
        res.status = status;
        res.objective = nuc + lam * l1;
        res.lambda = lam;
        res.rank_A = rank;
        res.outer_iters = outer;
        res.inner_iters = inner_total;
        res.svd_sweeps = sweeps;
        res.svd_warm = warm;
        res.svd_reorth = reorth;
        res.oob_pixels = sc->iscal[0];
        res.svt_qr = pr.tall;
        res.kkt_residual = c1;
    }
    __syncthreads();
}

}  // namespace tilt
