// Device code of the TILT-by-LADMAP solver: every function here is executed by all
// threads of one CTA, which owns one problem (window) for the duration of the call.
//
// Storage of an m x n window ("long-side contiguous"): R = max(m, n), C = min(m, n);
// element (i, j) lives at X(r, c) = c*R + r with (r, c) = (i, j) when m >= n and
// (r, c) = (j, i) otherwise.  The one-sided Jacobi SVD then works on the C contiguous
// columns of length R of the matrix X (X = M when m >= n, X = M^T otherwise; the singular
// value thresholding of Eq. A_1 commutes with transposition).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "tilt_tc.cuh"

namespace tilt {

constexpr int NT = 512;          // threads per CTA
constexpr int NW = NT / 32;      // warps per CTA
constexpr int PMAX = 8;          // largest transform (projective)
constexpr int MAX_SIDE = 512;

// Advances the (row r, column c) of a column-major pixel index e = c R + r by a stride given as
// stepc = stride / R whole columns plus stepr = stride % R rows, without a division (r < R).
__device__ __forceinline__ void next_rc(int& r, int& c, int R, int stepr, int stepc) {
    r += stepr;
    c += stepc;
    if (r >= R) { r -= R; ++c; }
}

// ------------------------------------------------------------------------------ parameters
struct Params {
    double lam, eps1, eps2, rho0, mu0, mu_max, eps_svd, outer_tol;
    int max_inner, max_outer;
    int svd_ws;            // 0: warm-started Jacobi; 1: Algorithm 2 (Cayley step) when the gate allows
};

// Per-problem result record (written once, at the end of the solve).
struct Result {
    int status;
    int p;
    double tau[8];
    double objective;
    double lambda;
    int rank_A, outer_iters, inner_iters, svd_sweeps, svd_warm, svd_reorth, svd_cayley, oob_pixels;
    double kkt_residual;
    // per-phase clock counters (SM cycles), for the time split of the fused solver
    unsigned long long cyc_warp, cyc_svd, cyc_recon, cyc_elem, cyc_other;
};

// Planes of one problem in device global memory (long-side-contiguous layout).
struct Planes {
    float* Dhat;   // S
    float* J;      // p * S
    float* A;      // S
    float* E;      // S
    float* Y;      // S   (the scaled multiplier Y~ = W^T Y of Sec. 4.3)
    float* P;      // S   (work plane: the power iteration's vector of an image set)
    float* Mp;     // S   (previous M, for the warm-start gate; kept only while the gate is on)
    float* Bg;     // ldb * Cp  (SVD work, global mode only)
    float* Vg;     // ldv * Cp
    float* Tg;     // ldb * Cp
    float* Zg;     // C * Cp   (X^T b_k of the kept columns, for the reconstruction; rows at stride Cp)
    float* Cay;    // cayley_floats() (Algorithm 2 workspace; only when Params::svd_ws = 1)
};

// One problem as the solver kernel sees it.
struct Problem {
    const float* img;
    long long ld;
    int H, W;
    int m, n, p, ttype;
    double tau[8];
    Params prm;
    Planes pl;
    int smem_svd;          // bits 0-3: B, V, T, Z live in shared memory (else Bg, Vg, Tg, Zg)
    int tc_nbuf;           // stage buffers of the tensor-core products (1 or 2, after B|V|T|Z);
                           // 0: the products run on the SIMT pipes
    int jsched;            // Jacobi schedule: bits 0-7 group width (lanes per column pair: 4, 8
                           // or 16), bit 8 block-cyclic pair ordering (else round-robin)
    Result* res;           // host-mapped result record
    volatile int* done;    // host-mapped completion flag
    const int* cancel;     // host-mapped: non-zero when the context is being destroyed
};

// ------------------------------------------------------------------------------ RASL
// RASL (Sec. 1): TILT's model with one image per column of the data matrix.  An image set of
// nimg images, each warped over an m x n window, gives an R x C matrix with R = m n pixels
// (row-major within the window) and C = nimg columns, stored like a TILT plane (column c
// contiguous); J holds, in column c, the Jacobian of that column with respect to tau_c.
constexpr int RASL_NMAX = 128;      // images per set

// FP64 state of one image of a set in device memory: a row of RASL_COLW doubles.
enum {
    RC_GI = 0,                      // (J_c^T J_c)^-1, p x p at row stride PMAX
    RC_G = PMAX * PMAX,             // J_c^T J_c (Gram staging, then the matrix)
    RC_JD = 2 * PMAX * PMAX,        // J_c^T D_hat_c
    RC_B = RC_JD + PMAX,            // (J_c^T J_c)^-1 J_c^T x_c of the current W^T W product
    RC_B2 = RC_B + PMAX,            // a second one (the prologue projects two planes at once)
    RC_CV = RC_B2 + PMAX,           // coefficients of the last W^T W product (dtau_c at exit)
    RC_TAU = RC_CV + PMAX,          // tau_c
    RC_DD = RC_TAU + PMAX,          // ||D_hat_c||^2
    RC_NORM = RC_DD + 1,            // ||I_c o tau_c||_F
    RC_SHIFT = RC_NORM + 1,         // corner shift of the last update
    RASL_COLW = RC_SHIFT + 2
};

struct RaslResult {
    int status;
    int outer_iters, inner_iters, svd_sweeps, svd_warm, svd_reorth, rank_A, oob_pixels;
    int svt_qr;            // the SVT took the QR path
    double objective, lambda, kkt_residual;
    unsigned long long cyc_warp, cyc_svd, cyc_recon, cyc_elem, cyc_other;
};

// One image set as the RASL kernel sees it.
struct RaslProblem {
    const float* imgs;     // image c at imgs + c * img_stride, rows at stride ld
    long long img_stride, ld;
    int H, W;
    int nimg, m, n, p, ttype;
    Params prm;
    Planes pl;             // R = m n, C = nimg
    double* col;           // nimg rows of RASL_COLW doubles
    double* tau;           // nimg x p, tau0 on entry, the result on exit
    int smem_svd, jsched;
    int tall;              // the SVT takes the QR path (V, T, B_c and its buffers in shared memory)
    RaslResult* res;
};

// Copy a small POD record word by word into shared memory (all threads).
template <typename T>
__device__ inline void copy_to_shared(T* dst, const T* src) {
    static_assert(sizeof(T) % 4 == 0, "record size");
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(dst);
    for (int w = threadIdx.x; w < (int)(sizeof(T) / 4); w += NT) d[w] = s[w];
    __syncthreads();
}

// Non-zero once the host has asked running problems to stop (read by thread 0).
__device__ inline int cancel_requested(const int* cancel) {
    if (!cancel) return 0;
    int v;
    asm volatile("ld.relaxed.sys.u32 %0, [%1];" : "=r"(v) : "l"(cancel) : "memory");
    return v;
}

struct Dims {
    int m, n, R, C, S, p;
    bool colmajor;         // m >= n
    int ldb, ldv, Cp;      // SVD buffer geometry (Cp = C rounded up to 4)
};

__host__ __device__ inline Dims make_dims(int m, int n, int p) {
    Dims d;
    d.m = m; d.n = n; d.p = p;
    d.colmajor = (m >= n);
    d.R = d.colmajor ? m : n;
    d.C = d.colmajor ? n : m;
    d.S = m * n;
    d.ldb = (d.R + 3) & ~3;
    d.Cp = (d.C + 3) & ~3;
    d.ldv = d.Cp;
    return d;
}

// Shared-memory bytes of the SVD buffers B, V, T.
__host__ __device__ inline size_t svd_smem_bytes(const Dims& d) {
    return sizeof(float) * ((size_t)2 * d.ldb * d.Cp + (size_t)d.ldv * d.Cp);
}

// Tensor-core products of the SVD and the SVT: K chunks of TC_KC, accumulators of up to
// min(C rounded up to 16, TC_NMAX) columns; every CTA holds TC_TMEM_COLS columns of tensor
// memory (two CTAs per SM at most: 512 columns).
constexpr int TC_KC = 8;
constexpr uint32_t TC_TMEM_COLS = 256;
// Windows whose products run on the tensor cores: below this short side the per-chunk
// staging and synchronisation of the tensor-core path cost more than the register-tiled
// SIMT products (measured on the 40-120 px windows of the affine batch: the SVT
// reconstruction took 15 % more cycles on the tensor cores).
constexpr int TC_MIN_C = 160;
__host__ __device__ inline bool use_tc_products(const Dims& d) { return d.C >= TC_MIN_C; }
__host__ __device__ inline int tc_np(const Dims& d) {
    const int np = (d.C + 15) & ~15;
    return np < TC_NMAX ? np : TC_NMAX;
}
__host__ __device__ inline size_t tc_stage_for(const Dims& d, int nbuf) { return tc_stage_bytes(tc_np(d), TC_KC, nbuf); }

// ------------------------------------------------------------------------------ CTA scratch
// Small per-CTA scalars kept in shared memory.
struct Scratch {
    double red[48 * NW];       // block-reduction staging (up to 48 values per reduction)
    double G[PMAX * PMAX];     // J^T J + Q^T Q
    double Gi[PMAX * PMAX];    // its inverse
    double Q[3 * PMAX];
    double jd[PMAX];           // J^T D_hat
    double ja[PMAX];           // J^T A
    double je[PMAX];           // J^T E
    double jy[PMAX];           // J^T Y (the ADM baseline)
    double cvec[PMAX];         // coefficients c = G^-1 J^T (.) of the current W^T W product
    double tau[PMAX];
    double dtau[PMAX];
    double scal[20];           // broadcast scalars
    float fs[16];              // per-iteration float scalars, computed by thread 0 (FS_*)
    int iscal[8];
    int flag[2];
    TcState tc;                // tensor-core products: mbarriers, tensor-memory address, error
};

// Dynamic shared memory layout: [Scratch][sigma: C floats][w: C floats][kept: C ints][B|V|T]
struct SmemLayout {
    Scratch* sc;
    float* sigma;
    float* w;
    int* kept;
    float* svd;
};

__host__ __device__ inline size_t smem_head_bytes() {
    size_t b = sizeof(Scratch);
    b += sizeof(float) * MAX_SIDE * 2 + sizeof(int) * MAX_SIDE;
    return (b + 255) & ~(size_t)255;
}

__device__ inline SmemLayout carve_smem(unsigned char* base) {
    SmemLayout L;
    L.sc = reinterpret_cast<Scratch*>(base);
    unsigned char* p = base + sizeof(Scratch);
    L.sigma = reinterpret_cast<float*>(p);
    L.w = L.sigma + MAX_SIDE;
    L.kept = reinterpret_cast<int*>(L.w + MAX_SIDE);
    L.svd = reinterpret_cast<float*>(base + smem_head_bytes());
    return L;
}

// ------------------------------------------------------------------------------ reductions
// Sum K values over the CTA; every thread gets the totals.  Within a warp the partials
// (FP32 per-thread sums) are added in FP32 by a shuffle tree; the NW warp totals are then
// added in FP64 by one thread per value (FP64 runs at 1/64 of the FP32 rate on this part, so
// it is kept to K * NW additions per reduction).  Fixed order -> deterministic.
template <int K>
__device__ inline void block_sum(double (&v)[K], double* red) {
    static_assert(K <= 44, "block_sum staging: 48 values per warp, the last 44 slots also hold the totals");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float f = (float)v[k];
        float lo = (float)(v[k] - (double)f);     // keep what FP32 drops of an FP64 partial
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            f += __shfl_xor_sync(0xffffffffu, f, off);
            lo += __shfl_xor_sync(0xffffffffu, lo, off);
        }
        if (lane == 0) red[k * NW + warp] = (double)f + (double)lo;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) s += red[threadIdx.x * NW + w];
        red[48 * NW - 1 - threadIdx.x] = s;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = red[48 * NW - 1 - k];
    __syncthreads();
}

// Per-iteration variant for FP32 partials: FP32 shuffle tree in every warp, then one thread
// per value adds the NW warp totals in FP64.  No per-thread FP64 arithmetic (on this part
// an FP64 operation issued by all 512 threads costs as much as ~32 of FP32).  The totals are
// left in red[48 NW - 1 - k] (read them after the final barrier).
template <int K>
__device__ inline void block_sum_f(float (&v)[K], double* red) {
    static_assert(K <= 44, "block_sum staging: 48 values per warp, the last 44 slots also hold the totals");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float f = v[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) f += __shfl_xor_sync(0xffffffffu, f, off);
        if (lane == 0) red[k * NW + warp] = (double)f;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) s += red[threadIdx.x * NW + w];
        red[48 * NW - 1 - threadIdx.x] = s;
    }
    __syncthreads();
}
__device__ inline double block_total(const double* red, int k) { return red[48 * NW - 1 - k]; }

// Exact-order FP64 variant for the once-per-outer-step reductions (norms of the warp, the
// Gram matrix, the warm-start projections): FP64 shuffle tree in every warp, FP64 sum of the
// warp totals by one thread per value.
template <int K>
__device__ inline void block_sum64(double (&v)[K], double* red) {
    static_assert(K <= 44, "block_sum staging: 48 values per warp, the last 44 slots also hold the totals");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
        if (lane == 0) red[k * NW + warp] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) s += red[threadIdx.x * NW + w];
        red[48 * NW - 1 - threadIdx.x] = s;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = red[48 * NW - 1 - k];
    __syncthreads();
}

__device__ inline float warp_sum(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Window pixel of storage index e.
__device__ inline void pixel_of(const Dims& d, int e, int& i, int& j) {
    int r = e % d.R, c = e / d.R;
    if (d.colmajor) { i = r; j = c; } else { i = c; j = r; }
}

// ------------------------------------------------------------------------------ transforms
// tau(u, v) -> (x, y) in FP64 with the operation order ((t0 u + t1 v) + t2), every
// operation rounded to nearest, so that the pixel-cell decision of the bilinear warp is
// bit-identical to a plain FP64 evaluation.
struct MapPt {
    double x, y, den;
};

__device__ inline MapPt map_point(const double* t, int ttype, double u, double v) {
    MapPt q;
    double nx = __dadd_rn(__dadd_rn(__dmul_rn(t[0], u), __dmul_rn(t[1], v)), t[2]);
    double ny = __dadd_rn(__dadd_rn(__dmul_rn(t[3], u), __dmul_rn(t[4], v)), t[5]);
    if (ttype == 8) {
        double den = __dadd_rn(__dadd_rn(__dmul_rn(t[6], u), __dmul_rn(t[7], v)), 1.0);
        q.x = __ddiv_rn(nx, den);
        q.y = __ddiv_rn(ny, den);
        q.den = den;
    } else {
        q.x = nx;
        q.y = ny;
        q.den = 1.0;
    }
    return q;
}

// d x / d tau and d y / d tau at (u, v) (FP64).
__device__ inline void map_derivs(const MapPt& q, int ttype, double u, double v, double* dx, double* dy) {
    if (ttype == 8) {
        double iu = u / q.den, iv = v / q.den, i1 = 1.0 / q.den;
        dx[0] = iu; dx[1] = iv; dx[2] = i1; dx[3] = 0; dx[4] = 0; dx[5] = 0; dx[6] = -q.x * iu; dx[7] = -q.x * iv;
        dy[0] = 0; dy[1] = 0; dy[2] = 0; dy[3] = iu; dy[4] = iv; dy[5] = i1; dy[6] = -q.y * iu; dy[7] = -q.y * iv;
    } else {
        dx[0] = u; dx[1] = v; dx[2] = 1; dx[3] = 0; dx[4] = 0; dx[5] = 0;
        dy[0] = 0; dy[1] = 0; dy[2] = 0; dy[3] = u; dy[4] = v; dy[5] = 1;
    }
}

// ------------------------------------------------------------------------------ K1
// Bilinear sample of img at the window point (u, v) mapped by tau, clamped at the image edge
// (R5), with the raw Jacobian row J_k = I_x dx/dtau_k + I_y dy/dtau_k (Sec. 4.1 layout); the
// derivative along a clamped axis is zero.  inside = false when a coordinate was clamped.
__device__ __forceinline__ float warp_sample(const float* __restrict__ img, long long ld, int H, int W, int ttype,
                                             const double* tau, double u, double v, float (&jr)[PMAX],
                                             bool& inside) {
    const double Wm1 = (double)(W - 1), Hm1 = (double)(H - 1);
    MapPt q = map_point(tau, ttype, u, v);
    const bool inx = (q.x >= 0.0) && (q.x <= Wm1);
    const bool iny = (q.y >= 0.0) && (q.y <= Hm1);
    const double xc = fmin(fmax(q.x, 0.0), Wm1);
    const double yc = fmin(fmax(q.y, 0.0), Hm1);
    const double x0 = fmin(floor(xc), (double)(W - 2));
    const double y0 = fmin(floor(yc), (double)(H - 2));
    const float fx = (float)(xc - x0), fy = (float)(yc - y0);
    const long long xi = (long long)x0, yi = (long long)y0;
    const float* row0 = img + yi * ld + xi;
    const float I00 = __ldg(row0), I01 = __ldg(row0 + 1);
    const float I10 = __ldg(row0 + ld), I11 = __ldg(row0 + ld + 1);
    const float val = (1.f - fy) * ((1.f - fx) * I00 + fx * I01) + fy * ((1.f - fx) * I10 + fx * I11);
    const float gx = inx ? ((1.f - fy) * (I01 - I00) + fy * (I11 - I10)) : 0.f;
    const float gy = iny ? ((1.f - fx) * (I10 - I00) + fx * (I11 - I01)) : 0.f;
    if (ttype == 8) {
        const float iu = (float)(u / q.den), iv = (float)(v / q.den), i1 = (float)(1.0 / q.den);
        const float gxy = gx * (float)q.x + gy * (float)q.y;
        jr[0] = gx * iu; jr[1] = gx * iv; jr[2] = gx * i1;
        jr[3] = gy * iu; jr[4] = gy * iv; jr[5] = gy * i1;
        jr[6] = -gxy * iu; jr[7] = -gxy * iv;
    } else {
        const float uf = (float)u, vf = (float)v;
        jr[0] = gx * uf; jr[1] = gx * vf; jr[2] = gx;
        jr[3] = gy * uf; jr[4] = gy * vf; jr[5] = gy;
        jr[6] = 0.f; jr[7] = 0.f;
    }
    inside = inx && iny;
    return val;
}

// Algorithm 1, Step 1: warp + normalise + Jacobian of the normalised warp.
// Writes D_hat and J; returns ||D o tau||_F (scal[0]) and the clamped-sample count (iscal[0]).
static __device__ void k1_warp_jacobian(const float* __restrict__ img, long long ld, int H, int W,
                                 const Dims& d, int ttype, const double* tau,
                                 float* __restrict__ Dhat, float* __restrict__ J, Scratch* sc) {
    const int p = d.p, S = d.S;
    const double hm = 0.5 * (d.m - 1), hn = 0.5 * (d.n - 1);
    double acc[2 + PMAX];
#pragma unroll
    for (int k = 0; k < 2 + PMAX; ++k) acc[k] = 0.0;
    for (int e = threadIdx.x; e < S; e += NT) {
        int i, j;
        pixel_of(d, e, i, j);
        const double u = (double)j - hn, v = (double)i - hm;
        float jr[PMAX];
        bool inside;
        const float val = warp_sample(img, ld, H, W, ttype, tau, u, v, jr, inside);
        Dhat[e] = val;
        acc[0] += (double)val * (double)val;
        acc[1] += inside ? 0.0 : 1.0;
#pragma unroll
        for (int k = 0; k < PMAX; ++k) {
            if (k < p) {
                J[(size_t)k * S + e] = jr[k];
                acc[2 + k] += (double)val * (double)jr[k];
            }
        }
    }
    block_sum64<2 + PMAX>(acc, sc->red);
    const double s = sqrt(acc[0]);
    if (threadIdx.x == 0) {
        sc->scal[0] = s;
        sc->iscal[0] = (int)acc[1];
    }
    const float inv = (s > 0.0) ? (float)(1.0 / s) : 0.f;
    float a[PMAX];
#pragma unroll
    for (int k = 0; k < PMAX; ++k) a[k] = (s > 0.0 && k < p) ? (float)(acc[2 + k] / (s * s)) : 0.f;
    for (int e = threadIdx.x; e < S; e += NT) {
        const float D = Dhat[e];
        Dhat[e] = D * inv;
#pragma unroll
        for (int k = 0; k < PMAX; ++k) {
            if (k < p) {
                float* jp = J + (size_t)k * S + e;
                *jp = (*jp - D * a[k]) * inv;
            }
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------------------------ K5 (Gram)
// Q rows (Sec. 4.3): derivatives of the centroid of the mapped window corners and of the
// signed area of the mapped quadrilateral (area row / ((m-1)(n-1))).  Thread 0 only.
__device__ inline void constraint_rows(const double* tau, int ttype, int m, int n, int p, double* Q) {
    const double a = 0.5 * (n - 1), b = 0.5 * (m - 1);
    const double cu[4] = {-a, a, a, -a}, cv[4] = {-b, -b, b, b};
    double x[4], y[4], dx[4][PMAX], dy[4][PMAX];
    for (int c = 0; c < 4; ++c) {
        MapPt q = map_point(tau, ttype, cu[c], cv[c]);
        x[c] = q.x; y[c] = q.y;
        map_derivs(q, ttype, cu[c], cv[c], dx[c], dy[c]);
    }
    const double norm = 1.0 / ((double)(m - 1) * (double)(n - 1));
    for (int k = 0; k < p; ++k) {
        double qx = 0, qy = 0, da = 0;
        for (int c = 0; c < 4; ++c) {
            const int c1 = (c + 1) & 3;
            qx += dx[c][k];
            qy += dy[c][k];
            da += dx[c][k] * y[c1] + x[c] * dy[c1][k] - dx[c1][k] * y[c] - x[c1] * dy[c][k];
        }
        Q[0 * PMAX + k] = 0.25 * qx;
        Q[1 * PMAX + k] = 0.25 * qy;
        Q[2 * PMAX + k] = 0.5 * da * norm;
    }
}

// Gauss-Jordan inverse with partial pivoting of a p x p FP64 matrix (row stride PMAX).
// Returns false when singular.  Thread 0 only.
__device__ inline bool invert_pp(const double* G, double* Gi, int p) {
    double a[PMAX][2 * PMAX];
    for (int r = 0; r < p; ++r)
        for (int c = 0; c < 2 * p; ++c) a[r][c] = (c < p) ? G[r * PMAX + c] : (c - p == r ? 1.0 : 0.0);
    double scale = 0.0;
    for (int r = 0; r < p; ++r) scale = fmax(scale, fabs(G[r * PMAX + r]));
    for (int col = 0; col < p; ++col) {
        int piv = col;
        for (int r = col + 1; r < p; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (!(fabs(a[piv][col]) > 1e-300) || !(fabs(a[piv][col]) > 1e-14 * scale)) return false;
        if (piv != col)
            for (int c = 0; c < 2 * p; ++c) { double t = a[col][c]; a[col][c] = a[piv][c]; a[piv][c] = t; }
        const double inv = 1.0 / a[col][col];
        for (int c = 0; c < 2 * p; ++c) a[col][c] *= inv;
        for (int r = 0; r < p; ++r) {
            if (r == col) continue;
            const double f = a[r][col];
            if (f != 0.0)
                for (int c = 0; c < 2 * p; ++c) a[r][c] -= f * a[col][c];
        }
    }
    for (int r = 0; r < p; ++r)
        for (int c = 0; c < p; ++c) Gi[r * PMAX + c] = a[r][p + c];
    return true;
}

// Products accumulated by the Gram pass: index q < 36 is J_a . J_b (a <= b, row-major
// upper triangle of an 8 x 8), 36 + a is J_a . D_hat, 44 is D_hat . D_hat.
__device__ inline void gram_index(int q, int& a, int& b) {
    if (q >= 44) { a = -1; b = -1; return; }
    if (q >= 36) { a = q - 36; b = -1; return; }
    int r = 0, rem = q;
    while (rem >= PMAX - r) { rem -= PMAX - r; ++r; }
    a = r;
    b = r + rem;
}

// G = J^T J + Q^T Q, G^-1, J^T D_hat and ||D_hat||^2, d0 = ||W^T W D_hat||_F (FP64; the
// 45 products are reduced in three passes of 15 to keep the per-thread accumulators few).
// Returns false when G is singular.  Results in sc->G, sc->Gi, sc->Q, sc->jd, scal[1] (d0),
// scal[2] (||D_hat||^2).  use_q = false: no constraint rows (Q = 0, G = J^T J; tau unused).
static __device__ bool k5_gram(const Dims& d, int ttype, const double* tau, const float* __restrict__ Dhat,
                               const float* __restrict__ J, Scratch* sc, bool use_q = true) {
    const int p = d.p, S = d.S;
    constexpr int NPROD = 45, CH = 15;
    double tot[NPROD];
#pragma unroll 1
    for (int q0 = 0; q0 < NPROD; q0 += CH) {
        double acc[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) acc[k] = 0.0;
        for (int e = threadIdx.x; e < S; e += NT) {
            const double dh = (double)Dhat[e];
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                int a, b;
                gram_index(q0 + k, a, b);
                if (a >= p || b >= p) continue;
                const double va = a < 0 ? dh : (double)J[(size_t)a * S + e];
                const double vb = b < 0 ? dh : (double)J[(size_t)b * S + e];
                acc[k] += va * vb;
            }
        }
        block_sum64<CH>(acc, sc->red);
#pragma unroll
        for (int k = 0; k < CH; ++k) tot[q0 + k] = acc[k];
    }
    __shared__ int ok_s;
    if (threadIdx.x == 0) {
        if (use_q)
            constraint_rows(tau, ttype, d.m, d.n, p, sc->Q);
        else
            for (int k = 0; k < 3 * PMAX; ++k) sc->Q[k] = 0.0;
        double JJ[PMAX][PMAX];
        for (int q = 0; q < 36; ++q) {
            int a, b;
            gram_index(q, a, b);
            if (a < p && b < p) { JJ[a][b] = tot[q]; JJ[b][a] = tot[q]; }
        }
        for (int a = 0; a < p; ++a)
            for (int b = 0; b < p; ++b) {
                double g = JJ[a][b];
                for (int l = 0; l < 3; ++l) g += sc->Q[l * PMAX + a] * sc->Q[l * PMAX + b];
                sc->G[a * PMAX + b] = g;
            }
        for (int a = 0; a < p; ++a) sc->jd[a] = tot[36 + a];
        const bool ok = invert_pp(sc->G, sc->Gi, p);
        ok_s = ok ? 1 : 0;
        // ||W^T W D||^2 = ||D||^2 - 2 jd^T c + c^T (J^T J) c with c = G^-1 jd
        double c[PMAX];
        for (int a = 0; a < p; ++a) {
            double v = 0;
            for (int b = 0; b < p; ++b) v += sc->Gi[a * PMAX + b] * sc->jd[b];
            c[a] = v;
        }
        double q2 = tot[44];
        for (int a = 0; a < p; ++a) {
            q2 -= 2.0 * sc->jd[a] * c[a];
            for (int b = 0; b < p; ++b) q2 += c[a] * c[b] * JJ[a][b];
        }
        sc->scal[1] = sqrt(fmax(q2, 0.0));
        sc->scal[2] = tot[44];
    }
    __syncthreads();
    const bool ok = ok_s != 0;
    __syncthreads();
    return ok;
}

// c = G^-1 v for a p-vector (thread 0 writes sc->cvec).
__device__ inline void ginv_apply(const Scratch* sc, int p, const double* v, double* out) {
    for (int a = 0; a < p; ++a) {
        double s = 0;
        for (int b = 0; b < p; ++b) s += sc->Gi[a * PMAX + b] * v[b];
        out[a] = s;
    }
}

// ------------------------------------------------------------------------------ ||D_hat||_2
// Largest singular value of the R x C matrix X (long-side-contiguous) by power iteration
// on X^T X in FP32 with FP64 norms; xv (C) and yv (R) are shared-memory work vectors.
static __device__ double spectral_norm(const float* __restrict__ X, const Dims& d, float* xv, float* yv, Scratch* sc) {
    const int R = d.R, C = d.C;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = threadIdx.x; c < C; c += NT) xv[c] = rsqrtf((float)C);
    __syncthreads();
    double prev = 0.0, sig = 0.0;
    int stable = 0;
    for (int it = 0; it < 300; ++it) {
        // y = X x
        double ny[1] = {0.0};
        for (int r = threadIdx.x; r < R; r += NT) {
            float s = 0.f;
            for (int c = 0; c < C; ++c) s += X[(size_t)c * R + r] * xv[c];
            yv[r] = s;
            ny[0] += (double)s * s;
        }
        block_sum<1>(ny, sc->red);
        sig = sqrt(ny[0]);
        // x = X^T y / ||X^T y||
        double nx[1] = {0.0};
        for (int c = warp; c < C; c += NW) {
            float s = 0.f;
            for (int r = lane; r < R; r += 32) s += X[(size_t)c * R + r] * yv[r];
            s = warp_sum(s);
            if (lane == 0) xv[c] = s;
        }
        __syncthreads();
        for (int c = threadIdx.x; c < C; c += NT) nx[0] += (double)xv[c] * xv[c];
        block_sum<1>(nx, sc->red);
        const float inv = nx[0] > 0 ? (float)(1.0 / sqrt(nx[0])) : 0.f;
        for (int c = threadIdx.x; c < C; c += NT) xv[c] *= inv;
        __syncthreads();
        if (fabs(sig - prev) <= 1e-7 * sig) {
            if (++stable >= 2) break;
        } else {
            stable = 0;
        }
        prev = sig;
    }
    return sig;
}

// ------------------------------------------------------------------------------ K2: SVD
// One-sided (Hestenes) Jacobi on the columns of B (R x C, column stride ldb, a multiple of
// 4), accumulating the rotations into V (C x C, stride ldv, a multiple of 4).
//
// Round-robin ordering: each round is a set of disjoint column pairs.  A pair is handled by
// a group of 8 lanes (4 pairs in flight per warp, 64 per CTA): lane g holds the float4
// chunks g, g+8, g+16, ... of both columns, so the dot product needs 3 shuffle levels
// and, when the columns fit in registers (R <= 128), the rotation reuses the loaded values.
// A pair is rotated when |b_i.b_j| > tol ||b_i|| ||b_j||, in Rutishauser's form
// x' = x - s (y + r x), y' = y + s (x - r y), r = tan(theta/2), so that small angles do not
// inflate the column norms (with c rounded to 1 the plain form grows them by t^2/2 per
// rotation).  The squared column norms are carried in a shared array instead of being
// recomputed at every pair: the rotation that zeroes b_i.b_j = g maps them to
// ||b_i||^2 - t g and ||b_j||^2 + t g (t = tan(theta)), the updates of Hestenes' method as
// in LAPACK's xGESVJ; a norm that the update shrinks below a quarter is recomputed from the
// rotated column (the difference would have cancelled), and every sweep starts from
// recomputed norms, so rounding cannot accumulate over more than one sweep.  Sweeps stop when
// one rotates nothing, or when the largest rotated cosine is below sqrt(tol) (cyclic Jacobi
// converges quadratically near the end, so the next sweep would find nothing above tol).
// Returns the number of sweeps.
struct RotParams {
    float s, r, t;
    bool rot;
    float cosabs;
};

__device__ inline RotParams rotation_for(float a, float b, float g, float tol) {
    // rotate when |g| > tol sqrt(a b), tested as g^2 > tol^2 a b (no square roots);
    // tan(theta) = t = 2g / (d + sgn(d) sqrt(d^2 + 4 g^2)), d = b - a (the smaller root);
    // with q = sqrt(1 + t^2): s = sin(theta) = t / q, r = tan(theta/2) = t / (1 + q)
    RotParams p;
    const float ab = a * b;
    p.rot = (ab > 0.f) && (g * g > tol * tol * ab);
    p.cosabs = 0.f;
    p.s = 0.f;
    p.r = 0.f;
    p.t = 0.f;
    if (p.rot) {
        // square roots as x rsqrt(x): s and r share q, so the applied transform
        // [[1 - s r, -s], [s, 1 - s r]] stays orthogonal to O(t^2 eps) whatever q's rounding
        p.cosabs = fabsf(g) * rsqrtf(ab);
        const float d = b - a;
        const float w = 2.f * g;
        const float h2 = fmaf(d, d, w * w);
        const float h = h2 * rsqrtf(h2);
        const float t = __fdividef(w, d + copysignf(h, d));
        const float q2 = fmaf(t, t, 1.f);
        const float q = q2 * rsqrtf(q2);
        p.s = __fdividef(t, q);
        p.r = __fdividef(t, 1.f + q);
        p.t = t;
    }
    return p;
}

__device__ inline float4 rot_x(float4 x, float4 y, float s, float r) {
    return make_float4(x.x - s * fmaf(r, x.x, y.x), x.y - s * fmaf(r, x.y, y.y), x.z - s * fmaf(r, x.z, y.z),
                       x.w - s * fmaf(r, x.w, y.w));
}
__device__ inline float4 rot_y(float4 x, float4 y, float s, float r) {
    return make_float4(y.x + s * fmaf(-r, y.x, x.x), y.y + s * fmaf(-r, y.y, x.y), y.z + s * fmaf(-r, y.z, x.z),
                       y.w + s * fmaf(-r, y.w, x.w));
}

__device__ inline float group_sum(float v, unsigned mask, int gw) {
#pragma unroll
    for (int off = 1; off < gw; off <<= 1) v += __shfl_xor_sync(mask, v, off, gw);
    return v;
}

// gw (4, 8 or 16) lanes per column pair: NT/gw pairs in flight per CTA, lane g of a group
// holds the float4 chunks g, g+gw, g+2gw, ... of both columns (in registers while
// R <= 4 gw NCH).  gw only changes how the work is spread, not the rotation sequence; the
// partial sums of the dot products are combined in a different order for each gw.

// One pair step of the one-sided Jacobi for columns i, j, executed by a group of gw lanes
// (lane g of the group holds float4 chunks g, g+gw, ... ; in registers while nqb <= gw NCH).
// TRACK: ni, nj hold the squared norms of the two columns, read and updated here; otherwise
// the norms are computed from the columns at every pair and ni, nj are unused.
constexpr float NORM_RECOMPUTE = 0.25f;   // recompute a norm that an update shrinks below this fraction

template <int NCH, int gw, bool TRACK = true>
__device__ inline void jacobi_pair_cols(float4* __restrict__ bi, float4* __restrict__ bj, float4* __restrict__ vi,
                                        float4* __restrict__ vj, float* ni, float* nj, int nqb, int nqv, int g,
                                        unsigned gmask, float tol, bool in_regs, bool& rotated, float& maxcos) {
    float a = 0.f, b = 0.f, gg = 0.f;
    if (TRACK) { a = *ni; b = *nj; }
    if (in_regs) {
        float4 x[NCH], y[NCH];
        float pa[NCH], pb[NCH], pg[NCH];
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
            const int q = g + gw * t;
            if (q < nqb) {
                x[t] = bi[q];
                y[t] = bj[q];
            } else {
                x[t] = make_float4(0.f, 0.f, 0.f, 0.f);
                y[t] = x[t];
            }
            if (!TRACK) {
                pa[t] = fmaf(x[t].x, x[t].x, fmaf(x[t].y, x[t].y, fmaf(x[t].z, x[t].z, x[t].w * x[t].w)));
                pb[t] = fmaf(y[t].x, y[t].x, fmaf(y[t].y, y[t].y, fmaf(y[t].z, y[t].z, y[t].w * y[t].w)));
            }
            pg[t] = fmaf(x[t].x, y[t].x, fmaf(x[t].y, y[t].y, fmaf(x[t].z, y[t].z, x[t].w * y[t].w)));
        }
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
            if (!TRACK) {
                a += pa[t];
                b += pb[t];
            }
            gg += pg[t];
        }
        if (!TRACK) {
            a = group_sum(a, gmask, gw);
            b = group_sum(b, gmask, gw);
        }
        gg = group_sum(gg, gmask, gw);
        const RotParams rp = rotation_for(a, b, gg, tol);
        if (rp.rot) {
#pragma unroll
            for (int t = 0; t < NCH; ++t) {
                const int q = g + gw * t;
                if (q < nqb) {
                    const float4 xn = rot_x(x[t], y[t], rp.s, rp.r);
                    const float4 yn = rot_y(x[t], y[t], rp.s, rp.r);
                    bi[q] = xn;
                    bj[q] = yn;
                    x[t] = xn;
                    y[t] = yn;
                }
            }
            if (TRACK) {
                float na = fmaf(-rp.t, gg, a), nb = fmaf(rp.t, gg, b);
                if (na < NORM_RECOMPUTE * a || nb < NORM_RECOMPUTE * b) {   // the same in every lane of the group
                    float sa = 0.f, sb = 0.f;
#pragma unroll
                    for (int t = 0; t < NCH; ++t) {
                        sa = fmaf(x[t].x, x[t].x, fmaf(x[t].y, x[t].y, fmaf(x[t].z, x[t].z, fmaf(x[t].w, x[t].w, sa))));
                        sb = fmaf(y[t].x, y[t].x, fmaf(y[t].y, y[t].y, fmaf(y[t].z, y[t].z, fmaf(y[t].w, y[t].w, sb))));
                    }
                    na = group_sum(sa, gmask, gw);
                    nb = group_sum(sb, gmask, gw);
                }
                if (g == 0) { *ni = na; *nj = nb; }
            }
            // V (C <= R rows): the same chunk pattern, unrolled so that all loads are in flight
#pragma unroll
            for (int t = 0; t < NCH; ++t) {
                const int q = g + gw * t;
                if (q < nqv) { x[t] = vi[q]; y[t] = vj[q]; }
            }
#pragma unroll
            for (int t = 0; t < NCH; ++t) {
                const int q = g + gw * t;
                if (q < nqv) {
                    vi[q] = rot_x(x[t], y[t], rp.s, rp.r);
                    vj[q] = rot_y(x[t], y[t], rp.s, rp.r);
                }
            }
            rotated = true;
            maxcos = fmaxf(maxcos, rp.cosabs);
        }
    } else {
        for (int q = g; q < nqb; q += gw) {
            const float4 x = bi[q], y = bj[q];
            if (!TRACK) {
                a = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, a))));
                b = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, b))));
            }
            gg = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, gg))));
        }
        if (!TRACK) {
            a = group_sum(a, gmask, gw);
            b = group_sum(b, gmask, gw);
        }
        gg = group_sum(gg, gmask, gw);
        const RotParams rp = rotation_for(a, b, gg, tol);
        if (rp.rot) {
            for (int q = g; q < nqb; q += gw) {
                const float4 x = bi[q], y = bj[q];
                bi[q] = rot_x(x, y, rp.s, rp.r);
                bj[q] = rot_y(x, y, rp.s, rp.r);
            }
            if (TRACK) {
                float na = fmaf(-rp.t, gg, a), nb = fmaf(rp.t, gg, b);
                if (na < NORM_RECOMPUTE * a || nb < NORM_RECOMPUTE * b) {   // the same in every lane of the group
                    float sa = 0.f, sb = 0.f;
                    for (int q = g; q < nqb; q += gw) {      // the chunks this lane has just written
                        const float4 x = bi[q], y = bj[q];
                        sa = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, sa))));
                        sb = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, sb))));
                    }
                    na = group_sum(sa, gmask, gw);
                    nb = group_sum(sb, gmask, gw);
                }
                if (g == 0) { *ni = na; *nj = nb; }
            }
            for (int q = g; q < nqv; q += gw) {
                const float4 x = vi[q], y = vj[q];
                vi[q] = rot_x(x, y, rp.s, rp.r);
                vj[q] = rot_y(x, y, rp.s, rp.r);
            }
            rotated = true;
            maxcos = fmaxf(maxcos, rp.cosabs);
        }
    }
}

template <int NCH, int gw, bool TRACK>
__device__ inline void jacobi_pair(float* B, int ldb, float* V, int ldv, float* nrm, int i, int j, int nqb, int nqv,
                                   int g, unsigned gmask, float tol, bool in_regs, bool& rotated, float& maxcos) {
    jacobi_pair_cols<NCH, gw, TRACK>(reinterpret_cast<float4*>(B + (size_t)i * ldb),
                              reinterpret_cast<float4*>(B + (size_t)j * ldb),
                              reinterpret_cast<float4*>(V + (size_t)i * ldv),
                              reinterpret_cast<float4*>(V + (size_t)j * ldv), nrm + i, nrm + j, nqb, nqv, g, gmask,
                              tol, in_regs, rotated, maxcos);
}

// Squared norms of the C columns of B (one warp per column), for the start of a sweep; the
// caller's next barrier publishes them.
__device__ inline void column_norms(const float* B, int ldb, int C, float* nrm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nqb = ldb / 4;
    for (int c = warp; c < C; c += NW) {
        const float4* col = reinterpret_cast<const float4*>(B + (size_t)c * ldb);
        float s = 0.f;
        for (int q = lane; q < nqb; q += 32) {
            const float4 x = col[q];
            s = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, s))));
        }
        s = warp_sum(s);
        if (lane == 0) nrm[c] = s;
    }
}

// End of a sweep: did any pair rotate, and the largest rotated cosine (all threads).
__device__ inline bool sweep_done(bool rotated, float maxcos, float tol, int* flag) {
    float* fl = reinterpret_cast<float*>(flag);
    const bool any_w = __any_sync(0xFFFFFFFFu, rotated);
    float mc_w = maxcos;
#pragma unroll
    for (int o = 16; o; o >>= 1) mc_w = fmaxf(mc_w, __shfl_xor_sync(0xFFFFFFFFu, mc_w, o));
    if (any_w && (threadIdx.x & 31) == 0) {
        flag[0] = 1;
        atomicMax(reinterpret_cast<int*>(&fl[1]), __float_as_int(mc_w));   // non-negative floats order as ints
    }
    __syncthreads();
    const int any = flag[0];
    const float mc = fl[1];
    __syncthreads();
    return !any || mc * mc < tol;
}

// Column-pair ordering of the sweeps.  0: round-robin over columns (C-1 rounds of disjoint
// pairs, a CTA barrier after each).  1: block-cyclic: the columns form 2 W blocks of b
// columns (W warps); in each of the 2W-1 block rounds a warp owns a block pair and works
// through its b^2 cross pairs (b sub-rounds of b disjoint pairs, __syncwarp between them;
// in the first block round of a sweep also the pairs inside each of its blocks), a CTA
// barrier after each block round.  Both visit every pair once per sweep.
// The group width is a template parameter: the shuffle widths and chunk indices sit on the
// critical path of every pair step.
template <int NCH, int gw, bool TRACK>
static __device__ int k2_jacobi_w(float* B, int ldb, float* V, int ldv, int R, int C, float tol, int max_sweeps,
                                  int* flag, int order, float* nrm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane & (gw - 1);
    const unsigned gmask = (gw == 32 ? 0xFFFFFFFFu : ((1u << gw) - 1u)) << (lane & ~(gw - 1));
    const int nqb = ldb / 4, nqv = ldv / 4;
    const bool in_regs = nqb <= gw * NCH;
    int sweep = 0;
    if (order == 0) {
        const int grp = threadIdx.x / gw;
        const int NG = NT / gw;
        const int Ce = C + (C & 1);
        const int npairs = Ce / 2;
        const int nr = Ce - 1;
        while (sweep < max_sweeps) {
            if (TRACK) column_norms(B, ldb, C, nrm);
            if (threadIdx.x == 0) { flag[0] = 0; reinterpret_cast<float*>(flag)[1] = 0.f; }
            __syncthreads();
            bool rotated = false;
            float maxcos = 0.f;
            for (int round = 0; round < nr; ++round) {
                for (int k = grp; k < npairs; k += NG) {
                    int i = 0;
                    if (k) { i = k - 1 + round; if (i >= nr) i -= nr; i += 1; }
                    int j = Ce - 2 - k + round;
                    if (j >= nr) j -= nr;
                    j += 1;
                    if (i >= C || j >= C) continue;
                    jacobi_pair<NCH, gw, TRACK>(B, ldb, V, ldv, nrm, i, j, nqb, nqv, g, gmask, tol, in_regs, rotated, maxcos);
                }
                __syncthreads();
            }
            ++sweep;
            if (sweep_done(rotated, maxcos, tol, flag)) break;
        }
        return sweep;
    }
    // block-cyclic
    const int gpw = 32 / gw;                       // groups per warp
    const int gi = lane / gw;                      // group index within the warp
    int b = (C + 2 * NW - 1) / (2 * NW);           // block width
    if (b < gpw) b = gpw;
    b += b & 1;                                    // even, for the round-robin inside a block
    int NB = (C + b - 1) / b;
    NB += NB & 1;
    const int nbr = NB - 1;                        // block rounds per sweep
    const int nwu = NB / 2;                        // warps with a block pair
    while (sweep < max_sweeps) {
        if (TRACK) column_norms(B, ldb, C, nrm);
        if (threadIdx.x == 0) { flag[0] = 0; reinterpret_cast<float*>(flag)[1] = 0.f; }
        __syncthreads();
        bool rotated = false;
        float maxcos = 0.f;
        for (int br = 0; br < nbr; ++br) {
            if (warp < nwu) {
                int P = 0;
                if (warp) { P = warp - 1 + br; if (P >= nbr) P -= nbr; P += 1; }
                int Q = NB - 2 - warp + br;
                if (Q >= nbr) Q -= nbr;
                Q += 1;
                if (br == 0) {
                    // pairs inside blocks P and Q: round-robin over b columns, b-1 sub-rounds of b/2
                    for (int sr = 0; sr < b - 1; ++sr) {
                        for (int k = gi; k < b; k += gpw) {
                            const int blk = (k < b / 2) ? P : Q;
                            const int kk = (k < b / 2) ? k : k - b / 2;
                            int li = 0;
                            if (kk) { li = kk - 1 + sr; if (li >= b - 1) li -= b - 1; li += 1; }
                            int lj = b - 2 - kk + sr;
                            if (lj >= b - 1) lj -= b - 1;
                            lj += 1;
                            const int ci = blk * b + li, cj = blk * b + lj;
                            if (ci < C && cj < C)
                                jacobi_pair<NCH, gw, TRACK>(B, ldb, V, ldv, nrm, ci, cj, nqb, nqv, g, gmask, tol, in_regs,
                                                     rotated, maxcos);
                        }
                        __syncwarp();
                    }
                }
                for (int s = 0; s < b; ++s) {
                    for (int a = gi; a < b; a += gpw) {
                        int c = a + s;
                        if (c >= b) c -= b;
                        const int ci = P * b + a, cj = Q * b + c;
                        if (ci < C && cj < C)
                            jacobi_pair<NCH, gw, TRACK>(B, ldb, V, ldv, nrm, ci, cj, nqb, nqv, g, gmask, tol, in_regs,
                                                 rotated, maxcos);
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
        }
        ++sweep;
        if (sweep_done(rotated, maxcos, tol, flag)) break;
    }
    return sweep;
}

// Staged sweeps for matrices whose B and V live in device memory (the largest windows):
// the columns form blocks of b; block pairs are visited row by row (P = 0 .. NB-1, then
// Q = P+1 .. NB-1: every column pair once per sweep, the pairs inside block P when P becomes
// the row block).  The row block P and the current block Q sit in shared memory, brought in
// and written back by bulk copies of whole columns (one per column of B and of V, issued by
// thread 0); Q alternates between two buffers, so the write-back of one block overlaps the
// work on the next.  Inside a block pair one warp rotates one column pair (32 lanes, float4
// chunks), b disjoint pairs per sub-round and a CTA barrier between sub-rounds, so the
// sweep reads each column of Q once per row instead of once per pair.  The squared norms of
// the staged columns are computed when a block arrives and carried through its pair steps (nrm:
// 3 b floats of shared memory, one per stage slot).  stage: 3 b (ldb + ldv) floats; st: the
// bulk-copy mbarrier.  Returns the number of sweeps, or -1 when a bounded
// wait for a copy gave up (st->error is set).
template <int NCH>
static __device__ int k2_jacobi_staged(float* B, int ldb, float* V, int ldv, int R, int C, float tol, int max_sweeps,
                                       int* flag, int b, float* stage, TcState* st, float* nrm) {
    (void)R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int NB = (C + b - 1) / b;
    const int nqb = ldb / 4, nqv = ldv / 4;
    const bool in_regs = nqb <= 32 * NCH;
    float* sB = stage;                               // 3 b columns of ldb floats
    float* sV = stage + (size_t)3 * b * ldb;         // 3 b columns of ldv floats
    auto colB = [&](int slot) { return reinterpret_cast<float4*>(sB + (size_t)slot * ldb); };
    auto colV = [&](int slot) { return reinterpret_cast<float4*>(sV + (size_t)slot * ldv); };
    auto ncols = [&](int blk) { return min(b, C - blk * b); };
    // thread 0: load block blk into slots base .. base + ncols - 1 (counted on st->jbar)
    auto load = [&](int blk, int base) {
        const int nc = ncols(blk);
        mbar_arrive_expect_tx(&st->jbar, (uint32_t)nc * (uint32_t)(ldb + ldv) * 4u);
        for (int c = 0; c < nc; ++c) {
            bulk_g2s(sB + (size_t)(base + c) * ldb, B + (size_t)(blk * b + c) * ldb, (uint32_t)ldb * 4u, &st->jbar);
            bulk_g2s(sV + (size_t)(base + c) * ldv, V + (size_t)(blk * b + c) * ldv, (uint32_t)ldv * 4u, &st->jbar);
        }
    };
    // thread 0: write block blk back from slots base ..; one bulk group
    auto store = [&](int blk, int base) {
        const int nc = ncols(blk);
        for (int c = 0; c < nc; ++c) {
            bulk_s2g(B + (size_t)(blk * b + c) * ldb, sB + (size_t)(base + c) * ldb, (uint32_t)ldb * 4u);
            bulk_s2g(V + (size_t)(blk * b + c) * ldv, sV + (size_t)(base + c) * ldv, (uint32_t)ldv * 4u);
        }
        bulk_commit();
    };
    // all threads: wait for the loads counted on st->jbar; false when the bounded wait gave up
    auto wait_loads = [&]() {
        const bool ok = mbar_wait(&st->jbar, st->jphase);
        const bool all = __syncthreads_and(ok);
        if (threadIdx.x == 0) st->jphase ^= 1;
        __syncthreads();
        return all;
    };
    // every thread's generic writes (to B, V in device memory, or to the stage) before the
    // bulk copies that read them
    fence_proxy_async();
    __syncthreads();
    int sweep = 0;
    bool ok = true;
    while (sweep < max_sweeps && ok) {
        if (threadIdx.x == 0) { flag[0] = 0; reinterpret_cast<float*>(flag)[1] = 0.f; }
        __syncthreads();
        bool rotated = false;
        float maxcos = 0.f;
        for (int P = 0; P < NB && ok; ++P) {
            // the row block: its last copy in device memory was written by an earlier bulk store
            if (threadIdx.x == 0) {
                bulk_wait_all();
                load(P, 0);
            }
            if (!(ok = wait_loads())) break;
            // pairs inside block P: round-robin over b columns, b - 1 sub-rounds of b/2 pairs
            const int nP = ncols(P);
            column_norms(sB, ldb, nP, nrm);
            __syncthreads();
            for (int sr = 0; sr < b - 1; ++sr) {
                if (warp < b / 2) {
                    int li = 0;
                    if (warp) { li = warp - 1 + sr; if (li >= b - 1) li -= b - 1; li += 1; }
                    int lj = b - 2 - warp + sr;
                    if (lj >= b - 1) lj -= b - 1;
                    lj += 1;
                    if (li < nP && lj < nP)
                        jacobi_pair_cols<NCH, 32, true>(colB(li), colB(lj), colV(li), colV(lj), nrm + li, nrm + lj, nqb,
                                                        nqv, lane, 0xFFFFFFFFu, tol, in_regs, rotated, maxcos);
                }
                __syncthreads();
            }
            if (P + 1 < NB) {
                if (threadIdx.x == 0) load(P + 1, b);
                if (!(ok = wait_loads())) break;
                column_norms(sB + (size_t)b * ldb, ldb, ncols(P + 1), nrm + b);
                __syncthreads();
            }
            int cur = b;                      // slot base of the buffer holding Q
            for (int Q = P + 1; Q < NB; ++Q) {
                const int nQ = ncols(Q);
                for (int s = 0; s < b; ++s) {
                    if (warp < b) {
                        const int a = warp;
                        int c = a + s;
                        if (c >= b) c -= b;
                        if (a < nP && c < nQ)
                            jacobi_pair_cols<NCH, 32, true>(colB(a), colB(cur + c), colV(a), colV(cur + c), nrm + a,
                                                            nrm + cur + c, nqb, nqv, lane, 0xFFFFFFFFu, tol, in_regs,
                                                            rotated, maxcos);
                    }
                    __syncthreads();
                }
                fence_proxy_async();
                __syncthreads();
                const int other = cur == b ? 2 * b : b;
                if (threadIdx.x == 0) {
                    store(Q, cur);
                    if (Q + 1 < NB) {
                        bulk_wait_read<1>();      // the write-back of Q - 1 has left the other buffer
                        load(Q + 1, other);
                    }
                }
                if (Q + 1 < NB) {
                    if (!(ok = wait_loads())) break;
                    column_norms(sB + (size_t)other * ldb, ldb, ncols(Q + 1), nrm + other);
                    __syncthreads();
                }
                cur = other;
            }
            if (!ok) break;
            fence_proxy_async();
            __syncthreads();
            if (threadIdx.x == 0) store(P, 0);
        }
        if (threadIdx.x == 0) {
            bulk_wait_all();
            fence_proxy_async();
        }
        __syncthreads();
        if (!ok) break;
        ++sweep;
        if (sweep_done(rotated, maxcos, tol, flag)) break;
    }
    if (!ok) {
        // a load that gave up may still be in flight: wait for it once more (bounded), and for
        // the issued write-backs, before the stage can be reused
        if (threadIdx.x == 0) {
            mbar_wait(&st->jbar, st->jphase ^ 1);
            bulk_wait_all();
            st->error = 1;
        }
        __syncthreads();
        return -1;
    }
    return sweep;
}

// TRACK: carry the squared column norms in nrm (C floats of shared memory) instead of
// recomputing them at every pair; columns of one float4 chunk per lane (the 32 x 32
// factor of the QR path) gain nothing from it and run with TRACK = false (nrm unused).
// (The staged sweeps carry the norms of their stage slots the same way.)
template <int NCH, bool TRACK = true>
static __device__ int k2_jacobi(float* B, int ldb, float* V, int ldv, int R, int C, float tol, int max_sweeps,
                                int* flag, int gw, int order, float* nrm) {
    if (C < 2) return 0;
    if (gw == 4) return k2_jacobi_w<NCH, 4, TRACK>(B, ldb, V, ldv, R, C, tol, max_sweeps, flag, order, nrm);
    if (gw == 16) return k2_jacobi_w<NCH, 16, TRACK>(B, ldb, V, ldv, R, C, tol, max_sweeps, flag, order, nrm);
    return k2_jacobi_w<NCH, 8, TRACK>(B, ldb, V, ldv, R, C, tol, max_sweeps, flag, order, nrm);
}

// Default group width for a C-column matrix: every pair of a round in flight at once when
// possible, otherwise the widest group that keeps at most two pairs per group.
__host__ __device__ inline int default_group_width(int R, int C) {
    const int pairs = (C + 1) / 2;
    if (pairs <= NT / 16 && R > 64) return 16;
    if (pairs <= NT / 8) return 8;
    return 4;
}

constexpr int JSCHED_BLOCK = 256;   // schedule bit: block-cyclic pair ordering
constexpr int JSCHED_STAGED = 512;  // schedule: staged block pairs (width field = block width b)
__host__ __device__ inline int jsched_width(int js) { return js & 255; }
__host__ __device__ inline int jsched_order(int js) { return js >> 8; }

// Device-memory floats of the workspace of the SVD warm start of Algorithm 2 (tilt_cayley.cuh):
// eight R x C planes, P_U (R x R), P_V and a C x C right-hand side, Sigma.
__host__ __device__ inline size_t cayley_floats(const Dims& d) {
    return (size_t)8 * d.ldb * d.Cp + (size_t)d.ldb * d.ldb + (size_t)2 * d.ldv * d.Cp + (size_t)d.Cp;
}

// Staged sweeps (matrices whose B and V live in device memory): shared-memory bytes of the
// three column blocks of width b, and the widest even b <= 16 whose blocks fit in `avail`
// bytes (0 when none does).
__host__ __device__ inline size_t jacobi_stage_bytes(const Dims& d, int b) {
    return (size_t)3 * b * (d.ldb + d.ldv) * sizeof(float);
}
__host__ __device__ inline int staged_block(const Dims& d, size_t avail) {
    for (int b = 16; b >= 2; b -= 2)
        if (jacobi_stage_bytes(d, b) <= avail) return b;
    return 0;
}

// Schedule of a size bucket the autotuner has not timed: block-cyclic ordering (one CTA
// barrier per block round instead of one per round), 16 lanes per pair for the long
// columns of wide matrices, 8 otherwise.  (The autotuner picks block-cyclic for most
// buckets; round-robin width 4 was 1.4x slower on 200 x 200 windows.)
__host__ __device__ inline int default_schedule(int R, int C) {
    return ((R > 128 && C >= 64) ? 16 : 8) | JSCHED_BLOCK;
}

// Whether the SVT of an R x C matrix may take the QR path of svt_tall_qr (tall matrices: the
// data matrices of RASL's image sets, one column per image).
__host__ __device__ inline bool tall_qr_ok(const Dims& d) { return d.R >= 4 * d.C + 4 && d.C >= 2; }
// Floats of the QR path's small buffers (buf.B): four C x C matrices at stride Cp and the
// reflectors' heads and scales.
__host__ __device__ inline size_t tall_small_floats(const Dims& d) { return ((size_t)4 * d.C + 2) * d.Cp; }

// Schedule of a RASL set (long columns of m n pixels, one per image) whose size bucket the
// autotuner has not timed: block-cyclic, 16 lanes per pair once the columns are 256 long
// (measured on 32 x 32 windows of 32 images: 0.83x the SVD cycles per iteration of width 8,
// 0.41x of width 4).
__host__ __device__ inline int rasl_schedule(int R, int C) {
    (void)C;
    return (R >= 256 ? 16 : 8) | JSCHED_BLOCK;
}

// The kept columns (w_k > 0) in ascending order, sum and max of (sigma_k - eps)_+ over them
// and the numerical rank at 1e-3 of the largest (scal[3], scal[4], iscal[2]; the kept count in
// iscal[1]).  All threads.
static __device__ void svt_select(int C, float eps, const float* sigma, const float* w, int* kept, Scratch* sc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0) {
        // kept columns in ascending order (ballot and prefix count), sum and max of
        // (sigma - eps)_+ over them, then the numerical rank at 1e-3 of the largest
        int nk = 0;
        float nuc = 0.f, mx = 0.f;
        for (int k0 = 0; k0 < C; k0 += 32) {
            const int k = k0 + lane;
            const bool keep = k < C && w[k] > 0.f;
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                kept[nk + __popc(m & ((1u << lane) - 1u))] = k;
                const float sv = sigma[k] - eps;
                nuc += sv;
                mx = fmaxf(mx, sv);
            }
            nk += __popc(m);
        }
        nuc = warp_sum(nuc);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        __syncwarp();
        int rk = 0;
        for (int q0 = 0; q0 < nk; q0 += 32) {
            const int q = q0 + lane;
            const bool big = q < nk && sigma[kept[q]] - eps > 1e-3f * mx;
            rk += __popc(__ballot_sync(0xffffffffu, big));
        }
        if (lane == 0) {
            sc->iscal[1] = nk;
            sc->scal[3] = (double)nuc;
            sc->scal[4] = (double)mx;
            sc->iscal[2] = rk;
        }
    }
    __syncthreads();
}

// Column norms sigma_k = ||b_k||, weights w_k = max(sigma_k - eps, 0) / sigma_k and the
// list of kept columns.  Returns (via scal) sum (sigma - eps)_+, max (sigma - eps)_+ and
// the kept count (iscal[1]).
static __device__ void svt_weights(const float* B, int ldb, int R, int C, float eps, float* sigma, float* w, int* kept,
                            Scratch* sc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = warp; k < C; k += NW) {
        const float* bk = B + (size_t)k * ldb;
        float s = 0.f;
        for (int r = lane; r < R; r += 32) s = fmaf(bk[r], bk[r], s);
        s = warp_sum(s);
        if (lane == 0) {
            const float sg = sqrtf(s);
            sigma[k] = sg;
            w[k] = (sg > eps) ? (sg - eps) / sg : 0.f;
        }
    }
    __syncthreads();
    svt_select(C, eps, sigma, w, kept, sc);
}

// Reconstruction coefficients of the singular value thresholding from the left factor:
// with B = U Sigma (orthogonal columns after the sweeps) and X = B V^T,
//   S_eps(X) = sum_k (sigma_k - eps)_+ u_k v_k^T = sum_k (w_k / sigma_k^2) b_k (X^T b_k)^T,
// which needs only the measured orthogonality of B, not the orthogonality of the
// accumulated V (FP32 rotations drift V away from orthogonal far faster than B).
// Z[q * ldz + c] = (w_k / sigma_k^2) (X^T b_k)_c for the kept columns k = kept[q]: the
// product B_K^T X (nk x R times R x C) on the tensor cores (3xTF32, FP32 accumulate).
// X and B have column stride ldx / ldb (rows R).  All threads; false if a wait gave up.
static __device__ bool svt_coeffs_tc(const float* __restrict__ X, int ldx, const float* __restrict__ B, int ldb,
                                     int R, int C, const float* sigma, const float* w, const int* kept, int nk,
                                     float* __restrict__ Z, int ldz, unsigned char* stage, int nbuf, TcState* tc) {
    if (nk <= 0) return true;
    auto la = [=](int q, int r) { return B[(size_t)kept[q] * ldb + r]; };   // B_K^T: contiguous along R
    auto lb = [=](int r, int c) { return X[(size_t)c * ldx + r]; };        // X: contiguous along R
    auto ep = [=](int q, int c, float v) {
        const int k = kept[q];
        Z[(size_t)q * ldz + c] = v * (w[k] / (sigma[k] * sigma[k]));
    };
    return tc_gemm<NT, true, true>(nk, C, R, la, lb, ep, stage, TC_KC, nbuf, tc);
}

// Warm start of the Jacobi SVD: B = T V (R x C times C x C, both column-major with strides
// ldb and ldv) on the tensor cores (3xTF32, FP32 accumulate).  Rows up to ldb are written,
// so B's padding rows (zero in T) stay zero.  All threads; false if a wait gave up.
static __device__ bool warm_start_tc(const float* __restrict__ T, int ldb, const float* __restrict__ V, int ldv,
                                     float* __restrict__ B, int C, unsigned char* stage, int nbuf, TcState* tc) {
    auto la = [=](int r, int j) { return T[(size_t)j * ldb + r]; };        // contiguous along rows
    auto lb = [=](int j, int c) { return V[(size_t)c * ldv + j]; };        // contiguous along K
    auto ep = [=](int r, int c, float v) { B[(size_t)c * ldb + r] = v; };
    return tc_gemm<NT, false, true>(ldb, C, C, la, lb, ep, stage, TC_KC, nbuf, tc);
}

// The coefficients Z[q * ldz + c] = (w_k / sigma_k^2) (X^T b_k)_c on the SIMT pipes for any
// column stride ldx of X (the step entry point reads X in place), one 8-lane group per
// coefficient.
static __device__ void svt_left_coeffs(const float* __restrict__ X, int ldx, const float* __restrict__ B, int ldb, int R,
                                       int C, const float* sigma, const float* w, const int* kept, int nk,
                                       float* __restrict__ Z, int ldz) {
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 3, g = lane & 7;
    const unsigned gmask = 0xFFu << (lane & 24);
    constexpr int NG = NT / 8;
    const bool vec = ((ldx & 3) == 0) && ((ldb & 3) == 0);
    for (int idx = grp; idx < nk * C; idx += NG) {
        const int q = idx / C, c = idx - q * C;
        const int k = kept[q];
        const float* x = X + (size_t)c * ldx;
        const float* b = B + (size_t)k * ldb;
        float s = 0.f;
        if (vec) {
            const int nq = (R + 3) >> 2;   // padding rows of B are zero, X rows beyond R exist (ldx >= R rounded)
            for (int t = g; t < nq; t += 8) {
                const float4 xv = reinterpret_cast<const float4*>(x)[t];
                const float4 bv = reinterpret_cast<const float4*>(b)[t];
                s = fmaf(xv.x, bv.x, fmaf(xv.y, bv.y, fmaf(xv.z, bv.z, fmaf(xv.w, bv.w, s))));
            }
        } else {
            for (int r = g; r < R; r += 8) s = fmaf(x[r], b[r], s);
        }
        s += __shfl_xor_sync(gmask, s, 1, 8);
        s += __shfl_xor_sync(gmask, s, 2, 8);
        s += __shfl_xor_sync(gmask, s, 4, 8);
        if (g == 0) {
            const float sg = sigma[k];
            Z[(size_t)q * ldz + c] = s * (w[k] / (sg * sg));
        }
    }
    __syncthreads();
}

// The same coefficients as a register-tiled FP32 product on the SIMT pipes (the windows too
// small for the tensor-core product to pay; rows of Z at stride ldz, a multiple of 4): a
// group of 8 lanes
// owns a 2 x 2 tile of Z (two kept columns of B times two columns of X); lane g takes the
// float4 row chunks g, g+8, ... of the four columns (consecutive chunks within a quarter
// warp: no bank conflicts whatever the column stride), so every shared-memory load feeds
// four FMAs, and the four sums reduce over 3 shuffle levels.  Padding rows (R..ldx) of X
// and B are zero.
static __device__ void svt_coeffs_tiled(const float* __restrict__ X, int ldx, const float* __restrict__ B, int ldb,
                                        int R, int C, const float* sigma, const float* w, const int* kept, int nk,
                                        float* __restrict__ Z, int ldz) {
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 3, g = lane & 7;
    const unsigned gmask = 0xFFu << (lane & 24);
    constexpr int NG = NT / 8;
    const int nq2 = (nk + 1) >> 1, nc2 = (C + 1) >> 1;
    const int nr4 = (R + 3) >> 2;
    for (int t = grp; t < nq2 * nc2; t += NG) {
        const int qp = t / nc2, cp = t - qp * nc2;
        const int q0 = 2 * qp, q1 = min(q0 + 1, nk - 1);
        const int c0 = 2 * cp, c1 = min(c0 + 1, C - 1);
        const int k0 = kept[q0], k1 = kept[q1];
        const float4* b0 = reinterpret_cast<const float4*>(B + (size_t)k0 * ldb);
        const float4* b1 = reinterpret_cast<const float4*>(B + (size_t)k1 * ldb);
        const float4* x0 = reinterpret_cast<const float4*>(X + (size_t)c0 * ldx);
        const float4* x1 = reinterpret_cast<const float4*>(X + (size_t)c1 * ldx);
        float s00 = 0.f, s01 = 0.f, s10 = 0.f, s11 = 0.f;
        for (int r = g; r < nr4; r += 8) {
            const float4 u0 = b0[r], u1 = b1[r], v0 = x0[r], v1 = x1[r];
            s00 = fmaf(u0.x, v0.x, fmaf(u0.y, v0.y, fmaf(u0.z, v0.z, fmaf(u0.w, v0.w, s00))));
            s01 = fmaf(u0.x, v1.x, fmaf(u0.y, v1.y, fmaf(u0.z, v1.z, fmaf(u0.w, v1.w, s01))));
            s10 = fmaf(u1.x, v0.x, fmaf(u1.y, v0.y, fmaf(u1.z, v0.z, fmaf(u1.w, v0.w, s10))));
            s11 = fmaf(u1.x, v1.x, fmaf(u1.y, v1.y, fmaf(u1.z, v1.z, fmaf(u1.w, v1.w, s11))));
        }
#pragma unroll
        for (int off = 1; off < 8; off <<= 1) {
            s00 += __shfl_xor_sync(gmask, s00, off, 8);
            s01 += __shfl_xor_sync(gmask, s01, off, 8);
            s10 += __shfl_xor_sync(gmask, s10, off, 8);
            s11 += __shfl_xor_sync(gmask, s11, off, 8);
        }
        if (g == 0) {
            const float f0 = w[k0] / (sigma[k0] * sigma[k0]), f1 = w[k1] / (sigma[k1] * sigma[k1]);
            Z[(size_t)q0 * ldz + c0] = s00 * f0;
            if (c1 != c0) Z[(size_t)q0 * ldz + c1] = s01 * f0;
            if (q1 != q0) {
                Z[(size_t)q1 * ldz + c0] = s10 * f1;
                if (c1 != c0) Z[(size_t)q1 * ldz + c1] = s11 * f1;
            }
        }
    }
    __syncthreads();
}

// B = T V (R x C times C x C), RT x 4 register tiles (RT = 4 or 8 rows: float4 reads of T,
// broadcast reads of V); T, B stride ldb (multiple of 4), V stride ldv.  Works on padded
// sizes (ldb rows, Cp columns).
template <int RT>
static __device__ void gemm_TV(const float* __restrict__ T, int ldb, const float* __restrict__ V, int ldv,
                               float* __restrict__ B, int Cp, int C) {
    static_assert(RT == 4 || RT == 8, "row tile");
    const int rt_n = (ldb + RT - 1) / RT, ct_n = Cp / 4;
    const int ntile = rt_n * ct_n;
    for (int t = threadIdx.x; t < ntile; t += NT) {
        const int rt = t % rt_n, ct = t / rt_n;
        const int r0 = rt * RT, c0 = ct * 4;
        const bool two = RT == 8 && r0 + 4 < ldb;     // second float4 of rows in range
        float acc[RT][4];
#pragma unroll
        for (int a = 0; a < RT; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
        for (int j = 0; j < C; ++j) {
            float tv[RT];
            const float4 t0 = *reinterpret_cast<const float4*>(T + (size_t)j * ldb + r0);
            tv[0] = t0.x; tv[1] = t0.y; tv[2] = t0.z; tv[3] = t0.w;
            if (RT == 8) {
                const float4 t1 = two ? *reinterpret_cast<const float4*>(T + (size_t)j * ldb + r0 + 4)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
                tv[RT - 4] = t1.x; tv[RT - 3] = t1.y; tv[RT - 2] = t1.z; tv[RT - 1] = t1.w;
            }
            float vv[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) vv[b] = V[(size_t)(c0 + b) * ldv + j];
#pragma unroll
            for (int a = 0; a < RT; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(tv[a], vv[b], acc[a][b]);
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            *reinterpret_cast<float4*>(B + (size_t)(c0 + b) * ldb + r0) =
                make_float4(acc[0][b], acc[1][b], acc[2][b], acc[3][b]);
            if (RT == 8 && two)
                *reinterpret_cast<float4*>(B + (size_t)(c0 + b) * ldb + r0 + 4) =
                    make_float4(acc[RT - 4][b], acc[RT - 3][b], acc[RT - 2][b], acc[RT - 1][b]);
        }
    }
    __syncthreads();
}

// Largest deviation of a column norm of V from 1 (how far the FP32 rotations have let V
// drift from orthogonal).
static __device__ float v_drift(const float* V, int ldv, int C, Scratch* sc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float mx = 0.f;
    for (int k = warp; k < C; k += NW) {
        const float* v = V + (size_t)k * ldv;
        float s = 0.f;
        for (int r = lane; r < C; r += 32) s = fmaf(v[r], v[r], s);
        s = warp_sum(s);
        mx = fmaxf(mx, fabsf(s - 1.f));
    }
    // max of the warp maxima through shared memory (as floats: no FP64 conversions per thread)
    float* fr = reinterpret_cast<float*>(sc->red);
    if (lane == 0) fr[warp] = mx;
    __syncthreads();
    float r = 0.f;
    for (int w = 0; w < NW; ++w) r = fmaxf(r, fr[w]);
    __syncthreads();
    return r;
}

// Re-orthonormalise the C columns of V (stride ldv) by modified Gram-Schmidt in FP64 before a
// warm start, when the FP32 rotations have let V drift from orthogonal: column j is
// normalised, then projected out of every later column, the dot products and updates in
// FP64 (V itself stays FP32, so the result is orthonormal to FP32 rounding).  About C^3
// FP64 multiply-adds and 2 C CTA barriers; all threads.
static __device__ void v_reorth_fp64(float* V, int ldv, int C, Scratch* sc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = 0; j < C; ++j) {
        float* vj = V + (size_t)j * ldv;
        double nn[1] = {0.0};
        for (int r = threadIdx.x; r < C; r += NT) nn[0] += (double)vj[r] * (double)vj[r];
        block_sum64<1>(nn, sc->red);
        const double inv = nn[0] > 0.0 ? 1.0 / sqrt(nn[0]) : 0.0;
        for (int r = threadIdx.x; r < C; r += NT) vj[r] = (float)((double)vj[r] * inv);
        __syncthreads();
        for (int k = j + 1 + warp; k < C; k += NW) {
            float* vk = V + (size_t)k * ldv;
            double dp = 0.0;
            for (int r = lane; r < C; r += 32) dp += (double)vj[r] * (double)vk[r];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) dp += __shfl_xor_sync(0xffffffffu, dp, off);
            for (int r = lane; r < C; r += 32) vk[r] = (float)((double)vk[r] - dp * (double)vj[r]);
        }
        __syncthreads();
    }
}

// V = I (Cp x Cp, stride ldv).
__device__ inline void set_identity(float* V, int ldv, int Cp) {
    for (int e = threadIdx.x; e < ldv * Cp; e += NT) {
        const int r = e % ldv, c = e / ldv;
        V[e] = (r == c) ? 1.f : 0.f;
    }
    __syncthreads();
}

// Singular values below this fraction of the largest are treated as converged noise
// by the rotation test (FP32 dot products cannot resolve more).
__device__ inline float jacobi_tol(int R) { return 1e-6f * fmaxf(1.f, sqrtf((float)R / 256.f)); }

}  // namespace tilt
