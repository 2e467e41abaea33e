/*
 * tilt.h -- C ABI of the GB300 (sm_103a) solver for Transform Invariant Low-rank Textures
 * by the Linearized Alternating Direction Method with Adaptive Penalty and warm starts
 * (Ren & Lin, arXiv 1205.5351).
 *
 * The solver rectifies an m x n window of an image: it finds the transform tau (affine,
 * p = 6, or projective, p = 8) and the split D o tau / ||D o tau||_F = A + E with A of low
 * rank and E sparse, by Algorithm 1 of the paper (outer loop: warp, normalise, Jacobian,
 * dtau; inner loop: LADMAP on the reformulated problem of Sec. 3.2 / 4.3 with singular
 * value thresholding, soft thresholding, the multiplier update and the adaptive penalty).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Images are float32, row-major, element (row y, column x) at img[y * ld + x], H >= 2,
 * W >= 2.  Window pixel (i, j), 0 <= i < m, 0 <= j < n, has centred coordinates
 * u = j - (n-1)/2, v = i - (m-1)/2.  tau maps (u, v) to image coordinates (x = column,
 * y = row):
 *   affine      tau = [a11 a12 a13 a21 a22 a23]:  x = a11 u + a12 v + a13,
 *                                                 y = a21 u + a22 v + a23
 *   projective  tau = [h1 .. h8]:  x = (h1 u + h2 v + h3) / (h7 u + h8 v + 1),
 *                                  y = (h4 u + h5 v + h6) / (h7 u + h8 v + 1)
 * D o tau is the bilinear interpolant of the image at those points; coordinates outside
 * the image are clamped to the edge (and counted).  Window sides: 2 <= m, n <= 512.
 *
 * Return codes are tilt_status values; on a negative code tilt_last_error() returns a
 * message for the calling thread.  No entry point is thread-safe on one context; use one
 * context per host thread.
 */
#ifndef TILT_H
#define TILT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tilt_ctx tilt_ctx;

typedef enum { TILT_AFFINE = 6, TILT_PROJECTIVE = 8 } tilt_transform;

typedef enum {
    TILT_OK = 0,
    TILT_PENDING = 1,       /* tilt_poll: the problem has not finished yet                    */
    TILT_E_INVAL = -1,      /* an argument is out of range                                    */
    TILT_E_NOMEM = -2,      /* the problem can never fit the context's device-memory budget  */
    TILT_E_BUSY = -3,       /* the admission queue is full; retry after polling              */
    TILT_E_CUDA = -4,       /* a CUDA call failed (message has the CUDA error string)         */
    TILT_E_TIMEOUT = -5,    /* a bounded wait expired                                         */
    TILT_E_NOTFOUND = -6    /* unknown or already retired ticket                              */
} tilt_status;

/* Context configuration.  Zero-initialise and set what you need. */
typedef struct {
    int device;                 /* CUDA device ordinal                                        */
    size_t hbm_budget_bytes;    /* device workspace pool; 0 -> 25 % of free memory at create  */
    int max_live;               /* problems admitted at once; 0 -> 65536                      */
    void* cuda_stream;          /* a cudaStream_t, or NULL: the context creates its own streams.
                                   Non-NULL: grouped launches (all launch classes, one after
                                   another), image uploads, plane reads and the step entry
                                   points are issued on this stream, which the context never
                                   destroys; tilt_destroy waits for it to drain.  The
                                   persistent workers of tilt_submit always run on a stream of
                                   the context's own, since they stay resident between
                                   submissions                                                */
    const char* autotune_cache; /* file of autotuned Jacobi schedules (read at create, written by
                                   tilt_autotune); NULL: tuning lives in the context only     */
} tilt_config;

/* Solver parameters (Algorithm 1 inputs).  tilt_default_params() fills the defaults;
 * a value <= 0 in lambda or mu0 selects the default rule. */
typedef struct {
    double lambda;     /* weight of ||E||_1; <= 0 -> 1/sqrt(max(m, n))                        */
    double eps1;       /* Eq. Cond1 threshold (default 1e-5)                                  */
    double eps2;       /* Eq. Cond2 / Eq. rho threshold (default 0.1)                         */
    double rho0;       /* Eq. rho growth factor, >= 1 (default 1.5)                           */
    double mu0;        /* initial penalty of every inner loop; <= 0 -> 1.25 / ||D_hat||_2     */
    double mu_max;     /* Eq. mu upper bound (default 1e10)                                   */
    double eps_svd;    /* SVD warm-start gate (the gate of Alg. 2): warm-start the Jacobi SVD
                          from the previous V when ||M_k - M_k-1||_F < eps_svd ||M_k||_F;
                          < 0 (default): whenever the previous V is valid.  The warm-started
                          Jacobi converges to the exact SVD for any change of M (it never
                          took more sweeps than a cold start in measurements), unlike the
                          approximate Cayley step that Alg. 2 gates                          */
    int max_inner;     /* inner iterations per outer step (default 500)                       */
    int max_outer;     /* outer steps (default 10)                                            */
    double outer_tol;  /* stop when dtau moves no window corner by more than this many
                          pixels (default 1e-2)                                               */
    int svd_ws;        /* SVD warm start: 0 (default) the previous right singular vectors feed
                          one-sided Jacobi sweeps, which end at an exact SVD; 1 the paper's
                          Algorithm 2: when ||M_k - M_k-1||_F < eps_svd ||M_k||_F (eps_svd < 0:
                          always) take one step along the Cayley curve from the previous
                          factors (tilt_svd_cayley) and threshold that approximate SVD, doing
                          a full SVD when the step is refused; the first SVD of every inner
                          loop is full.  Extra device memory per problem: about 8 R C + R^2
                          floats                                                          */
} tilt_params;

/* Result of one problem. */
typedef struct {
    int status;          /* 0 outer loop converged, 1 max_outer reached, 2 some inner loop hit
                            max_inner (tau still valid), < 0 numeric failure (-1 non-finite,
                            -2 singular J^T J + Q^T Q, -3 zero image window), -4 cancelled
                            by tilt_destroy (tau = the last completed outer step's), -5 a
                            bounded device wait expired (a tensor-core product did not
                            complete; tau = the last completed outer step's)                  */
    int p;               /* 6 or 8                                                             */
    double tau[8];       /* final transform (first p entries)                                 */
    double objective;    /* ||A||_* + lambda ||E||_1 of the last inner loop (Eq. TILT_2)       */
    double lambda;       /* lambda actually used                                              */
    int rank_A;          /* singular values of A above 1e-3 * the largest                     */
    int outer_iters;     /* outer steps taken                                                 */
    int inner_iters;     /* inner iterations summed over outer steps                          */
    int svd_sweeps;      /* one-sided Jacobi sweeps summed over all SVDs                      */
    int svd_warm;        /* SVDs that started from the previous right singular vectors (all but
                            the first of a solve)                                            */
    int oob_pixels;      /* samples clamped to the image edge in the last warp                */
    double kkt_residual; /* last Eq. Cond1 value                                              */
    float latency_ms;    /* submit -> completion, host clock                                  */
    uint64_t phase_cycles[5]; /* SM clock cycles of the solve by phase: warp + Jacobian, SVD
                                 (Jacobi sweeps + warm-start product), SVT reconstruction,
                                 elementwise passes (E, Y, M), other (Gram, ||D||_2)          */
    int launch_class;    /* grouped launch that solved it (tilt_submit_batch): 0 two CTAs per
                            SM, all SVD buffers in shared memory; 1 one CTA per SM, the SVD
                            buffers in shared memory as far as they fit (also class-0-sized
                            problems of a batch no larger than the SM count); 2 one CTA per
                            SM with the tensor-core products (short side >= 160), or with
                            every SVD buffer in device memory.  -1: solved by the persistent
                            workers                                                         */
    int svd_reorth;      /* warm starts whose right singular vectors had drifted from
                            orthogonal (a column norm off by more than 1e-4) and were
                            re-orthonormalised in FP64 first                                */
    int svd_cayley;      /* SVDs taken from an accepted step of Algorithm 2 (svd_ws = 1)     */
} tilt_result;

/* Fill *p with the default parameters. */
void tilt_default_params(tilt_params* p);

/* Create a context on cfg->device: allocates the device workspace pool (budget), its
 * streams and pinned completion records.  *out receives the context.  Errors:
 * TILT_E_INVAL (null pointer, bad device), TILT_E_CUDA. */
int tilt_create(const tilt_config* cfg, tilt_ctx** out);

/* Queue one problem (Algorithm 1 input: window D given by the image and m x n, initial
 * transform tau0[p], transform type, parameters; params may be NULL for defaults).
 * img is a host pointer (is_device_ptr = 0; copied before the call returns, so the caller
 * may reuse it at once) or a device pointer (is_device_ptr = 1; it must stay valid and
 * unchanged until the problem retires).  ld_elems is the image row stride in elements.
 * The problem starts on the GPU at once when it fits the budget, otherwise when earlier
 * problems retire.  *ticket_out identifies it for tilt_poll.  Errors: TILT_E_INVAL,
 * TILT_E_NOMEM (larger than the whole budget), TILT_E_BUSY (max_live reached), TILT_E_CUDA. */
int tilt_submit(tilt_ctx* ctx, const float* img, int H, int W, size_t ld_elems, int is_device_ptr,
                int m, int n, const double* tau0, tilt_transform type, const tilt_params* params,
                uint64_t* ticket_out);

/* One problem of a grouped submission. */
typedef struct {
    const float* img;    /* host or device pointer (see is_device_ptr of tilt_submit_batch)  */
    int H, W;
    size_t ld_elems;
    int m, n;
    int type;            /* tilt_transform                                                    */
    double tau0[8];
} tilt_problem;

/* Queue count problems as one grouped launch per size class (problems ordered by cost,
 * largest first, so that the block scheduler balances the load; a batch of at most one
 * problem per SM runs every problem one CTA per SM).  Same semantics as
 * count calls of tilt_submit; tickets_out[count] receives the tickets.  Either every
 * problem is admitted or none is (TILT_E_NOMEM / TILT_E_BUSY).  With the context's own
 * streams, consecutive batches alternate between two sets of streams: a batch submitted while
 * the previous one still runs starts on the SMs that batch frees (its longest solves finish
 * alongside). */
int tilt_submit_batch(tilt_ctx* ctx, int count, const tilt_problem* problems, int is_device_ptr,
                      const tilt_params* params, uint64_t* tickets_out);

/* Autotuner: for the size bucket ((R+15)/16, (C+15)/16), R = max(m, n), C = min(m, n), of
 * each of the count shapes (m, n pairs in shapes[2*count]) not tuned yet, time the Jacobi
 * schedules (group width 4, 8 or 16 lanes per column pair, times round-robin or
 * block-cyclic pair ordering) on a synthetic grouped launch (one problem per SM, one outer
 * step of 30 inner iterations) and keep the fastest for this context; chosen_out[count]
 * (may be NULL) receives the schedule of each shape: the width, plus 256 for block-cyclic
 * ordering.  Both orderings visit every column pair once per sweep.  The choice
 * depends only on the bucket, never on the batch a problem is submitted with.  When
 * tilt_config.autotune_cache names a file, it is read at tilt_create and rewritten here.
 * Each candidate runs twice and keeps its faster run.  Runs synchronously (about 0.2-4 s
 * per new bucket).  Errors: TILT_E_INVAL, TILT_E_CUDA. */
int tilt_autotune(tilt_ctx* ctx, const int* shapes, int count, tilt_transform type, int* chosen_out);

/* Multi-start selection: the same window solved from several initial transforms, results
 * stored group by group (results[g * starts + s]).  best_out[g] receives the s with the
 * lowest objective ||A||_* + lambda ||E||_1 among the results with status >= 0, or -1 when
 * none succeeded.  Ties keep the lower s.  Errors: TILT_E_INVAL. */
int tilt_best_of(const tilt_result* results, int n_groups, int starts, int* best_out);

/* Non-blocking completion check.  TILT_PENDING while running; TILT_OK once finished, in
 * which case *out (if non-NULL) receives the result, A_out / E_out (host, m x n row-major,
 * may be NULL) receive the final low-rank texture and sparse error of the normalised
 * window, and the ticket is retired (TILT_E_NOTFOUND afterwards).  Nothing is written
 * while the problem is pending. */
int tilt_poll(tilt_ctx* ctx, uint64_t ticket, tilt_result* out, float* A_out, float* E_out);

/* Blocking form of tilt_poll: waits up to timeout_ms (< 0: 60 s) and returns TILT_E_TIMEOUT
 * if the problem is still running then. */
int tilt_wait(tilt_ctx* ctx, uint64_t ticket, int timeout_ms, tilt_result* out, float* A_out,
              float* E_out);

/* Cancel and free: running solves stop after their current inner iteration, queued and
 * not yet started problems are retired unsolved (status -4), the persistent workers exit;
 * then wait (bounded, 120 s) for the device to finish and free everything.  Returns
 * TILT_E_TIMEOUT if work was still running when the wait expired (resources are then
 * leaked, never freed under a running kernel). */
int tilt_destroy(tilt_ctx* ctx);

/* Message of the last error on the calling thread ("" if none).  ctx is unused. */
const char* tilt_last_error(tilt_ctx* ctx);

/* Number of device kernels this context has launched (for launch accounting). */
uint64_t tilt_kernel_launches(tilt_ctx* ctx);

/* Device time of the grouped launches of the most recent tilt_submit_batch, measured with
 * CUDA events recorded around each launch on its own stream.  Waits (bounded, 600 s) for
 * those launches to finish, writes up to cap elapsed times in milliseconds to ms_out (one
 * per occupancy class launched) and returns their number, or a negative tilt_status. */
int tilt_batch_kernel_ms(tilt_ctx* ctx, float* ms_out, int cap);

/* ------------------------------------------------------------------------------------------
 * Step-level entry points.  They run one step of the method on one problem with the same
 * device code the solver uses, on the context's stream, and return when it has finished.
 * Device planes (m x n) are stored long-side contiguous: element (i, j) at j*m + i when
 * m >= n and at i*n + j when m < n.  J is p such planes back to back.
 * ---------------------------------------------------------------------------------------- */

/* Algorithm 1 Step 1: D_hat = D o tau / ||D o tau||_F and the Jacobian J of the normalised
 * warp w.r.t. tau (quotient rule).  img_dev: device image; Dhat_dev (m*n) and J_dev (p*m*n)
 * device outputs.  *norm_out = ||D o tau||_F, *oob_out = clamped samples (both may be NULL). */
int tilt_warp_jacobian(tilt_ctx* ctx, const float* img_dev, int H, int W, size_t ld_elems, int m,
                       int n, const double* tau, tilt_transform type, float* Dhat_dev, float* J_dev,
                       double* norm_out, int* oob_out);

/* Sec. 4.3: Q (3 x p: linearised centroid x, centroid y and signed area of the window
 * corners mapped by tau, the area row divided by (m-1)(n-1)), G = J^T J + Q^T Q and G^-1,
 * all row-major host outputs (any may be NULL), computed in FP64 on the device. */
int tilt_gram(tilt_ctx* ctx, const float* J_dev, int m, int n, const double* tau, tilt_transform type,
              double* Q_out, double* G_out, double* Ginv_out);

/* Eqs. A_1, S_operator: A = U max(Sigma - eps, 0) V^T for the m x n device matrix M_dev
 * (layout above) by one-sided Jacobi.  A_dev receives A; sigma_out (host, min(m, n), may be
 * NULL) the singular values of M in no particular order; *sweeps_out the sweeps used. */
int tilt_svt(tilt_ctx* ctx, const float* M_dev, int m, int n, float eps, float* A_dev,
             float* sigma_out, int* sweeps_out);

/* One step of the paper's SVD warm start, Algorithm 2 (Sec. 5, Appendix A): from the factors
 * U (R x C, columns orthonormal), Sigma (C, signed) and V (C x C, orthogonal) of the previous
 * matrix, compute the projected gradients P_U = X M^T - M X^T, P_V = X^T M - M^T X and
 * P_Sigma = Sigma - diag(U^T M V) with X = U Sigma V^T, the derivatives f'(0), f''(0) of
 * f(t) = 1/2 ||M - U(t) Sigma(t) V(t)^T||_F^2 along the Cayley curve of Eq. curve_to_search,
 * t = -f'(0) / f''(0), and the curve point (U(t) = (I + t/2 P_U)^-1 (I - t/2 P_U) U, Sigma(t) =
 * Sigma - t P_Sigma, V(t) likewise).  The step is accepted when f''(0) > 0 and f(t) <= f(0),
 * and then U_dev, S_dev, V_dev are overwritten with the curve point; otherwise they are left
 * as they were (the solver then computes a full SVD).  M_dev: the m x n matrix in the
 * long-side layout above, as the R x C matrix X (R = max(m, n), C = min(m, n)); U_dev R x C
 * column-major (stride R), S_dev C, V_dev C x C column-major (stride C), all device memory.
 * Outputs (host, may be NULL): f'(0), f''(0), t and whether the step was accepted.  FP32
 * products on the SIMT pipes, the two (R x R and C x C) linear systems by Gauss-Jordan
 * elimination with partial pivoting.  Errors: TILT_E_INVAL, TILT_E_CUDA. */
int tilt_svd_cayley(tilt_ctx* ctx, const float* M_dev, int m, int n, float* U_dev, float* S_dev, float* V_dev,
                    double* f1_out, double* f2_out, double* t_out, int* accepted_out);

/* tilt_svt warm-started as the solver warm-starts every SVD after the first (Sec. 5): from the
 * right singular vectors V of the previous iteration's M, re-orthonormalised first in FP64
 * (modified Gram-Schmidt) when a column norm of V is off by more than 1e-4 (FP32 rotations
 * let V drift from orthogonal), then B = X V and one-sided Jacobi sweeps from there.  X is
 * the m x n matrix M_dev when m >= n, its transpose otherwise (the long-side layout above);
 * V_dev: device, min(m, n) x min(m, n), column-major with stride min(m, n); on return it holds
 * the new right singular vectors of X.  *reorth_out (may be NULL) = 1 when V was
 * re-orthonormalised.  Other arguments and errors as tilt_svt. */
int tilt_svt_warm(tilt_ctx* ctx, const float* M_dev, int m, int n, float eps, float* V_dev, float* A_dev,
                  float* sigma_out, int* sweeps_out, int* reorth_out);

/* The inner loop of Algorithm 1 (Eqs. A, E, Y, mu, rho, Cond1, Cond2 in the W^T W form of
 * Eq. newvars2) on given D_hat, J and tau (tau gives Q; tau = NULL: no constraint rows, so
 * W^T W = J_perp of Sec. 4.1, as in the inner-loop-only experiment of Sec. 6.1).  A_dev, E_dev, Y_dev are the warm
 * start on entry (Y is projected by W^T W first, Eq. Y_new_warmstart) and the result on
 * exit.  mu0 <= 0 -> 1.25 / ||D_hat||_2.  Outputs (host, may be NULL): *iters_out,
 * dtau_out[p] (Eq. Delta_tau with Q), *c1_out, *c2_out, *mu_out (last mu used). */
int tilt_inner(tilt_ctx* ctx, const float* Dhat_dev, const float* J_dev, int m, int n,
               const double* tau, tilt_transform type, const tilt_params* params, double mu0,
               float* A_dev, float* E_dev, float* Y_dev, int* iters_out, double* dtau_out,
               double* c1_out, double* c2_out, double* mu_out);

/* The comparison method of Sec. 2.2: the alternating direction method (ADM) of Zhang et al.
 * for the inner loop, Eq. TILT_3 (min ||A||_* + lambda ||E||_1 s.t. D + J dtau = A + E), on
 * given D and J with no constraint rows.  It minimises the augmented Lagrangian over A, E and
 * dtau in turn (A' = S_{1/mu}(D + J dtau - E + Y/mu), E' = T_{lambda/mu}(D + J dtau - A' + Y/mu),
 * dtau' = (J^T J)^-1 J^T (A' + E' - D - Y/mu)), then Y' = Y + mu (D + J dtau' - A' - E') and
 * mu <- rho mu, from A = D, E = 0, dtau = 0, Y = 0, until ||D + J dtau - A - E||_F / ||D||_F <
 * tol.  The SVT is the solver's (one-sided Jacobi, warm-started from the previous V).
 * D_dev: m x n device plane (layout above); J_dev: p such planes, 0 <= p <= 8 (NULL when
 * p = 0).  params (may be NULL): lambda (<= 0 -> 1/sqrt(max(m, n))), eps1 = tol (default
 * 1e-5; Sec. 6.1's comparison uses 1e-7), rho0 = rho > 1 (default 1.5; 1.25 reproduces
 * Table 1's ADM column), max_inner = iteration cap; the other fields are ignored.
 * mu0 <= 0 -> 1.25 / ||D||_2.  A_dev, E_dev, Y_dev (device, m x n) receive the result.
 * Outputs (host, may be NULL): *iters_out, dtau_out[p], *residual_out (the last relative
 * constraint residual; >= tol when the cap was reached), *sweeps_out (Jacobi sweeps).
 * Errors: TILT_E_INVAL (also for a singular J^T J), TILT_E_TIMEOUT, TILT_E_CUDA. */
int tilt_inner_adm(tilt_ctx* ctx, const float* D_dev, const float* J_dev, int m, int n, int p,
                   const tilt_params* params, double mu0, float* A_dev, float* E_dev, float* Y_dev,
                   int* iters_out, double* dtau_out, double* residual_out, int* sweeps_out);

/* Counters of the most recent step entry point on this context (tilt_svt, tilt_svt_warm,
 * tilt_inner, tilt_inner_adm): Jacobi sweeps and, for tilt_inner with svd_ws = 1, the
 * iterations whose SVD came from an accepted step of Algorithm 2.  Either pointer may be NULL.
 * Errors: TILT_E_INVAL. */
int tilt_step_counters(tilt_ctx* ctx, int* sweeps_out, int* cayley_steps_out);

/* ------------------------------------------------------------------------------------------
 * RASL (Sec. 1): the TILT model with one image per column of the data matrix.  An image set
 * is nimg images of the same scene, each seen through its own transform tau_c; column c of
 * D_hat is image c sampled at tau_c over an m x n window (pixel i, j at row i n + j of the
 * column), divided by its own Frobenius norm, and J_c the Jacobian of that column with
 * respect to tau_c, so the Jacobian of the stacked problem is block-diagonal.  Constraint
 * rows Q = [I_p ... I_p] keep the sum of the increments dtau_c at zero (the low-rank
 * objective cannot see a transform applied to every image at once).  Each set runs the whole
 * of Algorithm 1 with this W^T W: the same LADMAP inner loop (Sec. 3.2, Eq. newvars2, warm
 * starts of Eqs. warm_start and Y_new_warmstart, Cond1 and Cond2), dtau_c per image,
 * tau_c <- tau_c + dtau_c, until no window corner of any image moves by outer_tol pixels.
 * lambda <= 0 -> 1/sqrt(max(m n, nimg)).
 *
 * SVT of a tall set (m n >= 4 nimg + 4, M small enough for shared memory: about 200 KB for M,
 * V and the buffers, e.g. 32 images of 32 x 32): M = Q R by Householder reflectors, the
 * one-sided Jacobi SVD of the nimg x nimg matrix R V (warm from the previous V), and
 * S_eps(M) = Q X with X formed from R's SVD (X = sum over kept k of (w_k / sigma_k^2) b_k
 * (R^T b_k)^T, b_k the columns of R V after the sweeps), Q applied in the compact WY form.
 * Other sets run the one-sided Jacobi on M itself, as TILT does. */
typedef struct tilt_rasl_result {
    int status;           /* as tilt_result.status (-2: a J_c^T J_c or the constraint system is singular) */
    int outer_iters, inner_iters;
    int svd_sweeps, svd_warm, svd_reorth;
    int rank;             /* numerical rank of A (singular values > 1e-3 of the largest) */
    int oob_pixels;       /* clamped samples at the last warp, over all images */
    int svt_qr;           /* 1: the SVTs ran through the QR factorisation of M (tall sets whose M fits
                           * in shared memory; see below), 0: one-sided Jacobi on M itself */
    double objective;     /* ||A||_* + lambda ||E||_1 at exit */
    double lambda;
    double kkt_residual;  /* Cond1 value of the last inner iteration */
    unsigned long long cycles[5];  /* SM cycles: warp, SVD, reconstruction, elementwise, other */
} tilt_rasl_result;

/* Solve `count` independent image sets of the same shape, one CTA per set, and wait for them
 * (on the context's first stream, or the caller's stream of tilt_config.cuda_stream).
 * imgs: count * nimg images of H x W floats, set s image c at imgs + (s nimg + c) H W, rows
 * contiguous; device memory when is_device_ptr, else host memory (pinned for speed) that is
 * copied to the device inside the call.  tau0, tau_out (host, may alias): count * nimg * p
 * doubles, set s image c at (s nimg + c) p.  A_out, E_out, D_out (host, may be NULL): the
 * result planes and the D_hat of the last outer step, count * nimg * m * n floats each,
 * set s at offset s nimg m n, column c (image c) contiguous.  results (host): count records.
 * kernel_ms_out (may be NULL): the launch's duration from CUDA events.  The device workspace
 * (about (8 + p) nimg m n floats per set) is the context's scratch and grows on demand.
 * Limits: 2 <= nimg <= 128, m n >= nimg, m, n, H, W >= 2, params->svd_ws = 0.  Errors:
 * TILT_E_INVAL, TILT_E_CUDA. */
int tilt_rasl(tilt_ctx* ctx, int count, int nimg, const float* imgs, int is_device_ptr, int H, int W, int m,
              int n, tilt_transform type, const double* tau0, const tilt_params* params, double* tau_out,
              float* A_out, float* E_out, float* D_out, tilt_rasl_result* results, float* kernel_ms_out);

/* ------------------------------------------------------------------------------------------
 * Allocation-free singular value thresholding.  (The paper has no counterpart: this is a
 * service of the library, not a step of the method.)
 *
 * Same operation and output as tilt_svt, for callers that cannot allocate device memory:
 * code whose device memory is owned by another memory manager with a fixed budget, and
 * latency-critical loops in which cudaMalloc / cudaFree would synchronise the device.  It
 * needs no tilt_ctx and allocates nothing.  Its scratch (the SVD work buffers of matrices
 * too large for shared memory, the reconstruction coefficients and a status record) is one
 * file-scope device array of about 772 KiB that every GPU which loads the library holds until the
 * process exits.
 *
 * M_dev (m x n, long-side-contiguous layout as above), A_dev (same layout) and sigma_dev
 * (min(m, n) floats, may be NULL) are device pointers owned by the caller.  The call is
 * asynchronous on `stream` (a cudaStream_t; NULL for the legacy default stream): it returns
 * after the launch, and the outputs are ready when the stream reaches that point.
 * Limits: 1 <= m, n <= 256, eps >= 0; anything else returns TILT_E_INVAL and launches
 * nothing.  Unlike tilt_svt it reports neither the number of Jacobi sweeps nor whether the
 * sweep cap (60) was reached: the status record it writes stays in the private scratch.  The first call on a device looks up the scratch array's device address with that
 * device current and sets the kernel's shared-memory limit; make that first call before any
 * stream capture.  Every call on a device shares the one scratch array, so calls whose
 * kernels overlap on the GPU (different streams, or host threads) race and corrupt each
 * other's results; serialise them on one stream.  Errors: TILT_E_INVAL, TILT_E_CUDA. */
int tilt_svt_noalloc(const float* M_dev, int m, int n, float eps, float* A_dev, float* sigma_dev,
                     void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TILT_H */
