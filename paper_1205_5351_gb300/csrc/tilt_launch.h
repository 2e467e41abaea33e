// Host-side declarations of the kernel launchers (defined in tilt_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "tilt_device.cuh"

namespace tilt {

// Output record of the step kernels (device memory).
struct StepOut {
    double norm;          // warp: ||D o tau||_F
    int oob;              // warp: clamped samples
    int sweeps;           // svt / inner
    int iters;            // inner
    int status;           // 0 ok, -2 singular G
    int reorth;           // svt: the warm start's V was re-orthonormalised in FP64
    int accepted;         // cayley: the step was taken
    double cay[5];        // cayley: f'(0), f''(0), t, f(0), f(t)
    double c1, c2, mu;    // inner
    double Q[3 * PMAX], G[PMAX * PMAX], Gi[PMAX * PMAX];
    double dtau[PMAX];
};

struct WarpArgs {
    const float* img;
    long long ld;
    int H, W, m, n, ttype;
    double tau[PMAX];
    float* Dhat;
    float* J;
    StepOut* out;
};

struct GramArgs {
    const float* J;
    const float* Dhat;   // may be a zero plane (only J^T J and Q are reported)
    int m, n, ttype;
    double tau[PMAX];
    StepOut* out;
};

struct SvtArgs {
    const float* M;
    float* A;
    int m, n;
    float eps;
    int smem_svd;
    float* Bg;    // global SVD buffers when !smem_svd
    float* Vg;
    float* Tg;
    float* Zg;    // device, C * Cp floats
    float* sigma; // device, C floats
    int jsched;   // Jacobi schedule (staged sweeps when the SVD buffers are in device memory)
    float* Vio;   // nullptr: cold start; else C x C right singular vectors (stride C) to warm-start
                  // from, overwritten with the new ones
    StepOut* out;
};

struct InnerArgs {
    const float* Dhat;
    const float* J;
    float* A;
    float* E;
    float* Y;
    float* Mp;     // scratch S
    float* Bg;     // global SVD buffers when !smem_svd
    float* Vg;
    float* Tg;
    float* Zg;     // scratch C * C
    float* Cay;    // Algorithm 2 workspace (cayley_floats) when prm.svd_ws = 1, else nullptr
    int m, n, ttype, smem_svd;
    int use_q;     // 0: no constraint rows (G = J^T J, W^T W = J_perp)
    int jsched;    // Jacobi schedule
    double tau[PMAX];
    Params prm;
    double mu0;
    StepOut* out;
};

struct AdmArgs {
    const float* D;
    const float* J;    // p planes (p may be 0)
    float* A;
    float* E;
    float* Y;
    float* Bg;         // global SVD buffers when !smem_svd
    float* Vg;
    float* Tg;
    float* Zg;         // scratch C * Cp
    int m, n, p, smem_svd, max_iter, jsched;
    double lam, tol, rho, mu0;
    StepOut* out;
};

struct CayArgs {
    const float* M;    // m x n, long-side layout (stride R)
    float* U;          // R x C, stride R (in/out)
    float* S;          // C (in/out)
    float* V;          // C x C, stride C (in/out)
    float* work;       // cayley_floats(d) + ldb * Cp + ldv * Cp floats of device memory
    int m, n;
    StepOut* out;
};

// Work queue of the persistent workers.  ring/tail/stop live in host-mapped memory (written
// by the host), head in device memory (claimed by the workers with atomicCAS).
struct WorkQueue {
    const int* ring;        // slot indices, cap entries
    int cap;
    const int* tail;        // entries published so far (host writes with release order)
    const int* stop;        // non-zero: workers exit when idle
    const int* cancel;      // non-zero: claimed problems are retired unsolved
    int* head;              // entries claimed so far
    int idle_spins;         // bounded idle wait (x ~2 us) before a worker exits
};

// Persistent workers: `ctas` CTAs claim problems from the queue until it stays empty for
// idle_spins polls (or stop is set), each solving one problem at a time.
cudaError_t launch_workers(Problem* probs, const WorkQueue& q, int ctas, size_t smem, cudaStream_t st);

// Solver: count CTAs, CTA b solves probs[order[b]].  minb selects the occupancy variant, tcp
// the 1-CTA variant that carries the tensor-core products (launch class 2).
cudaError_t launch_solver(Problem* probs, const int* order, int count, int minb, bool tcp, size_t smem,
                          cudaStream_t st);
cudaError_t launch_warp_step(const WarpArgs& a, cudaStream_t st);
cudaError_t launch_gram_step(const GramArgs& a, cudaStream_t st);
cudaError_t launch_svt_step(const SvtArgs& a, size_t smem, cudaStream_t st);
cudaError_t launch_inner_step(const InnerArgs& a, size_t smem, cudaStream_t st);
cudaError_t launch_adm_step(const AdmArgs& a, size_t smem, cudaStream_t st);
cudaError_t launch_cayley_step(const CayArgs& a, cudaStream_t st);
// RASL image sets: count CTAs, CTA b solves probs[b] (tcp: the variant with the staged
// Jacobi sweeps).
cudaError_t launch_rasl(RaslProblem* probs, int count, bool tcp, size_t smem, cudaStream_t st);
// One-time kernel attribute setup (dynamic shared memory opt-in).
cudaError_t configure_kernels(size_t max_smem);
cudaError_t configure_tc_kernels(size_t max_smem);
cudaError_t configure_worker_kernel(size_t max_smem);
cudaError_t configure_step_kernels(size_t max_smem);
cudaError_t configure_rasl_kernels(size_t max_smem);
// The tensor-core variant of the solver (launch class 2), called by launch_solver.
cudaError_t launch_solver_tc(Problem* probs, const int* order, int count, size_t smem, cudaStream_t st);

// Record an error message for tilt_last_error() on the calling thread; returns code.
int set_error(int code, const char* msg);

}  // namespace tilt
