// The persistent workers that serve single submissions, and their host launcher.
#include "tilt_cayley.cuh"
#include "tilt_launch.h"
#include "tilt_solver.cuh"

namespace tilt {

__device__ inline int load_acquire_sys(const int* p) {
    int v;
    asm volatile("ld.acquire.sys.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Persistent worker: thread 0 claims the next published problem (acquire load of the tail,
// compare-and-swap on the head), the CTA solves it and publishes the result; after
// idle_spins empty polls (each followed by a ~2 us sleep) or when stop is set, it exits.
// Once cancel is set, claimed problems are retired unsolved (status -4) and a running
// solve stops after its current inner iteration.
__global__ void __launch_bounds__(NT, 1) worker_kernel(Problem* probs, WorkQueue q) {
    extern __shared__ __align__(256) unsigned char smem_raw[];
    __shared__ Problem sp;
    __shared__ Result sres;
    __shared__ int claim;
    SmemLayout L = carve_smem(smem_raw);
    tc_setup(&L.sc->tc, TC_TMEM_COLS);
    for (;;) {
        if (threadIdx.x == 0) {
            int got = -1;
            for (int idle = 0; idle <= q.idle_spins;) {
                const int t = load_acquire_sys(q.tail);
                const int h = atomicAdd(q.head, 0);
                if (h < t) {
                    if (atomicCAS(q.head, h, h + 1) == h) {
                        got = load_acquire_sys(q.ring + (h % q.cap));
                        break;
                    }
                    continue;
                }
                if (load_acquire_sys(q.stop)) break;
                ++idle;
                __nanosleep(2000);
            }
            claim = got;
        }
        __syncthreads();
        const int slot = claim;
        __syncthreads();
        if (slot < 0) break;
        {   // the descriptor was written by the host before the tail was published
            const volatile int* s = reinterpret_cast<const volatile int*>(probs + slot);
            int* d = reinterpret_cast<int*>(&sp);
            for (int w = threadIdx.x; w < (int)(sizeof(Problem) / 4); w += NT) d[w] = s[w];
            __syncthreads();
        }
        if (cancel_requested(q.cancel)) {
            if (threadIdx.x == 0) {
                memset(&sres, 0, sizeof sres);
                sres.status = -4;
                sres.p = sp.p;
                for (int k = 0; k < PMAX; ++k) sres.tau[k] = sp.tau[k];
            }
            __syncthreads();
        } else {
            solve_problem<4>(sp, L, sres);
        }
        if (threadIdx.x == 0) {
            *sp.res = sres;
            __threadfence_system();
            *sp.done = 1;
        }
        __syncthreads();
    }
    tc_teardown(&L.sc->tc, TC_TMEM_COLS);
}

cudaError_t configure_worker_kernel(size_t max_smem) {
    return cudaFuncSetAttribute(worker_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem);
}

cudaError_t launch_workers(Problem* probs, const WorkQueue& q, int ctas, size_t smem, cudaStream_t st) {
    worker_kernel<<<ctas, NT, smem, st>>>(probs, q);
    return cudaGetLastError();
}

}  // namespace tilt
