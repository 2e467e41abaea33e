// Kernel of the RASL image-set solver (one CTA per set) and its host launcher.
#include "tilt_launch.h"
#include "tilt_rasl.cuh"

namespace tilt {

// One CTA per image set: the whole of Algorithm 1 with the set's W^T W.  TCP: the variant
// with the staged Jacobi sweeps (sets whose SVD buffers live in device memory), which need
// the bulk-copy mbarrier of the tensor-core state.
template <int NCH, bool TCP>
__global__ void __launch_bounds__(NT, 1) rasl_kernel(RaslProblem* probs) {
    extern __shared__ __align__(256) unsigned char smem_raw[];
    __shared__ RaslProblem sp;
    __shared__ RaslResult sres;
    SmemLayout L = carve_smem(smem_raw);
    if (TCP) tc_setup(&L.sc->tc, TC_TMEM_COLS);
    copy_to_shared(&sp, probs + blockIdx.x);
    solve_rasl<NCH, TCP>(sp, L, sres);
    if (threadIdx.x == 0) *sp.res = sres;
    if (TCP) tc_teardown(&L.sc->tc, TC_TMEM_COLS);
}

cudaError_t configure_rasl_kernels(size_t max_smem) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(rasl_kernel<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem)))
        return e;
    return cudaFuncSetAttribute(rasl_kernel<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem);
}

cudaError_t launch_rasl(RaslProblem* probs, int count, bool tcp, size_t smem, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    if (tcp)
        rasl_kernel<4, true><<<count, NT, smem, st>>>(probs);
    else
        rasl_kernel<4, false><<<count, NT, smem, st>>>(probs);
    return cudaGetLastError();
}

}  // namespace tilt
