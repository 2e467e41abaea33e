// The tensor-core variant of the solver kernel (launch class 2) and its host launcher.
#include "tilt_cayley.cuh"
#include "tilt_launch.h"
#include "tilt_solver.cuh"

namespace tilt {

cudaError_t configure_tc_kernels(size_t max_smem) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(solver_kernel<1, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)max_smem)))
        return e;
    return configure_worker_kernel(max_smem);
}

cudaError_t launch_solver_tc(Problem* probs, const int* order, int count, size_t smem, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    solver_kernel<1, 4, true><<<count, NT, smem, st>>>(probs, order);
    return cudaGetLastError();
}


}  // namespace tilt
