// Kernels of the TILT-by-LADMAP solver for sm_103a and their host launchers: the grouped
// launches of the SIMT variants (the tensor-core variant and the persistent workers are in
// tilt_kernels_tc.cu, the step kernels in tilt_steps.cu, so that the three compile in parallel).
#include "tilt_cayley.cuh"
#include "tilt_launch.h"
#include "tilt_solver.cuh"

namespace tilt {

cudaError_t configure_kernels(size_t max_smem) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(solver_kernel<1, 4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)max_smem)))
        return e;
    if ((e = cudaFuncSetAttribute(solver_kernel<2, 3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)max_smem)))
        return e;
    if ((e = configure_tc_kernels(max_smem))) return e;
    return configure_step_kernels(max_smem);
}

cudaError_t launch_solver(Problem* probs, const int* order, int count, int minb, bool tcp, size_t smem,
                          cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    if (tcp && minb < 2) return launch_solver_tc(probs, order, count, smem, st);
    if (minb >= 2)
        solver_kernel<2, 3, false><<<count, NT, smem, st>>>(probs, order);
    else
        solver_kernel<1, 4, false><<<count, NT, smem, st>>>(probs, order);
    return cudaGetLastError();
}

}  // namespace tilt
