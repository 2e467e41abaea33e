// Allocation-free singular value thresholding (tilt_svt_noalloc in include/tilt.h).
//
// For callers that may not allocate device memory: the scratch of the SVT step lives in one
// file-scope device array instead of the context pool.  Every call shares it.
#include <mutex>

#include "../../include/tilt.h"
#include "tilt_launch.h"

using namespace tilt;

namespace {

constexpr int NOALLOC_MAX_SIDE = 256;
constexpr size_t SQ = (size_t)NOALLOC_MAX_SIDE * NOALLOC_MAX_SIDE;   // one 256 x 256 buffer
constexpr size_t OFF_B = 0;                                          // B: ldb * Cp  (global mode)
constexpr size_t OFF_V = OFF_B + SQ;                                 // V: ldv * Cp  (global mode)
constexpr size_t OFF_Z = OFF_V + SQ;                                 // Z: C * Cp
constexpr size_t OFF_SIG = OFF_Z + SQ;                               // sigma: C
constexpr size_t OFF_OUT = OFF_SIG + 2 * NOALLOC_MAX_SIDE;           // StepOut record
constexpr size_t SCRATCH_FLOATS = OFF_OUT + (sizeof(StepOut) + 255) / 4;

// The scratch.  In host code this name is only a stand-in for the symbol: kernels get the
// device address obtained from cudaGetSymbolAddress.
static __device__ __align__(256) float g_svt_scratch[SCRATCH_FLOATS];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
float* g_scratch_ptr[MAX_DEVICES] = {};
size_t g_max_smem[MAX_DEVICES] = {};

// Once per device, with that device current: the scratch's device address and the
// shared-memory opt-in of the kernels.
int setup(int dev) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_ptr[dev]) return TILT_OK;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_svt_scratch);
    if (e != cudaSuccess) return set_error(TILT_E_CUDA, cudaGetErrorString(e));
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return set_error(TILT_E_CUDA, cudaGetErrorString(e));
    const size_t max_smem = (size_t)optin - 2048;
    e = configure_kernels(max_smem);
    if (e != cudaSuccess) return set_error(TILT_E_CUDA, cudaGetErrorString(e));
    g_max_smem[dev] = max_smem;
    g_scratch_ptr[dev] = static_cast<float*>(p);
    return TILT_OK;
}

}  // namespace

extern "C" int tilt_svt_noalloc(const float* M_dev, int m, int n, float eps, float* A_dev, float* sigma_dev,
                                void* stream) {
    if (!M_dev || !A_dev) return set_error(TILT_E_INVAL, "null M or A");
    if (m < 1 || n < 1 || m > NOALLOC_MAX_SIDE || n > NOALLOC_MAX_SIDE)
        return set_error(TILT_E_INVAL, "tilt_svt_noalloc: m and n must lie in 1..256");
    if (!(eps >= 0.f)) return set_error(TILT_E_INVAL, "eps must be >= 0");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(TILT_E_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return set_error(TILT_E_INVAL, "device ordinal out of range");
    int rc = setup(dev);
    if (rc) return rc;
    float* s = g_scratch_ptr[dev];
    const Dims d = make_dims(m, n, 0);
    const size_t svd = svd_smem_bytes(d), head = smem_head_bytes() + (use_tc_products(d) ? tc_stage_for(d, 1) : 0);
    SvtArgs a{};
    a.M = M_dev;
    a.A = A_dev;
    a.m = m;
    a.n = n;
    a.eps = eps;
    a.smem_svd = (svd + head <= g_max_smem[dev]) ? 1 : 0;
    a.jsched = default_group_width(d.R, d.C);
    a.Bg = s + OFF_B;
    a.Vg = s + OFF_V;
    a.Tg = nullptr;   // the SVT step keeps M in place of T
    a.Zg = s + OFF_Z;
    a.sigma = sigma_dev ? sigma_dev : s + OFF_SIG;
    a.out = reinterpret_cast<StepOut*>(s + OFF_OUT);
    e = launch_svt_step(a, a.smem_svd ? svd + head : head, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return set_error(TILT_E_CUDA, cudaGetErrorString(e));
    return TILT_OK;
}
