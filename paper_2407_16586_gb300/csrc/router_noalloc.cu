// Allocation-free variant of the router's loss-and-gradient evaluation.
//
// Some callers cannot call cudaMalloc / cudaFree at the point where they
// need this computation: code that runs while a CUDA stream is being captured
// into a graph (allocation calls are not allowed during a global-mode
// capture), code that shares a device with a framework whose caching
// allocator owns all free memory, and latency-critical callers that cannot
// afford the device synchronisation cudaFree may cause.  This entry point
// takes only caller-owned device buffers for its inputs and outputs; its
// per-block partial sums live in the file-scope device array below.
#include <cuda_runtime.h>

#include "router.cuh"

namespace tg {
namespace {

constexpr int kNoAllocMaxSamples = 65536;
constexpr int kNoAllocMaxBlocks = kNoAllocMaxSamples / TRB;  // 512
// per-block parameter gradients [block][NPARAM], then per-block losses [block]
constexpr size_t kNoAllocFloats = (size_t)kNoAllocMaxBlocks * NPARAM + kNoAllocMaxBlocks;

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

// device address of g_noalloc_scratch, resolved once per device
constexpr int kMaxDevices = 64;
float *g_scratch_ptr[kMaxDevices] = {nullptr};
bool g_attr_set[kMaxDevices] = {false};

}  // namespace
}  // namespace tg

using namespace tg;

extern "C" int tg_router_loss_grad_noalloc(int n, const float *X, const float *y, const float *mu, const float *sd,
                                           const float *params, float q, float *loss, float *grad, void *stream)
{
    if (n < 1 || !X || !y || !mu || !sd || !params || !loss || !grad || !(q > 0.f && q < 1.f)) return TG_EINVAL;
    if (n > kNoAllocMaxSamples) return TG_EUNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return TG_ECUDA;
    }
    if (!g_scratch_ptr[dev]) {
        // first call on this device: host code needs the array's device
        // address (the symbol name is only a host-side stand-in)
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return TG_ECUDA;
        }
        g_scratch_ptr[dev] = static_cast<float *>(p);
    }
    if (!g_attr_set[dev]) {
        if (cudaFuncSetAttribute(k_mlp_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_bwd_smem()) !=
            cudaSuccess) {
            cudaGetLastError();
            return TG_ECUDA;
        }
        g_attr_set[dev] = true;
    }
    float *gpart = g_scratch_ptr[dev];
    float *lpart = gpart + (size_t)kNoAllocMaxBlocks * NPARAM;
    const int nblk = (n + TRB - 1) / TRB;
    cudaStream_t st = (cudaStream_t)stream;
    // every block overwrites its own partial slots, so nothing needs clearing
    k_mlp_fwd_bwd<<<nblk, TRB, fwd_bwd_smem(), st>>>(n, X, y, mu, sd, params, q, gpart, lpart);
    k_sum_partials<<<(NPARAM + 127) / 128, 128, 0, st>>>(nblk, NPARAM, gpart, grad);
    k_sum_partials<<<1, 32, 0, st>>>(nblk, 1, lpart, loss);
    if (cudaGetLastError() != cudaSuccess) return TG_ECUDA;
    return TG_OK;
}
