// Fixed device scratch for pfc_advect_v_static (include/vlasov.h).
//
// The velocity pass needs one scratch row of 20 doubles per cell (the shear
// factors of the cell's velocity map, written by shear_setup_kernel and read
// by the block kernel). pfc_advect_v takes it from the caller's workspace;
// pfc_advect_v_static takes it from this file-scope array instead, so that
// callers which may not allocate device memory can still run the pass: hosts
// that own every device byte through an arena fixed before the run, and
// latency-bound callers for which an allocation (its time, or its failure
// part-way through a step) is not acceptable.
//
// The array is shared by every call in the process on a given device. It
// holds no state between calls: each call writes every row it reads before
// reading it, so nothing has to start at zero. Calls that overlap in time on
// one device (different streams or host threads) race on it.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace vl {

static __device__ __align__(256) double g_vpass_scratch[(size_t)VL_STATIC_SCRATCH_CELLS * 20];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};
}  // namespace

// Device address of the scratch array on the current device. The first call
// per device resolves it with cudaGetSymbolAddress (that device current) and
// caches it; later calls only read the cache.
cudaError_t static_scratch_address(void** out) {
    *out = nullptr;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_vpass_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace vl
