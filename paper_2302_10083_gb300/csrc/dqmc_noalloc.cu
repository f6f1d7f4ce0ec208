// dqmc_noalloc.cu -- the sweep for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: an application that hands all device
// memory to its own pool, or code on a latency path where an allocation (which
// may synchronise the device) is not acceptable.  dqmc_primes_dev_static gives
// them the prime bitmap of small functions (n <= 15) with a workspace that the
// library carries in a static device array, so nothing is allocated per call.
#include <mutex>

#include "dqmc.h"
#include "dqmc_internal.h"

namespace dqmc {

// 2 MiB: the workspace of n = 15 (3^10 padded state rows, control block) is
// 1.89 MB.  Every GPU that loads the library holds this array until the
// process exits.
constexpr uint64_t kStaticScratchBytes = 2ull << 20;
constexpr uint32_t kStaticMaxN = 15;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void *g_static_ptr[64];

}  // namespace dqmc

using namespace dqmc;

// The array's device address on the current device (looked up once per device,
// with that device current, and cached for the life of the process), or a
// negative status.
static int static_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return e == cudaSuccess ? DQMC_EINVAL : DQMC_ECUDA;
    }
    // Set-up: the name of the array in host code is only a host-side
    // stand-in, not a device pointer.
    std::lock_guard<std::mutex> g(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return DQMC_ECUDA;
        }
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return DQMC_OK;
}

extern "C" int dqmc_primes_dev_static(uint32_t n, const void *d_on, const void *d_dc, void *d_bitmap,
                                      uint64_t *d_count, void *stream)
{
    if (n > kStaticMaxN) return DQMC_EINVAL;
    if (workspace_layout((int)n).total > kStaticScratchBytes) return DQMC_EINVAL;
    void *ptr = nullptr;
    const int st = static_scratch(&ptr);
    if (st != DQMC_OK) return st;
    return dqmc_primes_dev(n, d_on, d_dc, d_bitmap, d_count, ptr, kStaticScratchBytes, stream);
}

// How the last static-workspace sweep on this device ended: the error word
// sits in the static array, whose address only the library knows.
extern "C" int dqmc_dev_status_static(uint32_t n, void *stream)
{
    if (n > kStaticMaxN) return DQMC_EINVAL;
    void *ptr = nullptr;
    const int st = static_scratch(&ptr);
    if (st != DQMC_OK) return st;
    return dqmc_dev_status(n, ptr, kStaticScratchBytes, stream);
}
