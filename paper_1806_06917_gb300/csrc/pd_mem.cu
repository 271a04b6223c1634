// pd_mem.cu -- device memory of the library: one stream-ordered pool per device
// (cudaMemPool) that keeps released memory for reuse (release threshold: never
// trim). Allocation and release are ordered on a stream instead of
// synchronising the whole device as cudaMalloc / cudaFree do, so simulations
// that come and go (the request server) do not stall the ones still running.
//
// Rules the callers follow: memory from lib_malloc(p, n, st) is used on other
// streams only after st has been synchronised, and lib_free(p, st) is issued
// only when no work on another stream still uses p.
#include <stdint.h>

#include <map>
#include <mutex>
#include <utility>

#include "pd_internal.cuh"

namespace pdk {

namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[MAX_DEVICES];
bool g_pool_ready[MAX_DEVICES];

cudaError_t device_pool(cudaMemPool_t *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool_ready[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if ((e = cudaMemPoolCreate(&g_pool[dev], &props)) != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;
        if ((e = cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess)
            return e;
        g_pool_ready[dev] = true;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}
}  // namespace

cudaError_t lib_malloc(void **p, size_t bytes, cudaStream_t st)
{
    cudaMemPool_t pool;
    cudaError_t e = device_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, st);
}

cudaError_t lib_free(void *p, cudaStream_t st) { return p ? cudaFreeAsync(p, st) : cudaSuccess; }


cudaError_t raise_smem_limit(const void *func, size_t bytes)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    size_t &cur = limit[std::make_pair(dev, func)];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

}  // namespace pdk
