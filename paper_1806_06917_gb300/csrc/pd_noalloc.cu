// pd_noalloc.cu -- pd_sum_noalloc: the fixed-order FP64 sum of pd_energy for
// callers that cannot allocate device memory.
//
// pd_energy reduces per-point values with two kernels (fixed-order block sums,
// then one block over the partials) whose partials live in a buffer the
// library allocates at pd_create. This entry point runs the same two kernels
// with the partials in a file-scope device array instead, so a call allocates
// nothing. The array holds PD_SUM_NOALLOC_PARTIALS doubles (8 KiB) on every
// device that loads the library, for the life of the process.
#include <mutex>

#include "pd_internal.cuh"

namespace pdk {
int reduce_sum(const double *x, long long n, double scale, double *partial, double *out, cudaStream_t st);
int reduce_blocks_for(long long n);
}  // namespace pdk

#define PD_SUM_NOALLOC_PARTIALS 1024

// One partial sum per block of 4096 input values. Every call writes all the
// partials it reads, so nothing has to start at zero.
static __device__ __align__(256) double g_sum_partials[PD_SUM_NOALLOC_PARTIALS];

static std::mutex g_sum_mu;
static double *g_sum_addr[256];   // device address of g_sum_partials, per device ordinal

// The address of g_sum_partials on the current device, looked up once per
// device (the name is only a host-side stand-in for the device array) and kept
// for the life of the process: it belongs to the device's context at the time
// of the lookup, so it is not valid after a cudaDeviceReset of that device.
static int partials_address(double **out)
{
    int dev = 0;
    PD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) {
        pdk::set_error("device ordinal %d out of range", dev);
        return PD_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_sum_mu);
    if (!g_sum_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_sum_partials);
        if (e != cudaSuccess) return pdk::cuda_fail(e, "cudaGetSymbolAddress(g_sum_partials)");
        g_sum_addr[dev] = static_cast<double *>(p);
    }
    *out = g_sum_addr[dev];
    return PD_OK;
}

extern "C" int pd_sum_noalloc(const double *x, int64_t n, double scale, double *out, void *stream)
{
    if (!out || (n > 0 && !x)) {
        pdk::set_error("pd_sum_noalloc: null pointer");
        return PD_EINVAL;
    }
    if (n < 0 || n > PD_SUM_NOALLOC_MAX_VALUES) {
        pdk::set_error("pd_sum_noalloc: n = %lld outside [0, %d] (its scratch holds %d partial sums of 4096 "
                       "values)", (long long)n, PD_SUM_NOALLOC_MAX_VALUES, PD_SUM_NOALLOC_PARTIALS);
        return PD_EINVAL;
    }
    static_assert(PD_SUM_NOALLOC_MAX_VALUES / 4096 <= PD_SUM_NOALLOC_PARTIALS, "scratch size");
    double *partials = nullptr;
    int rc = partials_address(&partials);
    if (rc != PD_OK) return rc;
    return pdk::reduce_sum(x, n, scale, partials, out, (cudaStream_t)stream);
}
