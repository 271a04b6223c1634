// pd_packed.cu -- the request server's packed kernel (pd_packed.cuh): one
// launch per explicit step of the quantum advances every active request by one
// step, its CTAs (a persistent grid of PACK_THREADS-thread CTAs) taking work
// items from the round's list in order. The items run the same tile bodies as
// the simulations' own kernels (pd_pmb_fast.cuh, pd_lps_fast.cuh), with the
// request's arguments copied into shared memory, so a request's arithmetic does
// not depend on what else is packed with it.
#include <algorithm>

#include "pd_lps_fast.cuh"
#include "pd_packed.cuh"
#include "pd_pmb_fast.cuh"

namespace pdk {

size_t pmb_fast_smem_split(const Geom &g, int split);
size_t lps_fast_smem(const Geom &g, bool dil);

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

// Requests with more than `round` steps in the quantum (nsteps descending).
__device__ __forceinline__ int active_count(const int *nsteps, int n, int round)
{
    int lo = 0, hi = n;                     // first index with nsteps <= round
    while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (__ldg(&nsteps[mid]) > round) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// The last request r < n with off[r] <= i (off[0] = 0 <= i < off[n]): the one
// whose items contain item i (requests without items in the group have
// off[r] == off[r + 1] and are skipped).
__device__ __forceinline__ int find_req(const int *off, int n, int i)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (__ldg(&off[mid]) <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Wait (warp 0 of the CTA, lane k polling neighbour k) until the 27 neighbour
// tiles of `tile` have finished this round's dilatation: one round trip per
// poll instead of 27 in a row. Bounded: after t.wait_ns (or once another CTA has
// reported a failure) lane 0 records the failure in t.status and the warp
// returns false. With stall, it waits for a flag value that nothing writes
// (tests).
__device__ bool wait_dil(const PackTable &t, const PackReq &q, int r, int tile, int round, bool stall)
{
    const unsigned lane = threadIdx.x & 31u;
    const unsigned want = stall ? 0xffffffffu : (unsigned)(q.step0 + round + 1);
    const int n = lane < 27u ? __ldg(&q.a[0].tile_nbr[27 * (size_t)tile + lane]) : -1;
    const long long t0 = globaltimer_ns();
    for (;;) {
        const bool ok = n < 0 || ld_acquire_u32(q.dil_done + n) >= want;
        if (__all_sync(0xffffffffu, ok)) return true;
        int fail = 0;
        if (lane == 0) {
            if (*(volatile unsigned *)t.status != PACK_OK) {
                fail = 1;
            } else if (globaltimer_ns() - t0 > t.wait_ns) {
                if (atomicCAS(t.status, (unsigned)PACK_OK, (unsigned)PACK_TIMEOUT) == (unsigned)PACK_OK) {
                    t.status[1] = (unsigned)r;
                    t.status[2] = (unsigned)tile;
                    t.status[3] = (unsigned)round;
                }
                fail = 1;
            }
        }
        if (__shfl_sync(0xffffffffu, fail, 0)) return false;
        __nanosleep(128);
    }
}

// The bodies, inlined into the kernel. (As separate functions each would get
// its own register allocation, 216 bytes of spills per thread down to at most
// 40, but the request mix measured slower that way: 2.38e11 against 2.47e11
// bond updates/s.)
static __device__ __forceinline__ void pk_lps_dil(const TileArgs &a, int tile, const float4 *tab)
{
    lps_dil_h2_body<false, true>(a, tile, tab);
}
static __device__ __forceinline__ void pk_lps_force(const TileArgs &a, int tile, const float4 *tab)
{
    lps_force_fast_body<false, true>(a, tile, tab);
}
static __device__ __forceinline__ void pk_pmb3s(const TileArgs &a, int tile) { pmb_fast_body<3, false, true, false>(a, tile, nullptr); }
static __device__ __forceinline__ void pk_pmb3(const TileArgs &a, int tile) { pmb_fast_body<3, false, false, false>(a, tile, nullptr); }
static __device__ __forceinline__ void pk_pmb2s(const TileArgs &a, int tile) { pmb_fast_body<2, false, true, false>(a, tile, nullptr); }
static __device__ __forceinline__ void pk_pmb2(const TileArgs &a, int tile) { pmb_fast_body<2, false, false, false>(a, tile, nullptr); }

__global__ void __launch_bounds__(PACK_THREADS, 2) pd_packed_round(const __grid_constant__ PackTable t, int round)
{
    __shared__ TileArgs s_a;
    __shared__ int s_item[4];               // request, tile, group, stop
    __shared__ int s_have;                  // the request whose arguments s_a holds (-1: none)
    if (threadIdx.x == 0) s_have = -1;      // published by the claim loop's first barrier
    const int A = active_count(t.nsteps, t.nreq, round);
    const int nA = __ldg(&t.offA[A]), nB = __ldg(&t.offB[A]);
    for (;;) {
        if (threadIdx.x < 32) {
            // lane 0 claims the next item; warp 0 waits for a force item's inputs.
            // (Claiming one item ahead, its atomic's round trip overlapping the
            // current item, measured slower in the request mix: 2.57e11 against
            // 2.70e11 bond updates/s. A claimed item then waits for its CTA's
            // current one instead of going to the next idle CTA, which lengthens
            // the tail of every round.)
            int r = 0, tile = 0, grp = 0, stop = 0, stall = 0;
            if (threadIdx.x == 0) {
                if (*(volatile unsigned *)t.status != PACK_OK) {
                    stop = 1;
                } else {
                    const int i = (int)atomicAdd(&t.counters[round], 1u);
                    if (i >= nA + nB) {
                        stop = 1;
                    } else if (i < nA) {
                        r = find_req(t.offA, A, i);
                        tile = i - __ldg(&t.offA[r]);
                    } else {
                        const int j = i - nA;
                        r = find_req(t.offB, A, j);
                        tile = j - __ldg(&t.offB[r]);
                        grp = 1;
                        stall = t.stall && round == 0 && j == 0;
                    }
                }
            }
            r = __shfl_sync(0xffffffffu, r, 0);
            tile = __shfl_sync(0xffffffffu, tile, 0);
            grp = __shfl_sync(0xffffffffu, grp, 0);
            stop = __shfl_sync(0xffffffffu, stop, 0);
            stall = __shfl_sync(0xffffffffu, stall, 0);
            if (!stop && grp && !wait_dil(t, t.req[r], r, tile, round, stall != 0)) stop = 1;
            if (threadIdx.x == 0) {
                s_item[0] = r;
                s_item[1] = tile;
                s_item[2] = grp;
                s_item[3] = stop;
            }
        }
        __syncthreads();
        if (s_item[3]) break;
        const int r = s_item[0], tile = s_item[1], grp = s_item[2];
        const PackReq &q = t.req[r];
        const int cur = q.cur0 ^ (round & 1);
        if (s_have != r) {
            // the request's arguments of this round (the same for all its items of
            // the launch: copied once per run of items of one request)
            const int *src = reinterpret_cast<const int *>(&q.a[cur]);
            int *dst = reinterpret_cast<int *>(&s_a);
            for (int k = threadIdx.x; k < (int)(sizeof(TileArgs) / sizeof(int)); k += blockDim.x)
                dst[k] = __ldg(&src[k]);
            __syncthreads();
            if (threadIdx.x == 0) {
                if (round == 0) {
                    s_a.v_is_half = q.vhalf0;
                    s_a.cd = q.cd0;
                }
                s_have = r;
            }
            __syncthreads();
        }
        const int kind = q.kind, split = q.split;
        if (kind == PK_LPS) {
            // the tables from the parameter bank (the host packs LPS requests of
            // m <= 3 only, whose tables it has placed there)
            if (grp == 0) pk_lps_dil(s_a, tile, t.tabs + q.tab_dil);
            else pk_lps_force(s_a, tile, t.tabs + q.tab_force);
        } else if (kind == PK_PMB3) {
            if (split == 2) pk_pmb3s(s_a, tile);
            else pk_pmb3(s_a, tile);
        } else {
            if (split == 2) pk_pmb2s(s_a, tile);
            else pk_pmb2(s_a, tile);
        }
        __syncthreads();
        if (kind == PK_LPS && grp == 0 && threadIdx.x == 0) {
            // theta of this tile is written (the barrier above): publish it
            __threadfence();
            st_release_u32(q.dil_done + tile, (unsigned)(q.step0 + round + 1));
        }
    }
}

size_t pack_smem(const Geom &g, int kind, int split)
{
    if (kind == PK_LPS) return std::max(lps_fast_smem(g, true), lps_fast_smem(g, false));
    return pmb_fast_smem_split(g, split);
}

int pack_occupancy(size_t smem, int *ctas_per_sm)
{
    // the kernel's own shared memory (the request's arguments, the bodies' tables
    // of neighbour tiles) comes out of the 227 KB a CTA may have
    cudaFuncAttributes fa;
    PD_CUDA(cudaFuncGetAttributes(&fa, pd_packed_round));
    const int dyn_max = 227 * 1024 - (int)fa.sharedSizeBytes;
    if ((long long)smem > dyn_max) {
        set_error("packed kernel: %zu bytes of shared memory requested, %d available", smem, dyn_max);
        return PD_EINVAL;
    }
    PD_CUDA(smem_limit(pd_packed_round, dyn_max));
    PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, pd_packed_round, PACK_THREADS, smem));
    return PD_OK;
}

int pack_launch_rounds(const PackTable &t, int rounds, int grid, size_t smem, cudaStream_t st)
{
    for (int s = 0; s < rounds; ++s) pd_packed_round<<<grid, PACK_THREADS, smem, st>>>(t, s);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

}  // namespace pdk
