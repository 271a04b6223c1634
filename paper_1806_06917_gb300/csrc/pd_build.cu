// pd_build.cu -- neighbour build and the per-simulation tables (done once, in the
// reference configuration, Sec. 4.2.1).
//
//   1. slots: tile-major Morton layout, user <-> slot maps, Morton ranks (scan);
//   2. cell list with cell edge m h >= delta: counting sort of the points by cell;
//   3. CSR: every point tests the points of the 3^d cells around it with the
//      integer predicate a^2 + b^2 + c^2 <= m^2 (Sec. 3.1, points at exactly
//      delta included). A CTA per cell stages the candidates of its 3^d cells
//      in shared memory once, sorts them by Morton rank (bitonic), and a warp
//      per row of the cell scans them in that order, so each row comes out
//      ascending; the same scan sets the row's stencil bits (the bond-intact
//      mask);
//   4. LPS weighted volume m~_i = sum_j |d|^2 V_ij (Algorithm 2, first loop, in
//      lattice units) and the stable-step sum of every point, both summed over
//      the point's mask bits in stencil order.
// Atomics are used only for counts and for the order of points inside a cell;
// the sorted CSR, the mask and every table are independent of that order.
#include "pd_tile.cuh"

namespace pdk {

// ------------------------------------------------------------------ scan

constexpr int SCAN_CHUNK = 1024;

__global__ void k_scan_sums(const int *in, long long n, long long *bsum)
{
    __shared__ long long sh[256];
    const long long lo = (long long)blockIdx.x * SCAN_CHUNK;
    long long acc = 0;
    for (int k = threadIdx.x; k < SCAN_CHUNK; k += blockDim.x)
        if (lo + k < n) acc += in[lo + k];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = sh[0];
}

// Exclusive scan of the block sums in place (one block, sequential carry).
__global__ void k_scan_offsets(long long *bsum, int nb, long long *total)
{
    __shared__ long long sh[256];
    long long carry = 0;
    for (int base = 0; base < nb; base += 256) {
        const int i = base + threadIdx.x;
        const long long v = i < nb ? bsum[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 256; off <<= 1) {
            long long t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) bsum[i] = carry + sh[threadIdx.x] - v;
        const long long tot = sh[255];
        __syncthreads();
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_apply(const int *in, long long n, const long long *boff, long long *out)
{
    __shared__ long long sh[256];
    const long long lo = (long long)blockIdx.x * SCAN_CHUNK;
    constexpr int PER = SCAN_CHUNK / 256;
    long long v[PER];
    long long acc = 0;
    for (int k = 0; k < PER; ++k) {
        const long long i = lo + threadIdx.x * PER + k;
        v[k] = i < n ? in[i] : 0;
        acc += v[k];
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
        long long t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    long long run = boff[blockIdx.x] + sh[threadIdx.x] - acc;
    for (int k = 0; k < PER; ++k) {
        const long long i = lo + threadIdx.x * PER + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
}

// out[0..n] = exclusive prefix sums of in[0..n), out[n] = total.
static int exclusive_scan(const int *in, long long n, long long *out, cudaStream_t st)
{
    const int nb = (int)((n + SCAN_CHUNK - 1) / SCAN_CHUNK);
    long long *bsum = nullptr;
    PD_CUDA(lib_malloc(reinterpret_cast<void **>(&bsum), sizeof(long long) * (nb > 0 ? nb : 1), st));
    if (nb > 0) {
        k_scan_sums<<<nb, 256, 0, st>>>(in, n, bsum);
        k_scan_offsets<<<1, 256, 0, st>>>(bsum, nb, out + n);
        k_scan_apply<<<nb, 256, 0, st>>>(in, n, bsum, out);
    } else {
        PD_CUDA(cudaMemsetAsync(out, 0, sizeof(long long), st));
    }
    cudaError_t e = cudaGetLastError();
    cudaStreamSynchronize(st);
    lib_free(bsum, st);
    if (e != cudaSuccess) return cuda_fail(e, "exclusive_scan");
    return PD_OK;
}

// ----------------------------------------------------------------- slots

__device__ __forceinline__ void slot_coord(const Geom &g, const int4 *tile_org, int s, int c[3])
{
    const int tile = s >> g.L;
    const int4 o = tile_org[tile];
    int l[3];
    morton_decode(g.dim, (uint64_t)(s & (g.T - 1)), l);
    c[0] = o.x + l[0];
    c[1] = o.y + l[1];
    c[2] = o.z + l[2];
}

__global__ void k_slots(Geom g, const int4 *tile_org, int *user_of_slot, int *slot_of_user, int *active)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.nslots) return;
    int c[3];
    slot_coord(g, tile_org, (int)s, c);
    const bool in = c[0] < g.nx && c[1] < g.ny && c[2] < g.nz;
    if (in) {
        const int u = c[0] + g.nx * (c[1] + g.ny * c[2]);
        user_of_slot[s] = u;
        slot_of_user[u] = (int)s;
    } else {
        user_of_slot[s] = -1;
    }
    active[s] = in ? 1 : 0;
}

__global__ void k_ranks(Geom g, const int *active, const long long *scan, int *rank_of_slot, int *slot_of_rank)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.nslots) return;
    if (active[s]) {
        const int r = (int)scan[s];
        rank_of_slot[s] = r;
        slot_of_rank[r] = (int)s;
    } else {
        rank_of_slot[s] = -1;
    }
}

int build_slots(const Geom &g, const Tables &t, int *user_of_slot, int *slot_of_user, int *rank_of_slot,
                int *slot_of_rank, cudaStream_t st)
{
    int *active = nullptr;
    long long *scan = nullptr;
    PD_CUDA(lib_malloc(reinterpret_cast<void **>(&active), sizeof(int) * (size_t)g.nslots, st));
    PD_CUDA(lib_malloc(reinterpret_cast<void **>(&scan), sizeof(long long) * ((size_t)g.nslots + 1), st));
    const int nb = (g.nslots + 255) / 256;
    k_slots<<<nb, 256, 0, st>>>(g, t.tile_org, user_of_slot, slot_of_user, active);
    int rc = exclusive_scan(active, g.nslots, scan, st);
    if (rc == PD_OK) {
        k_ranks<<<nb, 256, 0, st>>>(g, active, scan, rank_of_slot, slot_of_rank);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "build_slots");
    }
    lib_free(active, st);
    lib_free(scan, st);
    return rc;
}

// ------------------------------------------------------------- cell list

struct CellGrid {
    int m, cx, cy, cz;
};

__global__ void k_rank_coords(Geom g, const int4 *tile_org, const int *slot_of_rank, int4 *crd)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= g.npoints) return;
    int c[3];
    slot_coord(g, tile_org, slot_of_rank[r], c);
    crd[r] = make_int4(c[0], c[1], c[2], 0);
}

__device__ __forceinline__ int cell_of(const CellGrid &cg, int4 c)
{
    return c.x / cg.m + cg.cx * (c.y / cg.m + cg.cy * (c.z / cg.m));
}

__global__ void k_cell_count(Geom g, CellGrid cg, const int4 *crd, int *cell_count)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= g.npoints) return;
    atomicAdd(&cell_count[cell_of(cg, crd[r])], 1);
}

__global__ void k_cell_fill(Geom g, CellGrid cg, const int4 *crd, const long long *cell_start, int *cursor,
                            int *cell_pts)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= g.npoints) return;
    const int cell = cell_of(cg, crd[r]);
    const int pos = atomicAdd(&cursor[cell], 1);
    cell_pts[cell_start[cell] + pos] = (int)r;
}

// Candidates of a cell: the points of the 3^d cells around it, as (Morton rank,
// lattice coordinates relative to the cell's origin packed in 3 x 8 bits; they
// lie in [-m, 2m) with m <= 24).
constexpr int CELL_THREADS = 256;
constexpr int CELL_WARPS = CELL_THREADS / 32;
constexpr int REL_BIAS = 64;

__device__ __forceinline__ int pack_rel(int x, int y, int z)
{
    return (x + REL_BIAS) | ((y + REL_BIAS) << 8) | ((z + REL_BIAS) << 16);
}

// Largest candidate count: a cell of edge m holds at most m^d lattice points.
static long long cell_capacity(const Geom &g)
{
    long long c = 1;
    for (int d = 0; d < g.dim; ++d) c *= 3LL * g.m;
    long long n = 1;
    while (n < c) n <<= 1;
    return n;
}

static size_t cell_rows_smem(const Geom &g)
{
    return (size_t)cell_capacity(g) * 2 * sizeof(int) + (size_t)CELL_WARPS * g.W * sizeof(uint32_t);
}

// FILL = false: row_count[i] for the rows of the cell (no sort needed).
// FILL = true: col[row_ptr[i] ..] ascending, and the mask words of i's slot.
// err: 1 = a row differs from its counted length, 3 = a cell above capacity.
template <bool FILL>
__global__ void __launch_bounds__(CELL_THREADS) k_cell_rows(Geom g, CellGrid cg, int ncap, const int4 *crd,
                                                            const long long *cell_start, const int *cell_pts,
                                                            const int *slot_of_rank, const int *stencil_lut,
                                                            int *row_count, const int64_t *row_ptr, int *col,
                                                            uint32_t *mask, int *err)
{
    extern __shared__ int csm[];
    int *key = csm;
    int *val = csm + ncap;
    uint32_t *words = reinterpret_cast<uint32_t *>(csm + 2 * ncap);
    __shared__ long long s_start[27];
    __shared__ int s_off[28];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int cell = blockIdx.x;
    const int ca = cell % cg.cx, cb = (cell / cg.cx) % cg.cy, ce = cell / (cg.cx * cg.cy);
    const int nc = g.dim == 3 ? 27 : 9, centre = g.dim == 3 ? 13 : 4;
    if (warp == 0) {
        int cnt = 0;
        long long st0 = 0;
        if (lane < nc) {
            const int A = ca + lane % 3 - 1, B = cb + (lane / 3) % 3 - 1, E = ce + (g.dim == 3 ? lane / 9 - 1 : 0);
            if (A >= 0 && B >= 0 && E >= 0 && A < cg.cx && B < cg.cy && E < cg.cz) {
                const int c2 = A + cg.cx * (B + cg.cy * E);
                st0 = cell_start[c2];
                cnt = (int)(cell_start[c2 + 1] - st0);
            }
        }
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane < nc) {
            s_start[lane] = st0;
            s_off[lane + 1] = incl;
        }
        if (lane == 0) s_off[0] = 0;
    }
    __syncthreads();
    const int total = s_off[nc];
    if (total > ncap) {
        if (threadIdx.x == 0) atomicExch(err, 3);
        return;
    }
    int N = 1;
    while (N < total) N <<= 1;
    const int ox = ca * cg.m, oy = cb * cg.m, oz = ce * cg.m;
    for (int q = threadIdx.x; q < N; q += blockDim.x) {
        if (q < total) {
            int c = 0;
            while (s_off[c + 1] <= q) ++c;
            const int j = cell_pts[s_start[c] + (q - s_off[c])];
            const int4 cj = crd[j];
            key[q] = j;
            val[q] = pack_rel(cj.x - ox, cj.y - oy, cj.z - oz);
        } else {
            key[q] = 0x7fffffff;
            val[q] = 0;
        }
    }
    __syncthreads();
    if (FILL) {
        // bitonic sort of (key, val) by key; keys are distinct ranks, pads last
        for (int k = 2; k <= N; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int t = threadIdx.x; t < N / 2; t += blockDim.x) {
                    const int i = 2 * t - (t & (j - 1));
                    const int ixj = i + j;
                    const int ki = key[i], kj = key[ixj];
                    if ((ki > kj) == ((i & k) == 0)) {
                        key[i] = kj;
                        key[ixj] = ki;
                        const int v = val[i];
                        val[i] = val[ixj];
                        val[ixj] = v;
                    }
                }
                __syncthreads();
            }
    }
    const int n0 = s_off[centre + 1] - s_off[centre];
    const int mm = g.m * g.m, wdt = 2 * g.m + 1;
    uint32_t *ww = words + warp * g.W;
    for (int p = warp; p < n0; p += CELL_WARPS) {
        const int i = cell_pts[s_start[centre] + p];
        const int4 ci = crd[i];
        const int rx = ci.x - ox, ry = ci.y - oy, rz = ci.z - oz;
        long long base = 0;
        int want = 0;
        if (FILL) {
            base = row_ptr[i];
            want = (int)(row_ptr[i + 1] - base);
            for (int w = lane; w < g.W; w += 32) ww[w] = 0u;
            __syncwarp();
        }
        int cnt = 0;
        for (int q0 = 0; q0 < total; q0 += 32) {
            const int q = q0 + lane;
            bool hit = false;
            int j = 0, dx = 0, dy = 0, dz = 0;
            if (q < total) {
                j = key[q];
                const int v = val[q];
                dx = (v & 0xff) - REL_BIAS - rx;
                dy = ((v >> 8) & 0xff) - REL_BIAS - ry;
                dz = ((v >> 16) & 0xff) - REL_BIAS - rz;
                hit = j != i && dx * dx + dy * dy + dz * dz <= mm;
            }
            const unsigned ball = __ballot_sync(0xffffffffu, hit);
            if (FILL && hit) {
                const int pos = cnt + __popc(ball & ((1u << lane) - 1u));
                if (pos < want) col[base + pos] = j;        // never false unless the count pass disagreed
                const int k = stencil_lut[(dx + g.m) + wdt * ((dy + g.m) + wdt * (g.dim == 3 ? dz + g.m : 0))];
                atomicOr(&ww[k >> 5], 1u << (k & 31));
            }
            cnt += __popc(ball);
        }
        if (!FILL) {
            if (lane == 0) row_count[i] = cnt;
        } else {
            if (lane == 0 && cnt != want) atomicExch(err, 1);
            __syncwarp();
            const int sl = slot_of_rank[i];
            for (int w = lane; w < g.W; w += 32) mask[(size_t)w * g.nslots + sl] = ww[w];
            __syncwarp();
        }
    }
}

constexpr int MAX_WORDS = 64;

int build_csr(const Geom &g, const Tables &t, BuildOut *out, uint32_t *mask, cudaStream_t st)
{
    if (g.W > MAX_WORDS) {
        set_error("stencil of %d offsets exceeds %d mask words", g.S, MAX_WORDS);
        return PD_EINVAL;
    }
    CellGrid cg;
    cg.m = g.m;
    cg.cx = (g.nx + g.m - 1) / g.m;
    cg.cy = (g.ny + g.m - 1) / g.m;
    cg.cz = (g.nz + g.m - 1) / g.m;
    const long long ncell = (long long)cg.cx * cg.cy * cg.cz;
    const long long n = g.npoints;
    const int ncap = (int)cell_capacity(g);
    const size_t smem = cell_rows_smem(g);
    int4 *crd = nullptr;
    int *cell_count = nullptr, *cursor = nullptr, *cell_pts = nullptr, *row_count = nullptr, *err = nullptr;
    long long *cell_start = nullptr;
    int rc = PD_OK;
    out->row_ptr = nullptr;
    out->col = nullptr;
    out->nbonds = 0;
    if (smem > 227 * 1024) {
        set_error("neighbour build needs %zu bytes of shared memory per cell (m too large)", smem);
        return PD_EINVAL;
    }
#define B_ALLOC(p, bytes)                                              \
    do {                                                               \
        if (lib_malloc(reinterpret_cast<void **>(&(p)), (bytes), st) != cudaSuccess) { \
            rc = PD_ENOMEM;                                            \
            set_error("device allocation of %lld bytes failed", (long long)(bytes)); \
            goto done;                                                 \
        }                                                              \
    } while (0)
    B_ALLOC(crd, sizeof(int4) * n);
    B_ALLOC(cell_count, sizeof(int) * ncell);
    B_ALLOC(cursor, sizeof(int) * ncell);
    B_ALLOC(cell_start, sizeof(long long) * (ncell + 1));
    B_ALLOC(cell_pts, sizeof(int) * n);
    B_ALLOC(row_count, sizeof(int) * n);
    B_ALLOC(err, sizeof(int));
    B_ALLOC(out->row_ptr, sizeof(long long) * (n + 1));
    {
        const int nb = (int)((n + 255) / 256);
        cudaMemsetAsync(cell_count, 0, sizeof(int) * ncell, st);
        cudaMemsetAsync(cursor, 0, sizeof(int) * ncell, st);
        cudaMemsetAsync(err, 0, sizeof(int), st);
        cudaMemsetAsync(mask, 0, sizeof(uint32_t) * (size_t)g.W * g.nslots, st);
        PD_CUDA(smem_limit(k_cell_rows<false>, smem));
        PD_CUDA(smem_limit(k_cell_rows<true>, smem));
        k_rank_coords<<<nb, 256, 0, st>>>(g, t.tile_org, t.slot_of_rank, crd);
        k_cell_count<<<nb, 256, 0, st>>>(g, cg, crd, cell_count);
        rc = exclusive_scan(cell_count, ncell, cell_start, st);
        if (rc != PD_OK) goto done;
        k_cell_fill<<<nb, 256, 0, st>>>(g, cg, crd, cell_start, cursor, cell_pts);
        k_cell_rows<false><<<(unsigned)ncell, CELL_THREADS, smem, st>>>(
            g, cg, ncap, crd, cell_start, cell_pts, t.slot_of_rank, t.stencil_lut, row_count, nullptr, nullptr,
            nullptr, err);
        rc = exclusive_scan(row_count, n, (long long *)out->row_ptr, st);
        if (rc != PD_OK) goto done;
        long long nbonds = 0;
        if (cudaMemcpy(&nbonds, out->row_ptr + n, sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "row_ptr readback");
            goto done;
        }
        out->nbonds = nbonds;
        B_ALLOC(out->col, sizeof(int) * (nbonds > 0 ? nbonds : 1));
        k_cell_rows<true><<<(unsigned)ncell, CELL_THREADS, smem, st>>>(
            g, cg, ncap, crd, cell_start, cell_pts, t.slot_of_rank, t.stencil_lut, nullptr, out->row_ptr,
            out->col, mask, err);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "neighbour rows");
            goto done;
        }
        int herr = 0;
        cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
        if (herr) {
            rc = PD_EINVAL;
            set_error(herr == 3 ? "a cell holds more points than the lattice allows"
                                : "a neighbour row differs from its counted length");
        }
    }
done:
#undef B_ALLOC
    cudaStreamSynchronize(st);
    lib_free(crd, st);
    lib_free(cell_count, st);
    lib_free(cursor, st);
    lib_free(cell_start, st);
    lib_free(cell_pts, st);
    lib_free(row_count, st);
    lib_free(err, st);
    if (rc != PD_OK) {
        lib_free(out->row_ptr, st);
        lib_free(out->col, st);
        out->row_ptr = nullptr;
        out->col = nullptr;
    }
    return rc;
}

// --------------------------------------------------------- stencil mask

__device__ __forceinline__ int stencil_index(const Geom &g, const int *lut, int dx, int dy, int dz)
{
    const int w = 2 * g.m + 1;
    if (dx < -g.m || dx > g.m || dy < -g.m || dy > g.m || dz < -g.m || dz > g.m) return -1;
    return lut[(dx + g.m) + w * ((dy + g.m) + w * (g.dim == 3 ? dz + g.m : 0))];
}

// --------------------------------------------- weighted volume, step bound

// Per-point sums over the intact stencil bits, in stencil order, of a per-entry
// FP64 value built in shared memory from |d|: which = 0 gives the LPS weighted
// volume sum_j |d|^2 V_ij, which = 1 the stable-step sum sum_j V_ij / |d|.
__global__ void __launch_bounds__(256) k_stencil_sum(Geom g, int vol_corr, int which, const int *slot_of_rank,
                                                     const int4 *stencil, const double *stencil_r0,
                                                     const uint32_t *mask, double *mtil, float *minv32,
                                                     unsigned long long *smax)
{
    extern __shared__ double tabk[];
    for (int k = threadIdx.x; k < g.S; k += blockDim.x) {
        const double r0 = stencil_r0[k];
        const double v = vol_corr ? vol_factor_lattice(g.m, r0) : 1.0;
        tabk[k] = which == 0 ? (double)stencil[k].w * v : v / r0;     // .w = |d|^2, exact
    }
    __syncthreads();
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= g.npoints) return;
    const int s = slot_of_rank[r];
    double acc = 0.0;
    for (int w = 0; w < g.W; ++w) {
        uint32_t word = mask[(size_t)w * g.nslots + s];
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1u;
            acc += tabk[32 * w + b];
        }
    }
    if (which == 0) {
        mtil[s] = acc;
        minv32[s] = acc > 0.0 ? (float)(1.0 / acc) : 0.f;
    } else {
        // positive doubles order like their bit patterns
        atomicMax(smax, (unsigned long long)__double_as_longlong(acc));
    }
}

int build_weighted_volume(const Geom &g, const Material &mat, const Tables &t, const uint32_t *mask, double *mtil,
                          float *minv32, cudaStream_t st)
{
    k_stencil_sum<<<(g.npoints + 255) / 256, 256, sizeof(double) * g.S, st>>>(
        g, mat.vol_corr, 0, t.slot_of_rank, t.stencil, t.stencil_r0, mask, mtil, minv32, nullptr);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

// max_i sum_j V_ij / |d| (lattice units) over the intact bonds of the mask.
int build_dt_bound(const Geom &g, const Material &mat, const Tables &t, const uint32_t *mask, double *d_sum_max,
                   cudaStream_t st)
{
    PD_CUDA(cudaMemsetAsync(d_sum_max, 0, sizeof(double), st));
    k_stencil_sum<<<(g.npoints + 255) / 256, 256, sizeof(double) * g.S, st>>>(
        g, mat.vol_corr, 1, t.slot_of_rank, t.stencil, t.stencil_r0, mask, nullptr, nullptr,
        reinterpret_cast<unsigned long long *>(d_sum_max));
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

// ------------------------------------------------------- CSR bond state

__global__ void k_csr_broken(Geom g, const int4 *tile_org, const int *slot_of_rank, const int *stencil_lut,
                             const int64_t *row_ptr, const int *col, const uint32_t *mask, uint8_t *out)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= g.npoints) return;
    const int s = slot_of_rank[r];
    int c[3];
    slot_coord(g, tile_org, s, c);
    for (long long e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
        int cj[3];
        slot_coord(g, tile_org, slot_of_rank[col[e]], cj);
        const int k = stencil_index(g, stencil_lut, cj[0] - c[0], cj[1] - c[1], cj[2] - c[2]);
        if (k < 0) {
            out[e] = 1;
            continue;
        }
        const uint32_t word = mask[(size_t)(k >> 5) * g.nslots + s];
        out[e] = ((word >> (k & 31)) & 1u) ? 0 : 1;
    }
}

int csr_broken_flags(const Geom &g, const Tables &t, const BuildOut &csr, const uint32_t *mask, uint8_t *out,
                     cudaStream_t st)
{
    k_csr_broken<<<(g.npoints + 255) / 256, 256, 0, st>>>(g, t.tile_org, t.slot_of_rank, t.stencil_lut,
                                                          csr.row_ptr, csr.col, mask, out);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

// -------------------------------------------------------------- pre-notch

struct NotchDesc {
    int axis;
    double pos;
    double lo[3], hi[3];
};

// Segment X_i -> X_j crosses {x[axis] = pos} inside the rectangle. With
// D = c_j[axis] - c_i[axis], the crossing point satisfies
// P_b D = c_i[b] D + (pos - c_i[axis]) (c_j[b] - c_i[b]), exact in FP64 for
// lattice coordinates and a half-integer pos; compare against lo D and hi D.
__device__ __forceinline__ bool crosses(const NotchDesc &nd, int dim, const int ci[3], const int cj[3])
{
    const double si = __dadd_rn((double)ci[nd.axis], -nd.pos);
    const double sj = __dadd_rn((double)cj[nd.axis], -nd.pos);
    if (!((si < 0.0 && sj > 0.0) || (si > 0.0 && sj < 0.0))) return false;
    const int D = cj[nd.axis] - ci[nd.axis];
    const double ad = (double)(D < 0 ? -D : D);
    const double sgn = D < 0 ? -1.0 : 1.0;
    for (int b = 0; b < dim; ++b) {
        if (b == nd.axis) continue;
        const double pd = __dadd_rn(__dmul_rn((double)ci[b], (double)D),
                                    __dmul_rn(__dadd_rn(nd.pos, -(double)ci[nd.axis]), (double)(cj[b] - ci[b])));
        const double v = __dmul_rn(sgn, pd);
        if (v < __dmul_rn(nd.lo[b], ad) || v > __dmul_rn(nd.hi[b], ad)) return false;
    }
    return true;
}

__global__ void k_notch(Geom g, const int4 *tile_org, const int *user_of_slot, const int4 *stencil, NotchDesc nd,
                        uint32_t *mask, unsigned long long *count)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.nslots || user_of_slot[s] < 0) return;
    int c[3];
    slot_coord(g, tile_org, (int)s, c);
    // a bond spans at most m lattice units along the notch axis: points farther
    // than that from the plane have no crossing bond
    const double sd = __dadd_rn((double)c[nd.axis], -nd.pos);
    if (sd > (double)g.m || sd < -(double)g.m) return;
    unsigned long long local = 0;
    for (int w = 0; w < g.W; ++w) {
        uint32_t word = mask[(size_t)w * g.nslots + s];
        const uint32_t orig = word;
        const int nb = min(32, g.S - 32 * w);
        for (int b = 0; b < nb; ++b) {
            if (!((word >> b) & 1u)) continue;
            const int4 d = stencil[32 * w + b];
            const int cj[3] = {c[0] + d.x, c[1] + d.y, c[2] + d.z};
            if (crosses(nd, g.dim, c, cj)) {
                word &= ~(1u << b);
                ++local;
            }
        }
        if (word != orig) mask[(size_t)w * g.nslots + s] = word;
    }
    if (local) atomicAdd(count, local);
}

int break_notch(const Geom &g, const Tables &t, uint32_t *mask, int axis, double pos, const double lo[3],
                const double hi[3], unsigned long long *d_count, cudaStream_t st)
{
    NotchDesc nd;
    nd.axis = axis;
    nd.pos = pos;
    for (int b = 0; b < 3; ++b) {
        nd.lo[b] = lo[b];
        nd.hi[b] = hi[b];
    }
    PD_CUDA(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), st));
    k_notch<<<(g.nslots + 255) / 256, 256, 0, st>>>(g, t.tile_org, t.user_of_slot, t.stencil, nd, mask, d_count);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

// ---------------------------------------------------------- permutations

__global__ void k_scatter(Geom g, const int *slot_of_user, const double *user, double *s0, double *s1, double *s2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.npoints) return;
    const int s = slot_of_user[i];
    double *dst[3] = {s0, s1, s2};
    for (int c = 0; c < g.dim; ++c) dst[c][s] = user[i * g.dim + c];
}

// User order (n x dim FP64, AoS) to the slot of each point in one pass: the
// FP64 SoA arrays if given, and the staging form if given (FP32C double-float
// pair hi = fl(x), lo = fl(x - hi); FP64 double4). One thread per slot, so the
// slot-order writes are coalesced and the user array is read in runs of
// x-consecutive points (a Morton-ordered warp covers 4 x 4 x 2 points); slots
// off the lattice get zeros.
// The FP32 staging pair of an FP64 value: round-to-nearest high word (the
// double-float state's own representation) or, with bits, split_bits (the
// split the fused update writes for FP64 state, so that a staging pair made
// here equals the one a step would make from the same u).
__device__ __forceinline__ void split_pair(double x, bool bits, float &h, float &l)
{
    if (bits) {
        split_bits(x, h, l);
    } else {
        h = (float)x;
        l = (float)(x - (double)h);
    }
}

__device__ __forceinline__ void stage_slot(long long s, int d, double x, double y, double z, double *s0, double *s1,
                                           double *s2, float4 *hl, double4_32a *d4, bool bits)
{
    if (s0) {
        s0[s] = x;
        s1[s] = y;
        if (d == 3) s2[s] = z;
    }
    if (d4) d4[s] = make_double4_32a(x, y, z, 0.0);
    if (hl) {
        float hx, hy, hz, lx, ly, lz;
        split_pair(x, bits, hx, lx);
        split_pair(y, bits, hy, ly);
        split_pair(z, bits, hz, lz);
        hl[2 * s] = make_float4(hx, hy, hz, 0.f);
        hl[2 * s + 1] = make_float4(lx, ly, lz, 0.f);
    }
}

__global__ void k_scatter_stage(Geom g, const int *user_of_slot, const double *user, double *s0, double *s1,
                                double *s2, float4 *hl, double4_32a *d4, bool bits)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.nslots) return;
    const long long i = user_of_slot[s];
    const int d = g.dim;
    double x = 0.0, y = 0.0, z = 0.0;
    if (i >= 0) {
        x = user[i * d];
        y = user[i * d + 1];
        if (d == 3) z = user[i * d + 2];
    }
    stage_slot(s, d, x, y, z, s0, s1, s2, hl, d4, bits);
}

// The same for the user rows [r0, r1) alone, one thread per row (for a chunk of
// an upload that is still arriving). Slots off the lattice are not written: they
// hold zeros from the allocation on, as no kernel writes a slot off the lattice.
__global__ void k_scatter_rows(Geom g, const int *slot_of_user, const double *user, long long r0, long long r1,
                               double *s0, double *s1, double *s2, float4 *hl, double4_32a *d4, bool bits)
{
    const long long i = r0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= r1) return;
    const long long s = slot_of_user[i];
    const int d = g.dim;
    stage_slot(s, d, user[i * d], user[i * d + 1], d == 3 ? user[i * d + 2] : 0.0, s0, s1, s2, hl, d4, bits);
}

// The reverse: user order from the double-float pair (hl) or the FP64 SoA arrays.
__global__ void k_gather_unstage(Geom g, const int *slot_of_user, const float4 *hl, const double *s0,
                                 const double *s1, const double *s2, double *user, long long r0, long long r1)
{
    const long long i = r0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= r1) return;
    const int s = slot_of_user[i];
    const int d = g.dim;
    double x, y, z;
    if (hl) {
        const float4 hi = hl[2 * s], lo = hl[2 * s + 1];
        x = (double)hi.x + (double)lo.x;
        y = (double)hi.y + (double)lo.y;
        z = (double)hi.z + (double)lo.z;
    } else {
        x = s0[s];
        y = s1[s];
        z = d == 3 ? s2[s] : 0.0;
    }
    user[i * d] = x;
    user[i * d + 1] = y;
    if (d == 3) user[i * d + 2] = z;
}

int scatter_stage(const Geom &g, const int *user_of_slot, const double *user, double *const slot[3], float4 *hl,
                  double4_32a *d4, cudaStream_t st, bool bits)
{
    k_scatter_stage<<<(g.nslots + 255) / 256, 256, 0, st>>>(g, user_of_slot, user, slot ? slot[0] : nullptr,
                                                             slot ? slot[1] : nullptr, slot ? slot[2] : nullptr,
                                                             hl, d4, bits);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

int gather_unstage(const Geom &g, const int *slot_of_user, const float4 *hl, double *const slot[3], double *user,
                   cudaStream_t st)
{
    return gather_rows(g, slot_of_user, hl, slot, user, 0, g.npoints, st);
}

int gather_rows(const Geom &g, const int *slot_of_user, const float4 *hl, double *const slot[3], double *user,
                long long r0, long long r1, cudaStream_t st)
{
    if (r1 <= r0) return PD_OK;
    k_gather_unstage<<<(unsigned)((r1 - r0 + 255) / 256), 256, 0, st>>>(
        g, slot_of_user, hl, slot ? slot[0] : nullptr, slot ? slot[1] : nullptr, slot ? slot[2] : nullptr, user, r0,
        r1);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

int scatter_rows(const Geom &g, const int *slot_of_user, const double *user, long long r0, long long r1,
                 double *const slot[3], float4 *hl, double4_32a *d4, cudaStream_t st, bool bits)
{
    if (r1 <= r0) return PD_OK;
    k_scatter_rows<<<(unsigned)((r1 - r0 + 255) / 256), 256, 0, st>>>(
        g, slot_of_user, user, r0, r1, slot ? slot[0] : nullptr, slot ? slot[1] : nullptr, slot ? slot[2] : nullptr,
        hl, d4, bits);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

int scatter_user_to_slots(const Geom &g, const Tables &t, const double *user, double *const slot[3], double fill,
                          cudaStream_t st)
{
    (void)fill;
    k_scatter<<<(g.npoints + 255) / 256, 256, 0, st>>>(g, t.slot_of_user, user, slot[0], slot[1], slot[2]);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

__global__ void k_scatter_kinds(Geom g, const int *slot_of_user, const uint8_t *user, uint8_t *kind, int *err)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.npoints) return;
    const int s = slot_of_user[i];
    for (int c = 0; c < g.dim; ++c) {
        const uint8_t k = user[i * g.dim + c];
        if (k > PD_BC_DISPLACEMENT) atomicExch(err, 1);
        kind[(size_t)c * g.nslots + s] = k <= PD_BC_DISPLACEMENT ? k : 0;
    }
}

int scatter_kinds(const Geom &g, const Tables &t, const uint8_t *user, uint8_t *kind, int *err, cudaStream_t st)
{
    k_scatter_kinds<<<(g.npoints + 255) / 256, 256, 0, st>>>(g, t.slot_of_user, user, kind, err);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

// Staging buffer from FP64 SoA displacements (FP32 hi/lo pairs or double4_32a).
__global__ void k_pack_stage(Geom g, const double *u0, const double *u1, const double *u2, float4 *hl, double4_32a *d4,
                             bool bits)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.nslots) return;
    const double x = u0[s], y = u1[s], z = g.dim == 3 ? u2[s] : 0.0;
    if (d4) d4[s] = make_double4_32a(x, y, z, 0.0);
    else stage_slot(s, g.dim, x, y, z, nullptr, nullptr, nullptr, hl, nullptr, bits);
}

int pack_stage(const Geom &g, double *const u[3], float4 *hl, double4_32a *d4, cudaStream_t st, bool bits)
{
    k_pack_stage<<<(g.nslots + 255) / 256, 256, 0, st>>>(g, u[0], u[1], u[2], hl, d4, bits);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

// Double-float pairs back to FP64 SoA: x = hi + lo.
__global__ void k_unpack_pairs(Geom g, const float4 *in, double *x0, double *x1, double *x2)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.nslots) return;
    const float4 hi = in[2 * s], lo = in[2 * s + 1];
    x0[s] = (double)hi.x + (double)lo.x;
    x1[s] = (double)hi.y + (double)lo.y;
    if (g.dim == 3) x2[s] = (double)hi.z + (double)lo.z;
}

int unpack_pairs(const Geom &g, const float4 *in, double *const x[3], cudaStream_t st)
{
    k_unpack_pairs<<<(g.nslots + 255) / 256, 256, 0, st>>>(g, in, x[0], x[1], x[2]);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

// FP64 per-DOF values (component-major, 3 x nslots) to (hi, lo) float pairs.
__global__ void k_pack_dof_pairs(long long n, const double *in, float *out)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const double x = in[q];
    const float h = (float)x;
    out[2 * q] = h;
    out[2 * q + 1] = (float)(x - (double)h);
}

int pack_dof_pairs(long long n, const double *in, float *out, cudaStream_t st)
{
    k_pack_dof_pairs<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, in, out);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

// FP64 component-major per-DOF values to one float4 per slot.
__global__ void k_pack_f4(Geom g, const double *in, float4 *out)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.nslots) return;
    const size_t ns = g.nslots;
    out[s] = make_float4((float)in[s], (float)in[ns + s], g.dim == 3 ? (float)in[2 * ns + s] : 0.f, 0.f);
}

int pack_f4(const Geom &g, const double *in, float4 *out, cudaStream_t st)
{
    k_pack_f4<<<(g.nslots + 255) / 256, 256, 0, st>>>(g, in, out);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

// Zero the prescribed-displacement components of a slot-order vector (JVP masking),
// or copy them from src into dst (identity rows).
__global__ void k_dirichlet(Geom g, const uint8_t *kind, double *v0, double *v1, double *v2, const double *w0,
                            const double *w1, const double *w2, int copy)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.nslots) return;
    double *v[3] = {v0, v1, v2};
    const double *w[3] = {w0, w1, w2};
    for (int c = 0; c < g.dim; ++c)
        if (kind[(size_t)c * g.nslots + s] == PD_BC_DISPLACEMENT) v[c][s] = copy ? w[c][s] : 0.0;
}

int dirichlet_mask(const Geom &g, const uint8_t *kind, double *const v[3], const double *const w[3], int copy,
                   cudaStream_t st)
{
    k_dirichlet<<<(g.nslots + 255) / 256, 256, 0, st>>>(g, kind, v[0], v[1], v[2], w ? w[0] : nullptr,
                                                        w ? w[1] : nullptr, w ? w[2] : nullptr, copy);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

}  // namespace pdk
