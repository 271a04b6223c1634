// pd_tangent.cu -- the PMB tangent of Eq. (6) kept per bond for repeated
// products inside one Newton iteration.
//
// With n = y/|y| and s the stretch, a bond contributes D_ij (w_j - w_i) to
// (K w)_i with the symmetric d x d matrix
//   D_ij = (c V / h) V_ij [ (1/|d| - s/r) n n^T + (s/r) I ]      (lattice units, r = |y|)
// (the same algebra as the JVP kernel in pd_jvp.cu). tangent_prepare evaluates
// D for every intact bond of a linearisation point u once (3 entries in 2D, 6 in
// 3D, stored [k][entry][slot] so that a warp's accesses are coalesced) together
// with the slot of the neighbour; a broken or missing bond stores D = 0 and its
// own slot. tangent_apply then costs one coalesced read of D and one gather of
// w_j per bond and a few FMAs: on GB300, whose FP64 rate is 1/64 of FP32, this
// moves the FP64 tangent from the arithmetic pipe (rsqrt, divide, ~35 FP64 ops
// per bond per product) to memory that stays in L2 across a Krylov solve.
#include <type_traits>

#include "pd_tile.cuh"

namespace pdk {

size_t jvp_smem(const Geom &g, int precision);

template <class R>
__global__ void __launch_bounds__(256) tangent_prepare(const TileArgs a, R *coef, int *nbr)
{
    using R4 = typename std::conditional<sizeof(R) == 4, float4, double4_32a>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geom &g = a.g;
    const int m = g.m;
    const int HX = g.bx + 2 * m, HY = g.by + 2 * m, HZ = g.dim == 3 ? g.bz + 2 * m : 1;
    const int nbox = HX * HY * HZ;
    R4 *box = reinterpret_cast<R4 *>(smem_raw);
    const int tile = blockIdx.x;
    const int4 org = __ldg(&a.tile_org[tile]);
    if constexpr (sizeof(R) == 4)
        stage_box32(reinterpret_cast<float4 *>(box), HX, HY, nbox, m, a, org, tile_ref32(a, tile), (float)a.inv_h);
    else
        stage_box64(reinterpret_cast<double4_32a *>(box), HX, HY, nbox, m, a, org, tile_ref64(a, tile), a.inv_h);
    __syncthreads();

    const size_t ns = g.nslots;
    const int nc = g.dim == 3 ? 6 : 3;
    const R sc = (R)(a.cV * a.inv_h);
    for (int t = threadIdx.x; t < g.T; t += blockDim.x) {
        const int slot = tile * g.T + t;
        int l[3];
        morton_decode(g.dim, (uint64_t)t, l);
        const int x = org.x + l[0], y = org.y + l[1], z = org.z + l[2];
        const bool act = x < g.nx && y < g.ny && z < g.nz;
        const int bi = (l[0] + m) + HX * ((l[1] + m) + HY * (g.dim == 3 ? l[2] + m : 0));
        const R4 ui = box[act ? bi : 0];
        uint32_t word = 0;
        for (int k = 0; k < g.S; ++k) {
            if ((k & 31) == 0) word = act ? a.mask[(size_t)(k >> 5) * ns + slot] : 0u;
            R D[6] = {0, 0, 0, 0, 0, 0};
            int js = slot;
            if ((word >> (k & 31)) & 1u) {
                const int4 d = __ldg(&a.stencil[k]);
                const R r0 = (R)__ldg(&a.stencil_r0[k]);
                const R4 uj = box[bi + d.x + HX * (d.y + HY * d.z)];
                const R ex = uj.x - ui.x, ey = uj.y - ui.y, ez = uj.z - ui.z;
                const R yx = ex + (R)d.x, yy = ey + (R)d.y, yz = ez + (R)d.z;
                const R q = yx * yx + yy * yy + yz * yz;
                const R num = ex * ex + ey * ey + ez * ez + (R)2 * ((R)d.x * ex + (R)d.y * ey + (R)d.z * ez);
                const R rs = prsqrt1(q);
                const R s = pdiv1(num, r0 * (q * rs + r0));
                const R vij = a.vol_corr ? (R)vol_factor_lattice(m, (double)r0) : (R)1;
                const R al = sc * vij * ((R)1 / r0 - s * rs) * rs * rs;    // times y y^T
                const R be = sc * vij * s * rs;                             // times I
                D[0] = al * yx * yx + be;
                D[1] = al * yx * yy;
                D[2] = al * yy * yy + be;
                if (g.dim == 3) {
                    D[3] = al * yx * yz;
                    D[4] = al * yy * yz;
                    D[5] = al * yz * yz + be;
                }
                js = slot_at(g, a.tile_lut, x + d.x, y + d.y, z + d.z);
            }
            for (int c = 0; c < nc; ++c) coef[((size_t)k * nc + c) * ns + slot] = D[c];
            nbr[(size_t)k * ns + slot] = js;
        }
    }
}

// y = A w with A = -K on free DOFs and the identity on prescribed ones (the
// Newton operator of pd_solve_static); w, y component-major over slots. A block
// of 8 warps covers TA_SLOTS = 32 slots: warp k of the block takes every
// TA_PARTS-th stencil entry from k, so a warp's loads of D and nbr cover 32
// consecutive slots and the 8 warps share the slots' sums (the small grids of an implicit solve would otherwise run one warp per
// 32 slots, a few warps per SM, each waiting on its gathers in turn). The parts
// are added in part order through shared memory.
constexpr int TA_PARTS = 8;
constexpr int TA_SLOTS = 256 / TA_PARTS;

template <class R>
__global__ void __launch_bounds__(256) tangent_apply(Geom g, const R *coef, const int *nbr, const int *user_of_slot,
                                                     const uint8_t *kind, const double *w, double *y)
{
    __shared__ R part[TA_PARTS][3][TA_SLOTS];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int grp = warp / TA_PARTS, sub = warp % TA_PARTS;
    const int ls = grp * 32 + lane;                        // slot within the block
    const long long s = (long long)blockIdx.x * TA_SLOTS + ls;
    const size_t ns = g.nslots;
    const int d = g.dim;
    const bool act = s < g.nslots && user_of_slot[s] >= 0;
    R a0 = 0, a1 = 0, a2 = 0;
    if (act) {
        const int nc = d == 3 ? 6 : 3;
        const double wi0 = w[s], wi1 = w[ns + s], wi2 = d == 3 ? w[2 * ns + s] : 0.0;
#pragma unroll 2
        for (int k = sub; k < g.S; k += TA_PARTS) {
            const int j = __ldg(&nbr[(size_t)k * ns + s]);
            const R *Dk = coef + (size_t)k * nc * ns + s;
            const R d0 = (R)(w[j] - wi0), d1 = (R)(w[ns + j] - wi1);
            if (d == 3) {
                const R d2 = (R)(w[2 * ns + j] - wi2);
                const R xx = __ldg(&Dk[0]), xy = __ldg(&Dk[ns]), yy = __ldg(&Dk[2 * ns]);
                const R xz = __ldg(&Dk[3 * ns]), yz = __ldg(&Dk[4 * ns]), zz = __ldg(&Dk[5 * ns]);
                a0 += xx * d0 + xy * d1 + xz * d2;
                a1 += xy * d0 + yy * d1 + yz * d2;
                a2 += xz * d0 + yz * d1 + zz * d2;
            } else {
                const R xx = __ldg(&Dk[0]), xy = __ldg(&Dk[ns]), yy = __ldg(&Dk[2 * ns]);
                a0 += xx * d0 + xy * d1;
                a1 += xy * d0 + yy * d1;
            }
        }
    }
    part[sub][0][ls] = a0;
    part[sub][1][ls] = a1;
    part[sub][2][ls] = a2;
    __syncthreads();
    if (sub != 0 || s >= g.nslots) return;
    if (!act) {
        for (int c = 0; c < d; ++c) y[c * ns + s] = 0.0;
        return;
    }
    for (int c = 0; c < d; ++c) {
        R acc = part[0][c][ls];
        for (int p = 1; p < TA_PARTS; ++p) acc += part[p][c][ls];
        const size_t e = (size_t)c * ns + s;
        y[e] = kind[e] == PD_BC_DISPLACEMENT ? w[e] : -(double)acc;
    }
}

// Block-Jacobi preconditioner of A: the d x d diagonal block of point i is
// A_ii = sum_j D_ij (from (K w)_i = sum_j D_ij (w_j - w_i) and A = -K); a
// prescribed component gets an identity row and column, as A has. Its inverse is
// stored per slot (3 or 6 FP64 values); slots without a point store I.
template <class R>
__global__ void tangent_jacobi_prepare(Geom g, const R *coef, const int *user_of_slot, const uint8_t *kind,
                                       double *inv)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.nslots) return;
    const size_t ns = g.nslots;
    const int d = g.dim, nc = d == 3 ? 6 : 3;
    double B[6] = {0, 0, 0, 0, 0, 0};     // xx xy yy xz yz zz
    if (user_of_slot[s] >= 0)
        for (int k = 0; k < g.S; ++k)
            for (int c = 0; c < nc; ++c) B[c] += (double)coef[((size_t)k * nc + c) * ns + s];
    else {
        B[0] = B[2] = B[5] = 1.0;
    }
    // prescribed components: identity row and column
    const int diag[3] = {0, 2, 5};
    for (int c = 0; c < d; ++c) {
        if (user_of_slot[s] < 0 || kind[(size_t)c * ns + s] != PD_BC_DISPLACEMENT) continue;
        if (c == 0) { B[1] = 0.0; B[3] = 0.0; }
        if (c == 1) { B[1] = 0.0; B[4] = 0.0; }
        if (c == 2) { B[3] = 0.0; B[4] = 0.0; }
        B[diag[c]] = 1.0;
    }
    double *o = inv;
    if (d == 2) {
        const double det = B[0] * B[2] - B[1] * B[1];
        const double id = det != 0.0 ? 1.0 / det : 0.0;
        o[s] = B[2] * id;
        o[ns + s] = -B[1] * id;
        o[2 * ns + s] = B[0] * id;
    } else {
        // symmetric 3 x 3 inverse by cofactors
        const double a = B[0], b = B[1], c = B[3], e = B[2], f = B[4], i = B[5];
        const double A0 = e * i - f * f, A1 = -(b * i - c * f), A2 = b * f - c * e;
        const double det = a * A0 + b * A1 + c * A2;
        const double id = det != 0.0 ? 1.0 / det : 0.0;
        o[s] = A0 * id;                          // xx
        o[ns + s] = A1 * id;                     // xy
        o[2 * ns + s] = (a * i - c * c) * id;    // yy
        o[3 * ns + s] = A2 * id;                 // xz
        o[4 * ns + s] = -(a * f - b * c) * id;   // yz
        o[5 * ns + s] = (a * e - b * b) * id;    // zz
    }
}

// z = M^-1 r with the stored inverse blocks
__global__ void tangent_jacobi_apply(Geom g, const double *inv, const double *r, double *z)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.nslots) return;
    const size_t ns = g.nslots;
    const double r0 = r[s], r1 = r[ns + s];
    const double xx = inv[s], xy = inv[ns + s], yy = inv[2 * ns + s];
    if (g.dim == 2) {
        z[s] = xx * r0 + xy * r1;
        z[ns + s] = xy * r0 + yy * r1;
        return;
    }
    const double r2 = r[2 * ns + s];
    const double xz = inv[3 * ns + s], yz = inv[4 * ns + s], zz = inv[5 * ns + s];
    z[s] = xx * r0 + xy * r1 + xz * r2;
    z[ns + s] = xy * r0 + yy * r1 + yz * r2;
    z[2 * ns + s] = xz * r0 + yz * r1 + zz * r2;
}

// Cache layout: D [S][nc][nslots] (precision R), neighbour [S][nslots] int, and
// the preconditioner's inverse blocks [nc][nslots] FP64 (8-byte aligned).
static size_t cache_inv_offset(const Geom &g, int precision)
{
    const size_t nc = g.dim == 3 ? 6 : 3;
    const size_t r = precision == PD_FP64 ? sizeof(double) : sizeof(float);
    const size_t b = (size_t)g.S * g.nslots * (nc * r + sizeof(int));
    return (b + 7) & ~(size_t)7;
}

size_t tangent_cache_bytes(const Geom &g, int precision)
{
    const size_t nc = g.dim == 3 ? 6 : 3;
    return cache_inv_offset(g, precision) + nc * g.nslots * sizeof(double);
}

int launch_tangent_jacobi(const Geom &g, int precision, void *cache, const int *user_of_slot, const uint8_t *kind,
                          cudaStream_t st)
{
    double *inv = reinterpret_cast<double *>(static_cast<char *>(cache) + cache_inv_offset(g, precision));
    const unsigned nb = (unsigned)((g.nslots + 255) / 256);
    if (precision == PD_FP64)
        tangent_jacobi_prepare<double><<<nb, 256, 0, st>>>(g, static_cast<const double *>(cache), user_of_slot, kind, inv);
    else
        tangent_jacobi_prepare<float><<<nb, 256, 0, st>>>(g, static_cast<const float *>(cache), user_of_slot, kind, inv);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

int launch_tangent_precond(const Geom &g, int precision, const void *cache, const double *r, double *z,
                           cudaStream_t st)
{
    const double *inv =
        reinterpret_cast<const double *>(static_cast<const char *>(cache) + cache_inv_offset(g, precision));
    tangent_jacobi_apply<<<(unsigned)((g.nslots + 255) / 256), 256, 0, st>>>(g, inv, r, z);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

int launch_tangent_prepare(const TileArgs &a, int precision, void *cache, cudaStream_t st)
{
    const Geom &g = a.g;
    const size_t nc = g.dim == 3 ? 6 : 3;
    const size_t r = precision == PD_FP64 ? sizeof(double) : sizeof(float);
    int *nbr = reinterpret_cast<int *>(static_cast<char *>(cache) + (size_t)g.S * g.nslots * nc * r);
    const size_t smem = jvp_smem(g, precision) / 2;      // the u box alone
    if (smem > 227 * 1024) {
        set_error("the tangent cache's halo box (%zu bytes) does not fit in shared memory", smem);
        return PD_EINVAL;
    }
    if (precision == PD_FP64) {
        PD_CUDA(smem_limit(tangent_prepare<double>, smem));
        tangent_prepare<double><<<g.ntiles, 256, smem, st>>>(a, static_cast<double *>(cache), nbr);
    } else {
        PD_CUDA(smem_limit(tangent_prepare<float>, smem));
        tangent_prepare<float><<<g.ntiles, 256, smem, st>>>(a, static_cast<float *>(cache), nbr);
    }
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

int launch_tangent_apply(const Geom &g, int precision, const void *cache, const int *user_of_slot,
                         const uint8_t *kind, const double *w, double *y, cudaStream_t st)
{
    const size_t nc = g.dim == 3 ? 6 : 3;
    const size_t r = precision == PD_FP64 ? sizeof(double) : sizeof(float);
    const int *nbr = reinterpret_cast<const int *>(static_cast<const char *>(cache) + (size_t)g.S * g.nslots * nc * r);
    const unsigned nb = (unsigned)((g.nslots + TA_SLOTS - 1) / TA_SLOTS);
    if (precision == PD_FP64)
        tangent_apply<double><<<nb, 256, 0, st>>>(g, static_cast<const double *>(cache), nbr, user_of_slot, kind, w, y);
    else
        tangent_apply<float><<<nb, 256, 0, st>>>(g, static_cast<const float *>(cache), nbr, user_of_slot, kind, w, y);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

}  // namespace pdk
