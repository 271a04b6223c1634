// pd_tile.cuh -- machinery shared by the tile kernels (force, step, tangent,
// energy): packed arithmetic on P points per thread, the horizon stencil as
// compile-time constants, and shared-memory staging of a tile's halo box.
//
// A CTA owns one tile (a Morton brick of T = 2^L lattice points). It stages the
// displacements of the brick plus an m-wide halo into shared memory as a dense
// box in lattice coordinates, so the neighbour at stencil offset d of the point
// at box index b sits at box index b + d.x + HX (d.y + HY d.z): one
// conflict-free vector load per bond. Displacements are staged in lattice units
// relative to a per-tile reference displacement,
//     u~_j = (u_j - u_ref) / h,
// formed from FP32 hi/lo pairs (FP32C) or FP64 (FP64 path). Bond vectors are
// then eta = u~_j - u~_i and xi = d (integers), so the cancellation that a
// rigid translation or a large displacement would cause in FP32 never occurs:
// the error of eta is relative to the variation of u across one halo box.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "pd_internal.cuh"

// float4 words per stencil entry of the FP32C NP / LP table (np_word in
// pd_force_pmb.cu; built in pd_api.cu)
#define NP_TAB_WORDS(dim) ((dim) == 3 ? 3 : 2)

namespace pdk {

// ----------------------------------------------------------- packed values

// P values of type R, one per point handled by the thread. For float with P = 2
// every elementwise op is one Blackwell packed-FP32 instruction (f32x2).
template <class R, int P>
struct Pk {
    R v[P];
};

template <class R, int P>
__device__ __forceinline__ Pk<R, P> splat(R x)
{
    Pk<R, P> r;
#pragma unroll
    for (int p = 0; p < P; ++p) r.v[p] = x;
    return r;
}

#define PD_PK_BINOP(NAME, EXPR)                                                   \
    template <class R, int P>                                                     \
    __device__ __forceinline__ Pk<R, P> NAME(const Pk<R, P> &a, const Pk<R, P> &b) \
    {                                                                             \
        Pk<R, P> r;                                                               \
        _Pragma("unroll") for (int p = 0; p < P; ++p) r.v[p] = EXPR;              \
        return r;                                                                 \
    }
PD_PK_BINOP(padd, a.v[p] + b.v[p])
PD_PK_BINOP(psub, a.v[p] - b.v[p])
PD_PK_BINOP(pmul, a.v[p] * b.v[p])
#undef PD_PK_BINOP

template <class R, int P>
__device__ __forceinline__ Pk<R, P> pfma(const Pk<R, P> &a, const Pk<R, P> &b, const Pk<R, P> &c)
{
    Pk<R, P> r;
#pragma unroll
    for (int p = 0; p < P; ++p) r.v[p] = fma(a.v[p], b.v[p], c.v[p]);
    return r;
}

// float x 2: packed instructions.
__device__ __forceinline__ float2 f2(const Pk<float, 2> &a) { return make_float2(a.v[0], a.v[1]); }
__device__ __forceinline__ Pk<float, 2> pk2(float2 a)
{
    Pk<float, 2> r;
    r.v[0] = a.x;
    r.v[1] = a.y;
    return r;
}
template <>
__device__ __forceinline__ Pk<float, 2> padd(const Pk<float, 2> &a, const Pk<float, 2> &b)
{
    return pk2(__fadd2_rn(f2(a), f2(b)));
}
template <>
__device__ __forceinline__ Pk<float, 2> psub(const Pk<float, 2> &a, const Pk<float, 2> &b)
{
    return pk2(__fadd2_rn(f2(a), make_float2(-b.v[0], -b.v[1])));
}
template <>
__device__ __forceinline__ Pk<float, 2> pmul(const Pk<float, 2> &a, const Pk<float, 2> &b)
{
    return pk2(__fmul2_rn(f2(a), f2(b)));
}
template <>
__device__ __forceinline__ Pk<float, 2> pfma(const Pk<float, 2> &a, const Pk<float, 2> &b,
                                             const Pk<float, 2> &c)
{
    return pk2(__ffma2_rn(f2(a), f2(b), f2(c)));
}

// x + k and x * k for a compile-time or uniform scalar k.
template <class R, int P>
__device__ __forceinline__ Pk<R, P> padds(const Pk<R, P> &a, R k) { return padd(a, splat<R, P>(k)); }
template <class R, int P>
__device__ __forceinline__ Pk<R, P> pmuls(const Pk<R, P> &a, R k) { return pmul(a, splat<R, P>(k)); }
template <class R, int P>
__device__ __forceinline__ Pk<R, P> pfmas(const Pk<R, P> &a, R k, const Pk<R, P> &c)
{
    return pfma(a, splat<R, P>(k), c);
}

// 1/sqrt(q) and a/b: hardware approximations in FP32 (a few ulp), exact
// rounding in FP64.
__device__ __forceinline__ float prsqrt1(float q) { return rsqrtf(q); }
__device__ __forceinline__ double prsqrt1(double q) { return 1.0 / sqrt(q); }
__device__ __forceinline__ float pdiv1(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double pdiv1(double a, double b) { return a / b; }

template <class R, int P>
__device__ __forceinline__ Pk<R, P> prsqrt(const Pk<R, P> &q)
{
    Pk<R, P> r;
#pragma unroll
    for (int p = 0; p < P; ++p) r.v[p] = prsqrt1(q.v[p]);
    return r;
}
template <class R, int P>
__device__ __forceinline__ Pk<R, P> pdiv(const Pk<R, P> &a, const Pk<R, P> &b)
{
    Pk<R, P> r;
#pragma unroll
    for (int p = 0; p < P; ++p) r.v[p] = pdiv1(a.v[p], b.v[p]);
    return r;
}

// ------------------------------------------------------------------ stencil

// k-th offset of the horizon stencil {d : 0 < |d|^2 <= m^2}, ordered by
// (dz, dy, dx) ascending; comp 0..2 = dx, dy, dz, comp 3 = |d|^2.
__host__ __device__ constexpr int stencil_entry(int dim, int m, int k, int comp)
{
    int idx = 0;
    for (int dz = (dim == 3 ? -m : 0); dz <= (dim == 3 ? m : 0); ++dz)
        for (int dy = -m; dy <= m; ++dy)
            for (int dx = -m; dx <= m; ++dx) {
                int d2 = dx * dx + dy * dy + dz * dz;
                if (d2 == 0 || d2 > m * m) continue;
                if (idx == k) return comp == 0 ? dx : comp == 1 ? dy : comp == 2 ? dz : d2;
                ++idx;
            }
    return 0;
}

__host__ __device__ constexpr int stencil_size(int dim, int m)
{
    int idx = 0;
    for (int dz = (dim == 3 ? -m : 0); dz <= (dim == 3 ? m : 0); ++dz)
        for (int dy = -m; dy <= m; ++dy)
            for (int dx = -m; dx <= m; ++dx) {
                int d2 = dx * dx + dy * dy + dz * dz;
                if (d2 != 0 && d2 <= m * m) ++idx;
            }
    return idx;
}

// sqrt of a small non-negative integer, by Newton's method in double.
__host__ __device__ constexpr double csqrt(double x)
{
    double r = x > 1.0 ? x : 1.0;
    for (int i = 0; i < 64; ++i) r = 0.5 * (r + x / r);
    return x == 0.0 ? 0.0 : r;
}

// Partial-volume factor in lattice units: (m + 1/2 - |d|) for |d| > m - 1/2.
__host__ __device__ constexpr double vol_factor_lattice(int m, double r0)
{
    return r0 > m - 0.5 ? (m + 0.5 - r0) : 1.0;
}

template <int DIM, int L>
struct Brick {
    static constexpr int bx = 1 << ((L + DIM - 1) / DIM);
    static constexpr int by = 1 << ((L + DIM - 2) / DIM);
    static constexpr int bz = DIM == 3 ? (1 << (L / 3)) : 1;
    static constexpr int T = 1 << L;
    static_assert(bx * by * bz == T, "brick");
};

// Compile-time halo-box geometry for horizon M.
template <int DIM, int L, int M>
struct Box {
    using B = Brick<DIM, L>;
    static constexpr int HX = B::bx + 2 * M;
    static constexpr int HY = B::by + 2 * M;
    static constexpr int HZ = DIM == 3 ? B::bz + 2 * M : 1;
    static constexpr int N = HX * HY * HZ;
};

// Compile-time loop: f(std::integral_constant<int, K>) for K = 0..N-1.
template <class F, int... Ks>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, Ks...>)
{
    (f(std::integral_constant<int, Ks>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F &&f)
{
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// --------------------------------------------------------------- staging

// Local Morton code of brick-local coordinates (x, y, z) for a brick of 2^L codes.
__device__ __forceinline__ int local_code(int dim, int x, int y, int z)
{
    return (int)morton_encode(dim, (uint32_t)x, (uint32_t)y, (uint32_t)z);
}

// Reference displacement of a tile as FP32 hi/lo (FP32C) or FP64.
struct RefF { float3 hi, lo; };

// The staging source of one step: 32 bytes per slot. FP32C: float4 hi, float4 lo;
// FP64: double4_32a (x, y, z, 0).
struct StageSrc {
    const float4 *hl;      // FP32C
    const double4_32a *d4;     // FP64
};

__device__ __forceinline__ float4 stage_fp32c(const float4 *hl, int slot, const RefF &ref, float inv_h)
{
    float4 hi = __ldg(&hl[2 * slot]);
    float4 lo = __ldg(&hl[2 * slot + 1]);
    float4 r;
    r.x = ((hi.x - ref.hi.x) + (lo.x - ref.lo.x)) * inv_h;
    r.y = ((hi.y - ref.hi.y) + (lo.y - ref.lo.y)) * inv_h;
    r.z = ((hi.z - ref.hi.z) + (lo.z - ref.lo.z)) * inv_h;
    r.w = 0.f;
    return r;
}

__device__ __forceinline__ double4_32a stage_fp64(const double4_32a *d4, int slot, const double3 &ref, double inv_h)
{
    double4_32a a = d4[slot];
    double4_32a r;
    r.x = (a.x - ref.x) * inv_h;
    r.y = (a.y - ref.y) * inv_h;
    r.z = (a.z - ref.z) * inv_h;
    r.w = 0.0;
    return r;
}

// Global coordinates of box index b for a tile with origin org (runtime box dims).
__device__ __forceinline__ void box_coord(int b, int HX, int HY, int m, int dim, const int4 &org,
                                          int &x, int &y, int &z)
{
    int bxl = b % HX;
    int rest = b / HX;
    int byl = rest % HY;
    int bzl = rest / HY;
    x = org.x + bxl - m;
    y = org.y + byl - m;
    z = dim == 3 ? org.z + bzl - m : 0;
}

// --------------------------------------------------------- slot lookup

// Spread the bits of x so that bit b moves to bit 3b (x < 1024) or 2b (x < 65536).
__device__ __forceinline__ uint32_t spread3(uint32_t x)
{
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}
__device__ __forceinline__ uint32_t spread2(uint32_t x)
{
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

// Local Morton code of brick-local coordinates.
__device__ __forceinline__ int brick_code(int dim, int x, int y, int z)
{
    return dim == 3 ? (int)(spread3(x) | (spread3(y) << 1) | (spread3(z) << 2))
                    : (int)(spread2(x) | (spread2(y) << 1));
}

// Slot of lattice point (x, y, z), or -1 outside the grid.
__device__ __forceinline__ int slot_at(const Geom &g, const int *tile_lut, int x, int y, int z)
{
    if ((unsigned)x >= (unsigned)g.nx || (unsigned)y >= (unsigned)g.ny || (unsigned)z >= (unsigned)g.nz)
        return -1;
    int tx = x >> g.lbx, ty = y >> g.lby, tz = z >> g.lbz;
    int t = __ldg(&tile_lut[tx + g.tgx * (ty + g.tgy * tz)]);
    return t * g.T + brick_code(g.dim, x & (g.bx - 1), y & (g.by - 1), z & (g.bz - 1));
}

// ------------------------------------------------------- FP64 <-> FP32 pairs

// FP32 -> FP64 from the bits, on the integer pipes (exact, as the conversion
// instruction; FP32 denormals, which the FP32 arithmetic flushes, give zero).
__device__ __forceinline__ double f2d_bits(float x)
{
    const unsigned X = __float_as_uint(x);
    const unsigned e = (X >> 23) & 0xffu;
    const unsigned ed = e == 0xffu ? 0x7ffu : e + 896u;
    const unsigned hi = (X & 0x80000000u) | (e ? (ed << 20) | ((X >> 3) & 0xfffffu) : 0u);
    const unsigned lo = e ? X << 29 : 0u;
    return __hiloint2double((int)hi, (int)lo);
}

// u = hi + lo to about 47 bits, from the bits of u on the integer and FP32
// pipes: hi is u with its 29 low mantissa bits cut off (exactly an FP32
// value, same sign), lo the cut-off part, rest * 2^(e - 1075), rounded once to
// FP32 (its two 16-bit halves convert exactly through the 2^23 magic number).
// |u| < 2^-126 stages as 0; |u| >= 2^116 (never a displacement) takes the
// conversion instruction.
__device__ __forceinline__ void split_bits(double u, float &hi, float &lo)
{
    const unsigned H = (unsigned)__double2hiint(u), Lw = (unsigned)__double2loint(u);
    const unsigned sign = H & 0x80000000u;
    const int e = (int)((H >> 20) & 0x7ffu);
    const unsigned rest = Lw & 0x1fffffffu;
    const float r1 = __uint_as_float(0x4b000000u | (rest >> 16)) - 8388608.f;
    const float r0 = __uint_as_float(0x4b000000u | (rest & 0xffffu)) - 8388608.f;
    const float fr = fmaf(r1, 65536.f, r0);
    // 2^(e - 1075) as 2^(e - 1011) * 2^-64, both normal FP32 numbers for 897 <= e <= 1138
    const float s1 = __uint_as_float((unsigned)(e - 884) << 23);
    const float l = fr * s1 * 5.42101086242752217e-20f;
    if (e < 897) {
        hi = 0.f;
        lo = 0.f;
    } else if (e > 1138) {
        hi = __double2float_rn(u);
        lo = 0.f;
    } else {
        hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | ((H & 0xfffffu) << 3) | (Lw >> 29));
        lo = sign ? -l : l;
    }
}

// ------------------------------------------------------------ kernel args

// One POD argument block for every tile kernel.
struct TileArgs {
    Geom g;
    const int4 *tile_org;
    const int *tile_ref;
    const int *tile_lut;
    const int4 *stencil;        // runtime stencil (dx, dy, dz, |d|^2) for generic kernels
    const double *stencil_r0;   // |d| of each stencil entry
    const float4 *src_hl;       // staging source (FP32C hi/lo pairs)
    const double4_32a *src_d4;      // staging source (FP64)
    float4 *dst_hl;             // next staging buffer written by MODE_STEP
    double4_32a *dst_d4;
    uint32_t *mask;
    double *u[3];
    double *v[3];
    const uint8_t *bc_kind;
    const double *bc_val;
    const double *body;
    double *f[3];               // MODE_FORCE output
    const float *minv32;        // LPS 1/m~
    const double *mtil;         // LPS m~ (FP64)
    float *theta32;
    double *theta64;
    double psi_beta;            // NP / LP potential rate
    const double *w[3];         // tangent input (slot order)
    double *jv[3];              // tangent output
    double *epoint;             // per-point energy (slot order)
    float4 *vhl;                // FP32C velocity as double-float pairs (2 float4 per slot)
    const float *bc32;          // FP32C boundary values as (hi, lo) per DOF, component-major
    const float4 *body32;       // FP32C body force per slot
    const float4 *tab_a;        // FP32C stencil table of the PMB and NP kernels (4 or NP_TAB_WORDS float4 / entry),
                                // or of the LPS dilatation (3 float4 / entry)
    const float4 *tab_b;        // FP32C stencil table of the LPS force pass (3 float4 / entry)
    const int *tile_nbr;        // [ntiles * 27] the 3^d neighbour tiles of each tile (or -1)
    int nbr_ok;                 // halo within one tile in every direction: tile_nbr is usable
    const uint32_t *box_map;    // paired halo box: neighbour tile (5 bits) + brick code (9) of A, then of B
    int box_edge[3];            // box_map holds for tiles with org <= box_edge on every axis
    float kF, kB;               // FP32C kick factors: dt/2 * fscale / rho and dt/2 / rho
    float dt_h, dt_l;           // dt as a double-float pair
    double fscale;              // force density = fscale * F (PMB: c V; LPS: 1/h)
    double cV;                  // c V (PMB)
    double inv_rho, dt, s_c, inv_h, h;
    double A, B;                // LPS 3K - 5 mu and 15 mu
    double K;                   // LPS bulk modulus (energy)
    int model;                  // PD_MODEL_PMB or PD_MODEL_LPS
    int v_is_half, update_breaking, mode, vol_corr, use_body, adjoint;
    int cd;                     // MODE_STEP: central-difference drift from u^{k-1} at dst
    int split;                  // fused bond kernels: threads per point pair (1, 2 or 4)
    int state64;                // FP32C fused update: u, v in the FP64 arrays u[], v[] (else double-float pairs)
    // host copies of tab_a / tab_b (read by the host launchers only: tables of at
    // most PTAB_N float4 are passed to the kernels as a parameter, see ParamTab)
    const float4 *htab_a, *htab_b;
    int ntab_a, ntab_b;
};

// A stencil table passed as a kernel parameter: the kernel reads it from the
// constant bank, whose warp-uniform reads take none of the shared-memory
// bandwidth that bounds the bond loops (128^3 LPS force pass 0.392 -> 0.361 ms
// against the same table in shared memory). 8 KB: 3D stencils up to m = 3.
constexpr int PTAB_N = 512;
struct ParamTab {
    float4 e[PTAB_N];
};

// --------------------------------------------------------------- staging

struct Ref32 { float hx, hy, hz, lx, ly, lz; };

__device__ __forceinline__ Ref32 tile_ref32(const TileArgs &a, int tile)
{
    int rs = __ldg(&a.tile_ref[tile]);
    float4 hi = __ldg(&a.src_hl[2 * rs]);
    float4 lo = __ldg(&a.src_hl[2 * rs + 1]);
    return Ref32{hi.x, hi.y, hi.z, lo.x, lo.y, lo.z};
}

__device__ __forceinline__ double3 tile_ref64(const TileArgs &a, int tile)
{
    int rs = __ldg(&a.tile_ref[tile]);
    double4_32a d = a.src_d4[rs];
    return make_double3(d.x, d.y, d.z);
}

// Fill the halo box (dims HX x HY x HZ, m-wide halo around the brick at org)
// with staged displacements in lattice units; points outside the grid get 0.
__device__ __forceinline__ void stage_box32(float4 *box, int HX, int HY, int nbox, int m,
                                            const TileArgs &a, const int4 &org, const Ref32 &ref,
                                            float inv_h)
{
    for (int b = threadIdx.x; b < nbox; b += blockDim.x) {
        int bxl = b % HX, rest = b / HX;
        int byl = rest % HY, bzl = rest / HY;
        int x = org.x + bxl - m, y = org.y + byl - m;
        int z = a.g.dim == 3 ? org.z + bzl - m : 0;
        int s = slot_at(a.g, a.tile_lut, x, y, z);
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        if (s >= 0) {
            float4 hi = __ldg(&a.src_hl[2 * s]);
            float4 lo = __ldg(&a.src_hl[2 * s + 1]);
            r.x = ((hi.x - ref.hx) + (lo.x - ref.lx)) * inv_h;
            r.y = ((hi.y - ref.hy) + (lo.y - ref.ly)) * inv_h;
            r.z = ((hi.z - ref.hz) + (lo.z - ref.lz)) * inv_h;
        }
        box[b] = r;
    }
}

__device__ __forceinline__ void stage_box64(double4_32a *box, int HX, int HY, int nbox, int m,
                                            const TileArgs &a, const int4 &org, const double3 &ref,
                                            double inv_h)
{
    for (int b = threadIdx.x; b < nbox; b += blockDim.x) {
        int bxl = b % HX, rest = b / HX;
        int byl = rest % HY, bzl = rest / HY;
        int x = org.x + bxl - m, y = org.y + byl - m;
        int z = a.g.dim == 3 ? org.z + bzl - m : 0;
        int s = slot_at(a.g, a.tile_lut, x, y, z);
        double4_32a r = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        if (s >= 0) {
            double4_32a d = a.src_d4[s];
            r.x = (d.x - ref.x) * inv_h;
            r.y = (d.y - ref.y) * inv_h;
            r.z = (d.z - ref.z) * inv_h;
        }
        box[b] = r;
    }
}

// ------------------------------------------------------------- epilogue

// Integrator update of one point from its internal force density f (N/m^3):
// MODE_STEP   v <- v + (dt or dt/2) a, then drift u <- u + dt v with boundary
//             conditions, and write the next staging buffer;
// MODE_FINALIZE  v <- v + dt/2 a (completes a half step), no drift;
// MODE_FORCE  store f.
// a = (f + b) / rho. Eqs. (7)-(9): the second half-kick of step k-1 and the
// first half-kick of step k use the same force f^k and run in the same kernel.
// With a.cd set a free DOF drifts by the central difference of Eq. (10),
// u^{k+1} = 2 u^k - u^{k-1} + dt^2 a^k, u^{k-1} read from the staging buffer
// the step overwrites.
__device__ __forceinline__ void point_epilogue(const TileArgs &a, int slot, const double f[3],
                                               int dim, bool fp64)
{
    const int ns = a.g.nslots;
    if (a.mode == MODE_FORCE) {
        for (int c = 0; c < dim; ++c) a.f[c][slot] = f[c];
        return;
    }
    double un[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < dim; ++c) {
        double acc = f[c];
        if (a.use_body) acc += a.body[c * ns + slot];
        acc *= a.inv_rho;
        double v = a.v[c][slot];
        const int kind = a.bc_kind[c * ns + slot];
        if (a.mode == MODE_STEP) {
            // second half-kick of the previous step (Eq. (9)), then the first
            // half-kick of this one (Eq. (7)), as two roundings like the equations
            const double hk = 0.5 * a.dt;
            if (a.v_is_half) v = fma(hk, acc, v);
            v = fma(hk, acc, v);
            double u = a.u[c][slot];
            if (kind == PD_BC_VELOCITY) {
                v = a.bc_val[c * ns + slot];
                u = fma(a.dt, v, u);
            } else if (kind == PD_BC_DISPLACEMENT) {
                v = 0.0;
                u = a.bc_val[c * ns + slot];
            } else if (a.cd) {
                double up;
                if (fp64) {
                    const double4_32a p = a.dst_d4[slot];
                    up = c == 0 ? p.x : (c == 1 ? p.y : p.z);
                } else {
                    const float4 ph = a.dst_hl[2 * slot], pl = a.dst_hl[2 * slot + 1];
                    up = c == 0 ? (double)ph.x + pl.x : (c == 1 ? (double)ph.y + pl.y : (double)ph.z + pl.z);
                }
                u = fma(a.dt * a.dt, acc, 2.0 * u - up);
            } else {
                u = fma(a.dt, v, u);
            }
            a.u[c][slot] = u;
            un[c] = u;
        } else {
            if (a.v_is_half) v = fma(0.5 * a.dt, acc, v);
            if (kind == PD_BC_VELOCITY) v = a.bc_val[c * ns + slot];
            else if (kind == PD_BC_DISPLACEMENT) v = 0.0;
        }
        a.v[c][slot] = v;
    }
    if (a.mode == MODE_STEP) {
        if (fp64) {
            a.dst_d4[slot] = make_double4_32a(un[0], un[1], un[2], 0.0);
        } else {
            float hx = (float)un[0], hy = (float)un[1], hz = (float)un[2];
            a.dst_hl[2 * slot] = make_float4(hx, hy, hz, 0.f);
            a.dst_hl[2 * slot + 1] = make_float4((float)(un[0] - (double)hx), (float)(un[1] - (double)hy),
                                                 (float)(un[2] - (double)hz), 0.f);
        }
    }
}

}  // namespace pdk
