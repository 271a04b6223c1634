// pd_pair.cuh -- the FP32-compensated fast path: two points per thread in
// packed f32x2 arithmetic, pair-interleaved shared-memory staging, and the
// explicit update in double-float (FP32 hi/lo pairs) arithmetic.
//
// Point pairs. Thread t of a tile owns point A = (lx, ly, lz) and point
// B = A + (0, 0, bz/2) in 3D, or B = A + (0, by/2) in 2D. Both see the same
// stencil offset d at the same time, so the halo is staged as *pairs*: slot
// (x, y, z') of the paired box holds the displacements of (x, y, z') and
// (x, y, z' + bz/2), interleaved as {xA, xB, yA, yB} and {zA, zB, .., ..}. A
// bond then loads its two neighbours with one 16-byte and one 8-byte shared
// load straight into f32x2 register pairs.
//
// State. In the FP32C mode the integrator state is held as double-float
// numbers (hi + lo, two FP32 values, about 48 significant bits): GB300 runs FP64
// at 1/64 of the FP32 rate, and an FP64 update of u and v costs more than the
// bond loop of a small tile. The sums are Knuth's two-sum and Dekker's
// product with an FMA, which keep the accumulated rounding of a 1000-step run
// near 1e-12 relative, far below the 1e-4 tolerance on u.
#pragma once

#include "pd_tile.cuh"

namespace pdk {

// ------------------------------------------------------------ f32x2 helpers

// PD_PACKED selects the Blackwell packed-FP32 instructions (default) or plain
// scalar FP32 on the same two points.
#ifndef PD_PACKED
#define PD_PACKED 1
#endif
// Unroll depth of the bond loops and the CTAs per SM the kernels are built for.
#ifndef PD_UNROLL
#define PD_UNROLL 4
#endif
#ifndef PD_MINBLOCKS
#define PD_MINBLOCKS 4
#endif
#define PD_STR_(x) #x
#define PD_PRAGMA_UNROLL(n) _Pragma(PD_STR_(unroll n))
#if PD_PACKED
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
#else
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return make_float2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c)
{
    return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
}
#endif
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2rsqrt(float2 q) { return make_float2(rsqrtf(q.x), rsqrtf(q.y)); }
__device__ __forceinline__ float2 f2div(float2 a, float2 b)
{
    return make_float2(__fdividef(a.x, b.x), __fdividef(a.y, b.y));
}
__device__ __forceinline__ float2 f2lo(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 f2hi(float4 v) { return make_float2(v.z, v.w); }

// --------------------------------------------------------------- double-float

struct DF {
    float h, l;
};

// a + b with b a float (two-sum, then renormalise)
__device__ __forceinline__ DF df_add_f(DF a, float b)
{
    const float s = a.h + b;
    const float bb = s - a.h;
    float e = (a.h - (s - bb)) + (b - bb);
    e += a.l;
    const float h = s + e;
    return DF{h, e - (h - s)};
}

__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const float s = a.h + b.h;
    const float bb = s - a.h;
    float e = (a.h - (s - bb)) + (b.h - bb);
    e += a.l + b.l;
    const float h = s + e;
    return DF{h, e - (h - s)};
}

// a * b (Dekker's product with an FMA for the low part)
__device__ __forceinline__ DF df_mul(DF a, DF b)
{
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    const float h = p + e;
    return DF{h, e - (h - p)};
}

// ------------------------------------------------------------------ tables

// Paired-box geometry: x extent HX, y extent HY, and the pair planes along the
// split axis (3D: z' in [0, bz/2 + 2m); 2D: y' in [0, by/2 + 2m)).
struct PairBox {
    int HX, HY, HZ, n;
};

__device__ __forceinline__ PairBox pair_box(const Geom &g)
{
    PairBox b;
    b.HX = g.bx + 2 * g.m;
    if (g.dim == 3) {
        b.HY = g.by + 2 * g.m;
        b.HZ = g.bz / 2 + 2 * g.m;
    } else {
        b.HY = g.by / 2 + 2 * g.m;
        b.HZ = 1;
    }
    b.n = b.HX * b.HY * b.HZ;
    return b;
}

__device__ __forceinline__ float4 stage_one(const TileArgs &a, const float4 *hl, int s, const Ref32 &ref,
                                            float inv_h)
{
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    if (s >= 0) {
        const float4 hi = __ldg(&hl[2 * s]);
        const float4 lo = __ldg(&hl[2 * s + 1]);
        r.x = ((hi.x - ref.hx) + (lo.x - ref.lx)) * inv_h;
        r.y = ((hi.y - ref.hy) + (lo.y - ref.ly)) * inv_h;
        r.z = ((hi.z - ref.hz) + (lo.z - ref.lz)) * inv_h;
    }
    return r;
}

// Coordinates of the two points of pair-box index b.
__device__ __forceinline__ void pair_coords(const Geom &g, const PairBox &pb, const int4 &org, int b, int cA[3],
                                            int cB[3])
{
    const int bxl = b % pb.HX, rest = b / pb.HX;
    const int byl = rest % pb.HY, bzl = rest / pb.HY;
    cA[0] = cB[0] = org.x + bxl - g.m;
    if (g.dim == 3) {
        cA[1] = cB[1] = org.y + byl - g.m;
        cA[2] = org.z + bzl - g.m;
        cB[2] = cA[2] + g.bz / 2;
    } else {
        cA[1] = org.y + byl - g.m;
        cB[1] = cA[1] + g.by / 2;
        cA[2] = cB[2] = 0;
    }
}

// Stage the paired box of displacements: P4[b] = {xA, xB, yA, yB}, P2[b] = {zA, zB}.
__device__ __forceinline__ void stage_pairs(const TileArgs &a, const PairBox &pb, const int4 &org, int tile,
                                            float4 *P4, float2 *P2)
{
    const Ref32 ref = tile_ref32(a, tile);
    const float inv_h = (float)a.inv_h;
    for (int b = threadIdx.x; b < pb.n; b += blockDim.x) {
        int cA[3], cB[3];
        pair_coords(a.g, pb, org, b, cA, cB);
        const float4 rA = stage_one(a, a.src_hl, slot_at(a.g, a.tile_lut, cA[0], cA[1], cA[2]), ref, inv_h);
        const float4 rB = stage_one(a, a.src_hl, slot_at(a.g, a.tile_lut, cB[0], cB[1], cB[2]), ref, inv_h);
        P4[b] = make_float4(rA.x, rB.x, rA.y, rB.y);
        if (P2) P2[b] = make_float2(rA.z, rB.z);
    }
}

// Points of thread t: local coordinates of A and B, their slots, pair-box index.
struct PairPts {
    int slot[2];
    bool act[2];
    int bi;
};

__device__ __forceinline__ PairPts pair_points(const Geom &g, const PairBox &pb, const int4 &org, int tile, int t)
{
    PairPts q;
    const int lx = t & (g.bx - 1), r1 = t >> g.lbx;
    int ly[2], lz[2];
    if (g.dim == 3) {
        // the y rows of a warp's lanes 0-7 and 8-15 are by/2 apart, so that an
        // 8-byte shared load of 16 lanes covers all 32 banks (row pitch HX)
        const int yr = r1 & (g.by - 1);
        ly[0] = ly[1] = g.by >= 2 ? ((yr & 1) * (g.by / 2) + (yr >> 1)) : yr;
        lz[0] = r1 >> g.lby;
        lz[1] = lz[0] + g.bz / 2;
        q.bi = (lx + g.m) + pb.HX * ((ly[0] + g.m) + pb.HY * (lz[0] + g.m));
    } else {
        ly[0] = r1;
        ly[1] = r1 + g.by / 2;
        lz[0] = lz[1] = 0;
        q.bi = (lx + g.m) + pb.HX * (ly[0] + g.m);
    }
    for (int p = 0; p < 2; ++p) {
        q.slot[p] = tile * g.T + brick_code(g.dim, lx, ly[p], lz[p]);
        q.act[p] = org.x + lx < g.nx && org.y + ly[p] < g.ny && org.z + lz[p] < g.nz;
    }
    return q;
}

// ---------------------------------------------------------- update (FP32C)

// Velocity-Verlet update of one point in double-float arithmetic from its
// force F (FP32, in the kernel's units): the kick is kF * F (+ kB * b) with
// kF = dt/2 * (force scale)/rho and kB = dt/2/rho. MODE_STEP applies the
// second half-kick of the previous step (if v holds a half step), the first
// half-kick of this step, the drift u += dt v with boundary conditions, and
// writes u to the next staging buffer; MODE_FINALIZE applies only the pending
// half-kick; MODE_FORCE stores f = (force scale) * F in FP64.
__device__ __forceinline__ void pair_epilogue(const TileArgs &a, int slot, const float F[3], int dim)
{
    const int ns = a.g.nslots;
    if (a.mode == MODE_FORCE) {
        for (int c = 0; c < dim; ++c) a.f[c][slot] = a.fscale * (double)F[c];
        return;
    }
    const float4 vh4 = a.vhl[2 * slot], vl4 = a.vhl[2 * slot + 1];
    DF v[3] = {{vh4.x, vl4.x}, {vh4.y, vl4.y}, {vh4.z, vl4.z}};
    DF u[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    float4 bb = make_float4(0.f, 0.f, 0.f, 0.f);
    if (a.use_body) bb = a.body32[slot];
    const float bcomp[3] = {bb.x, bb.y, bb.z};
    if (a.mode == MODE_STEP) {
        const float4 uh4 = a.src_hl[2 * slot], ul4 = a.src_hl[2 * slot + 1];
        u[0] = DF{uh4.x, ul4.x};
        u[1] = DF{uh4.y, ul4.y};
        u[2] = DF{uh4.z, ul4.z};
    }
    for (int c = 0; c < dim; ++c) {
        const float kick = fmaf(a.kF, F[c], a.kB * bcomp[c]);
        const int kind = a.bc_kind[c * ns + slot];
        if (a.v_is_half) v[c] = df_add_f(v[c], kick);
        if (a.mode == MODE_STEP) {
            v[c] = df_add_f(v[c], kick);
            if (kind == PD_BC_VELOCITY) {
                v[c] = DF{a.bc32[2 * (size_t)(c * ns + slot)], a.bc32[2 * (size_t)(c * ns + slot) + 1]};
                u[c] = df_add(u[c], df_mul(DF{a.dt_h, a.dt_l}, v[c]));
            } else if (kind == PD_BC_DISPLACEMENT) {
                v[c] = DF{0.f, 0.f};
                u[c] = DF{a.bc32[2 * (size_t)(c * ns + slot)], a.bc32[2 * (size_t)(c * ns + slot) + 1]};
            } else {
                u[c] = df_add(u[c], df_mul(DF{a.dt_h, a.dt_l}, v[c]));
            }
        } else {
            if (kind == PD_BC_VELOCITY)
                v[c] = DF{a.bc32[2 * (size_t)(c * ns + slot)], a.bc32[2 * (size_t)(c * ns + slot) + 1]};
            else if (kind == PD_BC_DISPLACEMENT)
                v[c] = DF{0.f, 0.f};
        }
    }
    a.vhl[2 * slot] = make_float4(v[0].h, v[1].h, v[2].h, 0.f);
    a.vhl[2 * slot + 1] = make_float4(v[0].l, v[1].l, v[2].l, 0.f);
    if (a.mode == MODE_STEP) {
        a.dst_hl[2 * slot] = make_float4(u[0].h, u[1].h, u[2].h, 0.f);
        a.dst_hl[2 * slot + 1] = make_float4(u[0].l, u[1].l, u[2].l, 0.f);
    }
}

}  // namespace pdk
