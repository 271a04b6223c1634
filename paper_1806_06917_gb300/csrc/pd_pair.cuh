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
// State. In the FP32C mode the integrator state u, v is FP64 (PD_STATE_F64:
// two FP64 additions and one FMA per component and step, everything else of the
// update on the integer and FP32 pipes, since GB300 runs FP64 at 1/64 of the
// FP32 rate) or double-float numbers (PD_STATE_DF: hi + lo, two FP32 values,
// about 48 significant bits, Knuth's two-sum and Dekker's product with an FMA,
// no FP64 instruction at all). Either keeps the accumulated rounding of a
// 1000-step run near 1e-12 relative, far below the 1e-4 tolerance on u.
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

// Single special-function-unit approximations (PTX .approx.ftz forms).
__device__ __forceinline__ float sfu_rsqrt(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sfu_sqrt(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sfu_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sfu_ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float2 f2rsqrt(float2 q) { return make_float2(sfu_rsqrt(q.x), sfu_rsqrt(q.y)); }
__device__ __forceinline__ float2 f2ex2(float2 q) { return make_float2(sfu_ex2(q.x), sfu_ex2(q.y)); }
__device__ __forceinline__ float2 f2sqrt(float2 q) { return make_float2(sfu_sqrt(q.x), sfu_sqrt(q.y)); }
__device__ __forceinline__ float2 f2rcp(float2 q) { return make_float2(sfu_rcp(q.x), sfu_rcp(q.y)); }
__device__ __forceinline__ float2 f2div(float2 a, float2 b) { return f2mul(a, f2rcp(b)); }
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

// q = floor(b / d) for 0 <= b < 2^16 and 1 <= d <= 2^10 by a float product: b + 1/2
// lies at least 1/(2d) from a multiple of d, more than the product's error
// (b/d relative 2^-23), so truncation gives the exact quotient without an
// integer division sequence.
__device__ __forceinline__ int fdiv_small(int b, float inv_d) { return (int)(((float)b + 0.5f) * inv_d); }

// Coordinates of the two points of pair-box index b (b < 2^16).
__device__ __forceinline__ void pair_coords(const Geom &g, const PairBox &pb, const int4 &org, int b, int cA[3],
                                            int cB[3])
{
    const int rest = fdiv_small(b, __frcp_rn((float)pb.HX)), bxl = b - rest * pb.HX;
    const int bzl = fdiv_small(rest, __frcp_rn((float)pb.HY)), byl = rest - bzl * pb.HY;
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

// Load the tile's 3^d neighbour tiles (and, with them, the per-CTA tables) into
// shared memory; call before __syncthreads.
__device__ __forceinline__ void load_nbr(const TileArgs &a, int tile, int *s_nbr)
{
    if (a.nbr_ok)
        for (int k = threadIdx.x; k < 27; k += blockDim.x) s_nbr[k] = __ldg(&a.tile_nbr[27 * tile + k]);
}

// Slot of (x, y, z) through the neighbour-tile table (no global lookup), or -1.
__device__ __forceinline__ int slot_nbr(const Geom &g, const int *s_nbr, const int4 &org, int x, int y, int z)
{
    if ((unsigned)x >= (unsigned)g.nx || (unsigned)y >= (unsigned)g.ny || (unsigned)z >= (unsigned)g.nz)
        return -1;
    const int dtx = (x >> g.lbx) - (org.x >> g.lbx), dty = (y >> g.lby) - (org.y >> g.lby);
    const int dtz = (z >> g.lbz) - (org.z >> g.lbz);
    const int t = s_nbr[(dtx + 1) + 3 * (dty + 1) + 9 * (dtz + 1)];
    return t * g.T + brick_code(g.dim, x & (g.bx - 1), y & (g.by - 1), z & (g.bz - 1));
}

__device__ __forceinline__ int slot_of(const TileArgs &a, const int *s_nbr, const int4 &org, const int c[3])
{
    return a.nbr_ok ? slot_nbr(a.g, s_nbr, org, c[0], c[1], c[2]) : slot_at(a.g, a.tile_lut, c[0], c[1], c[2]);
}

// Whether the tile at org may take its staging slots from a.box_map: the map
// exists (the halo reaches one tile at most) and every neighbour tile of this
// one is whole or absent, so that a point of the box is off the grid exactly
// when its neighbour tile is absent.
__device__ __forceinline__ bool box_mapped(const TileArgs &a, const int4 &org)
{
    return a.box_map && org.x <= a.box_edge[0] && org.y <= a.box_edge[1] && org.z <= a.box_edge[2];
}

// Slots of the two points of a box-map entry e (or -1 off the grid).
__device__ __forceinline__ void map_slots(const TileArgs &a, const int *s_nbr, uint32_t e, int &sA, int &sB)
{
    const int tA = s_nbr[e & 31u], tB = s_nbr[(e >> 14) & 31u];
    sA = tA < 0 ? -1 : tA * a.g.T + (int)((e >> 5) & 511u);
    sB = tB < 0 ? -1 : tB * a.g.T + (int)((e >> 19) & 511u);
}

// Call body(b, sA, sB) for every pair-box entry b of this thread (b = threadIdx.x
// + k blockDim.x), with the slots of its two points (-1 off the grid). With
// mapped (CTA-uniform) the slots come from the box map, whose first NR entries
// of the thread are all loaded before the first is used (one memory round trip
// instead of one per entry); otherwise from the entry's coordinates.
template <int NR, class Body>
__device__ __forceinline__ void for_pair_slots(const TileArgs &a, const PairBox &pb, const int4 &org,
                                               const int *s_nbr, bool mapped, Body body)
{
    if (mapped) {
        uint32_t e[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            const int b = threadIdx.x + k * blockDim.x;
            e[k] = b < pb.n ? __ldg(&a.box_map[b]) : 0u;
        }
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            const int b = threadIdx.x + k * blockDim.x;
            if (b < pb.n) {
                int sA, sB;
                map_slots(a, s_nbr, e[k], sA, sB);
                body(b, sA, sB);
            }
        }
        for (int b = threadIdx.x + NR * blockDim.x; b < pb.n; b += blockDim.x) {
            int sA, sB;
            map_slots(a, s_nbr, __ldg(&a.box_map[b]), sA, sB);
            body(b, sA, sB);
        }
        return;
    }
#pragma unroll 2
    for (int b = threadIdx.x; b < pb.n; b += blockDim.x) {
        int cA[3], cB[3];
        pair_coords(a.g, pb, org, b, cA, cB);
        body(b, slot_of(a, s_nbr, org, cA), slot_of(a, s_nbr, org, cB));
    }
}

// Stage the paired box of displacements: P4[b] = {xA, xB, yA, yB}, P2[b] = {zA, zB}.
// s_nbr must be loaded and visible (a __syncthreads after load_nbr). use_map
// takes the slots from the box map where it holds: fewer instructions per entry,
// which pays where many waves of tiles keep the SMs issue-bound (128^3 LPS step
// 0.646 -> 0.614 ms with the LPS prefetch; 256^3 PMB step 2.544 -> 2.420 ms) and
// changes nothing in the one-wave 64^3 PMB step, whose staging waits on memory
// more than it issues. The coordinate loop is kept apart from for_pair_slots:
// through it the 2D NP kernel (443^2, m = 20, no map) measured 1 % slower.
__device__ __forceinline__ void stage_pairs(const TileArgs &a, const PairBox &pb, const int4 &org, int tile,
                                            const int *s_nbr, float4 *P4, float2 *P2, bool use_map)
{
    const Ref32 ref = tile_ref32(a, tile);
    const float inv_h = (float)a.inv_h;
    if (use_map && box_mapped(a, org)) {
        for_pair_slots<8>(a, pb, org, s_nbr, true, [&](int b, int sA, int sB) {
            const float4 rA = stage_one(a, a.src_hl, sA, ref, inv_h);
            const float4 rB = stage_one(a, a.src_hl, sB, ref, inv_h);
            P4[b] = make_float4(rA.x, rB.x, rA.y, rB.y);
            if (P2) P2[b] = make_float2(rA.z, rB.z);
        });
        return;
    }
#pragma unroll 2
    for (int b = threadIdx.x; b < pb.n; b += blockDim.x) {
        int cA[3], cB[3];
        pair_coords(a.g, pb, org, b, cA, cB);
        const float4 rA = stage_one(a, a.src_hl, slot_of(a, s_nbr, org, cA), ref, inv_h);
        const float4 rB = stage_one(a, a.src_hl, slot_of(a, s_nbr, org, cB), ref, inv_h);
        P4[b] = make_float4(rA.x, rB.x, rA.y, rB.y);
        if (P2) P2[b] = make_float2(rA.z, rB.z);
    }
}

// Bulk L2 prefetch of one byte range by the copy engine (cp.async.bulk.prefetch:
// no registers, nothing to wait for); ranges that are not 16-byte aligned in
// address and size are skipped. Callers pass ranges inside allocated arrays.
__device__ __forceinline__ void l2_prefetch(const void *p, uint32_t bytes)
{
    if (bytes && (((uintptr_t)p | bytes) & 15u) == 0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Bulk L2 prefetches of one tile's own slots [tile T, (tile + 1) T) of arrays
// that an LPS pass reads long after its staging loads (each range contiguous),
// issued by one thread so that those loads hit L2 when they come. The bond masks
// at the pass's start (the bond loop follows the staging); the update's state
// (FP64 u and v, or the double-float velocity, the boundary kinds, the body
// force, u^{k-1}) once the staging is done: issued at the start, beside the
// staging's own loads, the FP64 u and v measured slower (128^3 LPS step 0.596
// against 0.588 ms); after the staging, 0.568 -> 0.559 ms. The PMB and NP
// kernels measured no gain from the mask prefetch (64^3) or a 1 % loss (443^2,
// m = 20: 40 mask words per point) and do not issue it.
__device__ __forceinline__ void prefetch_tile_masks(const TileArgs &a, int tile)
{
    const uint32_t T = (uint32_t)a.g.T;
    const size_t ns = a.g.nslots, s0 = (size_t)tile * T;
    for (int w = 0; w < a.g.W; ++w) l2_prefetch(a.mask + w * ns + s0, 4 * T);
}

__device__ __forceinline__ void prefetch_tile_update(const TileArgs &a, int tile)
{
    if (a.mode == MODE_FORCE) return;
    const uint32_t T = (uint32_t)a.g.T;
    const size_t ns = a.g.nslots, s0 = (size_t)tile * T;
    if (a.state64)
        for (int c = 0; c < a.g.dim; ++c) {
            if (a.mode == MODE_STEP) l2_prefetch(a.u[c] + s0, 8 * T);
            l2_prefetch(a.v[c] + s0, 8 * T);
        }
    if (a.vhl) l2_prefetch(a.vhl + 2 * s0, 32 * T);
    for (int c = 0; c < a.g.dim; ++c) l2_prefetch(a.bc_kind + c * ns + s0, T);
    if (a.use_body && a.body32) l2_prefetch(a.body32 + s0, 16 * T);
    if (a.mode == MODE_STEP && a.cd && a.dst_hl) l2_prefetch(a.dst_hl + 2 * s0, 32 * T);
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

// The fused update with FP64 integrator state (PD_STATE_F64): u and v live in
// the FP64 component arrays a.u[c], a.v[c]. The kick dt/2 (f + b)/rho is formed
// in FP32 from the FP32 force, as in the double-float form, and added to v in
// FP64: from a half-step velocity, the previous step's second half-kick and this
// step's first (the same kick) as one add of 2 kick, the leapfrog form of Eq.
// (9); from a full-step velocity (a first step, or after MODE_FINALIZE) one
// kick; MODE_FINALIZE adds the pending half-kick alone. The drift
// u += dt v is one FP64 FMA; the next staging pair is u split into FP32 hi + lo
// (split_bits). Central difference (Eq. (10)) reads u^{k-1} from the staging
// pair it overwrites. One point at a time, its loads issued together (the
// FP64 values of both points at once would not fit beside the bond loop's
// registers).
__device__ __forceinline__ void point_update64(const TileArgs &a, int slot, const float F[3], int dim)
{
    const int ns = a.g.nslots;
    const bool step = a.mode == MODE_STEP, cd = step && a.cd;
    double v[3], u[3];
    int kind[3];
    const float4 bb = a.use_body ? a.body32[slot] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 uph = make_float4(0.f, 0.f, 0.f, 0.f), upl = uph;
    if (cd) {
        uph = a.dst_hl[2 * slot];
        upl = a.dst_hl[2 * slot + 1];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        v[c] = c < dim ? a.v[c][slot] : 0.0;
        u[c] = c < dim && step ? a.u[c][slot] : 0.0;
        kind[c] = c < dim ? a.bc_kind[c * ns + slot] : 0;
    }
    const float bcomp[3] = {bb.x, bb.y, bb.z};
    const float uphc[3] = {uph.x, uph.y, uph.z}, uplc[3] = {upl.x, upl.y, upl.z};
    float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (c >= dim) break;
        const float kick = fmaf(a.kF, F[c], a.kB * bcomp[c]);
        const double kd = f2d_bits(kick);
        double vc = v[c], uc = u[c];
        // the previous step's second half-kick and this step's first are the same
        // kick: one add of 2 kick (exact) from the half-step velocity, the leapfrog
        // form of Eq. (9), one rounding instead of two
        if (step && a.v_is_half) vc += 2.0 * kd;
        else if (a.v_is_half || step) vc += kd;
        if (step) {
            if (kind[c] == PD_BC_VELOCITY) {
                vc = a.bc_val[c * ns + slot];
                uc = fma(a.dt, vc, uc);
            } else if (kind[c] == PD_BC_DISPLACEMENT) {
                vc = 0.0;
                uc = a.bc_val[c * ns + slot];
            } else if (cd) {
                // u + (u - u^{k-1}) + dt^2 a^k, dt^2 a^k = 2 dt kick
                const double up = f2d_bits(uphc[c]) + f2d_bits(uplc[c]);
                uc = fma(a.dt, f2d_bits(2.f * kick), uc + (uc - up));
            } else {
                uc = fma(a.dt, vc, uc);
            }
            a.u[c][slot] = uc;
            split_bits(uc, hi[c], lo[c]);
        } else {
            if (kind[c] == PD_BC_VELOCITY) vc = a.bc_val[c * ns + slot];
            else if (kind[c] == PD_BC_DISPLACEMENT) vc = 0.0;
        }
        a.v[c][slot] = vc;
    }
    if (step) {
        a.dst_hl[2 * slot] = make_float4(hi[0], hi[1], hi[2], 0.f);
        a.dst_hl[2 * slot + 1] = make_float4(lo[0], lo[1], lo[2], 0.f);
    }
}

// Velocity-Verlet update of the thread's two points in double-float arithmetic
// from their forces F (FP32, in the kernel's units): the kick is kF * F (+ kB * b)
// with kF = dt/2 * (force scale)/rho and kB = dt/2/rho. MODE_STEP applies the
// second half-kick of the previous step (if v holds a half step), the first
// half-kick of this step, the drift u += dt v with boundary conditions, and
// writes u to the next staging buffer; MODE_FINALIZE applies only the pending
// half-kick; MODE_FORCE stores f = (force scale) * F in FP64. With a.cd set the
// drift of a free DOF is the central difference of Eq. (10) instead,
// u^{k+1} = u^k + (u^k - u^{k-1}) + dt^2 a^k with dt^2 a^k = 2 dt kick, and
// u^{k-1} read from the staging buffer it overwrites. Every other load of both
// points is issued before the arithmetic, so the two points share one memory
// round trip.
__device__ __forceinline__ void pair_epilogue2(const TileArgs &a, const PairPts &q, const float FA[3],
                                               const float FB[3], int dim)
{
    const int ns = a.g.nslots;
    if (a.mode == MODE_FORCE) {
        for (int p = 0; p < 2; ++p) {
            if (!q.act[p]) continue;
            const float *F = p ? FB : FA;
            for (int c = 0; c < dim; ++c) a.f[c][q.slot[p]] = a.fscale * (double)F[c];
        }
        return;
    }
    if (a.state64) {
        if (q.act[0]) point_update64(a, q.slot[0], FA, dim);
        if (q.act[1]) point_update64(a, q.slot[1], FB, dim);
        return;
    }
    float4 vh[2], vl[2], uh[2], ul[2], bb[2];
    int kind[2][3];
    const bool cd = a.mode == MODE_STEP && a.cd;
    for (int p = 0; p < 2; ++p) {
        const int s = q.act[p] ? q.slot[p] : q.slot[0];
        vh[p] = a.vhl[2 * s];
        vl[p] = a.vhl[2 * s + 1];
        uh[p] = a.src_hl[2 * s];
        ul[p] = a.src_hl[2 * s + 1];
        bb[p] = a.use_body ? a.body32[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int c = 0; c < 3; ++c) kind[p][c] = c < dim ? a.bc_kind[c * ns + s] : 0;
    }
    for (int p = 0; p < 2; ++p) {
        if (!q.act[p]) continue;
        const int slot = q.slot[p];
        const float *F = p ? FB : FA;
        DF v[3] = {{vh[p].x, vl[p].x}, {vh[p].y, vl[p].y}, {vh[p].z, vl[p].z}};
        DF u[3] = {{uh[p].x, ul[p].x}, {uh[p].y, ul[p].y}, {uh[p].z, ul[p].z}};
        const float bcomp[3] = {bb[p].x, bb[p].y, bb[p].z};
        DF up[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        if (cd) {   // -u^{k-1}, loaded here only under central difference
            const float4 ph = a.dst_hl[2 * slot], pl = a.dst_hl[2 * slot + 1];
            up[0] = DF{-ph.x, -pl.x};
            up[1] = DF{-ph.y, -pl.y};
            up[2] = DF{-ph.z, -pl.z};
        }
        for (int c = 0; c < dim; ++c) {
            const float kick = fmaf(a.kF, F[c], a.kB * bcomp[c]);
            const int kd = kind[p][c];
            if (a.v_is_half) v[c] = df_add_f(v[c], kick);
            const size_t bq = 2 * (size_t)(c * ns + slot);
            if (a.mode == MODE_STEP) {
                v[c] = df_add_f(v[c], kick);
                if (kd == PD_BC_VELOCITY) {
                    v[c] = DF{a.bc32[bq], a.bc32[bq + 1]};
                    u[c] = df_add(u[c], df_mul(DF{a.dt_h, a.dt_l}, v[c]));
                } else if (kd == PD_BC_DISPLACEMENT) {
                    v[c] = DF{0.f, 0.f};
                    u[c] = DF{a.bc32[bq], a.bc32[bq + 1]};
                } else if (cd) {
                    const DF du = df_add(u[c], up[c]);
                    u[c] = df_add(u[c], df_add(du, df_mul(DF{a.dt_h, a.dt_l}, DF{2.f * kick, 0.f})));
                } else {
                    u[c] = df_add(u[c], df_mul(DF{a.dt_h, a.dt_l}, v[c]));
                }
            } else {
                if (kd == PD_BC_VELOCITY) v[c] = DF{a.bc32[bq], a.bc32[bq + 1]};
                else if (kd == PD_BC_DISPLACEMENT) v[c] = DF{0.f, 0.f};
            }
        }
        a.vhl[2 * slot] = make_float4(v[0].h, v[1].h, v[2].h, 0.f);
        a.vhl[2 * slot + 1] = make_float4(v[0].l, v[1].l, v[2].l, 0.f);
        if (a.mode == MODE_STEP) {
            a.dst_hl[2 * slot] = make_float4(u[0].h, u[1].h, u[2].h, 0.f);
            a.dst_hl[2 * slot + 1] = make_float4(u[0].l, u[1].l, u[2].l, 0.f);
        }
    }
}

}  // namespace pdk
