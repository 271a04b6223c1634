// pd_lps_fast.cuh -- the FP32C state-based (LPS) passes of one tile: the
// dilatation pass and the force pass fused with the update (Eq. (4),
// Algorithm 2; Eqs. (7)-(9)). The bodies are shared by the kernels of
// pd_force_lps.cu and the request server's packed kernel (pd_packed.cu).
//
// In lattice units (xi = d, e~ = e / h, m~ = m / (h^2 V), omega = 1):
//   e~      = (2 d.eta + eta.eta) / (|y| + |d|)          cancellation-free extension
//   theta_i = (3 / m~_i) sum_j |d| e~ V_ij                Algorithm 2, second loop
//   f_i     = (1/h) sum_j [ (3K - 5mu) |d| (a_i + a_j) + 15 mu e~ (b_i + b_j) ] V_ij y/|y|
// with a = theta / m~, b = 1 / m~. The bracket is t_i<xi> + t_j<-xi> of Algorithm
// 2's third loop (t = 3K theta |xi| / m + 15 mu e^d / m, e^d = e - theta |xi| / 3)
// gathered at i: the "f_j -= t M V_i" scatter of row j lands on i as + t_j M_ij.
#pragma once

#include "pd_pair.cuh"

namespace pdk {

// ------------------------------------------------------------------ fast path

// FP32C, 3D, thread = point pair (A, B) in f32x2 arithmetic (pd_pair.cuh);
// rolled loop over a shared-memory table of pre-splatted stencil constants.
// One 32-bond word of the dilatation sum (MASKED = false: every bond of the
// warp's points exists and is intact, no per-bond mask operation).
// The table is the dilatation's: {2dx,2dx,2dy,2dy} {2dz,2dz,|d|,|d|} {|d|^2,|d|^2,offset,V_ij}:
// the extension needs 2 d.e + e.e = e.(e + 2d) and |y|, not y itself; the bond
// weight |d| V_ij is |d| itself without the partial volume (VOLCORR = false).
template <bool MASKED, bool VOLCORR>
__device__ __forceinline__ float2 lps_dil_word(const float4 *tw, int nb, const float4 *P4, const float2 *P2, int bi,
                                               float2 nux, float2 nuy, float2 nuz, uint32_t c0, uint32_t c1,
                                               float2 acc)
{
PD_PRAGMA_UNROLL(PD_UNROLL)
    for (int b = 0; b < nb; ++b) {
        const float4 ta = tw[3 * b], tb = tw[3 * b + 1], tc = tw[3 * b + 2];
        const int off = __float_as_int(tc.z);
        const float4 r4 = P4[bi + off];
        const float2 ex = f2add(f2lo(r4), nux), ey = f2add(f2hi(r4), nuy), ez = f2add(P2[bi + off], nuz);
        float2 num = f2mul(ex, f2add(ex, f2lo(ta)));
        num = f2fma(ey, f2add(ey, f2hi(ta)), num);
        num = f2fma(ez, f2add(ez, f2lo(tb)), num);
        const float2 qq = f2add(num, f2lo(tc));            // |y|^2 = |d|^2 + 2 d.e + e.e
        float2 e = f2mul(num, f2rcp(f2add(f2sqrt(qq), f2hi(tb))));
        if (MASKED) {
            e.x = ((c0 >> b) & 1u) ? e.x : 0.f;
            e.y = ((c1 >> b) & 1u) ? e.y : 0.f;
        }
        if (VOLCORR) e = f2mul(e, make_float2(tc.w, tc.w));
        acc = f2fma(e, f2hi(tb), acc);
    }
    return acc;
}

// Unroll depth of the force pass's bond loop: 8 measured 0.3569 ms per 128^3
// pass against 0.3598-0.3600 ms for 4 and 0.3680 ms for 2.
#ifndef PD_FORCE_UNROLL
#define PD_FORCE_UNROLL 8
#endif

// One 32-bond word of the LPS force sum. The staged a = (3K - 5mu) theta / m~ and
// b = 15 mu / m~ carry the moduli, so the bond weight is
//   (t_i + t_j) V_ij / |y| = (|d| (a_i + a_j) + e (b_i + b_j)) V_ij / |y|
// (VOLCORR = false: V_ij = 1, no multiply).
template <bool MASKED, bool VOLCORR>
__device__ __forceinline__ void lps_force_word(const float4 *tw, int nb, const float4 *P4, const float4 *PT,
                                               const float2 *P2, int bi, float2 nux, float2 nuy, float2 nuz,
                                               float2 ai, float2 bi_, uint32_t c0, uint32_t c1, float2 &Fx,
                                               float2 &Fy, float2 &Fz)
{
PD_PRAGMA_UNROLL(PD_FORCE_UNROLL)
    for (int b = 0; b < nb; ++b) {
        // table entry: {dx,dx,dy,dy} {dz,dz,|d|,|d|} {|d|^2,|d|^2,offset,V_ij}
        const float4 ta = tw[3 * b], tb = tw[3 * b + 1], td = tw[3 * b + 2];
        const int off = __float_as_int(td.z);
        const float4 r4 = P4[bi + off], t4 = PT[bi + off];
        const float2 ex = f2add(f2lo(r4), nux), ey = f2add(f2hi(r4), nuy), ez = f2add(P2[bi + off], nuz);
        const float2 yx = f2add(ex, f2lo(ta)), yy = f2add(ey, f2hi(ta)), yz = f2add(ez, f2lo(tb));
        float2 num = f2mul(ex, f2add(yx, f2lo(ta)));
        num = f2fma(ey, f2add(yy, f2hi(ta)), num);
        num = f2fma(ez, f2add(yz, f2lo(tb)), num);
        const float2 qq = f2add(num, f2lo(td));            // |y|^2 = |d|^2 + 2 d.e + e.e
        const float2 rs = f2rsqrt(qq);
        const float2 e = f2mul(num, f2rcp(f2add(f2mul(qq, rs), f2hi(tb))));
        float2 gg = f2mul(f2hi(tb), f2add(ai, f2lo(t4)));
        gg = f2fma(e, f2add(bi_, f2hi(t4)), gg);
        if (VOLCORR) gg = f2mul(gg, make_float2(td.w, td.w));
        float2 wgt = f2mul(gg, rs);
        if (MASKED) {
            wgt.x = ((c0 >> b) & 1u) ? wgt.x : 0.f;
            wgt.y = ((c1 >> b) & 1u) ? wgt.y : 0.f;
        }
        Fx = f2fma(wgt, yx, Fx);
        Fy = f2fma(wgt, yy, Fy);
        Fz = f2fma(wgt, yz, Fz);
    }
}

template <bool VOLCORR, bool PTAB>
__device__ __forceinline__ void lps_dil_fast_body(const TileArgs &a, int tile, const float4 *ptab)
{
    const Geom &g = a.g;
    const PairBox pb = pair_box(g);
    const int S = g.S;
    extern __shared__ float4 smem4[];
    float4 *P4 = smem4;
    float2 *P2 = reinterpret_cast<float2 *>(P4 + pb.n);
    float4 *tab = P4 + pb.n + (pb.n + 1) / 2;                  // 3 float4 per entry
    __shared__ int s_nbr[27];
    if (threadIdx.x == 0) prefetch_tile_masks(a, tile);
    const int4 org = __ldg(&a.tile_org[tile]);
    if (!PTAB)
        for (int k = threadIdx.x; k < 3 * S; k += blockDim.x) tab[k] = __ldg(&a.tab_a[k]);
    load_nbr(a, tile, s_nbr);
    __syncthreads();
    stage_pairs(a, pb, org, tile, s_nbr, P4, P2, true);
    __syncthreads();

    const int nthr = g.T / 2;            // a multiple of blockDim
    for (int t = threadIdx.x; t < nthr; t += blockDim.x) {
        const PairPts q = pair_points(g, pb, org, tile, t);
        const float4 ui4 = P4[q.bi];
        const float2 nux = f2neg(f2lo(ui4)), nuy = f2neg(f2hi(ui4)), nuz = f2neg(P2[q.bi]);
        float2 acc = make_float2(0.f, 0.f);
        uint32_t n0 = q.act[0] ? a.mask[q.slot[0]] : 0u;
        uint32_t n1 = q.act[1] ? a.mask[q.slot[1]] : 0u;
        for (int w = 0; w < g.W; ++w) {
            const uint32_t m0 = n0, m1 = n1;
            if (w + 1 < g.W) {
                const size_t mo = (size_t)(w + 1) * g.nslots;
                n0 = q.act[0] ? a.mask[mo + q.slot[0]] : 0u;
                n1 = q.act[1] ? a.mask[mo + q.slot[1]] : 0u;
            }
            const int nb = min(32, S - 32 * w);
            const uint32_t full = nb == 32 ? 0xffffffffu : ((1u << nb) - 1u);
            const float4 *tw = (PTAB ? ptab : tab) + 3 * 32 * w;
            if (__all_sync(0xffffffffu, m0 == full && m1 == full))
                acc = lps_dil_word<false, VOLCORR>(tw, nb, P4, P2, q.bi, nux, nuy, nuz, m0, m1, acc);
            else
                acc = lps_dil_word<true, VOLCORR>(tw, nb, P4, P2, q.bi, nux, nuy, nuz, m0, m1, acc);
        }
        for (int p = 0; p < 2; ++p)
            if (q.act[p]) a.theta32[q.slot[p]] = 3.f * __ldg(&a.minv32[q.slot[p]]) * (p ? acc.y : acc.x);
    }
}

// Dilatation with two point pairs per thread: pairs t and t + T/4 (2 z-layers
// apart in the box, the constant offset dbi), so every table entry read from
// shared memory serves four points; the CTA's two thread halves sum the two
// halves of the stencil words, added in a fixed order (half 0 + half 1). The
// one-pair kernel is bound by the L1 / shared-memory pipe (ncu: 92 % of its
// throughput, 14 wavefronts per 64 bonds, 7 of them table broadcasts); this
// form moves 19 per 128. The dilatation table has 3 float4 per entry (from 4:
// the 128^3 LPS step 0.614 -> 0.611 ms).
// Unroll depth of the two-pair dilatation's bond loop and its CTAs per SM:
// built for 3 CTAs per SM (80 registers, no spills) it measured 0.2176 ms per
// 128^3 pass against 0.2215 ms for 4 (64 registers, 36 bytes of spills);
// unrolled by 2 or 8 at 4 CTAs, 0.2179 and 0.2193 ms.
#ifndef PD_DIL2_UNROLL
#define PD_DIL2_UNROLL 4
#endif
#ifndef PD_DIL2_MINBLOCKS
#define PD_DIL2_MINBLOCKS 3
#endif

template <bool MASKED, bool VOLCORR>
__device__ __forceinline__ void lps_dil_word2(const float4 *tw, int nb, const float4 *P4, const float2 *P2, int bi,
                                              int dbi, float2 nux0, float2 nuy0, float2 nuz0, float2 nux1,
                                              float2 nuy1, float2 nuz1, uint32_t c0, uint32_t c1, uint32_t c2,
                                              uint32_t c3, float2 &acc0, float2 &acc1)
{
PD_PRAGMA_UNROLL(PD_DIL2_UNROLL)
    for (int b = 0; b < nb; ++b) {
        const float4 ta = tw[3 * b], tb = tw[3 * b + 1], tc = tw[3 * b + 2];
        const int off = __float_as_int(tc.z);
        const float4 r0 = P4[bi + off], r1 = P4[bi + dbi + off];
        const float2 z0 = P2[bi + off], z1 = P2[bi + dbi + off];
        float2 e0, e1;
        {
            const float2 ex = f2add(f2lo(r0), nux0), ey = f2add(f2hi(r0), nuy0), ez = f2add(z0, nuz0);
            float2 num = f2mul(ex, f2add(ex, f2lo(ta)));
            num = f2fma(ey, f2add(ey, f2hi(ta)), num);
            num = f2fma(ez, f2add(ez, f2lo(tb)), num);
            e0 = f2mul(num, f2rcp(f2add(f2sqrt(f2add(num, f2lo(tc))), f2hi(tb))));
        }
        {
            const float2 ex = f2add(f2lo(r1), nux1), ey = f2add(f2hi(r1), nuy1), ez = f2add(z1, nuz1);
            float2 num = f2mul(ex, f2add(ex, f2lo(ta)));
            num = f2fma(ey, f2add(ey, f2hi(ta)), num);
            num = f2fma(ez, f2add(ez, f2lo(tb)), num);
            e1 = f2mul(num, f2rcp(f2add(f2sqrt(f2add(num, f2lo(tc))), f2hi(tb))));
        }
        if (MASKED) {
            e0.x = ((c0 >> b) & 1u) ? e0.x : 0.f;
            e0.y = ((c1 >> b) & 1u) ? e0.y : 0.f;
            e1.x = ((c2 >> b) & 1u) ? e1.x : 0.f;
            e1.y = ((c3 >> b) & 1u) ? e1.y : 0.f;
        }
        if (VOLCORR) {
            e0 = f2mul(e0, make_float2(tc.w, tc.w));
            e1 = f2mul(e1, make_float2(tc.w, tc.w));
        }
        acc0 = f2fma(e0, f2hi(tb), acc0);
        acc1 = f2fma(e1, f2hi(tb), acc1);
    }
}

// Launch: one CTA per tile, T/2 threads (tiles of at least 2^7 points and two
// stencil words).
template <bool VOLCORR, bool PTAB>
__device__ __forceinline__ void lps_dil_fast2_body(const TileArgs &a, int tile, const float4 *ptab)
{
    const Geom &g = a.g;
    const PairBox pb = pair_box(g);
    const int S = g.S;
    extern __shared__ float4 smem4[];
    float4 *P4 = smem4;
    float2 *P2 = reinterpret_cast<float2 *>(P4 + pb.n);
    float4 *tab = P4 + pb.n + (pb.n + 1) / 2;                  // 3 float4 per entry
    __shared__ int s_nbr[27];
    if (threadIdx.x == 0) prefetch_tile_masks(a, tile);
    const int4 org = __ldg(&a.tile_org[tile]);
    if (!PTAB)
        for (int k = threadIdx.x; k < 3 * S; k += blockDim.x) tab[k] = __ldg(&a.tab_a[k]);
    load_nbr(a, tile, s_nbr);
    __syncthreads();
    stage_pairs(a, pb, org, tile, s_nbr, P4, P2, true);
    __syncthreads();
    // 1/m~ of the tile's points, read by the epilogue (128^3 LPS pass 0.2167 -> 0.2151 ms)
    if (threadIdx.x == 0) l2_prefetch(a.minv32 + (size_t)tile * g.T, 4 * g.T);

    const int nthr = g.T / 4;                                  // a multiple of 32
    const int half = threadIdx.x >= nthr, t = threadIdx.x - half * nthr;
    const int wsplit = (g.W + 1) / 2;
    const int w0 = half ? wsplit : 0, w1 = half ? g.W : wsplit;
    const PairPts q0 = pair_points(g, pb, org, tile, t), q1 = pair_points(g, pb, org, tile, t + nthr);
    const int dbi = q1.bi - q0.bi;
    float2 acc0 = make_float2(0.f, 0.f), acc1 = acc0;
    {
        const float4 u0 = P4[q0.bi], u1 = P4[q1.bi];
        const float2 nux0 = f2neg(f2lo(u0)), nuy0 = f2neg(f2hi(u0)), nuz0 = f2neg(P2[q0.bi]);
        const float2 nux1 = f2neg(f2lo(u1)), nuy1 = f2neg(f2hi(u1)), nuz1 = f2neg(P2[q1.bi]);
        const size_t mo0 = (size_t)w0 * g.nslots;
        uint32_t n0 = q0.act[0] && w0 < w1 ? a.mask[mo0 + q0.slot[0]] : 0u;
        uint32_t n1 = q0.act[1] && w0 < w1 ? a.mask[mo0 + q0.slot[1]] : 0u;
        uint32_t n2 = q1.act[0] && w0 < w1 ? a.mask[mo0 + q1.slot[0]] : 0u;
        uint32_t n3 = q1.act[1] && w0 < w1 ? a.mask[mo0 + q1.slot[1]] : 0u;
        for (int w = w0; w < w1; ++w) {
            const uint32_t m0 = n0, m1 = n1, m2 = n2, m3 = n3;
            if (w + 1 < w1) {
                const size_t mo = (size_t)(w + 1) * g.nslots;
                n0 = q0.act[0] ? a.mask[mo + q0.slot[0]] : 0u;
                n1 = q0.act[1] ? a.mask[mo + q0.slot[1]] : 0u;
                n2 = q1.act[0] ? a.mask[mo + q1.slot[0]] : 0u;
                n3 = q1.act[1] ? a.mask[mo + q1.slot[1]] : 0u;
            }
            const int nb = min(32, S - 32 * w);
            const uint32_t full = nb == 32 ? 0xffffffffu : ((1u << nb) - 1u);
            const float4 *tw = (PTAB ? ptab : tab) + 3 * 32 * w;
            if (__all_sync(0xffffffffu, m0 == full && m1 == full && m2 == full && m3 == full))
                lps_dil_word2<false, VOLCORR>(tw, nb, P4, P2, q0.bi, dbi, nux0, nuy0, nuz0, nux1, nuy1, nuz1, m0,
                                              m1, m2, m3, acc0, acc1);
            else
                lps_dil_word2<true, VOLCORR>(tw, nb, P4, P2, q0.bi, dbi, nux0, nuy0, nuz0, nux1, nuy1, nuz1, m0,
                                             m1, m2, m3, acc0, acc1);
        }
    }
    // combine the halves: half 1 publishes, half 0 adds and writes theta
    __syncthreads();
    float2 *ex = reinterpret_cast<float2 *>(smem4);            // reuses the staged box
    if (half) {
        ex[2 * t] = acc0;
        ex[2 * t + 1] = acc1;
    }
    __syncthreads();
    if (!half) {
        acc0 = f2add(acc0, ex[2 * t]);
        acc1 = f2add(acc1, ex[2 * t + 1]);
        for (int p = 0; p < 2; ++p) {
            if (q0.act[p]) a.theta32[q0.slot[p]] = 3.f * __ldg(&a.minv32[q0.slot[p]]) * (p ? acc0.y : acc0.x);
            if (q1.act[p]) a.theta32[q1.slot[p]] = 3.f * __ldg(&a.minv32[q1.slot[p]]) * (p ? acc1.y : acc1.x);
        }
    }
}

// The force pass needs 40 bytes of shared memory per point pair (u, and a, b of
// both points), which allows only two CTAs per SM. To keep 32 warps per SM it
// runs one thread per point (512 for a 2^9 tile): thread t of half h owns point
// pair t and sums the stencil words of its half; the two partial forces are
// added in a fixed order (half 0 + half 1) through shared memory before the
// update.
template <bool VOLCORR, bool PTAB>
__device__ __forceinline__ void lps_force_fast_body(const TileArgs &a, int tile, const float4 *ptab)
{
    const Geom &g = a.g;
    const PairBox pb = pair_box(g);
    const int S = g.S;
    extern __shared__ float4 smem4[];
    float4 *P4 = smem4;                                        // {xA, xB, yA, yB}
    float4 *PT = P4 + pb.n;                                     // {aA, aB, bA, bB}: a = theta/m~, b = 1/m~
    float2 *P2 = reinterpret_cast<float2 *>(PT + pb.n);        // {zA, zB}
    float4 *tab = PT + pb.n + (pb.n + 1) / 2;                  // 3 float4 per entry
    __shared__ int s_nbr[27];
    if (threadIdx.x == 0) prefetch_tile_masks(a, tile);
    const int4 org = __ldg(&a.tile_org[tile]);
    if (!PTAB)
        for (int k = threadIdx.x; k < 3 * S; k += blockDim.x) tab[k] = __ldg(&a.tab_b[k]);
    load_nbr(a, tile, s_nbr);
    __syncthreads();
    {
        const Ref32 ref = tile_ref32(a, tile);
        const float inv_h = (float)a.inv_h;
        const float kA = (float)a.A, kB = (float)a.B;           // 3K - 5mu, 15mu
        for_pair_slots<4>(a, pb, org, s_nbr, box_mapped(a, org), [&](int b, int sA, int sB) {
            const float4 rA = stage_one(a, a.src_hl, sA, ref, inv_h);
            const float4 rB = stage_one(a, a.src_hl, sB, ref, inv_h);
            const float mA = sA >= 0 ? __ldg(&a.minv32[sA]) : 0.f, mB = sB >= 0 ? __ldg(&a.minv32[sB]) : 0.f;
            // theta through L2 (ld.global.cg): in the request server's packed kernel
            // the dilatation items of the same launch write it
            const float aA = sA >= 0 ? kA * (__ldcg(&a.theta32[sA]) * mA) : 0.f;
            const float aB = sB >= 0 ? kA * (__ldcg(&a.theta32[sB]) * mB) : 0.f;
            P4[b] = make_float4(rA.x, rB.x, rA.y, rB.y);
            P2[b] = make_float2(rA.z, rB.z);
            PT[b] = make_float4(aA, aB, kB * mA, kB * mB);
        });
    }
    __syncthreads();
    if (threadIdx.x == 0) prefetch_tile_update(a, tile);

    const int np = g.T / 2;                                    // point pairs of the tile
    const int half = threadIdx.x >= np;
    const int t = threadIdx.x - half * np;
    const int wsplit = (g.W + 1) / 2;
    const int w0 = half ? wsplit : 0, w1 = half ? g.W : wsplit;
    // blockDim == g.T: one pair per thread of each half
    const PairPts q = pair_points(g, pb, org, tile, t);
    const float4 ui4 = P4[q.bi], ti4 = PT[q.bi];
    const float2 nux = f2neg(f2lo(ui4)), nuy = f2neg(f2hi(ui4)), nuz = f2neg(P2[q.bi]);
    const float2 ai = f2lo(ti4), bi = f2hi(ti4);
    float2 Fx = make_float2(0.f, 0.f), Fy = Fx, Fz = Fx;
    if (w0 < w1) {
        uint32_t n0 = q.act[0] ? a.mask[(size_t)w0 * g.nslots + q.slot[0]] : 0u;
        uint32_t n1 = q.act[1] ? a.mask[(size_t)w0 * g.nslots + q.slot[1]] : 0u;
        for (int w = w0; w < w1; ++w) {
            const uint32_t m0 = n0, m1 = n1;
            if (w + 1 < w1) {
                const size_t mo = (size_t)(w + 1) * g.nslots;
                n0 = q.act[0] ? a.mask[mo + q.slot[0]] : 0u;
                n1 = q.act[1] ? a.mask[mo + q.slot[1]] : 0u;
            }
            const int nb = min(32, S - 32 * w);
            const uint32_t full = nb == 32 ? 0xffffffffu : ((1u << nb) - 1u);
            const float4 *tw = (PTAB ? ptab : tab) + 3 * 32 * w;
            if (__all_sync(0xffffffffu, m0 == full && m1 == full))
                lps_force_word<false, VOLCORR>(tw, nb, P4, PT, P2, q.bi, nux, nuy, nuz, ai, bi, m0, m1, Fx, Fy, Fz);
            else
                lps_force_word<true, VOLCORR>(tw, nb, P4, PT, P2, q.bi, nux, nuy, nuz, ai, bi, m0, m1, Fx, Fy, Fz);
        }
    }
    // combine the halves: half 1 publishes its partial force, half 0 adds it
    __syncthreads();
    float2 *ex = reinterpret_cast<float2 *>(smem4);            // reuses the staged box
    if (half) {
        ex[3 * t] = Fx;
        ex[3 * t + 1] = Fy;
        ex[3 * t + 2] = Fz;
    }
    __syncthreads();
    if (!half) {
        Fx = f2add(Fx, ex[3 * t]);
        Fy = f2add(Fy, ex[3 * t + 1]);
        Fz = f2add(Fz, ex[3 * t + 2]);
        const float FA[3] = {Fx.x, Fy.x, Fz.x}, FB[3] = {Fx.y, Fy.y, Fz.y};
        pair_epilogue2(a, q, FA, FB, 3);
    }
}

// Dilatation with one point pair per thread and the stencil words split over
// the CTA's two thread halves (half 0 the first ceil(W/2) words, half 1 the
// rest), added in a fixed order (half 0 + half 1): per point the same sums in
// the same order as lps_dil_fast2, for a CTA of T threads (the request
// server's packed kernel, whose CTAs have the force pass's T threads).
template <bool VOLCORR, bool PTAB>
__device__ __forceinline__ void lps_dil_h2_body(const TileArgs &a, int tile, const float4 *ptab)
{
    const Geom &g = a.g;
    const PairBox pb = pair_box(g);
    const int S = g.S;
    extern __shared__ float4 smem4[];
    float4 *P4 = smem4;
    float2 *P2 = reinterpret_cast<float2 *>(P4 + pb.n);
    float4 *tab = P4 + pb.n + (pb.n + 1) / 2;                  // 3 float4 per entry
    __shared__ int s_nbr[27];
    if (threadIdx.x == 0) prefetch_tile_masks(a, tile);
    const int4 org = __ldg(&a.tile_org[tile]);
    if (!PTAB)
        for (int k = threadIdx.x; k < 3 * S; k += blockDim.x) tab[k] = __ldg(&a.tab_a[k]);
    load_nbr(a, tile, s_nbr);
    __syncthreads();
    stage_pairs(a, pb, org, tile, s_nbr, P4, P2, true);
    __syncthreads();
    if (threadIdx.x == 0) l2_prefetch(a.minv32 + (size_t)tile * g.T, 4 * g.T);

    const int np = g.T / 2;                                    // point pairs; blockDim == 2 np
    const int half = threadIdx.x >= np, t = threadIdx.x - half * np;
    const int wsplit = (g.W + 1) / 2;
    const int w0 = half ? wsplit : 0, w1 = half ? g.W : wsplit;
    const PairPts q = pair_points(g, pb, org, tile, t);
    float2 acc = make_float2(0.f, 0.f);
    {
        const float4 ui4 = P4[q.bi];
        const float2 nux = f2neg(f2lo(ui4)), nuy = f2neg(f2hi(ui4)), nuz = f2neg(P2[q.bi]);
        const size_t mo0 = (size_t)w0 * g.nslots;
        uint32_t n0 = q.act[0] && w0 < w1 ? a.mask[mo0 + q.slot[0]] : 0u;
        uint32_t n1 = q.act[1] && w0 < w1 ? a.mask[mo0 + q.slot[1]] : 0u;
        for (int w = w0; w < w1; ++w) {
            const uint32_t m0 = n0, m1 = n1;
            if (w + 1 < w1) {
                const size_t mo = (size_t)(w + 1) * g.nslots;
                n0 = q.act[0] ? a.mask[mo + q.slot[0]] : 0u;
                n1 = q.act[1] ? a.mask[mo + q.slot[1]] : 0u;
            }
            const int nb = min(32, S - 32 * w);
            const uint32_t full = nb == 32 ? 0xffffffffu : ((1u << nb) - 1u);
            const float4 *tw = (PTAB ? ptab : tab) + 3 * 32 * w;
            if (__all_sync(0xffffffffu, m0 == full && m1 == full))
                acc = lps_dil_word<false, VOLCORR>(tw, nb, P4, P2, q.bi, nux, nuy, nuz, m0, m1, acc);
            else
                acc = lps_dil_word<true, VOLCORR>(tw, nb, P4, P2, q.bi, nux, nuy, nuz, m0, m1, acc);
        }
    }
    __syncthreads();
    float2 *ex = reinterpret_cast<float2 *>(smem4);            // reuses the staged box
    if (half) ex[t] = acc;
    __syncthreads();
    if (!half) {
        acc = f2add(acc, ex[t]);
        for (int p = 0; p < 2; ++p)
            if (q.act[p]) a.theta32[q.slot[p]] = 3.f * __ldg(&a.minv32[q.slot[p]]) * (p ? acc.y : acc.x);
    }
}

template <bool VOLCORR>
__global__ void __launch_bounds__(256, PD_MINBLOCKS) lps_dil_fast(const TileArgs a)
{
    lps_dil_fast_body<VOLCORR, false>(a, blockIdx.x, nullptr);
}

template <bool VOLCORR>
__global__ void __launch_bounds__(256, PD_DIL2_MINBLOCKS) lps_dil_fast2(const TileArgs a)
{
    lps_dil_fast2_body<VOLCORR, false>(a, blockIdx.x, nullptr);
}

template <bool VOLCORR>
__global__ void __launch_bounds__(512, 2) lps_force_fast(const TileArgs a)
{
    lps_force_fast_body<VOLCORR, false>(a, blockIdx.x, nullptr);
}

// The same passes with the stencil table as a kernel parameter.
template <bool VOLCORR>
__global__ void __launch_bounds__(256, PD_MINBLOCKS)
    lps_dil_fast_pt(const __grid_constant__ TileArgs a, const __grid_constant__ ParamTab tp)
{
    lps_dil_fast_body<VOLCORR, true>(a, blockIdx.x, tp.e);
}

template <bool VOLCORR>
__global__ void __launch_bounds__(256, PD_DIL2_MINBLOCKS)
    lps_dil_fast2_pt(const __grid_constant__ TileArgs a, const __grid_constant__ ParamTab tp)
{
    lps_dil_fast2_body<VOLCORR, true>(a, blockIdx.x, tp.e);
}

template <bool VOLCORR>
__global__ void __launch_bounds__(512, 2)
    lps_force_fast_pt(const __grid_constant__ TileArgs a, const __grid_constant__ ParamTab tp)
{
    lps_force_fast_body<VOLCORR, true>(a, blockIdx.x, tp.e);
}

}  // namespace pdk
