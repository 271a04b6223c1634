// pd_pmb_fast.cuh -- the FP32C bond-based fused force + update of one tile
// (the PMB pair force of Eq. (3) with bond breaking, Algorithm 1's loop over
// the tile's points and their horizons, the update of Eqs. (7)-(9)): the body
// shared by the pmb_fast kernel (pd_force_pmb.cu) and the request server's
// packed kernel (pd_packed.cu).
//
// Per bond, in lattice units (xi = d, integer; eta = u~_j - u~_i):
//   y   = d + eta,   q = |y|^2,   r = |y| = q rsqrt(q)
//   s   = (2 d.eta + eta.eta) / (|d| (r + |d|))      cancellation-free stretch
//   f_i += c V V_ij s y / r                          (PMB pair force)
// A bond breaks for good when s > s_c, tested before it contributes. Each point
// sums its bonds sequentially in stencil order: no atomics, deterministic.
#pragma once

#include "pd_pair.cuh"

// Unroll depth of the bond-based step's bond loop: 8 measured 2.380 ms per
// 256^3 step against 2.418 ms for 4 (64^3: 0.0638 against 0.0650 ms).
#ifndef PD_PMB_UNROLL
#define PD_PMB_UNROLL 8
#endif

namespace pdk {

// ------------------------------------------------------------------ fast path

// FP32C. Thread t owns the point pair (A, B) of pd_pair.cuh and evaluates both
// in f32x2 arithmetic; the stencil loop is rolled over a shared-memory copy of a
// host-built table of pre-splatted constants, per entry
//   {dx, dx, dy, dy}, {dz, dz, |d|^2, |d|^2}, {R, R, C, C}, {offset, s_c V_ij, lo, hi}
// with R = |d| / V_ij and C = |d|^2 / V_ij. Per bond (lattice units, e = eta):
//   num = e.(e + 2d) = 2 d.e + e.e,   q = |y|^2 = |d|^2 + num,   r = sqrt(q)
//   w   = s V_ij / r = num / (R q + C r),   F += w y,
// since s = num / (|d| (r + |d|)) and (R r + C) r = R q + C r.
//
// Breaking decision of a bond near the threshold, the same from both of its
// ends. The bond loop forms s from displacements staged relative to each
// tile's reference, so the two rows of a bond that crosses a tile boundary
// round it differently and could decide differently when s is within rounding
// of s_c. A bond whose staged s V_ij lies within 2^-13 relative of s_c V_ij is
// therefore decided again here from the global staging pairs of its two
// points: eta = ((hi_j - hi_i) + (lo_j - lo_i)) / h changes sign exactly under
// (i, j) -> (j, i), as does d, so every product below keeps its value and s
// comes out bitwise the same from either end (explicit round-to-nearest
// operations: no contraction choice of the compiler enters). Rare: only such
// bonds take this path, with four global loads each.
static __device__ __noinline__ bool canon_break32(const TileArgs *ap, const int *s_nbr, int tile, int si, int p, int bj,
                                           float dx, float dy, float dz)
{
    const TileArgs &a = *ap;
    const int4 org = __ldg(&a.tile_org[tile]);
    const PairBox pb = pair_box(a.g);
    int sj;
    if (box_mapped(a, org)) {
        int sA, sB;
        map_slots(a, s_nbr, __ldg(&a.box_map[bj]), sA, sB);
        sj = p ? sB : sA;
    } else {
        int cA[3], cB[3];
        pair_coords(a.g, pb, org, bj, cA, cB);
        sj = slot_of(a, s_nbr, org, p ? cB : cA);
    }
    if (sj < 0) return false;
    const float4 hi = __ldg(&a.src_hl[2 * si]), li = __ldg(&a.src_hl[2 * si + 1]);
    const float4 hj = __ldg(&a.src_hl[2 * sj]), lj = __ldg(&a.src_hl[2 * sj + 1]);
    const float ih = (float)a.inv_h;
    const float ex = __fmul_rn(__fadd_rn(__fsub_rn(hj.x, hi.x), __fsub_rn(lj.x, li.x)), ih);
    const float ey = __fmul_rn(__fadd_rn(__fsub_rn(hj.y, hi.y), __fsub_rn(lj.y, li.y)), ih);
    const float ez = __fmul_rn(__fadd_rn(__fsub_rn(hj.z, hi.z), __fsub_rn(lj.z, li.z)), ih);
    // num = e.(e + 2d), as e.((e + d) + d)
    float num = __fmul_rn(ex, __fadd_rn(__fadd_rn(ex, dx), dx));
    num = __fmaf_rn(ey, __fadd_rn(__fadd_rn(ey, dy), dy), num);
    num = __fmaf_rn(ez, __fadd_rn(__fadd_rn(ez, dz), dz), num);
    const float d2 = dx * dx + dy * dy + dz * dz;             // exact (small integers)
    const float r0 = __fsqrt_rn(d2);
    const float r = __fsqrt_rn(__fadd_rn(num, d2));
    const float s = __fdiv_rn(num, __fmul_rn(r0, __fadd_rn(r, r0)));
    return s > (float)a.s_c;
}

// The words of a point pair whose masked pass took bonds out of the sum
// because their staged s V_ij exceeded td.z = s_c V_ij (1 - 2^-13) (bit w - w0
// of pend), decided after the pair's word loop, so that the loop pays one
// register for them. The mask words in memory still hold the bonds' states
// from before this pass. Per taken-out bond (recomputed with the arithmetic of
// pmb_word in scalar form: each f32x2 operation is two IEEE operations, the
// special-function approximations are the same instructions): above td.w =
// s_c V_ij (1 + 2^-13) it breaks; in between canon_break32 decides, and a bond
// that stays intact is added to the point's force (after the pair's other
// bonds). The final mask words are written here. Out of line and rare.
struct PendFix {
    float2 Fx, Fy, Fz;
};

template <int DIM>
__device__ __noinline__ PendFix pend_fix(const TileArgs *ap, const int *s_nbr, int tile, PairPts q, const float4 *tab,
                                         const float4 *P4, const float2 *P2, uint32_t pend, int w0, PendFix r)
{
    const TileArgs &a = *ap;
    const float4 ui4 = P4[q.bi];
    const float2 nux = f2neg(f2lo(ui4)), nuy = f2neg(f2hi(ui4));
    const float2 nuz = DIM == 3 ? f2neg(P2[q.bi]) : make_float2(0.f, 0.f);
    for (uint32_t pw = pend; pw; pw &= pw - 1u) {
        const int w = w0 + __ffs(pw) - 1;
        const float4 *tw = tab + 4 * 32 * w;
        const size_t mo = (size_t)w * a.g.nslots;
        for (int p = 0; p < 2; ++p) {
            if (!q.act[p]) continue;
            const uint32_t m = a.mask[mo + q.slot[p]];
            uint32_t k = m;
            for (uint32_t cm = m; cm; cm &= cm - 1u) {
                const int b = __ffs(cm) - 1;
                const float4 ta = tw[4 * b], tb = tw[4 * b + 1], tc = tw[4 * b + 2], td = tw[4 * b + 3];
                const int off = __float_as_int(td.x);
                const float4 r4 = P4[q.bi + off];
                const float ex = (p ? r4.y : r4.x) + (p ? nux.y : nux.x);
                const float ey = (p ? r4.w : r4.z) + (p ? nuy.y : nuy.x);
                const float yx = ex + ta.x, yy = ey + ta.z;
                float num = ex * (yx + ta.x);
                num = fmaf(ey, yy + ta.z, num);
                float yz = 0.f;
                if (DIM == 3) {
                    const float2 z2 = P2[q.bi + off];
                    const float ez = (p ? z2.y : z2.x) + (p ? nuz.y : nuz.x);
                    yz = ez + tb.x;
                    num = fmaf(ez, yz + tb.x, num);
                }
                const float qq = num + tb.z;
                const float rr = sfu_sqrt(qq);
                const float den = fmaf(qq, tc.x, rr * tc.z);
                const float wgt = num * sfu_rcp(den);
                const float sv = wgt * rr;
                if (!(sv > td.z)) continue;                               // counted in the loop
                if (sv > td.w || canon_break32(ap, s_nbr, tile, q.slot[p], p, q.bi + off, ta.x, ta.z, tb.x)) {
                    k &= ~(1u << b);                                      // breaks
                    continue;
                }
                float2 &Fx = r.Fx, &Fy = r.Fy, &Fz = r.Fz;
                if (p) {
                    Fx.y = fmaf(wgt, yx, Fx.y);
                    Fy.y = fmaf(wgt, yy, Fy.y);
                    if (DIM == 3) Fz.y = fmaf(wgt, yz, Fz.y);
                } else {
                    Fx.x = fmaf(wgt, yx, Fx.x);
                    Fy.x = fmaf(wgt, yy, Fy.x);
                    if (DIM == 3) Fz.x = fmaf(wgt, yz, Fz.x);
                }
            }
            if (k != m) a.mask[mo + q.slot[p]] = k;
        }
    }
    return r;
}

// One 32-bond word of the stencil at a time. MASKED = false is the path for
// words whose bonds all exist and are intact for every point of the warp (the
// common case: the warp then skips every per-bond mask operation); with
// breaking on, it only reports whether some bond came near s_c, and the warp then
// redoes the word on the masked path, which breaks the bond before it counts.
// The masked path takes every bond above td.z = s_c V_ij (1 - 2^-13) out of the
// sum and its mask bit (k0, k1); the caller passes those to near_fix, which
// keeps the ones that are not broken after all.
template <int DIM, bool MASKED, bool BRK>
__device__ __forceinline__ bool pmb_word(const float4 *tw, int nb, const float4 *P4, const float2 *P2, int bi,
                                         float2 nux, float2 nuy, float2 nuz, uint32_t c0, uint32_t c1,
                                         uint32_t &k0, uint32_t &k1, float2 &Fx, float2 &Fy, float2 &Fz)
{
    bool anybrk = false;
PD_PRAGMA_UNROLL(PD_PMB_UNROLL)
    for (int b = 0; b < nb; ++b) {
        const float4 ta = tw[4 * b], tb = tw[4 * b + 1], tc = tw[4 * b + 2], td = tw[4 * b + 3];
        const int off = __float_as_int(td.x);
        const float4 r4 = P4[bi + off];
        const float2 ex = f2add(f2lo(r4), nux), ey = f2add(f2hi(r4), nuy);
        const float2 yx = f2add(ex, f2lo(ta)), yy = f2add(ey, f2hi(ta));
        float2 num = f2mul(ex, f2add(yx, f2lo(ta)));
        num = f2fma(ey, f2add(yy, f2hi(ta)), num);
        float2 yz = make_float2(0.f, 0.f);
        if (DIM == 3) {
            const float2 ez = f2add(P2[bi + off], nuz);
            yz = f2add(ez, f2lo(tb));
            num = f2fma(ez, f2add(yz, f2lo(tb)), num);
        }
        const float2 qq = f2add(num, f2hi(tb));
        const float2 rr = f2sqrt(qq);
        const float2 den = f2fma(qq, f2lo(tc), f2mul(rr, f2hi(tc)));
        float2 wgt = f2mul(num, f2rcp(den));               // s V_ij / |y|
        if (MASKED) {
            const bool in0 = (c0 >> b) & 1u, in1 = (c1 >> b) & 1u;
            bool ok0 = in0, ok1 = in1;
            if (BRK) {
                // s > s_c, tested as s V_ij = w |y| > s_c V_ij; from td.z on the bond
                // leaves the sum here and near_fix decides
                const float2 sv = f2mul(wgt, rr);
                const bool b0 = in0 && sv.x > td.z, b1 = in1 && sv.y > td.z;
                if (b0) k0 &= ~(1u << b);
                if (b1) k1 &= ~(1u << b);
                ok0 = in0 && !b0;
                ok1 = in1 && !b1;
            }
            wgt.x = ok0 ? wgt.x : 0.f;
            wgt.y = ok1 ? wgt.y : 0.f;
        } else if (BRK) {
            const float2 sv = f2mul(wgt, rr);
            anybrk = anybrk || sv.x > td.z || sv.y > td.z;
        }
        Fx = f2fma(wgt, yx, Fx);
        Fy = f2fma(wgt, yy, Fy);
        if (DIM == 3) Fz = f2fma(wgt, yz, Fz);
    }
    return anybrk;
}

// Sum the a.split partial forces of a point pair (each part summed one
// contiguous range of stencil words): parts 1.. park theirs in red, part 0 adds
// them in part order (fixed: the result does not depend on timing). Every
// thread of the block calls this once.
__device__ __forceinline__ void pair_split_sum(const TileArgs &a, float2 *red, int npairs, int t, int part,
                                               float2 &Fx, float2 &Fy, float2 &Fz)
{
    if (part > 0) {
        float2 *r = red + 3 * ((part - 1) * npairs + t);
        r[0] = Fx;
        r[1] = Fy;
        r[2] = Fz;
    }
    __syncthreads();
    if (part == 0) {
        for (int j = 1; j < a.split; ++j) {
            const float2 *r = red + 3 * ((j - 1) * npairs + t);
            Fx = f2add(Fx, r[0]);
            Fy = f2add(Fy, r[1]);
            Fz = f2add(Fz, r[2]);
        }
    }
}

// Launch: one CTA per tile, (tile points / 2) * a.split threads. Thread
// (t, part) owns point pair t and the stencil words [part W / split,
// (part + 1) W / split). SPLIT = true (a.split of 2 or 4) at wide horizons,
// where one CTA's halo box and table fill the shared memory, so that more warps
// run per SM; SPLIT = false is the one-thread-per-pair kernel.
// The fused force + update of one tile. The kernel below runs it for tile
// blockIdx.x; the request server's packed kernel (pd_packed.cu) runs it for the
// tiles of its work items, with a in shared memory.
// PTAB: the table is read from ptab (a kernel parameter) instead of shared memory.
template <int DIM, bool BRK, bool SPLIT, bool PTAB>
__device__ __forceinline__ void pmb_fast_body(const TileArgs &a, int tile, const float4 *ptab)
{
    const Geom &g = a.g;
    const PairBox pb = pair_box(g);
    const int S = g.S;
    extern __shared__ float4 smem4[];
    float4 *P4 = smem4;
    float2 *P2 = reinterpret_cast<float2 *>(P4 + pb.n);
    float4 *tab = P4 + pb.n + (DIM == 3 ? (pb.n + 1) / 2 : 0);      // 4 float4 per stencil entry

    __shared__ int s_nbr[27];
    __shared__ uint32_t s_pend[BRK ? (SPLIT ? 1024 : 256) : 1];
    const int4 org = __ldg(&a.tile_org[tile]);
    // the table (at most two float4 per thread here) is loaded into registers
    // before the staging and stored after it, so its load latency overlaps the
    // staging's instead of preceding it
    const bool tab2 = !PTAB && 4 * S <= 2 * (int)blockDim.x;
    const int k0 = threadIdx.x, k1 = threadIdx.x + blockDim.x;
    float4 t0 = make_float4(0.f, 0.f, 0.f, 0.f), t1 = t0;
    if (tab2) {
        if (k0 < 4 * S) t0 = __ldg(&a.tab_a[k0]);
        if (k1 < 4 * S) t1 = __ldg(&a.tab_a[k1]);
    } else if (!PTAB) {
        for (int k = threadIdx.x; k < 4 * S; k += blockDim.x) tab[k] = __ldg(&a.tab_a[k]);
    }
    const int nthr = g.T / 2;            // point pairs: a multiple of 32, so a warp has one part
    const int part = SPLIT ? threadIdx.x / nthr : 0;
    const int w0 = SPLIT ? part * g.W / a.split : 0, w1 = SPLIT ? (part + 1) * g.W / a.split : g.W;
    // With the split (one pair per thread), the pair's first mask words are loaded
    // before the staging, so that their latency overlaps the staging's (64^3 at
    // 2^8 tiles: 62.6 -> 61.5 us). The one-thread-per-pair kernel loads them after
    // it: held across the staging they cost it registers in the bond loop (256^3
    // at 2^9 tiles: 2.42 -> 2.47 ms).
    PairPts q_pre;
    uint32_t n0_pre = 0u, n1_pre = 0u;
    if constexpr (SPLIT) {
        q_pre = pair_points(g, pb, org, tile, threadIdx.x % nthr);
        const size_t mo0 = (size_t)w0 * g.nslots;
        n0_pre = q_pre.act[0] && w0 < w1 ? a.mask[mo0 + q_pre.slot[0]] : 0u;
        n1_pre = q_pre.act[1] && w0 < w1 ? a.mask[mo0 + q_pre.slot[1]] : 0u;
    }
    load_nbr(a, tile, s_nbr);
    __syncthreads();
    stage_pairs(a, pb, org, tile, s_nbr, P4, DIM == 3 ? P2 : nullptr, true);
    if (tab2) {
        if (k0 < 4 * S) tab[k0] = t0;
        if (k1 < 4 * S) tab[k1] = t1;
    }
    __syncthreads();

    // one iteration per thread (T / 2 <= 256 = blockDim without the split)
    for (int t = SPLIT ? threadIdx.x % nthr : threadIdx.x; t < nthr; t += SPLIT ? nthr : blockDim.x) {
        const PairPts q = SPLIT ? q_pre : pair_points(g, pb, org, tile, t);
        const float4 ui4 = P4[q.bi];
        const float2 nux = f2neg(f2lo(ui4)), nuy = f2neg(f2hi(ui4));
        const float2 nuz = DIM == 3 ? f2neg(P2[q.bi]) : make_float2(0.f, 0.f);
        float2 Fx = make_float2(0.f, 0.f), Fy = Fx, Fz = Fx;
        const size_t mo0 = (size_t)w0 * g.nslots;
        uint32_t n0 = SPLIT ? n0_pre : (q.act[0] ? a.mask[mo0 + q.slot[0]] : 0u);
        uint32_t n1 = SPLIT ? n1_pre : (q.act[1] ? a.mask[mo0 + q.slot[1]] : 0u);
        // words with bonds taken out, a bit per word in shared memory (no register
        // in the bond loop); BRK launches keep a thread's words within 32
        if (BRK) s_pend[threadIdx.x] = 0u;
        for (int w = w0; w < w1; ++w) {
            const uint32_t m0 = n0, m1 = n1;
            if (w + 1 < w1) {
                const size_t mo = (size_t)(w + 1) * g.nslots;
                n0 = q.act[0] ? a.mask[mo + q.slot[0]] : 0u;
                n1 = q.act[1] ? a.mask[mo + q.slot[1]] : 0u;
            }
            const int nb = min(32, S - 32 * w);
            const uint32_t full = nb == 32 ? 0xffffffffu : ((1u << nb) - 1u);
            const float4 *tw = (PTAB ? ptab : tab) + 4 * 32 * w;
            uint32_t k0 = m0, k1 = m1;
            bool masked = !__all_sync(0xffffffffu, m0 == full && m1 == full);
            if (!masked) {
                const float2 sx = Fx, sy = Fy, sz = Fz;
                const bool brk = pmb_word<DIM, false, BRK>(tw, nb, P4, P2, q.bi, nux, nuy, nuz, m0, m1, k0, k1,
                                                           Fx, Fy, Fz);
                if (BRK && __any_sync(0xffffffffu, brk)) {
                    Fx = sx;
                    Fy = sy;
                    Fz = sz;
                    masked = true;
                }
            }
            if (masked) {
                pmb_word<DIM, true, BRK>(tw, nb, P4, P2, q.bi, nux, nuy, nuz, m0, m1, k0, k1, Fx, Fy, Fz);
                // bonds taken out: decided (and the mask word written) after the loop
                if (BRK && ((m0 & ~k0) | (m1 & ~k1))) s_pend[threadIdx.x] |= 1u << (w - w0);

            }
        }
        if (BRK && s_pend[threadIdx.x]) {
            const PendFix r = pend_fix<DIM>(&a, s_nbr, tile, q, PTAB ? ptab : tab, P4, P2, s_pend[threadIdx.x], w0,
                                            PendFix{Fx, Fy, Fz});
            Fx = r.Fx;
            Fy = r.Fy;
            Fz = r.Fz;
        }
        if (SPLIT) pair_split_sum(a, reinterpret_cast<float2 *>(tab + 4 * S), nthr, t, part, Fx, Fy, Fz);
        if (part == 0) {
            const float FA[3] = {Fx.x, Fy.x, Fz.x}, FB[3] = {Fx.y, Fy.y, Fz.y};
            pair_epilogue2(a, q, FA, FB, DIM);
        }
    }
}

template <int DIM, bool BRK, bool SPLIT>
__global__ void __launch_bounds__(SPLIT ? 1024 : 256, SPLIT ? 1 : PD_MINBLOCKS)
    pmb_fast(const __grid_constant__ TileArgs a)
{
    pmb_fast_body<DIM, BRK, SPLIT, false>(a, blockIdx.x, nullptr);
}

template <int DIM, bool BRK, bool SPLIT>
__global__ void __launch_bounds__(SPLIT ? 1024 : 256, SPLIT ? 1 : PD_MINBLOCKS)
    pmb_fast_pt(const __grid_constant__ TileArgs a, const __grid_constant__ ParamTab tp)
{
    pmb_fast_body<DIM, BRK, SPLIT, true>(a, blockIdx.x, tp.e);
}

}  // namespace pdk
