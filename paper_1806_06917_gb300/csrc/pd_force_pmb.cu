// pd_force_pmb.cu -- bond-based PMB internal force with bond breaking, fused
// with the explicit update (Eq. (3); Algorithm 1's loop over points and their
// horizons; Eqs. (7)-(9) for the update).
//
// Per bond, in lattice units (xi = d, integer; eta = u~_j - u~_i):
//   y   = d + eta,   q = |y|^2,   r = |y| = q rsqrt(q)
//   s   = (2 d.eta + eta.eta) / (|d| (r + |d|))      cancellation-free stretch
//   f_i += c V V_ij s y / r                          (PMB pair force)
// A bond breaks for good when s > s_c, tested before it contributes. Each point
// sums its bonds sequentially in stencil order: no atomics, deterministic.
#include <string.h>

#include <algorithm>
#include <type_traits>

#include "pd_pmb_fast.cuh"

// Unroll depth of the NP / LP bond loops (8 measured the same as 4 on the 443^2,
// m = 20 step: 0.1553 ms per launch).
#ifndef PD_NP_UNROLL
#define PD_NP_UNROLL PD_UNROLL
#endif

namespace pdk {

// Paired halo box (float4 {x_A, x_B, y_A, y_B}, plus float2 {z_A, z_B} in 3D)
// followed by the stencil table of `words` float4 per entry.
static size_t fast_smem(const Geom &g, int words)
{
    size_t n;
    if (g.dim == 3) n = (size_t)(g.bx + 2 * g.m) * (g.by + 2 * g.m) * (g.bz / 2 + 2 * g.m);
    else n = (size_t)(g.bx + 2 * g.m) * (g.by / 2 + 2 * g.m);
    const size_t p2 = g.dim == 3 ? ((n + 1) / 2) * sizeof(float4) : 0;
    return n * sizeof(float4) + p2 + (size_t)g.S * words * sizeof(float4);
}

size_t pmb_fast_smem(const Geom &g) { return fast_smem(g, 4); }

size_t np_fast_smem(const Geom &g) { return fast_smem(g, NP_TAB_WORDS(g.dim)); }

// ------------------------------------------------------------------ generic

// ------------------------------------------------------------- NP / LP, FP32C

// One 32-bond word of the NP / LP sum (Algorithm 1) for a point pair in f32x2.
// With S = eta.d / |d|^2 the bond term is t S [exp2(a S^2) for NP] d, t = J
// V_ij / |d| and a = -beta h |d| / ln 2 (see pd_api.cu); written in p = eta.d:
//   w = k p [exp2(a' p^2) for NP],  F += w d,   k = t / |d|^2,  a' = a / |d|^4.
// The direction is the reference bond d, so no square root or reciprocal is
// needed. Table entries of NP_TAB_WORDS(DIM) float4, the fewest shared-memory
// wavefronts per bond (a broadcast 16-byte load costs two):
//   2D: {dx,dx,dy,dy} {k,k,a',offset}
//   3D: {dx,dx,dy,dy} {dz,dz,k,k} {a',offset,-,-}
template <int DIM, bool MASKED, bool LINEAR>
__device__ __forceinline__ void np_word(const float4 *tw, int nb, const float4 *P4, const float2 *P2, int bi,
                                        float2 nux, float2 nuy, float2 nuz, uint32_t c0, uint32_t c1, float2 &Fx,
                                        float2 &Fy, float2 &Fz)
{
    constexpr int E = NP_TAB_WORDS(DIM);
PD_PRAGMA_UNROLL(PD_NP_UNROLL)
    for (int b = 0; b < nb; ++b) {
        const float4 ta = tw[E * b], tb = tw[E * b + 1];
        float ak;
        int off;
        if (DIM == 3) {
            const float2 tc = reinterpret_cast<const float2 *>(tw + E * b + 2)[0];
            ak = tc.x;
            off = __float_as_int(tc.y);
        } else {
            ak = tb.z;
            off = __float_as_int(tb.w);
        }
        const float4 r4 = P4[bi + off];
        const float2 ex = f2add(f2lo(r4), nux), ey = f2add(f2hi(r4), nuy);
        float2 dot = f2mul(ex, f2lo(ta));
        dot = f2fma(ey, f2hi(ta), dot);
        if (DIM == 3) dot = f2fma(f2add(P2[bi + off], nuz), f2lo(tb), dot);
        float2 wgt = f2mul(dot, DIM == 3 ? f2hi(tb) : f2lo(tb));
        if (!LINEAR) wgt = f2mul(wgt, f2ex2(f2mul(make_float2(ak, ak), f2mul(dot, dot))));
        if (MASKED) {
            wgt.x = ((c0 >> b) & 1u) ? wgt.x : 0.f;
            wgt.y = ((c1 >> b) & 1u) ? wgt.y : 0.f;
        }
        Fx = f2fma(wgt, f2lo(ta), Fx);
        Fy = f2fma(wgt, f2hi(ta), Fy);
        if (DIM == 3) Fz = f2fma(wgt, f2lo(tb), Fz);
    }
}

template <int DIM, bool LINEAR, bool SPLIT>
__global__ void __launch_bounds__(SPLIT ? 1024 : 256, SPLIT ? 1 : PD_MINBLOCKS) np_fast(const TileArgs a)
{
    const Geom &g = a.g;
    const PairBox pb = pair_box(g);
    const int S = g.S;
    extern __shared__ float4 smem4[];
    float4 *P4 = smem4;
    float2 *P2 = reinterpret_cast<float2 *>(P4 + pb.n);
    float4 *tab = P4 + pb.n + (DIM == 3 ? (pb.n + 1) / 2 : 0);      // the layout of np_fast_smem
    constexpr int E = NP_TAB_WORDS(DIM);
    __shared__ int s_nbr[27];
    const int tile = blockIdx.x;
    const int4 org = __ldg(&a.tile_org[tile]);
    for (int k = threadIdx.x; k < E * S; k += blockDim.x) tab[k] = __ldg(&a.tab_a[k]);
    load_nbr(a, tile, s_nbr);
    __syncthreads();
    stage_pairs(a, pb, org, tile, s_nbr, P4, DIM == 3 ? P2 : nullptr, true);
    __syncthreads();

    const int nthr = g.T / 2;            // point pairs; thread (t, part) as in pmb_fast
    const int part = SPLIT ? threadIdx.x / nthr : 0;
    const int w0 = SPLIT ? part * g.W / a.split : 0, w1 = SPLIT ? (part + 1) * g.W / a.split : g.W;
    // one iteration per thread (T / 2 <= 256 = blockDim without the split)
    for (int t = SPLIT ? threadIdx.x % nthr : threadIdx.x; t < nthr; t += SPLIT ? nthr : blockDim.x) {
        const PairPts q = pair_points(g, pb, org, tile, t);
        const float4 ui4 = P4[q.bi];
        const float2 nux = f2neg(f2lo(ui4)), nuy = f2neg(f2hi(ui4));
        const float2 nuz = DIM == 3 ? f2neg(P2[q.bi]) : make_float2(0.f, 0.f);
        float2 Fx = make_float2(0.f, 0.f), Fy = Fx, Fz = Fx;
        const size_t mo0 = (size_t)w0 * g.nslots;
        uint32_t n0 = q.act[0] && (!SPLIT || w0 < w1) ? a.mask[mo0 + q.slot[0]] : 0u;
        uint32_t n1 = q.act[1] && (!SPLIT || w0 < w1) ? a.mask[mo0 + q.slot[1]] : 0u;
        for (int w = w0; w < w1; ++w) {
            const uint32_t m0 = n0, m1 = n1;
            if (w + 1 < w1) {
                const size_t mo = (size_t)(w + 1) * g.nslots;
                n0 = q.act[0] ? a.mask[mo + q.slot[0]] : 0u;
                n1 = q.act[1] ? a.mask[mo + q.slot[1]] : 0u;
            }
            const int nb = min(32, S - 32 * w);
            const uint32_t full = nb == 32 ? 0xffffffffu : ((1u << nb) - 1u);
            const float4 *tw = tab + E * 32 * w;
            if (__all_sync(0xffffffffu, m0 == full && m1 == full))
                np_word<DIM, false, LINEAR>(tw, nb, P4, P2, q.bi, nux, nuy, nuz, m0, m1, Fx, Fy, Fz);
            else
                np_word<DIM, true, LINEAR>(tw, nb, P4, P2, q.bi, nux, nuy, nuz, m0, m1, Fx, Fy, Fz);
        }
        if (SPLIT) pair_split_sum(a, reinterpret_cast<float2 *>(tab + E * S), nthr, t, part, Fx, Fy, Fz);
        if (part == 0) {
            const float FA[3] = {Fx.x, Fy.x, Fz.x}, FB[3] = {Fx.y, Fy.y, Fz.y};
            pair_epilogue2(a, q, FA, FB, DIM);
        }
    }
}

// 2D wide horizons: each thread owns two point pairs, t and t + T/4 (by/4 box
// rows apart, the constant offset dbi), so that every table entry read from
// shared memory serves four points: per 32-lane step 2 broadcast table loads
// and 2 gathers move 128 bonds, against 2 + 1 for 64 bonds with one pair. The
// shared-memory data pipe bounds np_fast at m = 20; the arithmetic is np_word's.
template <bool MASKED, bool LINEAR>
__device__ __forceinline__ void np_word2(const float4 *tw, int nb, const float4 *P4, int bi, int dbi,
                                         float2 nux0, float2 nuy0, float2 nux1, float2 nuy1, uint32_t c0,
                                         uint32_t c1, uint32_t c2, uint32_t c3, float2 &Fx0, float2 &Fy0,
                                         float2 &Fx1, float2 &Fy1)
{
PD_PRAGMA_UNROLL(PD_NP_UNROLL)
    for (int b = 0; b < nb; ++b) {
        const float4 ta = tw[2 * b], tb = tw[2 * b + 1];
        const int off = __float_as_int(tb.w);
        const float4 r0 = P4[bi + off], r1 = P4[bi + dbi + off];
        const float2 ex0 = f2add(f2lo(r0), nux0), ey0 = f2add(f2hi(r0), nuy0);
        const float2 ex1 = f2add(f2lo(r1), nux1), ey1 = f2add(f2hi(r1), nuy1);
        float2 dot0 = f2mul(ex0, f2lo(ta)), dot1 = f2mul(ex1, f2lo(ta));
        dot0 = f2fma(ey0, f2hi(ta), dot0);
        dot1 = f2fma(ey1, f2hi(ta), dot1);
        float2 w0 = f2mul(dot0, f2lo(tb)), w1 = f2mul(dot1, f2lo(tb));
        if (!LINEAR) {
            const float2 ak = make_float2(tb.z, tb.z);
            w0 = f2mul(w0, f2ex2(f2mul(ak, f2mul(dot0, dot0))));
            w1 = f2mul(w1, f2ex2(f2mul(ak, f2mul(dot1, dot1))));
        }
        if (MASKED) {
            w0.x = ((c0 >> b) & 1u) ? w0.x : 0.f;
            w0.y = ((c1 >> b) & 1u) ? w0.y : 0.f;
            w1.x = ((c2 >> b) & 1u) ? w1.x : 0.f;
            w1.y = ((c3 >> b) & 1u) ? w1.y : 0.f;
        }
        Fx0 = f2fma(w0, f2lo(ta), Fx0);
        Fy0 = f2fma(w0, f2hi(ta), Fy0);
        Fx1 = f2fma(w1, f2lo(ta), Fx1);
        Fy1 = f2fma(w1, f2hi(ta), Fy1);
    }
}

// Launch: one CTA per tile, (tile points / 4) * a.split threads; thread (t, sub)
// owns pairs t and t + T/4 and the sub-th of a.split ranges of stencil words.
template <bool LINEAR>
__global__ void __launch_bounds__(1024, 1) np_fast2(const TileArgs a)
{
    const Geom &g = a.g;
    const PairBox pb = pair_box(g);
    const int S = g.S;
    extern __shared__ float4 smem4[];
    float4 *P4 = smem4;
    float4 *tab = P4 + pb.n;                  // the layout of np_fast_smem in 2D
    constexpr int E = NP_TAB_WORDS(2);
    __shared__ int s_nbr[27];
    const int tile = blockIdx.x;
    const int4 org = __ldg(&a.tile_org[tile]);
    for (int k = threadIdx.x; k < E * S; k += blockDim.x) tab[k] = __ldg(&a.tab_a[k]);
    load_nbr(a, tile, s_nbr);
    __syncthreads();
    stage_pairs(a, pb, org, tile, s_nbr, P4, nullptr, false);
    __syncthreads();

    const int npairs = g.T / 2, nthr = npairs / 2;     // nthr: a multiple of 32 (T >= 128)
    const int sub = threadIdx.x / nthr, t = threadIdx.x % nthr;
    const int w0 = sub * g.W / a.split, w1 = (sub + 1) * g.W / a.split;
    const PairPts q0 = pair_points(g, pb, org, tile, t), q1 = pair_points(g, pb, org, tile, t + nthr);
    const int dbi = q1.bi - q0.bi;
    float2 Fx0, Fy0, Fx1, Fy1;
    {
        const float4 u0 = P4[q0.bi], u1 = P4[q1.bi];
        const float2 nux0 = f2neg(f2lo(u0)), nuy0 = f2neg(f2hi(u0));
        const float2 nux1 = f2neg(f2lo(u1)), nuy1 = f2neg(f2hi(u1));
        Fx0 = Fy0 = Fx1 = Fy1 = make_float2(0.f, 0.f);
        const size_t mo0 = (size_t)w0 * g.nslots;
        uint32_t n0 = q0.act[0] ? a.mask[mo0 + q0.slot[0]] : 0u;
        uint32_t n1 = q0.act[1] ? a.mask[mo0 + q0.slot[1]] : 0u;
        uint32_t n2 = q1.act[0] ? a.mask[mo0 + q1.slot[0]] : 0u;
        uint32_t n3 = q1.act[1] ? a.mask[mo0 + q1.slot[1]] : 0u;
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
            const float4 *tw = tab + E * 32 * w;
            if (__all_sync(0xffffffffu, m0 == full && m1 == full && m2 == full && m3 == full))
                np_word2<false, LINEAR>(tw, nb, P4, q0.bi, dbi, nux0, nuy0, nux1, nuy1, m0, m1, m2, m3, Fx0, Fy0,
                                        Fx1, Fy1);
            else
                np_word2<true, LINEAR>(tw, nb, P4, q0.bi, dbi, nux0, nuy0, nux1, nuy1, m0, m1, m2, m3, Fx0, Fy0,
                                       Fx1, Fy1);
        }
    }
    float2 *red = reinterpret_cast<float2 *>(tab + E * S);
    float2 Fz0 = make_float2(0.f, 0.f), Fz1 = Fz0;
    if (a.split > 1) {
        pair_split_sum(a, red, npairs, t, sub, Fx0, Fy0, Fz0);
        pair_split_sum(a, red, npairs, t + nthr, sub, Fx1, Fy1, Fz1);
    }
    if (sub == 0) {
        const float FA0[3] = {Fx0.x, Fy0.x, 0.f}, FB0[3] = {Fx0.y, Fy0.y, 0.f};
        pair_epilogue2(a, q0, FA0, FB0, 2);
        const float FA1[3] = {Fx1.x, Fy1.x, 0.f}, FB1[3] = {Fx1.y, Fy1.y, 0.f};
        pair_epilogue2(a, q1, FA1, FB1, 2);
    }
}

// The FP64 stretch of bond (si, sj) with lattice offset d from the global FP64
// staging (the FP64 path's u), bitwise the same from both ends of the bond.
__device__ __forceinline__ double canon_stretch64(const TileArgs &a, int si, int sj, int4 d)
{
    const double4_32a ui = a.src_d4[si], uj = a.src_d4[sj];
    const double ex = __dmul_rn(__dsub_rn(uj.x, ui.x), a.inv_h);
    const double ey = __dmul_rn(__dsub_rn(uj.y, ui.y), a.inv_h);
    const double ez = __dmul_rn(__dsub_rn(uj.z, ui.z), a.inv_h);
    const double dx = d.x, dy = d.y, dz = d.z, d2 = d.w;
    double num = __dmul_rn(ex, __dadd_rn(__dadd_rn(ex, dx), dx));
    num = __fma_rn(ey, __dadd_rn(__dadd_rn(ey, dy), dy), num);
    num = __fma_rn(ez, __dadd_rn(__dadd_rn(ez, dz), dz), num);
    const double r0 = __dsqrt_rn(d2), r = __dsqrt_rn(__dadd_rn(num, d2));
    return __ddiv_rn(num, __dmul_rn(r0, __dadd_rn(r, r0)));
}

// Runtime stencil (any horizon), one point per thread. R = float (FP32C) or
// double (FP64). Stencil entries come from a.stencil; box dims from a.g.m.
template <class R>
__global__ void __launch_bounds__(256) pmb_generic(const TileArgs a)
{
    using R4 = typename std::conditional<sizeof(R) == 4, float4, double4_32a>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R4 *box = reinterpret_cast<R4 *>(smem_raw);
    const Geom &g = a.g;
    const int m = g.m;
    const int HX = g.bx + 2 * m, HY = g.by + 2 * m, HZ = g.dim == 3 ? g.bz + 2 * m : 1;
    const int nbox = HX * HY * HZ;
    const int tile = blockIdx.x;
    const int4 org = __ldg(&a.tile_org[tile]);
    if constexpr (sizeof(R) == 4) {
        stage_box32(reinterpret_cast<float4 *>(box), HX, HY, nbox, m, a, org, tile_ref32(a, tile),
                    (float)a.inv_h);
    } else {
        stage_box64(reinterpret_cast<double4_32a *>(box), HX, HY, nbox, m, a, org, tile_ref64(a, tile),
                    a.inv_h);
    }
    __syncthreads();

    const bool brk_on = a.update_breaking && a.s_c > 0.0;
    const bool np_law = a.model == PD_MODEL_NP || a.model == PD_MODEL_LP;
    const R s_c = (R)a.s_c;
    for (int t = threadIdx.x; t < g.T; t += blockDim.x) {
        const int lx = t % g.bx, ly = (t / g.bx) % g.by, lz = t / (g.bx * g.by);
        const int slot = tile * g.T + brick_code(g.dim, lx, ly, lz);
        const bool act = org.x + lx < g.nx && org.y + ly < g.ny && org.z + lz < g.nz;
        if (!act) continue;
        const int bi = (lx + m) + HX * ((ly + m) + HY * (g.dim == 3 ? lz + m : 0));
        const R4 ui = box[bi];
        R Fx = 0, Fy = 0, Fz = 0;
        for (int w = 0; w < g.W; ++w) {
            const uint32_t word = a.mask[(size_t)w * g.nslots + slot];
            uint32_t nword = word;
            const int nb = min(32, g.S - 32 * w);
            for (int b = 0; b < nb; ++b) {
                if (!((word >> b) & 1u)) continue;
                const int4 d = __ldg(&a.stencil[32 * w + b]);
                const R4 rj = box[bi + d.x + HX * (d.y + HY * d.z)];
                const R ex = rj.x - ui.x, ey = rj.y - ui.y, ez = rj.z - ui.z;
                if (np_law) {
                    // NP / LP (Algorithm 1): S = eta.d / |d|^2 in lattice units,
                    // f += J psi'(|xi| S^2)/(C beta) S d/|d| V_ij (times c V below)
                    if (d.w >= m * m) continue;                            // J = 0 on the boundary
                    const R r0 = (R)__ldg(&a.stencil_r0[32 * w + b]);
                    const R S = ((R)d.x * ex + (R)d.y * ey + (R)d.z * ez) / (R)d.w;
                    R wgt = S / r0;
                    if (a.model == PD_MODEL_NP) wgt *= exp(-(R)a.psi_beta * (R)a.h * r0 * S * S);
                    if (a.vol_corr) wgt *= (R)vol_factor_lattice(m, (double)r0);
                    Fx += wgt * (R)d.x;
                    Fy += wgt * (R)d.y;
                    Fz += wgt * (R)d.z;
                    continue;
                }
                const R yx = ex + (R)d.x, yy = ey + (R)d.y, yz = ez + (R)d.z;
                const R q = yx * yx + yy * yy + yz * yz;
                const R num = ex * ex + ey * ey + ez * ez +
                              (R)2 * ((R)d.x * ex + (R)d.y * ey + (R)d.z * ez);
                const R r0 = (R)__ldg(&a.stencil_r0[32 * w + b]);
                const R rs = prsqrt1(q);
                const R s = pdiv1(num, r0 * (q * rs + r0));
                bool brk = brk_on && s > s_c;
                // near s_c (2^-30 relative), decided from both points' global state
                // in an order that is bitwise symmetric in (i, j), as in canon_break32
                if (brk_on && fabs((double)s - a.s_c) <= 0x1p-30 * a.s_c) {
                    const int sj = slot_at(g, a.tile_lut, org.x + lx + d.x, org.y + ly + d.y,
                                           g.dim == 3 ? org.z + lz + d.z : 0);
                    brk = sj >= 0 && canon_stretch64(a, slot, sj, d) > a.s_c;
                }
                if (brk) {
                    nword &= ~(1u << b);
                    continue;
                }
                R wgt = s * rs;
                if (a.vol_corr) wgt *= (R)vol_factor_lattice(m, (double)r0);
                Fx += wgt * yx;
                Fy += wgt * yy;
                Fz += wgt * yz;
            }
            if (nword != word) a.mask[(size_t)w * g.nslots + slot] = nword;
        }
        const double f[3] = {a.cV * (double)Fx, a.cV * (double)Fy, a.cV * (double)Fz};
        point_epilogue(a, slot, f, g.dim, sizeof(R) == 8);
    }
}

// ---------------------------------------------------------------- dispatch

// Shared memory of pmb_fast / np_fast (base) with the stencil split over
// `split` threads per pair: the split-sum buffer (3 float2 per pair and extra part).
static size_t split_smem(const Geom &g, size_t base, int split)
{
    return base + (size_t)(split - 1) * (g.T / 2) * 3 * sizeof(float2);
}

size_t pmb_fast_smem_split(const Geom &g, int split) { return split_smem(g, pmb_fast_smem(g), split); }

// Threads per point pair: of 1, 2, 4 (at most the number of stencil words), the
// smallest that reaches the most resident threads per SM, counting the
// 1024-thread limit of 64 registers per thread and 228 KB of shared memory per
// SM (1 KB of it reserved per CTA).
static int choose_split(const Geom &g, size_t base, int pairs_per_thread = 1)
{
    const int nthr = g.T / 2 / pairs_per_thread;
    int best = 1, best_threads = 0;
    for (int split = 1; split <= 4 && split <= g.W; split *= 2) {
        const size_t smem = split_smem(g, base, split);
        if (smem > 227 * 1024) break;
        const int by_smem = (int)((228 * 1024) / (smem + 1024));
        const int ctas = std::min(by_smem, 1024 / (nthr * split));
        if (nthr * split * ctas > best_threads) {
            best = split;
            best_threads = nthr * split * ctas;
        }
    }
    return best;
}

// The stencil table as a kernel parameter when it fits one (PTAB_N float4) and
// the grid runs several waves of tiles: there the bond loops are bound by the
// shared-memory pipe that the table's reads would share (256^3 PMB step 2.43 ->
// 2.33 ms), while a grid of about one wave, bound by latency, measured slower
// with it (64^3: 0.064 -> 0.069 ms).
constexpr int PTAB_MIN_TILES = 2048;

static bool param_table(const float4 *host, int n, int ntiles, ParamTab &tp)
{
    if (!host || n <= 0 || n > PTAB_N || ntiles < PTAB_MIN_TILES) return false;
    memcpy(tp.e, host, sizeof(float4) * (size_t)n);
    return true;
}

template <int DIM, bool BRK, bool SPLIT>
static int launch_fast_split(const TileArgs &a, cudaStream_t st)
{
    const size_t smem = split_smem(a.g, pmb_fast_smem(a.g), a.split);
    static thread_local ParamTab tp;
    if (param_table(a.htab_a, a.ntab_a, a.g.ntiles, tp)) {
        PD_CUDA(smem_limit(pmb_fast_pt<DIM, BRK, SPLIT>, smem));
        pmb_fast_pt<DIM, BRK, SPLIT><<<a.g.ntiles, a.g.T / 2 * a.split, smem, st>>>(a, tp);
    } else {
        PD_CUDA(smem_limit(pmb_fast<DIM, BRK, SPLIT>, smem));
        pmb_fast<DIM, BRK, SPLIT><<<a.g.ntiles, a.g.T / 2 * a.split, smem, st>>>(a);
    }
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

template <int DIM, bool BRK>
static int launch_fast(const TileArgs &a0, cudaStream_t st)
{
    TileArgs a = a0;
    if (a.split == 0) {
        a.split = choose_split(a.g, pmb_fast_smem(a.g));
        // with breaking a thread records its words with decisions pending in 32 bits
        while (BRK && (a.g.W + a.split - 1) / a.split > 32 && 2 * a.split <= std::min(4, a.g.W)) a.split *= 2;
    }
    if (a.split > a.g.W || split_smem(a.g, pmb_fast_smem(a.g), a.split) > 227 * 1024 || a.g.T / 2 * a.split > 1024 ||
        (BRK && (a.g.W + a.split - 1) / a.split > 32)) {
        set_error("pair_threads = %d: more than the %d stencil words, more than 32 words per thread with "
                  "breaking, or the CTA exceeds its limits", a.split, a.g.W);
        return PD_EINVAL;
    }
    return a.split > 1 ? launch_fast_split<DIM, BRK, true>(a, st) : launch_fast_split<DIM, BRK, false>(a, st);
}

size_t pmb_generic_smem(const Geom &g, int precision)
{
    const int HX = g.bx + 2 * g.m, HY = g.by + 2 * g.m, HZ = g.dim == 3 ? g.bz + 2 * g.m : 1;
    return (size_t)HX * HY * HZ * (precision == PD_FP64 ? sizeof(double4_32a) : sizeof(float4));
}

template <int DIM, bool LINEAR, bool SPLIT>
static int launch_np_split(const TileArgs &a, cudaStream_t st)
{
    const size_t smem = split_smem(a.g, np_fast_smem(a.g), a.split);
    PD_CUDA(smem_limit(np_fast<DIM, LINEAR, SPLIT>, smem));
    np_fast<DIM, LINEAR, SPLIT><<<a.g.ntiles, a.g.T / 2 * a.split, smem, st>>>(a);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

template <bool LINEAR>
static int launch_np_fast2(const TileArgs &a, cudaStream_t st)
{
    const size_t smem = split_smem(a.g, np_fast_smem(a.g), a.split);
    PD_CUDA(smem_limit(np_fast2<LINEAR>, smem));
    np_fast2<LINEAR><<<a.g.ntiles, a.g.T / 4 * a.split, smem, st>>>(a);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

template <int DIM, bool LINEAR>
static int launch_np_fast(const TileArgs &a0, cudaStream_t st)
{
    TileArgs a = a0;   // pair_threads applies to PMB only: the split is chosen here
    a.split = choose_split(a.g, np_fast_smem(a.g));
    // 2D wide horizons (the one-pair kernel would split): two pairs per thread
    if (DIM == 2 && a.split > 1 && a.g.T >= 128) {
        a.split = choose_split(a.g, np_fast_smem(a.g), 2);
        return launch_np_fast2<LINEAR>(a, st);
    }
    return a.split > 1 ? launch_np_split<DIM, LINEAR, true>(a, st) : launch_np_split<DIM, LINEAR, false>(a, st);
}

// Every bond-based law: PMB, NP, LP.
int launch_pmb_args(const TileArgs &a, int precision, cudaStream_t st)
{
    const Geom &g = a.g;
    const bool brk = a.update_breaking && a.s_c > 0.0;
    if (precision == PD_FP32C && (a.model == PD_MODEL_NP || a.model == PD_MODEL_LP)) {
        const bool lin = a.model == PD_MODEL_LP;
        if (g.dim == 3) return lin ? launch_np_fast<3, true>(a, st) : launch_np_fast<3, false>(a, st);
        return lin ? launch_np_fast<2, true>(a, st) : launch_np_fast<2, false>(a, st);
    }
    if (precision == PD_FP32C) {
        if (g.dim == 3) return brk ? launch_fast<3, true>(a, st) : launch_fast<3, false>(a, st);
        return brk ? launch_fast<2, true>(a, st) : launch_fast<2, false>(a, st);
    }
    const size_t smem = pmb_generic_smem(g, precision);
    PD_CUDA(smem_limit(pmb_generic<double>, smem));
    pmb_generic<double><<<g.ntiles, 256, smem, st>>>(a);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

}  // namespace pdk
