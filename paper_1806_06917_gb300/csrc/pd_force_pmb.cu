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
#include <type_traits>

#include "pd_tile.cuh"

namespace pdk {

// ------------------------------------------------------------------ fast path

// FP32C, P points per thread (P = 2: packed f32x2 arithmetic on the points
// (lx, ly, lz) and (lx, ly, lz + bz/2) in 3D, (lx, ly) and (lx, ly + by/2) in
// 2D), horizon and halo box at run time. The stencil lives in shared memory as
// (dx, dy, dz, |d|) and (box offset, V_ij); the loop over it is rolled (partly
// unrolled), which keeps the kernel near 50 registers.
template <int DIM, int P, bool BRK>
__global__ void __launch_bounds__(256, 3) pmb_fast(const TileArgs a)
{
    const Geom &g = a.g;
    const int m = g.m, S = g.S;
    const int HX = g.bx + 2 * m, HY = g.by + 2 * m, HZ = DIM == 3 ? g.bz + 2 * m : 1;
    const int nbox = HX * HY * HZ;
    extern __shared__ float4 smem4[];
    float4 *box = smem4;
    float4 *tabA = box + nbox;                                  // dx, dy, dz, |d|
    int2 *tabB = reinterpret_cast<int2 *>(tabA + S);            // box offset, V_ij bits

    const int tile = blockIdx.x;
    const int4 org = __ldg(&a.tile_org[tile]);
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
        const int4 d = __ldg(&a.stencil[k]);
        const float r0 = (float)__ldg(&a.stencil_r0[k]);
        tabA[k] = make_float4((float)d.x, (float)d.y, (float)d.z, r0);
        const float vij = a.vol_corr ? (float)vol_factor_lattice(m, (double)r0) : 1.f;
        tabB[k] = make_int2(d.x + HX * (d.y + HY * d.z), __float_as_int(vij));
    }
    stage_box32(box, HX, HY, nbox, m, a, org, tile_ref32(a, tile), (float)a.inv_h);
    __syncthreads();

    const int nthr = g.T / P;
    const float s_c = (float)a.s_c;
    for (int t = threadIdx.x; t < nthr; t += blockDim.x) {
        const int lx = t & (g.bx - 1);
        const int r1 = t >> g.lbx;
        int bi[P], slot[P];
        bool act[P];
        Pk<float, P> ux, uy, uz;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            int ly, lz;
            if (DIM == 3) {
                ly = r1 & (g.by - 1);
                lz = (r1 >> g.lby) + p * (g.bz / P);
            } else {
                ly = r1 + p * (g.by / P);
                lz = 0;
            }
            bi[p] = (lx + m) + HX * ((ly + m) + HY * (DIM == 3 ? lz + m : 0));
            slot[p] = tile * g.T + brick_code(DIM, lx, ly, lz);
            act[p] = org.x + lx < g.nx && org.y + ly < g.ny && org.z + lz < g.nz;
            const float4 ui = box[bi[p]];
            ux.v[p] = ui.x;
            uy.v[p] = ui.y;
            uz.v[p] = ui.z;
        }
        Pk<float, P> Fx = splat<float, P>(0.f), Fy = Fx, Fz = Fx;
        for (int w = 0; w < g.W; ++w) {
            uint32_t word[P], cur[P];
#pragma unroll
            for (int p = 0; p < P; ++p) word[p] = cur[p] = act[p] ? a.mask[(size_t)w * g.nslots + slot[p]] : 0u;
            uint32_t keep[P];
#pragma unroll
            for (int p = 0; p < P; ++p) keep[p] = word[p];
            const int nb = min(32, S - 32 * w);
#pragma unroll 4
            for (int b = 0; b < nb; ++b) {
                const int k = 32 * w + b;
                const float4 ta = tabA[k];
                const int2 tb = tabB[k];
                Pk<float, P> ex, ey, ez;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const float4 rj = box[bi[p] + tb.x];
                    ex.v[p] = rj.x;
                    ey.v[p] = rj.y;
                    ez.v[p] = rj.z;
                }
                ex = psub(ex, ux);
                ey = psub(ey, uy);
                ez = psub(ez, uz);
                const Pk<float, P> yx = padds(ex, ta.x), yy = padds(ey, ta.y);
                const Pk<float, P> yz = DIM == 3 ? padds(ez, ta.z) : ez;
                Pk<float, P> q = pmul(yx, yx);
                q = pfma(yy, yy, q);
                if (DIM == 3) q = pfma(yz, yz, q);
                // 2 d.eta + eta.eta = eta.(y + d)
                Pk<float, P> num = pmul(ex, padds(yx, ta.x));
                num = pfma(ey, padds(yy, ta.y), num);
                if (DIM == 3) num = pfma(ez, padds(yz, ta.z), num);
                const Pk<float, P> rs = prsqrt(q);
                const Pk<float, P> den = pmuls(padds(pmul(q, rs), ta.w), ta.w);
                const Pk<float, P> s = pdiv(num, den);
                Pk<float, P> wgt = pmuls(pmul(s, rs), __int_as_float(tb.y));
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    bool intact = cur[p] & 1u;
                    if (BRK) {
                        const bool brk = intact && s.v[p] > s_c;
                        if (brk) keep[p] &= ~(1u << b);
                        intact = intact && !brk;
                    }
                    cur[p] >>= 1;
                    wgt.v[p] = intact ? wgt.v[p] : 0.f;
                }
                Fx = pfma(wgt, yx, Fx);
                Fy = pfma(wgt, yy, Fy);
                if (DIM == 3) Fz = pfma(wgt, yz, Fz);
            }
            if (BRK) {
#pragma unroll
                for (int p = 0; p < P; ++p)
                    if (act[p] && keep[p] != word[p]) a.mask[(size_t)w * g.nslots + slot[p]] = keep[p];
            }
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (!act[p]) continue;
            const double f[3] = {a.cV * (double)Fx.v[p], a.cV * (double)Fy.v[p], a.cV * (double)Fz.v[p]};
            point_epilogue(a, slot[p], f, DIM, false);
        }
    }
}

size_t pmb_fast_smem(const Geom &g)
{
    const size_t nbox = (size_t)(g.bx + 2 * g.m) * (g.by + 2 * g.m) * (g.dim == 3 ? g.bz + 2 * g.m : 1);
    return nbox * sizeof(float4) + (size_t)g.S * (sizeof(float4) + sizeof(int2));
}

// ------------------------------------------------------------------ generic

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
                const R yx = ex + (R)d.x, yy = ey + (R)d.y, yz = ez + (R)d.z;
                const R q = yx * yx + yy * yy + yz * yz;
                const R num = ex * ex + ey * ey + ez * ez +
                              (R)2 * ((R)d.x * ex + (R)d.y * ey + (R)d.z * ez);
                const R r0 = (R)__ldg(&a.stencil_r0[32 * w + b]);
                const R rs = prsqrt1(q);
                const R s = pdiv1(num, r0 * (q * rs + r0));
                if (brk_on && s > s_c) {
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

template <int DIM, int P, bool BRK>
static int launch_fast(const TileArgs &a, cudaStream_t st)
{
    const size_t smem = pmb_fast_smem(a.g);
    PD_CUDA(cudaFuncSetAttribute(pmb_fast<DIM, P, BRK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int threads = a.g.T / P < 256 ? a.g.T / P : 256;
    pmb_fast<DIM, P, BRK><<<a.g.ntiles, threads, smem, st>>>(a);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

size_t pmb_generic_smem(const Geom &g, int precision)
{
    const int HX = g.bx + 2 * g.m, HY = g.by + 2 * g.m, HZ = g.dim == 3 ? g.bz + 2 * g.m : 1;
    return (size_t)HX * HY * HZ * (precision == PD_FP64 ? sizeof(double4_32a) : sizeof(float4));
}

int launch_pmb_args(const TileArgs &a, int precision, cudaStream_t st)
{
    const Geom &g = a.g;
    const bool brk = a.update_breaking && a.s_c > 0.0;
    if (precision == PD_FP32C) {
        if (g.dim == 3) return brk ? launch_fast<3, 2, true>(a, st) : launch_fast<3, 2, false>(a, st);
        return brk ? launch_fast<2, 2, true>(a, st) : launch_fast<2, 2, false>(a, st);
    }
    const size_t smem = pmb_generic_smem(g, precision);
    PD_CUDA(cudaFuncSetAttribute(pmb_generic<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    pmb_generic<double><<<g.ntiles, 256, smem, st>>>(a);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

}  // namespace pdk
