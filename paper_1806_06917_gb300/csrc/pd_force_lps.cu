// pd_force_lps.cu -- state-based linear peridynamic solid (LPS): the dilatation
// pass and the force pass of Algorithm 2, the latter fused with the explicit
// update (Eq. (4); Eqs. (7)-(9)).
//
// In lattice units (xi = d, e~ = e / h, m~ = m / (h^2 V), omega = 1):
//   e~      = (2 d.eta + eta.eta) / (|y| + |d|)          cancellation-free extension
//   theta_i = (3 / m~_i) sum_j |d| e~ V_ij                Algorithm 2, second loop
//   f_i     = (1/h) sum_j [ (3K - 5mu) |d| (a_i + a_j) + 15 mu e~ (b_i + b_j) ] V_ij y/|y|
// with a = theta / m~, b = 1 / m~. The bracket is t_i<xi> + t_j<-xi> of Algorithm
// 2's third loop (t = 3K theta |xi| / m + 15 mu e^d / m, e^d = e - theta |xi| / 3)
// gathered at i: the "f_j -= t M V_i" scatter of row j lands on i as + t_j M_ij.
// The weighted volume m~ is computed once at the neighbour build.
#include <type_traits>

#include "pd_tile.cuh"

namespace pdk {

// Staging of the force pass: float4 (u~x, u~y, u~z, a_j) and float b_j.
__device__ __forceinline__ void stage_box32_lps(float4 *box, float *boxb, int HX, int HY, int nbox,
                                                int m, const TileArgs &a, const int4 &org,
                                                const Ref32 &ref, float inv_h)
{
    for (int b = threadIdx.x; b < nbox; b += blockDim.x) {
        int bxl = b % HX, rest = b / HX;
        int byl = rest % HY, bzl = rest / HY;
        int x = org.x + bxl - m, y = org.y + byl - m, z = org.z + bzl - m;
        int s = slot_at(a.g, a.tile_lut, x, y, z);
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        float rb = 0.f;
        if (s >= 0) {
            float4 hi = __ldg(&a.src_hl[2 * s]);
            float4 lo = __ldg(&a.src_hl[2 * s + 1]);
            r.x = ((hi.x - ref.hx) + (lo.x - ref.lx)) * inv_h;
            r.y = ((hi.y - ref.hy) + (lo.y - ref.ly)) * inv_h;
            r.z = ((hi.z - ref.hz) + (lo.z - ref.lz)) * inv_h;
            rb = __ldg(&a.minv32[s]);
            r.w = a.theta32[s] * rb;
        }
        box[b] = r;
        boxb[b] = rb;
    }
}

// ------------------------------------------------------------------ fast path

// FP32C, 3D, P points per thread, horizon at run time; rolled loop over a
// shared-memory stencil table (dx, dy, dz, |d|) and (box offset, V_ij).
__device__ __forceinline__ void build_tab(const TileArgs &a, int HX, int HY, float4 *tabA, int2 *tabB)
{
    for (int k = threadIdx.x; k < a.g.S; k += blockDim.x) {
        const int4 d = __ldg(&a.stencil[k]);
        const float r0 = (float)__ldg(&a.stencil_r0[k]);
        tabA[k] = make_float4((float)d.x, (float)d.y, (float)d.z, r0);
        const float vij = a.vol_corr ? (float)vol_factor_lattice(a.g.m, (double)r0) : 1.f;
        tabB[k] = make_int2(d.x + HX * (d.y + HY * d.z), __float_as_int(vij));
    }
}

template <int P>
__global__ void __launch_bounds__(256, 3) lps_dil_fast(const TileArgs a)
{
    const Geom &g = a.g;
    const int m = g.m, S = g.S;
    const int HX = g.bx + 2 * m, HY = g.by + 2 * m, HZ = g.bz + 2 * m;
    const int nbox = HX * HY * HZ;
    extern __shared__ float4 smem4[];
    float4 *box = smem4;
    float4 *tabA = box + nbox;
    int2 *tabB = reinterpret_cast<int2 *>(tabA + S);
    const int tile = blockIdx.x;
    const int4 org = __ldg(&a.tile_org[tile]);
    build_tab(a, HX, HY, tabA, tabB);
    stage_box32(box, HX, HY, nbox, m, a, org, tile_ref32(a, tile), (float)a.inv_h);
    __syncthreads();

    const int nthr = g.T / P;
    for (int t = threadIdx.x; t < nthr; t += blockDim.x) {
        const int lx = t & (g.bx - 1), r1 = t >> g.lbx;
        const int ly = r1 & (g.by - 1), lz0 = r1 >> g.lby;
        int bi[P], slot[P];
        bool act[P];
        Pk<float, P> ux, uy, uz;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int lz = lz0 + p * (g.bz / P);
            bi[p] = (lx + m) + HX * ((ly + m) + HY * (lz + m));
            slot[p] = tile * g.T + brick_code(3, lx, ly, lz);
            act[p] = org.x + lx < g.nx && org.y + ly < g.ny && org.z + lz < g.nz;
            const float4 ui = box[bi[p]];
            ux.v[p] = ui.x;
            uy.v[p] = ui.y;
            uz.v[p] = ui.z;
        }
        Pk<float, P> acc = splat<float, P>(0.f);
        for (int w = 0; w < g.W; ++w) {
            uint32_t cur[P];
#pragma unroll
            for (int p = 0; p < P; ++p) cur[p] = act[p] ? a.mask[(size_t)w * g.nslots + slot[p]] : 0u;
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
                const Pk<float, P> yx = padds(ex, ta.x), yy = padds(ey, ta.y), yz = padds(ez, ta.z);
                Pk<float, P> q = pmul(yx, yx);
                q = pfma(yy, yy, q);
                q = pfma(yz, yz, q);
                Pk<float, P> num = pmul(ex, padds(yx, ta.x));
                num = pfma(ey, padds(yy, ta.y), num);
                num = pfma(ez, padds(yz, ta.z), num);
                Pk<float, P> e = pdiv(num, padds(pmul(q, prsqrt(q)), ta.w));
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    e.v[p] = (cur[p] & 1u) ? e.v[p] : 0.f;
                    cur[p] >>= 1;
                }
                acc = pfmas(e, ta.w * __int_as_float(tb.y), acc);
            }
        }
#pragma unroll
        for (int p = 0; p < P; ++p)
            if (act[p]) a.theta32[slot[p]] = 3.f * __ldg(&a.minv32[slot[p]]) * acc.v[p];
    }
}

template <int P>
__global__ void __launch_bounds__(256, 3) lps_force_fast(const TileArgs a)
{
    const Geom &g = a.g;
    const int m = g.m, S = g.S;
    const int HX = g.bx + 2 * m, HY = g.by + 2 * m, HZ = g.bz + 2 * m;
    const int nbox = HX * HY * HZ;
    extern __shared__ float4 smem4[];
    float4 *box = smem4;
    float4 *tabA = box + nbox;
    int2 *tabB = reinterpret_cast<int2 *>(tabA + S);
    float *boxb = reinterpret_cast<float *>(tabB + S);
    const int tile = blockIdx.x;
    const int4 org = __ldg(&a.tile_org[tile]);
    build_tab(a, HX, HY, tabA, tabB);
    stage_box32_lps(box, boxb, HX, HY, nbox, m, a, org, tile_ref32(a, tile), (float)a.inv_h);
    __syncthreads();

    const float A = (float)a.A, B = (float)a.B;
    const int nthr = g.T / P;
    for (int t = threadIdx.x; t < nthr; t += blockDim.x) {
        const int lx = t & (g.bx - 1), r1 = t >> g.lbx;
        const int ly = r1 & (g.by - 1), lz0 = r1 >> g.lby;
        int bi[P], slot[P];
        bool act[P];
        Pk<float, P> ux, uy, uz, ai, bi_;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int lz = lz0 + p * (g.bz / P);
            bi[p] = (lx + m) + HX * ((ly + m) + HY * (lz + m));
            slot[p] = tile * g.T + brick_code(3, lx, ly, lz);
            act[p] = org.x + lx < g.nx && org.y + ly < g.ny && org.z + lz < g.nz;
            const float4 ui = box[bi[p]];
            ux.v[p] = ui.x;
            uy.v[p] = ui.y;
            uz.v[p] = ui.z;
            ai.v[p] = ui.w;
            bi_.v[p] = boxb[bi[p]];
        }
        Pk<float, P> Fx = splat<float, P>(0.f), Fy = Fx, Fz = Fx;
        for (int w = 0; w < g.W; ++w) {
            uint32_t cur[P];
#pragma unroll
            for (int p = 0; p < P; ++p) cur[p] = act[p] ? a.mask[(size_t)w * g.nslots + slot[p]] : 0u;
            const int nb = min(32, S - 32 * w);
#pragma unroll 4
            for (int b = 0; b < nb; ++b) {
                const int k = 32 * w + b;
                const float4 ta = tabA[k];
                const int2 tb = tabB[k];
                Pk<float, P> ex, ey, ez, aj, bj;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const float4 rj = box[bi[p] + tb.x];
                    ex.v[p] = rj.x;
                    ey.v[p] = rj.y;
                    ez.v[p] = rj.z;
                    aj.v[p] = rj.w;
                    bj.v[p] = boxb[bi[p] + tb.x];
                }
                ex = psub(ex, ux);
                ey = psub(ey, uy);
                ez = psub(ez, uz);
                const Pk<float, P> yx = padds(ex, ta.x), yy = padds(ey, ta.y), yz = padds(ez, ta.z);
                Pk<float, P> q = pmul(yx, yx);
                q = pfma(yy, yy, q);
                q = pfma(yz, yz, q);
                Pk<float, P> num = pmul(ex, padds(yx, ta.x));
                num = pfma(ey, padds(yy, ta.y), num);
                num = pfma(ez, padds(yz, ta.z), num);
                const Pk<float, P> rs = prsqrt(q);
                const Pk<float, P> e = pdiv(num, padds(pmul(q, rs), ta.w));
                // t_i + t_j = A |d| (a_i + a_j) + B e (b_i + b_j)
                Pk<float, P> gg = pmuls(padd(ai, aj), A * ta.w);
                gg = pfma(pmuls(e, B), padd(bi_, bj), gg);
                Pk<float, P> wgt = pmuls(pmul(gg, rs), __int_as_float(tb.y));
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    wgt.v[p] = (cur[p] & 1u) ? wgt.v[p] : 0.f;
                    cur[p] >>= 1;
                }
                Fx = pfma(wgt, yx, Fx);
                Fy = pfma(wgt, yy, Fy);
                Fz = pfma(wgt, yz, Fz);
            }
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (!act[p]) continue;
            const double f[3] = {a.inv_h * (double)Fx.v[p], a.inv_h * (double)Fy.v[p], a.inv_h * (double)Fz.v[p]};
            point_epilogue(a, slot[p], f, 3, false);
        }
    }
}

size_t lps_fast_smem(const Geom &g, bool dil)
{
    const size_t nbox = (size_t)(g.bx + 2 * g.m) * (g.by + 2 * g.m) * (g.bz + 2 * g.m);
    return nbox * (sizeof(float4) + (dil ? 0 : sizeof(float))) + (size_t)g.S * (sizeof(float4) + sizeof(int2));
}

// ------------------------------------------------------------------ generic

template <class R>
__global__ void __launch_bounds__(256) lps_dil_generic(const TileArgs a)
{
    using R4 = typename std::conditional<sizeof(R) == 4, float4, double4_32a>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R4 *box = reinterpret_cast<R4 *>(smem_raw);
    const Geom &g = a.g;
    const int m = g.m;
    const int HX = g.bx + 2 * m, HY = g.by + 2 * m, HZ = g.bz + 2 * m;
    const int nbox = HX * HY * HZ;
    const int tile = blockIdx.x;
    const int4 org = __ldg(&a.tile_org[tile]);
    if constexpr (sizeof(R) == 4)
        stage_box32(reinterpret_cast<float4 *>(box), HX, HY, nbox, m, a, org, tile_ref32(a, tile), (float)a.inv_h);
    else
        stage_box64(reinterpret_cast<double4_32a *>(box), HX, HY, nbox, m, a, org, tile_ref64(a, tile), a.inv_h);
    __syncthreads();
    for (int t = threadIdx.x; t < g.T; t += blockDim.x) {
        const int lx = t % g.bx, ly = (t / g.bx) % g.by, lz = t / (g.bx * g.by);
        const int slot = tile * g.T + brick_code(3, lx, ly, lz);
        if (!(org.x + lx < g.nx && org.y + ly < g.ny && org.z + lz < g.nz)) continue;
        const int bi = (lx + m) + HX * ((ly + m) + HY * (lz + m));
        const R4 ui = box[bi];
        R acc = 0;
        for (int w = 0; w < g.W; ++w) {
            const uint32_t word = a.mask[(size_t)w * g.nslots + slot];
            const int nb = min(32, g.S - 32 * w);
            for (int b = 0; b < nb; ++b) {
                if (!((word >> b) & 1u)) continue;
                const int4 d = __ldg(&a.stencil[32 * w + b]);
                const R r0 = (R)__ldg(&a.stencil_r0[32 * w + b]);
                const R4 rj = box[bi + d.x + HX * (d.y + HY * d.z)];
                const R ex = rj.x - ui.x, ey = rj.y - ui.y, ez = rj.z - ui.z;
                const R yx = ex + (R)d.x, yy = ey + (R)d.y, yz = ez + (R)d.z;
                const R q = yx * yx + yy * yy + yz * yz;
                const R num = ex * ex + ey * ey + ez * ez + (R)2 * ((R)d.x * ex + (R)d.y * ey + (R)d.z * ez);
                const R e = pdiv1(num, q * prsqrt1(q) + r0);
                R vij = a.vol_corr ? (R)vol_factor_lattice(m, (double)r0) : (R)1;
                acc += r0 * vij * e;
            }
        }
        if constexpr (sizeof(R) == 4)
            a.theta32[slot] = 3.f * a.minv32[slot] * acc;
        else
            a.theta64[slot] = 3.0 * acc / a.mtil[slot];
    }
}

template <class R>
__global__ void __launch_bounds__(256) lps_force_generic(const TileArgs a)
{
    using R4 = typename std::conditional<sizeof(R) == 4, float4, double4_32a>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geom &g = a.g;
    const int m = g.m;
    const int HX = g.bx + 2 * m, HY = g.by + 2 * m, HZ = g.bz + 2 * m;
    const int nbox = HX * HY * HZ;
    R4 *box = reinterpret_cast<R4 *>(smem_raw);
    R *boxb = reinterpret_cast<R *>(box + nbox);
    const int tile = blockIdx.x;
    const int4 org = __ldg(&a.tile_org[tile]);
    if constexpr (sizeof(R) == 4) {
        stage_box32_lps(reinterpret_cast<float4 *>(box), reinterpret_cast<float *>(boxb), HX, HY, nbox, m,
                        a, org, tile_ref32(a, tile), (float)a.inv_h);
    } else {
        const double3 ref = tile_ref64(a, tile);
        for (int b = threadIdx.x; b < nbox; b += blockDim.x) {
            int x, y, z;
            box_coord(b, HX, HY, m, 3, org, x, y, z);
            int s = slot_at(g, a.tile_lut, x, y, z);
            double4_32a r = make_double4_32a(0.0, 0.0, 0.0, 0.0);
            double rb = 0.0;
            if (s >= 0) {
                double4_32a d = a.src_d4[s];
                r.x = (d.x - ref.x) * a.inv_h;
                r.y = (d.y - ref.y) * a.inv_h;
                r.z = (d.z - ref.z) * a.inv_h;
                rb = 1.0 / a.mtil[s];
                r.w = a.theta64[s] * rb;
            }
            reinterpret_cast<double4_32a *>(box)[b] = r;
            reinterpret_cast<double *>(boxb)[b] = rb;
        }
    }
    __syncthreads();
    const R A = (R)a.A, B = (R)a.B;
    for (int t = threadIdx.x; t < g.T; t += blockDim.x) {
        const int lx = t % g.bx, ly = (t / g.bx) % g.by, lz = t / (g.bx * g.by);
        const int slot = tile * g.T + brick_code(3, lx, ly, lz);
        if (!(org.x + lx < g.nx && org.y + ly < g.ny && org.z + lz < g.nz)) continue;
        const int bi = (lx + m) + HX * ((ly + m) + HY * (lz + m));
        const R4 ui = box[bi];
        const R bi_ = boxb[bi];
        R Fx = 0, Fy = 0, Fz = 0;
        for (int w = 0; w < g.W; ++w) {
            const uint32_t word = a.mask[(size_t)w * g.nslots + slot];
            const int nb = min(32, g.S - 32 * w);
            for (int b = 0; b < nb; ++b) {
                if (!((word >> b) & 1u)) continue;
                const int4 d = __ldg(&a.stencil[32 * w + b]);
                const R r0 = (R)__ldg(&a.stencil_r0[32 * w + b]);
                const int bj = bi + d.x + HX * (d.y + HY * d.z);
                const R4 rj = box[bj];
                const R ex = rj.x - ui.x, ey = rj.y - ui.y, ez = rj.z - ui.z;
                const R yx = ex + (R)d.x, yy = ey + (R)d.y, yz = ez + (R)d.z;
                const R q = yx * yx + yy * yy + yz * yz;
                const R num = ex * ex + ey * ey + ez * ez + (R)2 * ((R)d.x * ex + (R)d.y * ey + (R)d.z * ez);
                const R rs = prsqrt1(q);
                const R e = pdiv1(num, q * rs + r0);
                const R gg = A * r0 * (ui.w + rj.w) + B * e * (bi_ + boxb[bj]);
                R wgt = gg * rs;
                if (a.vol_corr) wgt *= (R)vol_factor_lattice(m, (double)r0);
                Fx += wgt * yx;
                Fy += wgt * yy;
                Fz += wgt * yz;
            }
        }
        const double f[3] = {a.inv_h * (double)Fx, a.inv_h * (double)Fy, a.inv_h * (double)Fz};
        point_epilogue(a, slot, f, 3, sizeof(R) == 8);
    }
}

// ---------------------------------------------------------------- dispatch

size_t lps_generic_smem(const Geom &g, int precision, bool dil)
{
    if (precision != PD_FP64) return lps_fast_smem(g, dil);
    const size_t nbox = (size_t)(g.bx + 2 * g.m) * (g.by + 2 * g.m) * (g.bz + 2 * g.m);
    return nbox * (sizeof(double4_32a) + (dil ? 0 : sizeof(double)));
}

// dil = 1: dilatation pass; dil = 0: force pass (+ update per a.mode).
int launch_lps_args(const TileArgs &a, int precision, int dil, cudaStream_t st)
{
    const Geom &g = a.g;
    const size_t smem = lps_generic_smem(g, precision, dil);
    if (precision == PD_FP32C) {
        auto k = dil ? lps_dil_fast<2> : lps_force_fast<2>;
        PD_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int threads = g.T / 2 < 256 ? g.T / 2 : 256;
        k<<<g.ntiles, threads, smem, st>>>(a);
    } else {
        auto k = dil ? lps_dil_generic<double> : lps_force_generic<double>;
        PD_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k<<<g.ntiles, 256, smem, st>>>(a);
    }
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

}  // namespace pdk
