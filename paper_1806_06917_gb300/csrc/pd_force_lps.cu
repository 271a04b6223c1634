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
#include <string.h>

#include <type_traits>

#include "pd_lps_fast.cuh"

namespace pdk {

size_t lps_fast_smem(const Geom &g, bool dil)
{
    const size_t n = (size_t)(g.bx + 2 * g.m) * (g.by + 2 * g.m) * (g.bz / 2 + 2 * g.m);
    const size_t p2 = ((n + 1) / 2) * sizeof(float4);
    if (dil) return n * sizeof(float4) + p2 + (size_t)g.S * 3 * sizeof(float4);
    return 2 * n * sizeof(float4) + p2 + (size_t)g.S * 3 * sizeof(float4);
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
    {
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
        // dilatation: two pairs per thread from 2^7-point tiles and two stencil words on
        const bool dil2 = dil && g.T >= 128 && g.W >= 2;
        const int threads = dil ? (g.T / 2 < 256 ? g.T / 2 : 256) : g.T;
        static thread_local ParamTab tp;
        // the table as a kernel parameter on grids of several waves (as for PMB,
        // pd_force_pmb.cu): 128^3 force pass 0.392 -> 0.361 ms
        // (the dilatation's table is tab_a, the force pass's tab_b)
        const float4 *ht = dil ? a.htab_a : a.htab_b;
        const int nt = dil ? a.ntab_a : a.ntab_b;
        const bool pt = ht && nt > 0 && nt <= PTAB_N && g.ntiles >= 2048;
        if (pt) {
            memcpy(tp.e, ht, sizeof(float4) * (size_t)nt);
            auto k = dil ? (dil2 ? (a.vol_corr ? lps_dil_fast2_pt<true> : lps_dil_fast2_pt<false>)
                                 : (a.vol_corr ? lps_dil_fast_pt<true> : lps_dil_fast_pt<false>))
                         : (a.vol_corr ? lps_force_fast_pt<true> : lps_force_fast_pt<false>);
            PD_CUDA(smem_limit(k, smem));
            k<<<g.ntiles, threads, smem, st>>>(a, tp);
        } else {
            auto k = dil ? (dil2 ? (a.vol_corr ? lps_dil_fast2<true> : lps_dil_fast2<false>)
                                 : (a.vol_corr ? lps_dil_fast<true> : lps_dil_fast<false>))
                         : (a.vol_corr ? lps_force_fast<true> : lps_force_fast<false>);
            PD_CUDA(smem_limit(k, smem));
            k<<<g.ntiles, threads, smem, st>>>(a);
        }
    } else {
        auto k = dil ? lps_dil_generic<double> : lps_force_generic<double>;
        PD_CUDA(smem_limit(k, smem));
        k<<<g.ntiles, 256, smem, st>>>(a);
    }
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

}  // namespace pdk
