// pd_reduce.cu -- strain and kinetic energy per point and their FP64 sums.
//
// Per point (lattice units, same staging as the force kernels):
//   PMB: W_i = 1/2 sum_j c s^2 |xi| / 2 V_j V_ij = (c V h / 4) sum_j s^2 |d| V_ij
//   LPS: W_i = K theta_i^2 / 2 + 15 mu / (2 m~_i) sum_j (e~ - theta_i |d| / 3)^2 V_ij
// (pair potential c s^2 |xi| / 2, whose eta-gradient is the PMB pair force; LPS
// energy of Silling 2007). Kinetic: rho |v_i|^2 V / 2.
// The sums over points run in FP64 in a fixed order: each block reduces a fixed
// contiguous range of slots with a fixed tree, then one block reduces the block
// partials the same way. Same inputs, same bits.
#include <type_traits>

#include "pd_tile.cuh"

namespace pdk {

template <class R>
__global__ void __launch_bounds__(256) energy_generic(const TileArgs a)
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
    const bool lps = a.model == PD_MODEL_LPS;
    const bool np_law = a.model == PD_MODEL_NP || a.model == PD_MODEL_LP;
    for (int t = threadIdx.x; t < g.T; t += blockDim.x) {
        const int lx = t % g.bx, ly = (t / g.bx) % g.by, lz = t / (g.bx * g.by);
        const int slot = tile * g.T + brick_code(g.dim, lx, ly, lz);
        if (!(org.x + lx < g.nx && org.y + ly < g.ny && org.z + lz < g.nz)) {
            a.epoint[slot] = 0.0;
            continue;
        }
        const int bi = (lx + m) + HX * ((ly + m) + HY * (g.dim == 3 ? lz + m : 0));
        const R4 ui = box[bi];
        R th = 0;
        if (lps) th = sizeof(R) == 4 ? (R)a.theta32[slot] : (R)a.theta64[slot];
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
                if (np_law) {
                    // Algorithm 1's energy: J psi(|xi| S^2) V_ij; with r = h |d| S^2,
                    // NP: psi / (C beta) = (1 - exp(-beta r)) / beta, LP: psi / (C beta) = r
                    if (d.w >= m * m) continue;
                    const R S = ((R)d.x * ex + (R)d.y * ey + (R)d.z * ez) / (R)d.w;
                    const R rr = (R)a.h * r0 * S * S;
                    const R vij = a.vol_corr ? (R)vol_factor_lattice(m, (double)r0) : (R)1;
                    acc += (a.model == PD_MODEL_NP ? -expm1(-(R)a.psi_beta * rr) / (R)a.psi_beta : rr) * vij;
                    continue;
                }
                const R yx = ex + (R)d.x, yy = ey + (R)d.y, yz = ez + (R)d.z;
                const R q = yx * yx + yy * yy + yz * yz;
                const R num = ex * ex + ey * ey + ez * ez + (R)2 * ((R)d.x * ex + (R)d.y * ey + (R)d.z * ez);
                const R rr = q * prsqrt1(q);
                const R vij = a.vol_corr ? (R)vol_factor_lattice(m, (double)r0) : (R)1;
                if (lps) {
                    const R ed = pdiv1(num, rr + r0) - th * r0 / (R)3;
                    acc += ed * ed * vij;
                } else {
                    const R s = pdiv1(num, r0 * (rr + r0));
                    acc += s * s * r0 * vij;
                }
            }
        }
        double W;
        if (lps) {
            const double mt = sizeof(R) == 4 ? 1.0 / (double)a.minv32[slot] : a.mtil[slot];
            W = 0.5 * a.K * (double)th * (double)th + 0.5 * a.B / mt * (double)acc;
        } else if (np_law) {
            // W_i = sum_j J psi V_j V_ij / (delta |B|) = (c V / 4) sum_j J (psi / (C beta)) V_ij
            W = 0.25 * a.cV * (double)acc;
        } else {
            W = 0.25 * a.cV * a.h * (double)acc;
        }
        a.epoint[slot] = W;
    }
}

__global__ void kinetic_points(const TileArgs a, double *out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.g.nslots) return;
    double v2 = 0.0;
    for (int c = 0; c < a.g.dim; ++c) v2 += a.v[c][s] * a.v[c][s];
    out[s] = v2;   // inactive slots hold v = 0
}

// Fixed-order block sums of x[0..n): block b owns [b*chunk, (b+1)*chunk).
__global__ void __launch_bounds__(256) reduce_blocks(const double *x, long long n, long long chunk,
                                                      double *partial)
{
    __shared__ double sh[256];
    const long long lo = (long long)blockIdx.x * chunk;
    const long long hi = min(n, lo + chunk);
    double acc = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += x[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(256) reduce_final(const double *partial, int nb, double scale,
                                                     double *out)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = scale * sh[0];
}

// Number of block partials reduce_sum() uses for n values.
int reduce_blocks_for(long long n)
{
    long long nb = (n + 4095) / 4096;
    if (nb < 1) nb = 1;
    if (nb > 1024) nb = 1024;
    return (int)nb;
}

// out = scale * sum(x[0..n)) in a fixed order; partial needs reduce_blocks_for(n) doubles.
int reduce_sum(const double *x, long long n, double scale, double *partial, double *out, cudaStream_t st)
{
    const int nb = reduce_blocks_for(n);
    const long long chunk = (n + nb - 1) / nb;
    reduce_blocks<<<nb, 256, 0, st>>>(x, n, chunk, partial);
    PD_CUDA(cudaGetLastError());
    reduce_final<<<1, 256, 0, st>>>(partial, nb, scale, out);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

size_t energy_smem(const Geom &g, int precision)
{
    const size_t nbox = (size_t)(g.bx + 2 * g.m) * (g.by + 2 * g.m) * (g.dim == 3 ? g.bz + 2 * g.m : 1);
    return nbox * (precision == PD_FP64 ? sizeof(double4_32a) : sizeof(float4));
}

// Strain energy per point into a.epoint, kinetic |v|^2 per point into kin.
int launch_energy_points(const TileArgs &a, int precision, double *kin, cudaStream_t st)
{
    const size_t smem = energy_smem(a.g, precision);
    if (precision == PD_FP64) {
        PD_CUDA(smem_limit(energy_generic<double>, smem));
        energy_generic<double><<<a.g.ntiles, 256, smem, st>>>(a);
    } else {
        PD_CUDA(smem_limit(energy_generic<float>, smem));
        energy_generic<float><<<a.g.ntiles, 256, smem, st>>>(a);
    }
    PD_CUDA(cudaGetLastError());
    kinetic_points<<<(a.g.nslots + 255) / 256, 256, 0, st>>>(a, kin);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

}  // namespace pdk
