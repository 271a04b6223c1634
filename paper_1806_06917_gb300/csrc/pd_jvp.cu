// pd_jvp.cu -- tangent Jacobian-vector product of the PMB internal force and its
// adjoint: the matrix-free replacement of the central-difference stiffness
// assembly of Eq. (6) / Algorithm 3.
//
// With f_pair(eta) = c s n, n = y/|y|, s = (|y| - |xi|)/|xi| and y = xi + eta,
//   d f_pair / d eta = c [ n n^T / |xi| + s (I - n n^T) / |y| ] =: D_ij,
//   (K w)_i = sum_j D_ij (w_j - w_i) V_j V_ij.
// In lattice units (|xi| = h|d|, |y| = h r):
//   (K w)_i = (c V / h) sum_j V_ij [ (n.dw)(1/|d| - s/r) n + (s/r) dw ].
// The adjoint kernel evaluates the transposed gather
//   (K^T v)_i = sum_j D_ji V_i V_ij v_j - sum_j D_ij V_j V_ij v_i
// with D_ji computed from the bond as seen from j (xi -> -xi, eta -> -eta).
// Displacements are staged as in the force kernels; the direction w is staged
// relative to the tile's reference value so that w_j - w_i keeps its precision.
#include <type_traits>

#include "pd_tile.cuh"

namespace pdk {

template <class R>
__global__ void __launch_bounds__(256) jvp_generic(const TileArgs a)
{
    using R4 = typename std::conditional<sizeof(R) == 4, float4, double4_32a>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geom &g = a.g;
    const int m = g.m;
    const int HX = g.bx + 2 * m, HY = g.by + 2 * m, HZ = g.dim == 3 ? g.bz + 2 * m : 1;
    const int nbox = HX * HY * HZ;
    R4 *box = reinterpret_cast<R4 *>(smem_raw);
    R4 *wbox = box + nbox;
    const int tile = blockIdx.x;
    const int4 org = __ldg(&a.tile_org[tile]);
    if constexpr (sizeof(R) == 4)
        stage_box32(reinterpret_cast<float4 *>(box), HX, HY, nbox, m, a, org, tile_ref32(a, tile), (float)a.inv_h);
    else
        stage_box64(reinterpret_cast<double4_32a *>(box), HX, HY, nbox, m, a, org, tile_ref64(a, tile), a.inv_h);
    const int rs_slot = __ldg(&a.tile_ref[tile]);
    const double wr[3] = {a.w[0][rs_slot], a.w[1][rs_slot], g.dim == 3 ? a.w[2][rs_slot] : 0.0};
    for (int b = threadIdx.x; b < nbox; b += blockDim.x) {
        int x, y, z;
        box_coord(b, HX, HY, m, g.dim, org, x, y, z);
        const int s = slot_at(g, a.tile_lut, x, y, z);
        R4 r;
        r.x = r.y = r.z = r.w = (R)0;
        if (s >= 0) {
            r.x = (R)(a.w[0][s] - wr[0]);
            r.y = (R)(a.w[1][s] - wr[1]);
            if (g.dim == 3) r.z = (R)(a.w[2][s] - wr[2]);
        }
        wbox[b] = r;
    }
    __syncthreads();

    const int adj = a.adjoint;
    for (int t = threadIdx.x; t < g.T; t += blockDim.x) {
        const int lx = t % g.bx, ly = (t / g.bx) % g.by, lz = t / (g.bx * g.by);
        const int slot = tile * g.T + brick_code(g.dim, lx, ly, lz);
        if (!(org.x + lx < g.nx && org.y + ly < g.ny && org.z + lz < g.nz)) continue;
        const int bi = (lx + m) + HX * ((ly + m) + HY * (g.dim == 3 ? lz + m : 0));
        const R4 ui = box[bi];
        const R4 wi = wbox[bi];
        R ox = 0, oy = 0, oz = 0;
        for (int w = 0; w < g.W; ++w) {
            const uint32_t word = a.mask[(size_t)w * g.nslots + slot];
            const int nb = min(32, g.S - 32 * w);
            for (int b = 0; b < nb; ++b) {
                if (!((word >> b) & 1u)) continue;
                const int4 d = __ldg(&a.stencil[32 * w + b]);
                const R r0 = (R)__ldg(&a.stencil_r0[32 * w + b]);
                const int bj = bi + d.x + HX * (d.y + HY * d.z);
                const R4 uj = box[bj];
                const R4 wj = wbox[bj];
                // bond geometry from i's side, or from j's side for the adjoint
                const R sg = adj ? (R)-1 : (R)1;
                const R ex = sg * (uj.x - ui.x), ey = sg * (uj.y - ui.y), ez = sg * (uj.z - ui.z);
                const R dx = sg * (R)d.x, dy = sg * (R)d.y, dz = sg * (R)d.z;
                const R yx = ex + dx, yy = ey + dy, yz = ez + dz;
                const R q = yx * yx + yy * yy + yz * yz;
                const R num = ex * ex + ey * ey + ez * ez + (R)2 * (dx * ex + dy * ey + dz * ez);
                const R rs = prsqrt1(q);
                const R s = pdiv1(num, r0 * (q * rs + r0));
                // D (w_j - w_i); volumes are uniform, so V_i / V_j placement is 1
                const R dwx = wj.x - wi.x, dwy = wj.y - wi.y, dwz = wj.z - wi.z;
                const R ndw = (yx * dwx + yy * dwy + yz * dwz) * rs;
                const R cn = ndw * ((R)1 / r0 - s * rs) * rs;
                const R cs = s * rs;
                R vij = a.vol_corr ? (R)vol_factor_lattice(m, (double)r0) : (R)1;
                ox += vij * (cn * yx + cs * dwx);
                oy += vij * (cn * yy + cs * dwy);
                oz += vij * (cn * yz + cs * dwz);
            }
        }
        const double sc = a.cV * a.inv_h;
        a.jv[0][slot] = sc * (double)ox;
        a.jv[1][slot] = sc * (double)oy;
        if (g.dim == 3) a.jv[2][slot] = sc * (double)oz;
    }
}

size_t jvp_smem(const Geom &g, int precision)
{
    const size_t nbox = (size_t)(g.bx + 2 * g.m) * (g.by + 2 * g.m) * (g.dim == 3 ? g.bz + 2 * g.m : 1);
    return 2 * nbox * (precision == PD_FP64 ? sizeof(double4_32a) : sizeof(float4));
}

int launch_jvp_args(const TileArgs &a, int precision, cudaStream_t st)
{
    const size_t smem = jvp_smem(a.g, precision);
    if (precision == PD_FP64) {
        PD_CUDA(smem_limit(jvp_generic<double>, smem));
        jvp_generic<double><<<a.g.ntiles, 256, smem, st>>>(a);
    } else {
        PD_CUDA(smem_limit(jvp_generic<float>, smem));
        jvp_generic<float><<<a.g.ntiles, 256, smem, st>>>(a);
    }
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

}  // namespace pdk
