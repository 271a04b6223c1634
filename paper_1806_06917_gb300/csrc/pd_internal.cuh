// pd_internal.cuh -- internal layout and launcher declarations of libpd.
//
// Internal point order ("slots"). The lattice is cut into tiles: aligned blocks
// of T = 2^L consecutive Morton codes, i.e. Morton bricks (L = 9 in 3D: 8x8x8;
// L = 9 in 2D: 32x16). Tiles that intersect the grid are numbered in increasing
// Morton code; slot = tile * T + local Morton code. Slots outside the grid (only
// in edge tiles of grids whose sides are not multiples of the brick) are
// inactive. Walking active slots in order is the global Morton order, and the
// Morton rank of a point is its position among active slots.
//
// Bonds. The CSR neighbour list (Morton ranks) is the canonical bond list. On a
// lattice the row of point i is the horizon stencil {d : 0 < |d|^2 <= m^2}
// translated to i and clipped to the grid, so the force kernels read it as one
// bit per (point, stencil slot): bit k of mask[w][slot] (k = 32 w + bit) is set
// when the bond to slot + d_k exists and is intact. Stencil slots are ordered
// by (dz, dy, dx) ascending.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pd.h"

namespace pdk {

// ------------------------------------------------------------ error plumbing

void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

#define PD_CUDA(call)                                               \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return ::pdk::cuda_fail(e_, #call);  \
    } while (0)

// A kernel's dynamic shared-memory limit (cudaFuncAttributeMaxDynamicSharedMemorySize)
// is one value per kernel and device, shared by every host thread: one thread
// lowering it between another's setting and launch would fail that launch
// ("too many resources requested for launch"; the request server's setup and
// worker threads launch the same kernels with different sizes). So the limit
// is only ever raised, under a lock (pd_mem.cu), to at least `bytes`.
cudaError_t raise_smem_limit(const void *func, size_t bytes);
template <class F>
inline cudaError_t smem_limit(F *func, size_t bytes)
{
    return raise_smem_limit(reinterpret_cast<const void *>(func), bytes);
}

// ------------------------------------------------------------------- Morton

// Bit b of coordinate a goes to bit DIM*b + a of the code (x least significant).
__host__ __device__ inline uint64_t morton_encode(int dim, uint32_t x, uint32_t y, uint32_t z)
{
    uint64_t code = 0;
    for (int b = 0; b < 21; ++b) {
        code |= (uint64_t)((x >> b) & 1u) << (dim * b);
        code |= (uint64_t)((y >> b) & 1u) << (dim * b + 1);
        if (dim == 3) code |= (uint64_t)((z >> b) & 1u) << (dim * b + 2);
    }
    return code;
}

__host__ __device__ inline void morton_decode(int dim, uint64_t code, int c[3])
{
    c[0] = c[1] = c[2] = 0;
    for (int b = 0; b < 21; ++b) {
        c[0] |= (int)((code >> (dim * b)) & 1u) << b;
        c[1] |= (int)((code >> (dim * b + 1)) & 1u) << b;
        if (dim == 3) c[2] |= (int)((code >> (dim * b + 2)) & 1u) << b;
    }
}

// Brick dimensions of a tile of 2^L codes: code bit p belongs to axis p % dim.
__host__ __device__ inline void brick_dims(int dim, int L, int b[3])
{
    b[0] = b[1] = b[2] = 1;
    for (int p = 0; p < L; ++p) b[p % dim] *= 2;
}

// ------------------------------------------------------------------ layout

// Everything a kernel needs about the lattice and the slot layout (POD, passed
// by value).
struct Geom {
    int dim, m;
    int S, W;            // stencil size, 32-bit mask words per point
    int L, T;            // tile log2 and points per tile
    int bx, by, bz;      // brick dims
    int lbx, lby, lbz;   // log2 of the brick dims
    int nx, ny, nz;      // lattice dims
    int tgx, tgy, tgz;   // tile grid dims
    int ntiles;
    int nslots;          // ntiles * T
    int npoints;
    double h;
};

struct Material {
    int model, vol_corr;
    double E, rho, K, mu, s_c, thickness;
    double psi_c, psi_beta;   // NP / LP potential
    double c;            // PMB micromodulus; NP / LP bond stiffness 4 C beta / (delta |B|)
    double V;            // nodal volume
};

// Device tables built once per simulation.
struct Tables {
    const int4 *tile_org;       // [ntiles] tile origin (x, y, z, 0) in lattice units
    const int *tile_ref;        // [ntiles] slot whose displacement is the tile's reference
    const int *tile_lut;        // [tgx*tgy*tgz] tile grid (row-major) -> tile or -1
    const int *user_of_slot;    // [nslots] user index or -1
    const int *slot_of_user;    // [npoints]
    const int *rank_of_slot;    // [nslots] Morton rank or -1
    const int *slot_of_rank;    // [npoints]
    const int4 *stencil;        // [S] (dx, dy, dz, |d|^2)
    const int *stencil_lut;     // [(2m+1)^dim] offset -> stencil slot or -1
    const double *stencil_r0;   // [S] |d| of each stencil entry
};

enum Mode { MODE_FORCE = 0, MODE_STEP = 1, MODE_FINALIZE = 2 };

// ------------------------------------------------------------- launchers

// Neighbour build (pd_build.cu).
struct BuildOut {
    int64_t *row_ptr;   // device [npoints + 1]
    int32_t *col;       // device [nbonds]
    int64_t nbonds;
};
int build_slots(const Geom &g, const Tables &t, int *d_user_of_slot, int *d_slot_of_user,
                int *d_rank_of_slot, int *d_slot_of_rank, cudaStream_t st);
// CSR rows (ascending Morton ranks) and the bond-intact stencil mask of every slot.
int build_csr(const Geom &g, const Tables &t, BuildOut *out, uint32_t *mask, cudaStream_t st);
int build_weighted_volume(const Geom &g, const Material &mat, const Tables &t,
                          const uint32_t *mask, double *mtil, float *minv32, cudaStream_t st);
int build_dt_bound(const Geom &g, const Material &mat, const Tables &t, const uint32_t *mask,
                   double *d_sum_max, cudaStream_t st);
int csr_broken_flags(const Geom &g, const Tables &t, const BuildOut &csr, const uint32_t *mask,
                     uint8_t *out, cudaStream_t st);
int break_notch(const Geom &g, const Tables &t, uint32_t *mask, int axis, double pos,
                const double lo[3], const double hi[3], unsigned long long *d_count,
                cudaStream_t st);

// Library device memory (pd_mem.cu): a stream-ordered pool per device.
cudaError_t lib_malloc(void **p, size_t bytes, cudaStream_t st);
cudaError_t lib_free(void *p, cudaStream_t st);

// Description checks of pd_create (pd_api.cu), for the request server.
int validate_description(const pd_grid *gr, const pd_material *mt, const pd_run *rn);

// Krylov solvers (pd_krylov.cu). Vectors: n FP64 values on the device.
struct KrylovOp {
    int (*apply)(void *ctx, const double *x, double *y, cudaStream_t st);   // y = A x
    void *ctx;
    int (*precond)(void *ctx, const double *r, double *z, cudaStream_t st); // z = M^-1 r, or null
};
// Device scalars a Krylov solve needs at least (dot results and CG's state).
constexpr size_t KRYLOV_DSC_MIN = 24;
struct KrylovWork {
    double *basis;      // GMRES: (restart + 1) * n; CG: 3 * n
    double *tmp;        // n
    double *aux;        // 2 * n (preconditioned solves)
    double *partial;    // krylov_partial_doubles(n, restart)
    double *dsc;        // krylov_dsc_doubles(...)
    cudaStream_t cap;   // a stream for graph capture (CG), or null
};
struct KrylovStats {
    int iters;
    int converged;
    double res0, res;   // ||b||, final ||b - A x|| (GMRES: at the last restart or the rotation estimate)
};
int krylov_gmres(const KrylovOp &op, const double *b, double *x, long long n, int restart, int maxit,
                 double rtol, KrylovWork &wk, KrylovStats *stats, cudaStream_t st);
int krylov_cg(const KrylovOp &op, const double *b, double *x, long long n, int maxit, double rtol,
              KrylovWork &wk, KrylovStats *stats, cudaStream_t st);
size_t krylov_partial_doubles(long long n, int kmax);
// Device scalars (KrylovWork::dsc) a solve needs: GMRES(restart) or, with 0, CG.
size_t krylov_dsc_doubles(int krylov_gmres_restart);
int krylov_norm(const double *x, long long n, KrylovWork &wk, double *out, cudaStream_t st);

// User order to slots with the staging form in one pass, and back (pd_build.cu).
// bits: the FP32 staging pair by split_bits (FP64 integrator state) instead of
// the round-to-nearest double-float split.
int scatter_stage(const Geom &g, const int *user_of_slot, const double *user, double *const slot[3], float4 *hl,
                  double4_32a *d4, cudaStream_t st, bool bits = false);
int gather_unstage(const Geom &g, const int *slot_of_user, const float4 *hl, double *const slot[3], double *user,
                   cudaStream_t st);
// The same for the user rows [r0, r1) only (chunks of a pipelined host transfer).
int scatter_rows(const Geom &g, const int *slot_of_user, const double *user, long long r0, long long r1,
                 double *const slot[3], float4 *hl, double4_32a *d4, cudaStream_t st, bool bits = false);
int gather_rows(const Geom &g, const int *slot_of_user, const float4 *hl, double *const slot[3], double *user,
                long long r0, long long r1, cudaStream_t st);

// Permutations between user order (AoS n x dim) and slot order (SoA).
int scatter_user_to_slots(const Geom &g, const Tables &t, const double *user, double *const slot[3],
                          double fill, cudaStream_t st);
// Boundary-condition kinds (n x dim bytes, user order) into component-major
// slot order; err[0] is set if a kind is unknown.
int scatter_kinds(const Geom &g, const Tables &t, const uint8_t *user, uint8_t *kind, int *err, cudaStream_t st);

}  // namespace pdk
