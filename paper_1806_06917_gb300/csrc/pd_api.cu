// pd_api.cu -- the C ABI of libpd (include/pd.h): simulation lifecycle, the
// per-simulation tables, host/device transfers in user order, graph-captured
// explicit stepping, force, tangent and energy entry points.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <vector>

#include "pd_packed.cuh"

namespace pdk {

// ------------------------------------------------------------ error plumbing

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PD_ENOMEM : PD_ECUDA;
}

// launchers defined in the kernel files
int launch_pmb_args(const TileArgs &a, int precision, cudaStream_t st);
int launch_lps_args(const TileArgs &a, int precision, int dil, cudaStream_t st);
int launch_jvp_args(const TileArgs &a, int precision, cudaStream_t st);
int launch_energy_points(const TileArgs &a, int precision, double *kin, cudaStream_t st);
int reduce_sum(const double *x, long long n, double scale, double *partial, double *out, cudaStream_t st);
int reduce_blocks_for(long long n);
size_t pmb_generic_smem(const Geom &g, int precision);
size_t pmb_fast_smem(const Geom &g);
size_t np_fast_smem(const Geom &g);
size_t lps_generic_smem(const Geom &g, int precision, bool dil);
size_t jvp_smem(const Geom &g, int precision);
// Per-bond tangent cache (pd_tangent.cu): prepare at a linearisation point,
// then y = A w (A = -K on free DOFs, identity on prescribed ones) from the cache.
size_t tangent_cache_bytes(const Geom &g, int precision);
int launch_tangent_prepare(const TileArgs &a, int precision, void *cache, cudaStream_t st);
int launch_tangent_apply(const Geom &g, int precision, const void *cache, const int *user_of_slot,
                         const uint8_t *kind, const double *w, double *y, cudaStream_t st);
int launch_tangent_jacobi(const Geom &g, int precision, void *cache, const int *user_of_slot, const uint8_t *kind,
                          cudaStream_t st);
int launch_tangent_precond(const Geom &g, int precision, const void *cache, const double *r, double *z,
                           cudaStream_t st);
size_t energy_smem(const Geom &g, int precision);
int pack_stage(const Geom &g, double *const u[3], float4 *hl, double4_32a *d4, cudaStream_t st, bool bits = false);
int dirichlet_mask(const Geom &g, const uint8_t *kind, double *const v[3], const double *const w[3], int copy,
                   cudaStream_t st);
int unpack_pairs(const Geom &g, const float4 *in, double *const x[3], cudaStream_t st);
int pack_dof_pairs(long long n, const double *in, float *out, cudaStream_t st);
int pack_f4(const Geom &g, const double *in, float4 *out, cudaStream_t st);

}  // namespace pdk

using namespace pdk;

constexpr int GRAPH_CHUNK = 16;   // steps per captured graph (even: parity-preserving)
constexpr size_t SMEM_LIMIT = 227 * 1024;

// Chunks of a pipelined host transfer of one state field (pd_set_state / pd_get_state).
constexpr int IO_CHUNKS = 4;

struct pd_sim {
    pd_grid grid;
    pd_material pmat;
    pd_run run;
    Geom g;
    Material mat;
    int precision = PD_FP32C;
    bool state64 = true;        // FP32C: u, v in the FP64 arrays (PD_STATE_F64), else double-float pairs
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    // host transfers of pd_set_state / pd_get_state (see xfer_chunks): uploads copy
    // into io_up on copy_stream, downloads copy out of io_dn on copy_out (room for
    // both fields each), each chunk's scatter or gather on the caller's stream;
    // events per field and chunk
    cudaStream_t copy_stream = nullptr, copy_out = nullptr;
    cudaEvent_t ev_in = nullptr, ev_copy[2][IO_CHUNKS] = {}, ev_done[2][IO_CHUNKS] = {};
    cudaEvent_t ev_out = nullptr, ev_dgath[2][IO_CHUNKS] = {}, ev_dcopy[2][IO_CHUNKS] = {};
    double *io_up = nullptr, *io_dn = nullptr;
    bool built = false;
    double dt = 0.0, dt_crit = 0.0;
    int64_t step = 0;
    int v_is_half = 0;
    bool u_prev_ok = false;     // the other staging buffer holds u^{k-1} of the same dt
    int cur = 0;
    bool tangent_ok = true;     // the tangent's halo box fits at this tile size
    bool use_body = false;
    double c_dt = 0.0;          // micromodulus used by the stable-step bound

    // tables
    int4 *tile_org = nullptr;
    int *tile_ref = nullptr, *tile_lut = nullptr;
    int *user_of_slot = nullptr, *slot_of_user = nullptr, *rank_of_slot = nullptr, *slot_of_rank = nullptr;
    int4 *stencil = nullptr;
    double *stencil_r0 = nullptr;
    int *stencil_lut = nullptr;
    float4 *tab_a = nullptr;        // FP32C stencil table: PMB, or LPS dilatation
    float4 *tab_b = nullptr;        // FP32C stencil table: LPS force
    std::vector<float4> htab_a, htab_b;   // host copies (passed as kernel parameters when small)
    int *tile_nbr = nullptr;        // [ntiles * 27]
    int nbr_ok = 0;
    uint32_t *box_map = nullptr;    // [paired halo box] neighbour tile + brick code of both points
    int box_edge[3] = {0, 0, 0};    // largest tile origin per axis for which box_map holds
    // CSR
    BuildOut csr{nullptr, nullptr, 0};
    // state
    double *u[3] = {nullptr, nullptr, nullptr}, *v[3] = {nullptr, nullptr, nullptr};
    float4 *hl[2] = {nullptr, nullptr};
    double4_32a *d4[2] = {nullptr, nullptr};
    float4 *lin_hl = nullptr;
    double4_32a *lin_d4 = nullptr;
    float4 *vhl = nullptr;          // FP32C double-float state: velocity pairs
    float *bc32 = nullptr;          // FP32C double-float state: boundary values, (hi, lo) per DOF
    float4 *body32 = nullptr;       // FP32C body force
    uint8_t *bc_kind = nullptr;
    double *bc_val = nullptr, *body = nullptr;
    uint32_t *mask = nullptr;
    double *mtil = nullptr;
    float *minv32 = nullptr, *theta32 = nullptr;
    double *theta64 = nullptr;
    double *f[3] = {nullptr, nullptr, nullptr}, *w[3] = {nullptr, nullptr, nullptr};
    double *jv[3] = {nullptr, nullptr, nullptr}, *ulin[3] = {nullptr, nullptr, nullptr};
    double *epoint = nullptr, *ekin = nullptr, *red = nullptr, *dout = nullptr;
    double *io = nullptr;
    int *d_err = nullptr;
    unsigned long long *d_count = nullptr;
    std::vector<void *> allocs;
    // Newton-Krylov work of pd_solve_static, allocated on first use
    double *nk_basis = nullptr, *nk_tmp = nullptr, *nk_partial = nullptr, *nk_dsc = nullptr;
    double *nk_r = nullptr, *nk_du = nullptr, *nk_aux = nullptr;
    size_t nk_basis_n = 0, nk_partial_n = 0, nk_dsc_n = 0;
    void *nk_tan = nullptr;         // per-bond tangent cache
    size_t nk_tan_n = 0;
    // graphs: [start parity]
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
};

static int pd_alloc(pd_sim *s, void **p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    cudaError_t e = lib_malloc(p, bytes, s->stream);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "device allocation");
    }
    s->allocs.push_back(*p);
    e = cudaMemsetAsync(*p, 0, bytes, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);    // usable on every stream from here
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
    return PD_OK;
}

#define ALLOC(ptr, bytes)                                                  \
    do {                                                                   \
        int rc_ = pd_alloc(s, (void **)&(ptr), (size_t)(bytes));           \
        if (rc_ != PD_OK) return rc_;                                      \
    } while (0)

static cudaStream_t pick(pd_sim *s, void *stream) { return stream ? (cudaStream_t)stream : s->stream; }

static void drop_graphs(pd_sim *s)
{
    for (int p = 0; p < 2; ++p)
        if (s->graph[p]) {
            cudaGraphExecDestroy(s->graph[p]);
            s->graph[p] = nullptr;
        }
}

// Shared memory of the largest halo box any kernel of the simulation stages;
// with_tangent includes the tangent (PMB only), which stages u and w.
static size_t max_smem(const Geom &g, int precision, int model, bool with_tangent)
{
    size_t m = energy_smem(g, precision);
    if (with_tangent) m = std::max(m, jvp_smem(g, precision));
    if (model == PD_MODEL_NP || model == PD_MODEL_LP)
        m = std::max(m, precision == PD_FP64 ? pmb_generic_smem(g, precision) : np_fast_smem(g));
    else if (model != PD_MODEL_LPS)
        m = std::max(m, precision == PD_FP64 ? pmb_generic_smem(g, precision) : pmb_fast_smem(g));
    else m = std::max(m, lps_generic_smem(g, precision, false));
    return m;
}

// ---------------------------------------------------------------- create

static int validate(const pd_grid *gr, const pd_material *mt, const pd_run *rn)
{
    if (!gr || !mt || !rn) { set_error("null description"); return PD_EINVAL; }
    if (gr->dim != 2 && gr->dim != 3) { set_error("dim must be 2 or 3"); return PD_EINVAL; }
    for (int a = 0; a < 3; ++a)
        if (gr->n[a] < 1) { set_error("n[%d] must be >= 1", a); return PD_EINVAL; }
    if (gr->dim == 2 && gr->n[2] != 1) { set_error("2D grids need n[2] == 1"); return PD_EINVAL; }
    if (gr->m < 1 || gr->m > 24) { set_error("horizon factor m must be in [1, 24]"); return PD_EINVAL; }
    if (!(gr->h > 0.0) || !isfinite(gr->h)) { set_error("h must be > 0"); return PD_EINVAL; }
    if (gr->reserved != 0) { set_error("pd_grid.reserved must be 0"); return PD_EINVAL; }
    if ((double)gr->n[0] * gr->n[1] * gr->n[2] > 1.0e9) { set_error("more than 1e9 points"); return PD_EINVAL; }
    if (mt->model < PD_MODEL_PMB || mt->model > PD_MODEL_LP) { set_error("unknown model"); return PD_EINVAL; }
    if (mt->model == PD_MODEL_NP || mt->model == PD_MODEL_LP) {
        if (!(mt->psi_c > 0.0) || !(mt->psi_beta > 0.0)) { set_error("NP / LP need psi_c > 0 and psi_beta > 0"); return PD_EINVAL; }
        if (mt->s_c != 0.0) { set_error("NP / LP have no bond breaking (s_c must be 0)"); return PD_EINVAL; }
    }
    if (!(mt->rho > 0.0)) { set_error("rho must be > 0"); return PD_EINVAL; }
    if (mt->model == PD_MODEL_PMB && !(mt->E > 0.0)) { set_error("E must be > 0"); return PD_EINVAL; }
    if (mt->model == PD_MODEL_LPS) {
        if (gr->dim != 3) { set_error("LPS is 3D only"); return PD_EINVAL; }
        if (!(mt->K > 0.0) || !(mt->mu > 0.0)) { set_error("LPS needs K > 0 and mu > 0"); return PD_EINVAL; }
        if (mt->s_c != 0.0) { set_error("LPS has no bond breaking (s_c must be 0)"); return PD_EINVAL; }
    }
    if (mt->s_c < 0.0) { set_error("s_c must be >= 0"); return PD_EINVAL; }
    if (gr->dim == 2 && !(mt->thickness > 0.0)) { set_error("2D needs thickness > 0"); return PD_EINVAL; }
    if (rn->precision != PD_FP32C && rn->precision != PD_FP64) { set_error("unknown precision"); return PD_EINVAL; }
    if (rn->tile_log2 != 0 && (rn->tile_log2 < 6 || rn->tile_log2 > 9)) {
        set_error("tile_log2 must be 0 or in [6, 9]");
        return PD_EINVAL;
    }
    if (rn->dt < 0.0 || rn->dt_factor < 0.0) { set_error("dt and dt_factor must be >= 0"); return PD_EINVAL; }
    if (rn->integrator != PD_INTEGRATOR_VERLET && rn->integrator != PD_INTEGRATOR_CD) {
        set_error("unknown integrator");
        return PD_EINVAL;
    }
    if (rn->state != PD_STATE_F64 && rn->state != PD_STATE_DF) { set_error("unknown state precision"); return PD_EINVAL; }
    if (rn->pair_threads != 0 && rn->pair_threads != 1 && rn->pair_threads != 2 && rn->pair_threads != 4) {
        set_error("pair_threads must be 0, 1, 2 or 4");
        return PD_EINVAL;
    }
    if (rn->reserved != 0) { set_error("pd_run.reserved must be 0"); return PD_EINVAL; }
    if (rn->precision == PD_FP64 && rn->state != PD_STATE_F64) {
        set_error("the FP64 path keeps FP64 state (pd_run.state must be 0)");
        return PD_EINVAL;
    }
    return PD_OK;
}

int pdk::validate_description(const pd_grid *gr, const pd_material *mt, const pd_run *rn)
{
    if (!gr || !mt || !rn) { set_error("null description"); return PD_EINVAL; }
    return validate(gr, mt, rn);
}

static int create_impl(pd_sim *s)
{
    const pd_grid &gr = s->grid;
    Geom &g = s->g;
    memset(&g, 0, sizeof(g));
    g.dim = gr.dim;
    g.m = gr.m;
    g.nx = gr.n[0];
    g.ny = gr.n[1];
    g.nz = gr.dim == 3 ? gr.n[2] : 1;
    g.h = gr.h;
    g.npoints = g.nx * g.ny * g.nz;
    auto set_tile = [&g](int L) {
        g.L = L;
        g.T = 1 << L;
        int b[3];
        brick_dims(g.dim, L, b);
        g.bx = b[0];
        g.by = b[1];
        g.bz = b[2];
        g.lbx = __builtin_ctz(b[0]);
        g.lby = __builtin_ctz(b[1]);
        g.lbz = __builtin_ctz(b[2]);
        g.tgx = (g.nx + g.bx - 1) / g.bx;
        g.tgy = (g.ny + g.by - 1) / g.by;
        g.tgz = (g.nz + g.bz - 1) / g.bz;
    };

    // stencil: offsets 0 < |d|^2 <= m^2 ordered by (dz, dy, dx)
    std::vector<int4> st;
    std::vector<double> r0;
    const int wdt = 2 * g.m + 1;
    std::vector<int> lut((size_t)wdt * wdt * (g.dim == 3 ? wdt : 1), -1);
    for (int dz = (g.dim == 3 ? -g.m : 0); dz <= (g.dim == 3 ? g.m : 0); ++dz)
        for (int dy = -g.m; dy <= g.m; ++dy)
            for (int dx = -g.m; dx <= g.m; ++dx) {
                const int d2 = dx * dx + dy * dy + dz * dz;
                if (d2 == 0 || d2 > g.m * g.m) continue;
                lut[(dx + g.m) + wdt * ((dy + g.m) + wdt * (g.dim == 3 ? dz + g.m : 0))] = (int)st.size();
                st.push_back(make_int4(dx, dy, dz, d2));
                r0.push_back(sqrt((double)d2));
            }
    g.S = (int)st.size();
    g.W = (g.S + 31) / 32;
    if (g.W > 64) { set_error("horizon stencil too large"); return PD_EINVAL; }

    // tile size: the requested one, or the largest brick (up to 2^9 points)
    // whose halo box fits in shared memory for every kernel of this simulation
    // (the tangent's, if it fits at all: at wide horizons in FP64 its two boxes
    // do not fit even in the smallest tile, and the tangent calls then refuse)
    const int model = s->pmat.model;
    bool tangent = model == PD_MODEL_PMB;
    if (s->run.tile_log2) {
        set_tile(s->run.tile_log2);
        tangent = tangent && max_smem(g, s->precision, model, true) <= SMEM_LIMIT;
    } else {
        int L = 9;
        set_tile(L);
        while (L > 6 && max_smem(g, s->precision, model, tangent) > SMEM_LIMIT) set_tile(--L);
        if (tangent && max_smem(g, s->precision, model, true) > SMEM_LIMIT) {
            tangent = false;
            L = 9;
            set_tile(L);
            while (L > 6 && max_smem(g, s->precision, model, false) > SMEM_LIMIT) set_tile(--L);
        }
    }
    s->tangent_ok = tangent;

    // tiles: bricks intersecting the grid, ordered by the Morton code of their origin
    struct TileKey { uint64_t code; int tx, ty, tz; };
    std::vector<TileKey> tiles;
    tiles.reserve((size_t)g.tgx * g.tgy * g.tgz);
    for (int tz = 0; tz < g.tgz; ++tz)
        for (int ty = 0; ty < g.tgy; ++ty)
            for (int tx = 0; tx < g.tgx; ++tx)
                tiles.push_back({morton_encode(g.dim, tx * g.bx, ty * g.by, tz * g.bz), tx, ty, tz});
    std::sort(tiles.begin(), tiles.end(), [](const TileKey &x, const TileKey &y) { return x.code < y.code; });
    g.ntiles = (int)tiles.size();
    const long long nslots = (long long)g.ntiles * g.T;
    if (nslots >= (1LL << 31)) { set_error("lattice too large for 32-bit slots"); return PD_EINVAL; }
    g.nslots = (int)nslots;
    std::vector<int4> org(g.ntiles);
    std::vector<int> ref(g.ntiles), tlut((size_t)g.tgx * g.tgy * g.tgz, -1);
    for (int t = 0; t < g.ntiles; ++t) {
        org[t] = make_int4(tiles[t].tx * g.bx, tiles[t].ty * g.by, tiles[t].tz * g.bz, 0);
        ref[t] = t * g.T;   // the brick's origin corner is always inside the grid
        tlut[tiles[t].tx + g.tgx * (tiles[t].ty + g.tgy * tiles[t].tz)] = t;
    }

    const size_t smem = max_smem(g, s->precision, s->pmat.model, false);
    if (smem > SMEM_LIMIT) {
        set_error("halo box needs %zu bytes of shared memory (> %zu); use a smaller tile_log2", smem, SMEM_LIMIT);
        return PD_EINVAL;
    }

    // material constants
    Material &mt = s->mat;
    mt.model = s->pmat.model;
    mt.vol_corr = s->pmat.vol_corr;
    mt.E = s->pmat.E;
    mt.rho = s->pmat.rho;
    mt.K = s->pmat.K;
    mt.mu = s->pmat.mu;
    mt.s_c = s->pmat.s_c;
    mt.thickness = s->pmat.thickness;
    mt.psi_c = s->pmat.psi_c;
    mt.psi_beta = s->pmat.psi_beta;
    const double delta = g.m * g.h;
    const double PI = 3.14159265358979323846;
    auto pmb_c = [&](double E) {
        if (g.dim == 3) {
            const double Kp = E / (3.0 * (1.0 - 2.0 * 0.25));   // nu = 1/4
            return 18.0 * Kp / (PI * delta * delta * delta * delta);
        }
        return 9.0 * E / (PI * mt.thickness * delta * delta * delta);
    };
    mt.V = g.dim == 3 ? g.h * g.h * g.h : g.h * g.h * mt.thickness;
    const bool np_law = mt.model == PD_MODEL_NP || mt.model == PD_MODEL_LP;
    // NP / LP: 4 C beta / (delta |B_delta(0)|), the bond stiffness at zero strain
    const double ball = g.dim == 3 ? 4.0 * PI * delta * delta * delta / 3.0 : PI * delta * delta;
    mt.c = mt.model == PD_MODEL_PMB ? pmb_c(mt.E) : np_law ? 4.0 * mt.psi_c * mt.psi_beta / (delta * ball) : 0.0;
    s->c_dt = mt.model == PD_MODEL_LPS ? pmb_c(9.0 * mt.K * mt.mu / (3.0 * mt.K + mt.mu)) : mt.c;

    PD_CUDA(cudaGetDevice(&s->device));
    PD_CUDA(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    PD_CUDA(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
    PD_CUDA(cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking));
    PD_CUDA(cudaStreamCreateWithFlags(&s->copy_out, cudaStreamNonBlocking));
    PD_CUDA(cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming));
    PD_CUDA(cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming));
    for (int f = 0; f < 2; ++f)
        for (int k = 0; k < IO_CHUNKS; ++k) {
            PD_CUDA(cudaEventCreateWithFlags(&s->ev_copy[f][k], cudaEventDisableTiming));
            PD_CUDA(cudaEventCreateWithFlags(&s->ev_done[f][k], cudaEventDisableTiming));
            PD_CUDA(cudaEventCreateWithFlags(&s->ev_dgath[f][k], cudaEventDisableTiming));
            PD_CUDA(cudaEventCreateWithFlags(&s->ev_dcopy[f][k], cudaEventDisableTiming));
        }

    const size_t NS = (size_t)g.nslots, NP = (size_t)g.npoints;
    std::vector<uint32_t> box_map;      // uploaded after the other arrays (see the end)
    ALLOC(s->tile_org, sizeof(int4) * g.ntiles);
    ALLOC(s->tile_ref, sizeof(int) * g.ntiles);
    ALLOC(s->tile_lut, sizeof(int) * tlut.size());
    ALLOC(s->user_of_slot, sizeof(int) * NS);
    ALLOC(s->slot_of_user, sizeof(int) * NP);
    ALLOC(s->rank_of_slot, sizeof(int) * NS);
    ALLOC(s->slot_of_rank, sizeof(int) * NP);
    ALLOC(s->stencil, sizeof(int4) * g.S);
    ALLOC(s->stencil_r0, sizeof(double) * g.S);
    ALLOC(s->stencil_lut, sizeof(int) * lut.size());
    PD_CUDA(cudaMemcpy(s->tile_org, org.data(), sizeof(int4) * g.ntiles, cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(s->tile_ref, ref.data(), sizeof(int) * g.ntiles, cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(s->tile_lut, tlut.data(), sizeof(int) * tlut.size(), cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(s->stencil, st.data(), sizeof(int4) * g.S, cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(s->stencil_r0, r0.data(), sizeof(double) * g.S, cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(s->stencil_lut, lut.data(), sizeof(int) * lut.size(), cudaMemcpyHostToDevice));

    // FP32C stencil tables in the kernels' pre-splatted form; offsets index the
    // paired halo box (x extent bx + 2m; y extent by + 2m in 3D, by/2 + 2m in 2D)
    {
        const int PHX = g.bx + 2 * g.m, PHY = g.dim == 3 ? g.by + 2 * g.m : g.by / 2 + 2 * g.m;
        std::vector<float4> ta(4 * (size_t)g.S), tb(3 * (size_t)g.S), tc(3 * (size_t)g.S);
        for (int k = 0; k < g.S; ++k) {
            const int4 d = st[k];
            const double rr = r0[k], d2 = d.w;
            const double vij = mt.vol_corr && rr > g.m - 0.5 ? (g.m + 0.5 - rr) : 1.0;
            const int off = d.x + PHX * (d.y + PHY * d.z);
            float offf;
            memcpy(&offf, &off, sizeof(float));
            const float4 dxy = make_float4((float)d.x, (float)d.x, (float)d.y, (float)d.y);
            if (!np_law) ta[4 * k] = dxy;
            // LPS force, 3 float4 per entry: {dx,dx,dy,dy} {dz,dz,|d|,|d|} {|d|^2,|d|^2,offset,V_ij}
            // (the moduli 3K - 5mu and 15mu go with the staged theta / m~ and 1 / m~)
            tb[3 * k] = dxy;
            tb[3 * k + 1] = make_float4((float)d.z, (float)d.z, (float)rr, (float)rr);
            tb[3 * k + 2] = make_float4((float)d2, (float)d2, offf, (float)vij);
            // LPS dilatation, 3 float4 per entry: {2dx,2dx,2dy,2dy} {2dz,2dz,|d|,|d|}
            // {|d|^2,|d|^2,offset,V_ij} (its extension needs e.(e + 2d), not y)
            tc[3 * k] = make_float4(2.f * d.x, 2.f * d.x, 2.f * d.y, 2.f * d.y);
            tc[3 * k + 1] = make_float4(2.f * d.z, 2.f * d.z, (float)rr, (float)rr);
            tc[3 * k + 2] = tb[3 * k + 2];
            if (mt.model == PD_MODEL_NP || mt.model == PD_MODEL_LP) {
                // compact entries (NP_TAB_WORDS float4 each, written over the first
                // entries of the table): the bond weight t = J V_ij / |d| and the
                // exponent a = -beta h |d| log2(e) (so that psi'(|xi| S^2) / (C beta)
                // = exp2(a S^2)) folded with S = p / |d|^2, p = eta.d, into
                // k = t / |d|^2 and a' = a / |d|^4:
                //   2D {dx,dx,dy,dy} {k,k,a',offset}; 3D {dx,dx,dy,dy} {dz,dz,k,k} {a',offset,-,-}
                const double J = d2 < (double)g.m * g.m ? 1.0 : 0.0;
                const float kk = (float)(J * vij / rr / d2);
                const float ak = (float)(-mt.psi_beta * g.h * rr / log(2.0) / (d2 * d2));
                const int E = NP_TAB_WORDS(g.dim);
                ta[E * k] = dxy;
                if (g.dim == 3) {
                    ta[E * k + 1] = make_float4((float)d.z, (float)d.z, kk, kk);
                    ta[E * k + 2] = make_float4(ak, offf, 0.f, 0.f);
                } else {
                    ta[E * k + 1] = make_float4(kk, kk, ak, offf);
                }
            } else if (mt.model == PD_MODEL_PMB) {
                // {dz,dz,|d|^2,|d|^2} {|d|/V_ij x2, |d|^2/V_ij x2} {offset, s_c V_ij, lo, hi}: between
                // lo = s_c V_ij (1 - 2^-13) and hi = s_c V_ij (1 + 2^-13) the kernel decides a
                // bond's breaking from both ends' global state (the same decision in both rows)
                ta[4 * k + 1] = make_float4((float)d.z, (float)d.z, (float)d2, (float)d2);
                ta[4 * k + 2] = make_float4((float)(rr / vij), (float)(rr / vij), (float)(d2 / vij), (float)(d2 / vij));
                ta[4 * k + 3] = make_float4(offf, (float)(mt.s_c * vij), (float)(mt.s_c * vij * (1.0 - 0x1p-13)),
                                            (float)(mt.s_c * vij * (1.0 + 0x1p-13)));
            }
        }
        // LPS: the force pass reads tb, the dilatation tc (held in tab_a, which no
        // LPS kernel reads otherwise)
        if (mt.model == PD_MODEL_LPS) {
            std::fill(ta.begin(), ta.end(), make_float4(0.f, 0.f, 0.f, 0.f));
            std::copy(tc.begin(), tc.end(), ta.begin());
        }
        ALLOC(s->tab_a, sizeof(float4) * ta.size());
        ALLOC(s->tab_b, sizeof(float4) * tb.size());
        PD_CUDA(cudaMemcpy(s->tab_a, ta.data(), sizeof(float4) * ta.size(), cudaMemcpyHostToDevice));
        PD_CUDA(cudaMemcpy(s->tab_b, tb.data(), sizeof(float4) * tb.size(), cudaMemcpyHostToDevice));
        // the entries the kernels read: PMB 4 float4 each (NP / LP keep theirs in
        // shared memory), LPS 3
        if (mt.model == PD_MODEL_PMB) s->htab_a.assign(ta.begin(), ta.begin() + 4 * (size_t)g.S);
        if (mt.model == PD_MODEL_LPS) {
            s->htab_a = tc;
            s->htab_b = tb;
        }
        // neighbour tiles (index (dx+1) + 3 (dy+1) + 9 (dz+1)); usable when the halo
        // reaches at most one tile in every direction
        std::vector<int> nbr(27 * (size_t)g.ntiles, -1);
        for (int t = 0; t < g.ntiles; ++t)
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int x = tiles[t].tx + dx, y = tiles[t].ty + dy, z = tiles[t].tz + dz;
                        if (x < 0 || y < 0 || z < 0 || x >= g.tgx || y >= g.tgy || z >= g.tgz) continue;
                        nbr[27 * (size_t)t + (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)] =
                            tlut[x + g.tgx * (y + g.tgy * z)];
                    }
        s->nbr_ok = g.m <= g.bx && g.m <= g.by && (g.dim == 2 || g.m <= g.bz);
        ALLOC(s->tile_nbr, sizeof(int) * nbr.size());
        PD_CUDA(cudaMemcpy(s->tile_nbr, nbr.data(), sizeof(int) * nbr.size(), cudaMemcpyHostToDevice));
        if (s->nbr_ok) {
            // The paired halo box relative to a tile-aligned origin is the same for
            // every tile: entry b holds, for its points A and B, the index of the
            // neighbour tile (0..26, as in tile_nbr) and the brick code inside it,
            // A in bits 0-13 and B in bits 14-27 (5 + 9 bits each; T <= 2^9). It
            // replaces the staging's per-entry coordinate arithmetic in tiles whose
            // 3^d neighbours are whole tiles or absent (box_edge).
            const int dims[3] = {g.bx, g.by, g.dim == 3 ? g.bz : 1};
            const int HX = g.bx + 2 * g.m, HY = g.dim == 3 ? g.by + 2 * g.m : g.by / 2 + 2 * g.m;
            const int HZ = g.dim == 3 ? g.bz / 2 + 2 * g.m : 1;
            std::vector<uint32_t> &map = box_map;
            map.resize((size_t)HX * HY * HZ);
            for (int b = 0; b < (int)map.size(); ++b) {
                const int bxl = b % HX, byl = (b / HX) % HY, bzl = b / HX / HY;
                int r[2][3] = {{bxl - g.m, byl - g.m, g.dim == 3 ? bzl - g.m : 0}, {0, 0, 0}};
                for (int c = 0; c < 3; ++c) r[1][c] = r[0][c];
                if (g.dim == 3) r[1][2] += g.bz / 2;
                else r[1][1] += g.by / 2;
                uint32_t e = 0;
                for (int p = 0; p < 2; ++p) {
                    int dt[3], l[3];
                    for (int c = 0; c < 3; ++c) {
                        dt[c] = r[p][c] < 0 ? -1 : r[p][c] / dims[c];
                        l[c] = r[p][c] - dt[c] * dims[c];
                    }
                    const uint32_t k = (uint32_t)((dt[0] + 1) + 3 * (dt[1] + 1) + 9 * (dt[2] + 1));
                    const uint32_t code = (uint32_t)morton_encode(g.dim, l[0], l[1], l[2]);
                    e |= (k | code << 5) << (14 * p);
                }
                map[b] = e;
            }
            const int n3[3] = {g.nx, g.ny, g.nz};
            for (int c = 0; c < 3; ++c) s->box_edge[c] = n3[c] % dims[c] == 0 ? INT_MAX : n3[c] - 2 * dims[c];
        }
    }

    for (int c = 0; c < 3; ++c) {
        ALLOC(s->u[c], sizeof(double) * NS);
        ALLOC(s->v[c], sizeof(double) * NS);
        ALLOC(s->f[c], sizeof(double) * NS);
        ALLOC(s->w[c], sizeof(double) * NS);
        ALLOC(s->jv[c], sizeof(double) * NS);
        ALLOC(s->ulin[c], sizeof(double) * NS);
    }
    if (s->precision == PD_FP64) {
        ALLOC(s->d4[0], sizeof(double4_32a) * NS);
        ALLOC(s->d4[1], sizeof(double4_32a) * NS);
        ALLOC(s->lin_d4, sizeof(double4_32a) * NS);
    } else {
        ALLOC(s->hl[0], 2 * sizeof(float4) * NS);
        ALLOC(s->hl[1], 2 * sizeof(float4) * NS);
        ALLOC(s->lin_hl, 2 * sizeof(float4) * NS);
        if (!s->state64) {
            ALLOC(s->vhl, 2 * sizeof(float4) * NS);
            ALLOC(s->bc32, 2 * 3 * sizeof(float) * NS);
        }
    }
    ALLOC(s->bc_kind, 3 * NS);
    ALLOC(s->bc_val, 3 * sizeof(double) * NS);
    ALLOC(s->mask, sizeof(uint32_t) * g.W * NS);
    if (mt.model == PD_MODEL_LPS) {
        ALLOC(s->mtil, sizeof(double) * NS);
        ALLOC(s->minv32, sizeof(float) * NS);
        ALLOC(s->theta32, sizeof(float) * NS);
        ALLOC(s->theta64, sizeof(double) * NS);
    }
    ALLOC(s->epoint, sizeof(double) * NS);
    ALLOC(s->ekin, sizeof(double) * NS);
    ALLOC(s->red, sizeof(double) * reduce_blocks_for(NS));
    ALLOC(s->dout, sizeof(double) * 8);
    ALLOC(s->io, sizeof(double) * 3 * std::max(NP, NS));
    ALLOC(s->io_up, sizeof(double) * 2 * 3 * NP);
    ALLOC(s->io_dn, sizeof(double) * 2 * 3 * NP);
    ALLOC(s->d_err, sizeof(int));
    ALLOC(s->d_count, sizeof(unsigned long long));
    // last, so that it moves no other array of the pool
    if (!box_map.empty()) {
        ALLOC(s->box_map, sizeof(uint32_t) * box_map.size());
        PD_CUDA(cudaMemcpy(s->box_map, box_map.data(), sizeof(uint32_t) * box_map.size(), cudaMemcpyHostToDevice));
    }
    return PD_OK;
}

static TileArgs make_args(pd_sim *s, int mode, const float4 *src_hl, const double4_32a *src_d4)
{
    TileArgs a;
    memset(&a, 0, sizeof(a));
    a.g = s->g;
    a.tile_org = s->tile_org;
    a.tile_ref = s->tile_ref;
    a.tile_lut = s->tile_lut;
    a.stencil = s->stencil;
    a.stencil_r0 = s->stencil_r0;
    a.src_hl = src_hl;
    a.src_d4 = src_d4;
    a.dst_hl = s->hl[s->cur ^ 1];
    a.dst_d4 = s->d4[s->cur ^ 1];
    a.mask = s->mask;
    for (int c = 0; c < 3; ++c) {
        a.u[c] = s->u[c];
        a.v[c] = s->v[c];
        a.f[c] = s->f[c];
        a.w[c] = s->w[c];
        a.jv[c] = s->jv[c];
    }
    a.bc_kind = s->bc_kind;
    a.bc_val = s->bc_val;
    a.body = s->body;
    a.minv32 = s->minv32;
    a.mtil = s->mtil;
    a.theta32 = s->theta32;
    a.theta64 = s->theta64;
    a.epoint = s->epoint;
    a.cV = s->mat.c * s->mat.V;
    a.inv_rho = 1.0 / s->mat.rho;
    a.dt = s->dt;
    a.s_c = s->mat.s_c;
    a.h = s->g.h;
    a.inv_h = 1.0 / s->g.h;
    a.A = 3.0 * s->mat.K - 5.0 * s->mat.mu;
    a.B = 15.0 * s->mat.mu;
    a.K = s->mat.K;
    a.model = s->mat.model;
    a.v_is_half = s->v_is_half;
    a.cd = s->run.integrator == PD_INTEGRATOR_CD && s->u_prev_ok ? 1 : 0;
    a.state64 = s->precision == PD_FP32C && s->state64 ? 1 : 0;
    a.split = s->run.pair_threads;   // 0: the launcher's choice
    a.update_breaking = s->mat.s_c > 0.0 ? 1 : 0;
    a.mode = mode;
    a.vol_corr = s->mat.vol_corr;
    a.use_body = s->use_body ? 1 : 0;
    a.adjoint = 0;
    a.vhl = s->vhl;
    a.tab_a = s->tab_a;
    a.tab_b = s->tab_b;
    a.htab_a = s->htab_a.empty() ? nullptr : s->htab_a.data();
    a.htab_b = s->htab_b.empty() ? nullptr : s->htab_b.data();
    a.ntab_a = (int)s->htab_a.size();
    a.ntab_b = (int)s->htab_b.size();
    a.tile_nbr = s->tile_nbr;
    a.nbr_ok = s->nbr_ok;
    a.box_map = s->box_map;
    for (int c = 0; c < 3; ++c) a.box_edge[c] = s->box_edge[c];
    a.bc32 = s->bc32;
    a.body32 = s->body32;
    a.fscale = s->mat.model == PD_MODEL_LPS ? 1.0 / s->g.h : s->mat.c * s->mat.V;
    a.psi_beta = s->mat.psi_beta;
    a.kF = (float)(0.5 * s->dt * a.fscale / s->mat.rho);
    a.kB = (float)(0.5 * s->dt / s->mat.rho);
    a.dt_h = (float)s->dt;
    a.dt_l = (float)(s->dt - (double)a.dt_h);
    return a;
}

// ------------------------------------------------- the server's packed kernel

int pdk::sim_pack_info(pd_sim *s, PackInfo *pi)
{
    memset(pi, 0, sizeof(*pi));
    if (!s->built) { set_error("neighbours not built"); return PD_ESTATE; }
    const Geom &g = s->g;
    const int model = s->mat.model;
    const int split = pack_split_for(g.W);
    int kind = -1;
    if (model == PD_MODEL_PMB && s->mat.s_c == 0.0) kind = g.dim == 3 ? PK_PMB3 : PK_PMB2;
    if (model == PD_MODEL_LPS && !s->mat.vol_corr) kind = PK_LPS;
    pi->eligible = s->precision == PD_FP32C && kind >= 0 && g.L == 9 && s->nbr_ok &&
                   (kind == PK_LPS || s->run.pair_threads == split) &&
                   (kind != PK_LPS || (g.dim == 3 && g.m <= PACK_LPS_MMAX &&
                                       s->htab_a.size() == 3 * (size_t)pack_lps_stencil(g.m) &&
                                       s->htab_b.size() == 3 * (size_t)pack_lps_stencil(g.m)));
    if (!pi->eligible) return PD_OK;
    pi->kind = kind;
    pi->m = g.m;
    if (kind == PK_LPS) {
        pi->htab_dil = s->htab_a.data();
        pi->htab_force = s->htab_b.data();
    }
    pi->split = kind == PK_LPS ? 2 : split;
    pi->ntiles = g.ntiles;
    pi->smem = pack_smem(g, kind, split);
    // items that would leave the packed kernel fewer than two CTAs per SM stay on
    // their own stream
    int ctas = 0;
    const int rc = pack_occupancy(pi->smem, &ctas);
    if (rc != PD_OK && rc != PD_EINVAL) return rc;
    if (rc == PD_EINVAL || ctas < 2) {
        pi->eligible = 0;
        return PD_OK;
    }
    for (int p = 0; p < 2; ++p) {
        TileArgs a = make_args(s, MODE_STEP, s->hl[p], s->d4[p]);
        a.dst_hl = s->hl[p ^ 1];
        a.dst_d4 = s->d4[p ^ 1];
        a.v_is_half = 1;
        a.cd = s->run.integrator == PD_INTEGRATOR_CD ? 1 : 0;
        a.update_breaking = 0;
        a.split = pi->split;
        a.htab_a = a.htab_b = nullptr;      // the packed bodies read the device tables
        a.ntab_a = a.ntab_b = 0;
        pi->a[p] = a;
    }
    pi->cur = s->cur;
    pi->vhalf = s->v_is_half;
    pi->cd0 = s->run.integrator == PD_INTEGRATOR_CD && s->u_prev_ok ? 1 : 0;
    pi->cd = s->run.integrator == PD_INTEGRATOR_CD ? 1 : 0;
    pi->step = s->step;
    return PD_OK;
}

void pdk::sim_pack_advance(pd_sim *s, long long n)
{
    if (n <= 0) return;
    s->cur ^= (int)(n & 1);
    s->step += n;
    s->v_is_half = 1;
    s->u_prev_ok = true;
}

// Internal force at the staging buffer src (+ update per mode).
static int run_force(pd_sim *s, int mode, const float4 *src_hl, const double4_32a *src_d4, int update_breaking,
                     cudaStream_t st)
{
    TileArgs a = make_args(s, mode, src_hl, src_d4);
    a.update_breaking = update_breaking && s->mat.s_c > 0.0;
    if (s->mat.model != PD_MODEL_LPS) return launch_pmb_args(a, s->precision, st);   // bond-based laws
    int rc = launch_lps_args(a, s->precision, 1, st);
    if (rc != PD_OK) return rc;
    return launch_lps_args(a, s->precision, 0, st);
}

// Complete a half-step velocity (Eq. (9)) with the force at the current u.
static int finalize(pd_sim *s, cudaStream_t st)
{
    if (!s->v_is_half) return PD_OK;
    int rc = run_force(s, MODE_FINALIZE, s->hl[s->cur], s->d4[s->cur], 1, st);
    if (rc != PD_OK) return rc;
    s->v_is_half = 0;
    return PD_OK;
}

static int one_step(pd_sim *s, cudaStream_t st)
{
    int rc = run_force(s, MODE_STEP, s->hl[s->cur], s->d4[s->cur], 1, st);
    if (rc != PD_OK) return rc;
    s->cur ^= 1;
    s->v_is_half = 1;
    s->u_prev_ok = true;
    s->step += 1;
    return PD_OK;
}

static int capture_graph(pd_sim *s, int parity)
{
    const int cur0 = s->cur;
    const int64_t step0 = s->step;
    s->cur = parity;
    PD_CUDA(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = PD_OK;
    for (int k = 0; k < GRAPH_CHUNK && rc == PD_OK; ++k) rc = one_step(s, s->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s->cap_stream, &graph);
    s->cur = cur0;
    s->step = step0;
    if (rc != PD_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&s->graph[parity], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return PD_OK;
}

static int upload_user(pd_sim *s, const void *src, size_t bytes, cudaStream_t st)
{
    PD_CUDA(cudaMemcpyAsync(s->io, src, bytes, cudaMemcpyDefault, st));
    return PD_OK;
}

// An address of the caller's array that the simulation's kernels can use in
// place: device or managed memory of this device (no staging copy). Host
// memory, pinned or not, goes through a copy into the library's staging buffer:
// on GB300 the copy engine moves a pinned host array at the link's rate, and
// kernels reading pinned host memory directly measured no faster.
static void *direct_ptr(const pd_sim *s, const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();     // clear the error of an unknown pointer
        return nullptr;
    }
    if ((at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == s->device)
        return at.devicePointer;
    return nullptr;
}

// The user array as the kernels read it: in place when possible, else uploaded.
static int user_source(pd_sim *s, const double *user, const double **src, cudaStream_t st)
{
    *src = static_cast<const double *>(direct_ptr(s, user));
    if (*src) return PD_OK;
    int rc = upload_user(s, user, sizeof(double) * s->g.npoints * s->g.dim, st);
    *src = s->io;
    return rc;
}

// Scatter a user-order (n x dim) FP64 vector into slot-order SoA arrays.
static int user_to_slots(pd_sim *s, const double *user, double *const dst[3], cudaStream_t st)
{
    const double *src = nullptr;
    int rc = user_source(s, user, &src, st);
    if (rc != PD_OK) return rc;
    Tables t = {};
    t.slot_of_user = s->slot_of_user;
    return scatter_user_to_slots(s->g, t, src, dst, 0.0, st);
}

// Slot arrays (hl: double-float pairs instead) to the caller's array, written in
// place when the kernels can reach it, else through the staging buffer.
static int to_user(pd_sim *s, const float4 *hl, double *const src[3], double *user, cudaStream_t st)
{
    double *dst = static_cast<double *>(direct_ptr(s, user));
    int rc = gather_unstage(s->g, s->slot_of_user, hl, src, dst ? dst : s->io, st);
    if (rc != PD_OK) return rc;
    if (!dst) PD_CUDA(cudaMemcpyAsync(user, s->io, sizeof(double) * s->g.npoints * s->g.dim, cudaMemcpyDefault, st));
    return PD_OK;
}

static int slots_to_user(pd_sim *s, double *const src[3], double *user, cudaStream_t st)
{
    return to_user(s, nullptr, src, user, st);
}

static int stage_lin(pd_sim *s, const double *u, const float4 **hl, const double4_32a **d4, cudaStream_t st)
{
    if (!u) {
        *hl = s->hl[s->cur];
        *d4 = s->d4[s->cur];
        return PD_OK;
    }
    int rc = user_to_slots(s, u, s->ulin, st);
    if (rc != PD_OK) return rc;
    // the same split as the state's staging, so that a force at a passed u equals
    // the force at the same u set as the state
    rc = pack_stage(s->g, s->ulin, s->lin_hl, s->lin_d4, st, s->precision == PD_FP32C && s->state64);
    *hl = s->lin_hl;
    *d4 = s->lin_d4;
    return rc;
}

__global__ void k_scalar_gather(Geom g, const int *slot_of_user, const float *a32, const double *a64, double *out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.npoints) return;
    const int s = slot_of_user[i];
    out[i] = a64 ? a64[s] : (double)a32[s];
}

__global__ void k_perm(Geom g, const int *slot_of_rank, const int *user_of_slot, long long *perm)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= g.npoints) return;
    perm[r] = user_of_slot[slot_of_rank[r]];
}

#define CHECK_SIM(s)                                                   \
    do {                                                               \
        if (!(s)) { set_error("null simulation"); return PD_EINVAL; }  \
    } while (0)
#define CHECK_BUILT(s)                                                          \
    do {                                                                        \
        CHECK_SIM(s);                                                           \
        if (!(s)->built) { set_error("call pd_build_neighbors first"); return PD_ESTATE; } \
    } while (0)

// ============================================================ Newton-Krylov

// r = f + b on free DOFs of points, 0 elsewhere (component-major, c * nslots + s)
__global__ void k_nk_residual(Geom g, const int *user_of_slot, const uint8_t *kind, const double *f0,
                              const double *f1, const double *f2, const double *body, double *r)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.nslots) return;
    const bool act = user_of_slot[s] >= 0;
    const double *f[3] = {f0, f1, f2};
    for (int c = 0; c < g.dim; ++c) {
        const size_t e = (size_t)c * g.nslots + s;
        r[e] = (act && kind[e] != PD_BC_DISPLACEMENT) ? f[c][s] + (body ? body[e] : 0.0) : 0.0;
    }
}

// y = A x from y = K x: -y on free DOFs, x on prescribed ones, 0 off the lattice
__global__ void k_nk_post(Geom g, const int *user_of_slot, const uint8_t *kind, const double *x, double *y)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.nslots) return;
    const bool act = user_of_slot[s] >= 0;
    for (int c = 0; c < g.dim; ++c) {
        const size_t e = (size_t)c * g.nslots + s;
        y[e] = !act ? 0.0 : (kind[e] == PD_BC_DISPLACEMENT ? x[e] : -y[e]);
    }
}

// u = prescribed value on PD_BC_DISPLACEMENT DOFs; with du: u += du elsewhere
__global__ void k_nk_update(Geom g, const uint8_t *kind, const double *val, const double *du, double *u0, double *u1,
                            double *u2)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.nslots) return;
    double *u[3] = {u0, u1, u2};
    for (int c = 0; c < g.dim; ++c) {
        const size_t e = (size_t)c * g.nslots + s;
        if (kind[e] == PD_BC_DISPLACEMENT) u[c][s] = val[e];
        else if (du) u[c][s] += du[e];
    }
}

static int nk_apply(void *ctx, const double *x, double *y, cudaStream_t st)
{
    pd_sim *s = static_cast<pd_sim *>(ctx);
    const Geom &g = s->g;
    TileArgs a = make_args(s, MODE_FORCE, s->hl[s->cur], s->d4[s->cur]);
    for (int c = 0; c < g.dim; ++c) {
        a.w[c] = x + (size_t)c * g.nslots;
        a.jv[c] = y + (size_t)c * g.nslots;
    }
    int rc = launch_jvp_args(a, s->precision, st);
    if (rc != PD_OK) return rc;
    k_nk_post<<<(g.nslots + 255) / 256, 256, 0, st>>>(g, s->user_of_slot, s->bc_kind, x, y);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

// The same operator from the per-bond tangent cache of the current iterate.
static int nk_apply_cached(void *ctx, const double *x, double *y, cudaStream_t st)
{
    pd_sim *s = static_cast<pd_sim *>(ctx);
    return launch_tangent_apply(s->g, s->precision, s->nk_tan, s->user_of_slot, s->bc_kind, x, y, st);
}

// z = M^-1 r with the block-Jacobi blocks of the cached tangent.
static int nk_precond(void *ctx, const double *r, double *z, cudaStream_t st)
{
    pd_sim *s = static_cast<pd_sim *>(ctx);
    return launch_tangent_precond(s->g, s->precision, s->nk_tan, r, z, st);
}

static int nk_reserve(double **p, size_t *have, size_t want, cudaStream_t st)
{
    if (*p && *have >= want) return PD_OK;
    lib_free(*p, st);
    *p = nullptr;
    *have = 0;
    cudaError_t e = lib_malloc(reinterpret_cast<void **>(p), sizeof(double) * (want ? want : 1), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("device allocation of %zu doubles for the Newton-Krylov work failed", want);
        return PD_ENOMEM;
    }
    *have = want;
    return PD_OK;
}

// ==================================================================== C ABI

extern "C" {

int pd_last_error(char *buf, size_t len)
{
    const int n = (int)strlen(g_err);
    if (buf && len) {
        strncpy(buf, g_err, len - 1);
        buf[len - 1] = '\0';
    }
    return n;
}

int pd_create(pd_sim **out, const pd_grid *grid, const pd_material *mat, const pd_run *run)
{
    if (!out) { set_error("null out"); return PD_EINVAL; }
    *out = nullptr;
    int rc = validate(grid, mat, run);
    if (rc != PD_OK) return rc;
    pd_sim *s = new (std::nothrow) pd_sim();
    if (!s) { set_error("host allocation failed"); return PD_ENOMEM; }
    s->grid = *grid;
    s->pmat = *mat;
    s->run = *run;
    s->precision = run->precision;
    s->state64 = run->state == PD_STATE_F64;
    rc = create_impl(s);
    if (rc != PD_OK) {
        pd_destroy(s);
        return rc;
    }
    *out = s;
    return PD_OK;
}

int pd_destroy(pd_sim *s)
{
    if (!s) return PD_OK;
    drop_graphs(s);
    if (s->copy_stream) cudaStreamSynchronize(s->copy_stream);
    if (s->copy_out) cudaStreamSynchronize(s->copy_out);
    if (s->stream) cudaStreamSynchronize(s->stream);
    cudaStream_t fs = s->stream;     // stream-ordered release after the simulation's own work
    for (void *p : s->allocs) lib_free(p, fs);
    for (double *p : {s->nk_basis, s->nk_tmp, s->nk_partial, s->nk_dsc, s->nk_r, s->nk_du, s->nk_aux}) lib_free(p, fs);
    lib_free(s->nk_tan, fs);
    lib_free(s->csr.row_ptr, fs);
    lib_free(s->csr.col, fs);
    if (fs) cudaStreamSynchronize(fs);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    if (s->copy_out) cudaStreamDestroy(s->copy_out);
    if (s->ev_in) cudaEventDestroy(s->ev_in);
    if (s->ev_out) cudaEventDestroy(s->ev_out);
    for (int f = 0; f < 2; ++f)
        for (int k = 0; k < IO_CHUNKS; ++k) {
            if (s->ev_copy[f][k]) cudaEventDestroy(s->ev_copy[f][k]);
            if (s->ev_done[f][k]) cudaEventDestroy(s->ev_done[f][k]);
            if (s->ev_dgath[f][k]) cudaEventDestroy(s->ev_dgath[f][k]);
            if (s->ev_dcopy[f][k]) cudaEventDestroy(s->ev_dcopy[f][k]);
        }
    delete s;
    return PD_OK;
}

int pd_tune(const pd_grid *grid, const pd_material *mat, const pd_run *run, int32_t steps, int32_t *tile_log2,
            int32_t *pair_threads, void *stream)
{
    if (!grid || !mat || !run || !tile_log2 || steps < 1) {
        set_error("pd_tune: null argument or steps < 1");
        return PD_EINVAL;
    }
    {   // the description is checked once, before any device call
        pd_run r = *run;
        r.tile_log2 = 0;
        r.pair_threads = 0;
        const int rc = validate(grid, mat, &r);
        if (rc != PD_OK) return rc;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PD_CUDA(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ce, "cudaEventCreate");
    }
    // threads per point pair are a choice of the FP32C PMB kernel only; 1, 2, 4
    // up to the stencil's 32-bond words
    const int W = (stencil_size(grid->dim, grid->m) + 31) / 32;
    const bool splits = pair_threads && run->precision == PD_FP32C && mat->model == PD_MODEL_PMB;
    int best = 0, best_pt = 0, last_rc = PD_OK;
    float best_ms = 0.f;
    for (int L = 9; L >= 6; --L) {
        for (int pt = splits ? 1 : 0; pt <= (splits ? std::min(4, W) : 0); pt = pt ? 2 * pt : 1) {
            pd_run r = *run;
            r.tile_log2 = L;
            r.pair_threads = pt;
            pd_sim *s = nullptr;
            int rc = pd_create(&s, grid, mat, &r);
            if (rc == PD_OK) rc = pd_build_neighbors(s, stream);
            if (rc == PD_OK) rc = pd_step_explicit(s, 2, stream);
            // the best of three timed runs of `steps` steps
            float ms = 0.f;
            for (int rep = 0; rep < 3 && rc == PD_OK; ++rep) {
                cudaStream_t st = pick(s, stream);
                float t = 0.f;
                cudaError_t e = cudaEventRecord(e0, st);
                if (e == cudaSuccess) rc = pd_step_explicit(s, steps, stream);
                if (e == cudaSuccess && rc == PD_OK) e = cudaEventRecord(e1, st);
                if (e == cudaSuccess && rc == PD_OK) e = cudaEventSynchronize(e1);
                if (e == cudaSuccess && rc == PD_OK) e = cudaEventElapsedTime(&t, e0, e1);
                if (e != cudaSuccess && rc == PD_OK) rc = cuda_fail(e, "pd_tune timing");
                if (rc == PD_OK && (rep == 0 || t < ms)) ms = t;
            }
            pd_destroy(s);
            if (rc != PD_OK) {
                last_rc = rc;
                continue;
            }
            // a smaller tile or more threads per pair only when at least 1 % faster
            if (!best || ms < 0.99f * best_ms) {
                best = L;
                best_pt = pt;
                best_ms = ms;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!best) return last_rc != PD_OK ? last_rc : PD_EINVAL;
    *tile_log2 = best;
    if (pair_threads) *pair_threads = best_pt;
    return PD_OK;
}

int pd_tune_tile(const pd_grid *grid, const pd_material *mat, const pd_run *run, int32_t steps,
                 int32_t *tile_log2, void *stream)
{
    return pd_tune(grid, mat, run, steps, tile_log2, nullptr, stream);
}

int pd_build_neighbors(pd_sim *s, void *stream)
{
    CHECK_SIM(s);
    cudaStream_t st = pick(s, stream);
    drop_graphs(s);
    cudaStreamSynchronize(st);
    lib_free(s->csr.row_ptr, st);
    lib_free(s->csr.col, st);
    s->csr = BuildOut{nullptr, nullptr, 0};
    s->built = false;
    Tables t = {};
    t.tile_org = s->tile_org;
    t.tile_ref = s->tile_ref;
    t.tile_lut = s->tile_lut;
    t.stencil = s->stencil;
    t.stencil_lut = s->stencil_lut;
    t.stencil_r0 = s->stencil_r0;
    int rc = build_slots(s->g, t, s->user_of_slot, s->slot_of_user, s->rank_of_slot, s->slot_of_rank, st);
    if (rc != PD_OK) return rc;
    t.user_of_slot = s->user_of_slot;
    t.slot_of_user = s->slot_of_user;
    t.rank_of_slot = s->rank_of_slot;
    t.slot_of_rank = s->slot_of_rank;
    rc = build_csr(s->g, t, &s->csr, s->mask, st);
    if (rc != PD_OK) return rc;
    if (s->mat.model == PD_MODEL_LPS) {
        rc = build_weighted_volume(s->g, s->mat, t, s->mask, s->mtil, s->minv32, st);
        if (rc != PD_OK) return rc;
    }
    rc = build_dt_bound(s->g, s->mat, t, s->mask, s->dout, st);
    if (rc != PD_OK) return rc;
    double smax = 0.0;
    PD_CUDA(cudaMemcpyAsync(&smax, s->dout, sizeof(double), cudaMemcpyDeviceToHost, st));
    PD_CUDA(cudaStreamSynchronize(st));
    // sum_j c V V_ij / |xi| = (c V / h) sum_j V_ij / |d|
    const double denom = s->c_dt * s->mat.V / s->g.h * smax;
    s->dt_crit = denom > 0.0 ? sqrt(2.0 * s->mat.rho / denom) : 0.0;
    if (s->run.dt > 0.0) s->dt = s->run.dt;
    else s->dt = (s->run.dt_factor > 0.0 ? s->run.dt_factor : 0.5) * s->dt_crit;
    if (!(s->dt > 0.0)) { set_error("time step could not be determined (no bonds?)"); return PD_EINVAL; }
    rc = pack_stage(s->g, s->u, s->hl[s->cur], s->d4[s->cur], st, s->state64);
    if (rc != PD_OK) return rc;
    PD_CUDA(cudaStreamSynchronize(st));
    s->u_prev_ok = false;
    s->built = true;
    return PD_OK;
}

int pd_bond_count(const pd_sim *s, int64_t *nb)
{
    CHECK_BUILT(s);
    if (!nb) { set_error("null output"); return PD_EINVAL; }
    *nb = s->csr.nbonds;
    return PD_OK;
}

int pd_get_neighbors(pd_sim *s, int64_t *row_ptr, int32_t *col, int64_t *perm, void *stream)
{
    CHECK_BUILT(s);
    cudaStream_t st = pick(s, stream);
    if (row_ptr)
        PD_CUDA(cudaMemcpyAsync(row_ptr, s->csr.row_ptr, sizeof(int64_t) * (s->g.npoints + 1), cudaMemcpyDefault, st));
    if (col && s->csr.nbonds)
        PD_CUDA(cudaMemcpyAsync(col, s->csr.col, sizeof(int32_t) * s->csr.nbonds, cudaMemcpyDefault, st));
    if (perm) {
        long long *tmp = reinterpret_cast<long long *>(s->io);
        k_perm<<<(s->g.npoints + 255) / 256, 256, 0, st>>>(s->g, s->slot_of_rank, s->user_of_slot, tmp);
        PD_CUDA(cudaGetLastError());
        PD_CUDA(cudaMemcpyAsync(perm, tmp, sizeof(int64_t) * s->g.npoints, cudaMemcpyDefault, st));
    }
    PD_CUDA(cudaStreamSynchronize(st));
    return PD_OK;
}

int pd_get_broken(pd_sim *s, uint8_t *broken, void *stream)
{
    CHECK_BUILT(s);
    if (!broken) { set_error("null output"); return PD_EINVAL; }
    cudaStream_t st = pick(s, stream);
    uint8_t *tmp = nullptr;
    PD_CUDA(lib_malloc(reinterpret_cast<void **>(&tmp), s->csr.nbonds > 0 ? s->csr.nbonds : 1, st));
    Tables t = {};
    t.tile_org = s->tile_org;
    t.slot_of_rank = s->slot_of_rank;
    t.stencil_lut = s->stencil_lut;
    int rc = csr_broken_flags(s->g, t, s->csr, s->mask, tmp, st);
    if (rc == PD_OK && s->csr.nbonds) {
        cudaError_t e = cudaMemcpyAsync(broken, tmp, s->csr.nbonds, cudaMemcpyDefault, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "broken copy");
    }
    cudaError_t e = cudaStreamSynchronize(st);
    lib_free(tmp, st);
    if (rc == PD_OK && e != cudaSuccess) rc = cuda_fail(e, "pd_get_broken");
    return rc;
}

int pd_break_bonds(pd_sim *s, int axis, double pos, const double lo[3], const double hi[3], int64_t *nbroken,
                   void *stream)
{
    CHECK_BUILT(s);
    if (axis < 0 || axis >= s->g.dim || !lo || !hi) { set_error("bad notch description"); return PD_EINVAL; }
    cudaStream_t st = pick(s, stream);
    Tables t = {};
    t.tile_org = s->tile_org;
    t.user_of_slot = s->user_of_slot;
    t.stencil = s->stencil;
    int rc = break_notch(s->g, t, s->mask, axis, pos, lo, hi, s->d_count, st);
    if (rc != PD_OK) return rc;
    unsigned long long cnt = 0;
    PD_CUDA(cudaMemcpyAsync(&cnt, s->d_count, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    PD_CUDA(cudaStreamSynchronize(st));
    if (nbroken) *nbroken = (int64_t)cnt;
    return PD_OK;
}

// Pipelined host transfer of up to two state fields (u: the staging pair of the
// current step, or the FP64 arrays; v: the velocity pair or array), in IO_CHUNKS
// chunks of user rows, each field in its own half of the staging buffer.
// Upload: chunk k of a field is copied into io_up on copy_stream, then scattered
// on st once its copy event fired, so the copy of chunk k + 1 overlaps the
// scatter of chunk k; a copy into a chunk first waits for the last scatter of
// that chunk (of an earlier upload) to have read it. Download: chunk k is
// gathered on st into io_dn, then copied out on copy_out; a gather into a chunk
// first waits for the last copy out of that chunk. Uploads and downloads have
// their own buffers and copy streams, so an upload may run while an earlier
// download is still copying out, in the other direction of the link, and both
// fields of an upload may cross the link while st still computes.
// Synchronous calls: the copies also wait for the work already queued on st (the
// caller's arrays may be written by it) and st waits for them at the end.
// Pipelined (async) calls move each field in one copy and one conversion pass,
// waiting only for the staging buffer. Every wait is an event in stream order:
// no host synchronisation here.
static int xfer_chunks(pd_sim *s, const double *const host[2], const bool is_u[2], bool upload, cudaStream_t st,
                       bool async)
{
    const Geom &g = s->g;
    // double-float state: the pairs alone; FP64 state: the FP64 arrays (and for
    // u the staging pair); the FP64 path: the FP64 arrays (and for u the double4 staging)
    const bool pairs = s->precision == PD_FP32C && !s->state64;
    const bool f32c = s->precision == PD_FP32C;
    const long long n = g.npoints, d = g.dim;
    const size_t row_bytes = sizeof(double) * d;
    // one chunk below 1 MB per field: a pipeline of small copies gains nothing
    const int nc = n * (long long)row_bytes < (1 << 20) ? 1 : IO_CHUNKS;
    const long long rows = ((n + nc - 1) / nc + 255) / 256 * 256;
    cudaStream_t cs = upload ? s->copy_stream : s->copy_out;
    cudaEvent_t ev_join = upload ? s->ev_in : s->ev_out;
    if (async) {
        // pipelined calls: each field in one copy and one conversion pass (its
        // copy overlaps the previous step, so chunks would only add launches on
        // st); the upload with one thread per slot, so that its slot-order writes
        // (u, v and the staging pair) are coalesced, the download with one per
        // user row (coalesced user-order writes): both measured faster than the
        // other way round. Every chunk's event is recorded, so that a later
        // chunked call waits for the whole pass
        for (int f = 0; f < 2; ++f) {
            if (!host[f]) continue;
            double *const *slot = pairs ? nullptr : (is_u[f] ? s->u : s->v);
            float4 *hl = pairs ? (is_u[f] ? s->hl[s->cur] : s->vhl)
                               : (f32c && is_u[f] && upload ? s->hl[s->cur] : nullptr);
            double4_32a *d4 = !f32c && is_u[f] ? s->d4[s->cur] : nullptr;
            const size_t bytes = (size_t)n * row_bytes;
            if (upload) {
                double *base = s->io_up + (size_t)f * n * d;
                for (int k = 0; k < IO_CHUNKS; ++k) PD_CUDA(cudaStreamWaitEvent(cs, s->ev_done[f][k], 0));
                PD_CUDA(cudaMemcpyAsync(base, host[f], bytes, cudaMemcpyDefault, cs));
                PD_CUDA(cudaEventRecord(s->ev_copy[f][0], cs));
                PD_CUDA(cudaStreamWaitEvent(st, s->ev_copy[f][0], 0));
                int rc = scatter_stage(g, s->user_of_slot, base, slot, hl, d4, st, f32c && s->state64);
                if (rc != PD_OK) return rc;
                for (int k = 0; k < IO_CHUNKS; ++k) PD_CUDA(cudaEventRecord(s->ev_done[f][k], st));
            } else {
                double *base = s->io_dn + (size_t)f * n * d;
                for (int k = 0; k < IO_CHUNKS; ++k) PD_CUDA(cudaStreamWaitEvent(st, s->ev_dcopy[f][k], 0));
                int rc = gather_rows(g, s->slot_of_user, hl, slot, base, 0, n, st);
                if (rc != PD_OK) return rc;
                PD_CUDA(cudaEventRecord(s->ev_dgath[f][0], st));
                PD_CUDA(cudaStreamWaitEvent(cs, s->ev_dgath[f][0], 0));
                PD_CUDA(cudaMemcpyAsync(const_cast<double *>(host[f]), base, bytes, cudaMemcpyDefault, cs));
                for (int k = 0; k < IO_CHUNKS; ++k) PD_CUDA(cudaEventRecord(s->ev_dcopy[f][k], cs));
            }
        }
        return PD_OK;
    }
    PD_CUDA(cudaEventRecord(ev_join, st));
    PD_CUDA(cudaStreamWaitEvent(cs, ev_join, 0));
    for (int f = 0; f < 2; ++f) {
        if (!host[f]) continue;
        double *const *slot = pairs ? nullptr : (is_u[f] ? s->u : s->v);
        float4 *hl = pairs ? (is_u[f] ? s->hl[s->cur] : s->vhl) : (f32c && is_u[f] && upload ? s->hl[s->cur] : nullptr);
        double4_32a *d4 = !f32c && is_u[f] ? s->d4[s->cur] : nullptr;
        for (int k = 0; k < nc; ++k) {
            const long long r0 = std::min(n, k * rows), r1 = std::min(n, r0 + rows);
            if (r1 <= r0) continue;
            const size_t bytes = (size_t)(r1 - r0) * row_bytes;
            if (upload) {
                double *base = s->io_up + (size_t)f * n * d;
                PD_CUDA(cudaStreamWaitEvent(cs, s->ev_done[f][k], 0));
                PD_CUDA(cudaMemcpyAsync(base + r0 * d, host[f] + r0 * d, bytes, cudaMemcpyDefault, cs));
                PD_CUDA(cudaEventRecord(s->ev_copy[f][k], cs));
                PD_CUDA(cudaStreamWaitEvent(st, s->ev_copy[f][k], 0));
                int rc = scatter_rows(g, s->slot_of_user, base, r0, r1, slot, hl, d4, st, f32c && s->state64);
                if (rc != PD_OK) return rc;
                PD_CUDA(cudaEventRecord(s->ev_done[f][k], st));
            } else {
                double *base = s->io_dn + (size_t)f * n * d;
                PD_CUDA(cudaStreamWaitEvent(st, s->ev_dcopy[f][k], 0));
                int rc = gather_rows(g, s->slot_of_user, hl, slot, base, r0, r1, st);
                if (rc != PD_OK) return rc;
                PD_CUDA(cudaEventRecord(s->ev_dgath[f][k], st));
                PD_CUDA(cudaStreamWaitEvent(cs, s->ev_dgath[f][k], 0));
                PD_CUDA(cudaMemcpyAsync(const_cast<double *>(host[f]) + r0 * d, base + r0 * d, bytes,
                                        cudaMemcpyDefault, cs));
                PD_CUDA(cudaEventRecord(s->ev_dcopy[f][k], cs));
            }
        }
    }
    // the caller's stream finishes after every copy of this call
    PD_CUDA(cudaEventRecord(ev_join, cs));
    PD_CUDA(cudaStreamWaitEvent(st, ev_join, 0));
    return PD_OK;
}

static int set_state_impl(pd_sim *s, const double *u, const double *v, void *stream, bool async)
{
    CHECK_BUILT(s);
    cudaStream_t st = pick(s, stream);
    int rc = PD_OK;
    // a kept v must first be completed to the integer step; a replaced one not
    if (v) s->v_is_half = 0;
    else if ((rc = finalize(s, st)) != PD_OK) return rc;
    s->u_prev_ok = false;       // a central-difference run restarts from the new state
    // one pass per field from the uploaded user array: FP32C writes the
    // double-float pairs the kernels read (its FP64 arrays are a view refreshed
    // on demand), FP64 writes its SoA arrays and the double4 staging
    const bool f32c = s->precision == PD_FP32C, pairs = f32c && !s->state64;
    const double *src = nullptr;
    // host arrays: both fields in chunks through the staging buffer, copies
    // overlapping the scatters of the chunks before them
    const bool host_u = u && !direct_ptr(s, u), host_v = v && !direct_ptr(s, v);
    if (host_u || host_v) {
        const double *hu[2] = {host_u ? u : nullptr, host_v ? v : nullptr};
        const bool is_u[2] = {true, false};
        if ((rc = xfer_chunks(s, hu, is_u, true, st, async)) != PD_OK) return rc;
    }
    if (u && !host_u) {
        if ((rc = user_source(s, u, &src, st)) != PD_OK) return rc;
        rc = scatter_stage(s->g, s->user_of_slot, src, pairs ? nullptr : s->u, f32c ? s->hl[s->cur] : nullptr,
                           f32c ? nullptr : s->d4[s->cur], st, f32c && s->state64);
        if (rc != PD_OK) return rc;
    }
    if (v && !host_v) {
        if ((rc = user_source(s, v, &src, st)) != PD_OK) return rc;
        rc = scatter_stage(s->g, s->user_of_slot, src, pairs ? nullptr : s->v, pairs ? s->vhl : nullptr, nullptr, st);
        if (rc != PD_OK) return rc;
    }
    return PD_OK;
}

int pd_set_state(pd_sim *s, const double *u, const double *v, void *stream)
{
    return set_state_impl(s, u, v, stream, false);
}

int pd_set_state_async(pd_sim *s, const double *u, const double *v, void *stream)
{
    return set_state_impl(s, u, v, stream, true);
}

// FP32C with double-float state keeps u and v as pairs; refresh the FP64 SoA
// copies (with FP64 state those arrays are the state itself).
static int unpack_state(pd_sim *s, cudaStream_t st, bool want_u = true, bool want_v = true)
{
    if (s->precision != PD_FP32C || s->state64) return PD_OK;
    int rc = PD_OK;
    if (want_u && (rc = unpack_pairs(s->g, s->hl[s->cur], s->u, st)) != PD_OK) return rc;
    if (want_v && (rc = unpack_pairs(s->g, s->vhl, s->v, st)) != PD_OK) return rc;
    return PD_OK;
}

static int get_state_impl(pd_sim *s, double *u, double *v, void *stream, bool async)
{
    CHECK_BUILT(s);
    cudaStream_t st = pick(s, stream);
    int rc = PD_OK;
    // u is always at the integer step; only v may need the completing half kick
    if (v && (rc = finalize(s, st)) != PD_OK) return rc;
    // one pass per field into user order: from the double-float pairs (FP32C)
    // or the FP64 arrays, then one copy to the caller
    const bool pairs = s->precision == PD_FP32C && !s->state64;
    const bool host_u = u && !direct_ptr(s, u), host_v = v && !direct_ptr(s, v);
    if (u && !host_u && (rc = to_user(s, pairs ? s->hl[s->cur] : nullptr, s->u, u, st)) != PD_OK) return rc;
    if (v && !host_v && (rc = to_user(s, pairs ? s->vhl : nullptr, s->v, v, st)) != PD_OK) return rc;
    if (host_u || host_v) {
        // gathers in chunks on st, each chunk's copy out on copy_stream behind it
        const double *hu[2] = {host_u ? u : nullptr, host_v ? v : nullptr};
        const bool is_u[2] = {true, false};
        if ((rc = xfer_chunks(s, hu, is_u, false, st, async)) != PD_OK) return rc;
        if (!async) PD_CUDA(cudaStreamSynchronize(s->copy_out));
    }
    if (!async) PD_CUDA(cudaStreamSynchronize(st));
    return PD_OK;
}

int pd_get_state(pd_sim *s, double *u, double *v, void *stream)
{
    return get_state_impl(s, u, v, stream, false);
}

int pd_get_state_async(pd_sim *s, double *u, double *v, void *stream)
{
    return get_state_impl(s, u, v, stream, true);
}

int pd_io_sync(pd_sim *s)
{
    CHECK_BUILT(s);
    PD_CUDA(cudaStreamSynchronize(s->copy_stream));
    PD_CUDA(cudaStreamSynchronize(s->copy_out));
    return PD_OK;
}

int pd_set_bc(pd_sim *s, const uint8_t *kind, const double *value, void *stream)
{
    CHECK_BUILT(s);
    cudaStream_t st = pick(s, stream);
    const size_t NS = s->g.nslots;
    if (!kind) {
        PD_CUDA(cudaMemsetAsync(s->bc_kind, 0, 3 * NS, st));
        return PD_OK;
    }
    if (!value) { set_error("pd_set_bc needs values with kinds"); return PD_EINVAL; }
    const size_t n = (size_t)s->g.npoints * s->g.dim;
    PD_CUDA(cudaMemsetAsync(s->bc_kind, 0, 3 * NS, st));
    PD_CUDA(cudaMemsetAsync(s->d_err, 0, sizeof(int), st));
    uint8_t *kbuf = reinterpret_cast<uint8_t *>(s->ekin);   // n bytes of scratch
    PD_CUDA(cudaMemcpyAsync(kbuf, kind, n, cudaMemcpyDefault, st));
    Tables t = {};
    t.slot_of_user = s->slot_of_user;
    int rc = scatter_kinds(s->g, t, kbuf, s->bc_kind, s->d_err, st);
    if (rc != PD_OK) return rc;
    double *vals[3] = {s->bc_val, s->bc_val + NS, s->bc_val + 2 * NS};
    rc = user_to_slots(s, value, vals, st);
    if (rc != PD_OK) return rc;
    if (s->bc32 && (rc = pack_dof_pairs(3 * (long long)NS, s->bc_val, s->bc32, st)) != PD_OK) return rc;
    int herr = 0;
    PD_CUDA(cudaMemcpyAsync(&herr, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    PD_CUDA(cudaStreamSynchronize(st));
    if (herr) {
        PD_CUDA(cudaMemset(s->bc_kind, 0, 3 * NS));
        set_error("unknown boundary-condition kind");
        return PD_EINVAL;
    }
    return PD_OK;
}

int pd_set_body_force(pd_sim *s, const double *b, void *stream)
{
    CHECK_BUILT(s);
    cudaStream_t st = pick(s, stream);
    drop_graphs(s);
    if (!b) {
        s->use_body = false;
        return PD_OK;
    }
    if (!s->body) ALLOC(s->body, 3 * sizeof(double) * s->g.nslots);
    double *dst[3] = {s->body, s->body + s->g.nslots, s->body + 2 * (size_t)s->g.nslots};
    int rc = user_to_slots(s, b, dst, st);
    if (rc != PD_OK) return rc;
    if (s->precision == PD_FP32C) {
        if (!s->body32) ALLOC(s->body32, sizeof(float4) * s->g.nslots);
        if ((rc = pack_f4(s->g, s->body, s->body32, st)) != PD_OK) return rc;
    }
    s->use_body = true;
    return PD_OK;
}

int pd_get_dt(const pd_sim *s, double *dt)
{
    CHECK_BUILT(s);
    if (!dt) { set_error("null output"); return PD_EINVAL; }
    *dt = s->dt;
    return PD_OK;
}

int pd_set_dt(pd_sim *s, double dt)
{
    CHECK_BUILT(s);
    if (!(dt > 0.0)) { set_error("dt must be > 0"); return PD_EINVAL; }
    if (s->v_is_half) {
        int rc = finalize(s, s->stream);
        if (rc != PD_OK) return rc;
    }
    s->dt = dt;
    s->u_prev_ok = false;
    drop_graphs(s);
    return PD_OK;
}

int pd_get_step(const pd_sim *s, int64_t *step)
{
    CHECK_SIM(s);
    if (!step) { set_error("null output"); return PD_EINVAL; }
    *step = s->step;
    return PD_OK;
}

int pd_force(pd_sim *s, const double *u, double *f_out, unsigned flags, void *stream)
{
    CHECK_BUILT(s);
    if (!f_out) { set_error("null output"); return PD_EINVAL; }
    cudaStream_t st = pick(s, stream);
    const float4 *hl;
    const double4_32a *d4;
    int rc = stage_lin(s, u, &hl, &d4, st);
    if (rc != PD_OK) return rc;
    rc = run_force(s, MODE_FORCE, hl, d4, (flags & PD_FORCE_UPDATE_BREAKING) ? 1 : 0, st);
    if (rc != PD_OK) return rc;
    return slots_to_user(s, s->f, f_out, st);
}

int pd_dilatation(pd_sim *s, const double *u, double *theta_out, void *stream)
{
    CHECK_BUILT(s);
    if (s->mat.model != PD_MODEL_LPS) { set_error("dilatation is defined for LPS only"); return PD_EINVAL; }
    if (!theta_out) { set_error("null output"); return PD_EINVAL; }
    cudaStream_t st = pick(s, stream);
    const float4 *hl;
    const double4_32a *d4;
    int rc = stage_lin(s, u, &hl, &d4, st);
    if (rc != PD_OK) return rc;
    TileArgs a = make_args(s, MODE_FORCE, hl, d4);
    rc = launch_lps_args(a, s->precision, 1, st);
    if (rc != PD_OK) return rc;
    k_scalar_gather<<<(s->g.npoints + 255) / 256, 256, 0, st>>>(
        s->g, s->slot_of_user, s->theta32, s->precision == PD_FP64 ? s->theta64 : nullptr, s->io);
    PD_CUDA(cudaGetLastError());
    PD_CUDA(cudaMemcpyAsync(theta_out, s->io, sizeof(double) * s->g.npoints, cudaMemcpyDefault, st));
    return PD_OK;
}

int pd_step_explicit_timed(pd_sim *s, int64_t nsteps, double pass_ms[2], void *stream)
{
    CHECK_BUILT(s);
    if (nsteps < 0 || !pass_ms) { set_error("nsteps must be >= 0 and pass_ms non-null"); return PD_EINVAL; }
    cudaStream_t st = pick(s, stream);
    pass_ms[0] = pass_ms[1] = 0.0;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    for (int k = 0; k < 3; ++k)
        if (cudaEventCreate(&ev[k]) != cudaSuccess) {
            for (int j = 0; j < k; ++j) cudaEventDestroy(ev[j]);
            return cuda_fail(cudaGetLastError(), "cudaEventCreate");
        }
    const bool lps = s->mat.model == PD_MODEL_LPS;
    int rc = PD_OK;
    for (int64_t n = 0; n < nsteps && rc == PD_OK; ++n) {
        TileArgs a = make_args(s, MODE_STEP, s->hl[s->cur], s->d4[s->cur]);
        a.update_breaking = s->mat.s_c > 0.0;
        cudaError_t e = cudaEventRecord(ev[0], st);
        if (e == cudaSuccess) {
            if (lps) {
                rc = launch_lps_args(a, s->precision, 1, st);
                if (rc == PD_OK) e = cudaEventRecord(ev[1], st);
                if (rc == PD_OK && e == cudaSuccess) rc = launch_lps_args(a, s->precision, 0, st);
            } else {
                rc = launch_pmb_args(a, s->precision, st);
            }
        }
        if (rc == PD_OK && e == cudaSuccess) e = cudaEventRecord(ev[2], st);
        if (rc == PD_OK && e == cudaSuccess) e = cudaEventSynchronize(ev[2]);
        if (rc == PD_OK && e != cudaSuccess) rc = cuda_fail(e, "step timing events");
        if (rc != PD_OK) break;
        float t0 = 0.f, t1 = 0.f;
        if (lps) {
            cudaEventElapsedTime(&t0, ev[0], ev[1]);
            cudaEventElapsedTime(&t1, ev[1], ev[2]);
        } else {
            cudaEventElapsedTime(&t0, ev[0], ev[2]);
        }
        pass_ms[0] += t0;
        pass_ms[1] += t1;
        s->cur ^= 1;
        s->v_is_half = 1;
        s->u_prev_ok = true;
        s->step += 1;
    }
    for (int k = 0; k < 3; ++k) cudaEventDestroy(ev[k]);
    return rc;
}

int pd_step_explicit(pd_sim *s, int64_t nsteps, void *stream)
{
    CHECK_BUILT(s);
    if (nsteps < 0) { set_error("nsteps must be >= 0"); return PD_EINVAL; }
    cudaStream_t st = pick(s, stream);
    int rc = PD_OK;
    // the first step after a restart is a velocity-Verlet step; graphs hold
    // steps that start from a half-step velocity (and, under central
    // difference, a valid u^{k-1})
    if (nsteps > 0 && (!s->v_is_half || !s->u_prev_ok)) {
        rc = one_step(s, st);
        if (rc != PD_OK) return rc;
        --nsteps;
    }
    while (nsteps >= GRAPH_CHUNK) {
        if (!s->graph[s->cur]) {
            rc = capture_graph(s, s->cur);
            if (rc != PD_OK) return rc;
        }
        PD_CUDA(cudaGraphLaunch(s->graph[s->cur], st));
        s->step += GRAPH_CHUNK;   // GRAPH_CHUNK is even: parity unchanged
        nsteps -= GRAPH_CHUNK;
    }
    while (nsteps-- > 0) {
        rc = one_step(s, st);
        if (rc != PD_OK) return rc;
    }
    return PD_OK;
}

static int tangent(pd_sim *s, const double *u_lin, const double *w, double *out, unsigned flags, int adjoint,
                   void *stream)
{
    CHECK_BUILT(s);
    if (s->mat.model != PD_MODEL_PMB) { set_error("the tangent is implemented for PMB only"); return PD_EINVAL; }
    if (!s->tangent_ok) {
        set_error("the tangent's halo box does not fit in shared memory at this horizon and precision");
        return PD_EINVAL;
    }
    if (!w || !out) { set_error("null vector"); return PD_EINVAL; }
    cudaStream_t st = pick(s, stream);
    const float4 *hl;
    const double4_32a *d4;
    int rc = stage_lin(s, u_lin, &hl, &d4, st);
    if (rc != PD_OK) return rc;
    rc = user_to_slots(s, w, s->f, st);      // unmasked copy kept in f
    if (rc != PD_OK) return rc;
    for (int c = 0; c < s->g.dim; ++c)
        PD_CUDA(cudaMemcpyAsync(s->w[c], s->f[c], sizeof(double) * s->g.nslots, cudaMemcpyDeviceToDevice, st));
    const bool mask = (flags & PD_JVP_MASK_DIRICHLET) != 0;
    if (mask && (rc = dirichlet_mask(s->g, s->bc_kind, s->w, nullptr, 0, st)) != PD_OK) return rc;
    TileArgs a = make_args(s, MODE_FORCE, hl, d4);
    a.adjoint = adjoint;
    rc = launch_jvp_args(a, s->precision, st);
    if (rc != PD_OK) return rc;
    if (mask) {
        const double *src[3] = {s->f[0], s->f[1], s->f[2]};
        if ((rc = dirichlet_mask(s->g, s->bc_kind, s->jv, src, 1, st)) != PD_OK) return rc;
    }
    return slots_to_user(s, s->jv, out, st);
}

int pd_jvp(pd_sim *s, const double *u_lin, const double *w, double *out, unsigned flags, void *stream)
{
    return tangent(s, u_lin, w, out, flags, 0, stream);
}

int pd_vjp(pd_sim *s, const double *u_lin, const double *v, double *out, unsigned flags, void *stream)
{
    return tangent(s, u_lin, v, out, flags, 1, stream);
}

int pd_solve_static(pd_sim *s, const pd_newton_opts *opts, pd_newton_stats *stats, void *stream)
{
    CHECK_BUILT(s);
    if (s->mat.model != PD_MODEL_PMB) { set_error("the static solve needs the PMB tangent"); return PD_EINVAL; }
    pd_newton_opts o = {PD_KRYLOV_GMRES, 50, 20000, 20, PD_TANGENT_CACHED, PD_PRECOND_NONE, 1e-8, 1e-8, 0.0};
    if (opts) o = *opts;
    if (o.krylov != PD_KRYLOV_GMRES && o.krylov != PD_KRYLOV_CG) { set_error("unknown Krylov method"); return PD_EINVAL; }
    if (o.restart < 1 || o.restart > 500) { set_error("restart must be in [1, 500]"); return PD_EINVAL; }
    if (o.max_linear_iters < 1 || o.max_newton_iters < 1) { set_error("iteration limits must be >= 1"); return PD_EINVAL; }
    if (o.tangent != PD_TANGENT_CACHED && o.tangent != PD_TANGENT_JVP) { set_error("unknown tangent mode"); return PD_EINVAL; }
    const bool cached = o.tangent == PD_TANGENT_CACHED;
    if (o.precond != PD_PRECOND_NONE && o.precond != PD_PRECOND_BLOCK_JACOBI) { set_error("unknown preconditioner"); return PD_EINVAL; }
    const bool jacobi = o.precond == PD_PRECOND_BLOCK_JACOBI;
    if (jacobi && !cached) { set_error("the block-Jacobi preconditioner needs the cached tangent"); return PD_EINVAL; }
    if (!cached && !s->tangent_ok) {
        set_error("the tangent's halo box does not fit in shared memory at this horizon and precision");
        return PD_EINVAL;
    }
    if (!(o.linear_rtol > 0.0) || !(o.newton_rtol >= 0.0) || !(o.newton_atol >= 0.0)) {
        set_error("tolerances must be linear_rtol > 0, newton_rtol >= 0, newton_atol >= 0");
        return PD_EINVAL;
    }
    cudaStream_t st = pick(s, stream);
    const Geom &g = s->g;
    const long long n = (long long)g.dim * g.nslots;
    const int kdim = o.krylov == PD_KRYLOV_GMRES ? o.restart : 2;
    size_t hr = 0, hd = 0;
    int rc = PD_OK;
    if ((rc = nk_reserve(&s->nk_basis, &s->nk_basis_n, (size_t)(kdim + 1) * n, st)) != PD_OK) return rc;
    if ((rc = nk_reserve(&s->nk_partial, &s->nk_partial_n, krylov_partial_doubles(n, kdim + 1), st)) != PD_OK) return rc;
    if ((rc = nk_reserve(&s->nk_dsc, &s->nk_dsc_n,
                         krylov_dsc_doubles(o.krylov == PD_KRYLOV_GMRES ? o.restart : 0), st)) != PD_OK)
        return rc;
    if (!s->nk_tmp) {
        if ((rc = nk_reserve(&s->nk_tmp, &hr, (size_t)n, st)) != PD_OK) return rc;
        if ((rc = nk_reserve(&s->nk_r, &hr, (size_t)n, st)) != PD_OK) return rc;
        if ((rc = nk_reserve(&s->nk_du, &hd, (size_t)n, st)) != PD_OK) return rc;
        if ((rc = nk_reserve(&s->nk_aux, &hd, 2 * (size_t)n, st)) != PD_OK) return rc;
    }
    const size_t tan_bytes = cached ? tangent_cache_bytes(g, s->precision) : 0;
    if (s->nk_tan_n < tan_bytes) {
        lib_free(s->nk_tan, st);
        s->nk_tan = nullptr;
        s->nk_tan_n = 0;
        if (lib_malloc(&s->nk_tan, tan_bytes, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
            s->nk_tan = nullptr;
            set_error("device allocation of %zu bytes for the tangent cache failed", tan_bytes);
            return PD_ENOMEM;
        }
        s->nk_tan_n = tan_bytes;
    }
    KrylovWork wk{s->nk_basis, s->nk_tmp, s->nk_aux, s->nk_partial, s->nk_dsc, s->cap_stream};
    KrylovOp op{cached ? nk_apply_cached : nk_apply, s, jacobi ? nk_precond : nullptr};
    const unsigned nbs = (unsigned)((g.nslots + 255) / 256);

    // the iterate lives in the FP64 slot arrays u; the prescribed values first
    if ((rc = unpack_state(s, st, true, false)) != PD_OK) return rc;
    k_nk_update<<<nbs, 256, 0, st>>>(g, s->bc_kind, s->bc_val, nullptr, s->u[0], s->u[1], s->u[2]);
    PD_CUDA(cudaGetLastError());
    pd_newton_stats ns = {0, 0, 0, 0, 0.0, 0.0};
    for (int it = 0;; ++it) {
        if ((rc = pack_stage(g, s->u, s->hl[s->cur], s->d4[s->cur], st, s->state64)) != PD_OK) return rc;
        if ((rc = run_force(s, MODE_FORCE, s->hl[s->cur], s->d4[s->cur], 0, st)) != PD_OK) return rc;
        k_nk_residual<<<nbs, 256, 0, st>>>(g, s->user_of_slot, s->bc_kind, s->f[0], s->f[1], s->f[2],
                                           s->use_body ? s->body : nullptr, s->nk_r);
        PD_CUDA(cudaGetLastError());
        double rn = 0.0;
        if ((rc = krylov_norm(s->nk_r, n, wk, &rn, st)) != PD_OK) return rc;
        if (it == 0) ns.res0 = rn;
        ns.res = rn;
        if (rn <= o.newton_rtol * ns.res0 + o.newton_atol) {
            ns.converged = 1;
            break;
        }
        if (it >= o.max_newton_iters) break;
        // the tangent at this iterate, once for the whole linear solve
        if (cached) {
            TileArgs ta = make_args(s, MODE_FORCE, s->hl[s->cur], s->d4[s->cur]);
            if ((rc = launch_tangent_prepare(ta, s->precision, s->nk_tan, st)) != PD_OK) return rc;
            if (jacobi && (rc = launch_tangent_jacobi(g, s->precision, s->nk_tan, s->user_of_slot, s->bc_kind, st)) != PD_OK)
                return rc;
        }
        KrylovStats ks = {0, 0, 0.0, 0.0};
        rc = o.krylov == PD_KRYLOV_GMRES
                 ? krylov_gmres(op, s->nk_r, s->nk_du, n, o.restart, o.max_linear_iters, o.linear_rtol, wk, &ks, st)
                 : krylov_cg(op, s->nk_r, s->nk_du, n, o.max_linear_iters, o.linear_rtol, wk, &ks, st);
        if (rc != PD_OK) return rc;
        ns.newton_iters += 1;
        ns.linear_iters += ks.iters;
        ns.linear_failures += ks.converged ? 0 : 1;
        k_nk_update<<<nbs, 256, 0, st>>>(g, s->bc_kind, s->bc_val, s->nk_du, s->u[0], s->u[1], s->u[2]);
        PD_CUDA(cudaGetLastError());
    }
    // static state: v = 0 at an integer step
    for (int c = 0; c < 3; ++c)
        if (s->v[c]) PD_CUDA(cudaMemsetAsync(s->v[c], 0, sizeof(double) * g.nslots, st));
    if (s->vhl) PD_CUDA(cudaMemsetAsync(s->vhl, 0, 2 * sizeof(float4) * g.nslots, st));
    s->v_is_half = 0;
    s->u_prev_ok = false;
    PD_CUDA(cudaStreamSynchronize(st));
    if (stats) *stats = ns;
    return PD_OK;
}

int pd_energy(pd_sim *s, double *kinetic, double *strain, void *stream)
{
    CHECK_BUILT(s);
    cudaStream_t st = pick(s, stream);
    int rc = finalize(s, st);
    if (rc != PD_OK) return rc;
    if ((rc = unpack_state(s, st)) != PD_OK) return rc;
    TileArgs a = make_args(s, MODE_FORCE, s->hl[s->cur], s->d4[s->cur]);
    if (s->mat.model == PD_MODEL_LPS && (rc = launch_lps_args(a, s->precision, 1, st)) != PD_OK) return rc;
    if ((rc = launch_energy_points(a, s->precision, s->ekin, st)) != PD_OK) return rc;
    if ((rc = reduce_sum(s->epoint, s->g.nslots, s->mat.V, s->red, s->dout, st)) != PD_OK) return rc;
    if ((rc = reduce_sum(s->ekin, s->g.nslots, 0.5 * s->mat.rho * s->mat.V, s->red, s->dout + 1, st)) != PD_OK)
        return rc;
    double h[2];
    PD_CUDA(cudaMemcpyAsync(h, s->dout, sizeof(h), cudaMemcpyDeviceToHost, st));
    PD_CUDA(cudaStreamSynchronize(st));
    if (strain) *strain = h[0];
    if (kinetic) *kinetic = h[1];
    return PD_OK;
}

}  // extern "C"
