// pd_krylov.cu -- Krylov solvers of the matrix-free Newton step that replaces the
// assembled-stiffness Newton iteration of Sec. 5 (Eq. (6), Algorithm 3): the
// tangent is applied by the JVP kernel (pd_jvp.cu), never assembled.
//
// Vectors are FP64, component-major over slots: v[c * nslots + s], c < dim;
// slots without a point hold 0 and every operation keeps them 0. All sums are
// deterministic: a fixed block partition, a fixed in-block tree, and a fixed
// final tree over the block partials. The scalar steps run on the device too
// (one-thread kernels): GMRES's Hessenberg column is formed from the
// Gram-Schmidt dot products' final sums, and its Givens rotations and the
// residual estimate from the Arnoldi vector's norm; CG's alpha and beta are
// formed from p.Ap and r.r. The host reads the scalars back once per chunk of
// iterations (GM_CHUNK Arnoldi steps, CG_CHUNK CG iterations), each chunk
// replayed as a captured CUDA graph.
#include <math.h>

#include <algorithm>
#include <vector>

#include "pd_tile.cuh"

namespace pdk {

constexpr int KT = 256;               // threads per block
constexpr int KPER = 8;               // elements per thread in a reduction block
constexpr int KCHUNK = KT * KPER;     // elements per reduction block

static int kblocks(long long n) { return (int)((n + KCHUNK - 1) / KCHUNK); }

// Fixed-order sum of one value per thread of the block; the result is valid in
// thread 0.
__device__ __forceinline__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    __syncthreads();            // red may still be read from a previous call
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < KT / 32; ++w) t += red[w];
    return t;
}

// partial[i * nb + b] = sum over block b of V_i . w (V_i = V + i * ldv); grid
// (nb, k): block (b, i) sums chunk b of vector i, so all k products run at once.
__global__ void __launch_bounds__(KT) k_mdot(const double *V, long long ldv, const double *w, long long n,
                                             double *partial)
{
    __shared__ double red[KT / 32];
    const long long base = (long long)blockIdx.x * KCHUNK + threadIdx.x;
    const double *vi = V + (long long)blockIdx.y * ldv;
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < KPER; ++q) {
        const long long e = base + (long long)q * KT;
        if (e < n) acc = fma(vi[e], w[e], acc);
    }
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) partial[(long long)blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// out[i] = sum_b partial[i * nb + b], one block per i, fixed order.
__global__ void __launch_bounds__(KT) k_partial_sum(const double *partial, int nb, double *out)
{
    __shared__ double red[KT / 32];
    const double *p = partial + (long long)blockIdx.x * nb;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += KT) acc += p[b];
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) out[blockIdx.x] = t;
}

// y = alpha * y + sum_{i<k} coef[i] * V_i  (coef on the device; alpha on the host)
__global__ void k_lincomb(double *y, double alpha, const double *V, long long ldv, int k, const double *coef,
                          double csign, long long n)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double acc = alpha == 0.0 ? 0.0 : alpha * y[e];
#pragma unroll 8
    for (int i = 0; i < k; ++i) acc = fma(csign * coef[i], V[(long long)i * ldv + e], acc);
    y[e] = acc;
}

// y = a * x + b * y
__global__ void k_axpby(double a, const double *x, double b, double *y, long long n)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    y[e] = a * x[e] + (b == 0.0 ? 0.0 : b * y[e]);
}

// ------------------------------------------------------------------ helpers

struct KrylovCtx {
    long long n;               // dim * nslots
    cudaStream_t st;
    double *partial;           // kblocks(n) * (kmax + 1)
    double *dsc;               // device scalars, kmax + 2
    std::vector<double> hsc;   // host copies
};

static int dots(KrylovCtx &c, const double *V, long long ldv, int k, const double *w, double *host_out)
{
    const int nb = kblocks(c.n);
    k_mdot<<<dim3(nb, k), KT, 0, c.st>>>(V, ldv, w, c.n, c.partial);
    k_partial_sum<<<k, KT, 0, c.st>>>(c.partial, nb, c.dsc);
    PD_CUDA(cudaGetLastError());
    if (host_out) {
        PD_CUDA(cudaMemcpyAsync(host_out, c.dsc, sizeof(double) * k, cudaMemcpyDeviceToHost, c.st));
        PD_CUDA(cudaStreamSynchronize(c.st));
    }
    return PD_OK;
}

static int axpby(KrylovCtx &c, double a, const double *x, double b, double *y)
{
    k_axpby<<<(unsigned)((c.n + 255) / 256), 256, 0, c.st>>>(a, x, b, y, c.n);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

// y = alpha y + csign * sum_i coef[i] V_i with coef already in c.dsc
static int lincomb_dev(KrylovCtx &c, double *y, double alpha, const double *V, long long ldv, int k, double csign)
{
    k_lincomb<<<(unsigned)((c.n + 255) / 256), 256, 0, c.st>>>(y, alpha, V, ldv, k, c.dsc, csign, c.n);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

static int norm2(KrylovCtx &c, const double *x, double *out)
{
    double d = 0.0;
    int rc = dots(c, x, 0, 1, x, &d);
    if (rc != PD_OK) return rc;
    *out = sqrt(d);
    return PD_OK;
}

// ------------------------------------------------------------------ GMRES(m)

// Device layout of GMRES's small arrays in dsc (m = restart): the dot results
// [0, m+1), the Hessenberg matrix H (column-major, (m+1) x m), the rotations cs
// and sn, the rotated right-hand side g (m+1), the solution y of the small
// triangular system (m), and the scalars. The host enqueues GM_CHUNK Arnoldi
// steps at a time and reads back once per chunk; a step after the one that
// met the target (or broke down) changes nothing that the update of x uses.
struct GmLayout {
    int m, H, cs, sn, g, y, sc;
    __host__ __device__ explicit GmLayout(int m_)
        : m(m_), H(m_ + 1), cs(H + (m_ + 1) * m_), sn(cs + m_), g(sn + m_), y(g + m_ + 1), sc(y + m_)
    {
    }
    __host__ __device__ int size() const { return sc + 8; }
};
enum { GM_TARGET = 0, GM_DONE, GM_K, GM_RES, GM_INVH, GM_ITERS };
constexpr int GM_CHUNK = 8;

size_t krylov_dsc_doubles(int krylov_gmres_restart)
{
    const size_t g = krylov_gmres_restart > 0 ? (size_t)GmLayout(krylov_gmres_restart).size() : 0;
    return std::max(g, KRYLOV_DSC_MIN);
}

// The block sums of k_partial_sum for dot i (block i, the same fixed order), and
// with them column j of the Hessenberg matrix: H[i, j] = dot i (first
// Gram-Schmidt pass) or += (second pass), unless the cycle is done.
__global__ void __launch_bounds__(KT) k_partial_sum_hcol(const double *partial, int nb, double *d, int m, int j,
                                                       int add)
{
    __shared__ double red[KT / 32];
    const GmLayout L(m);
    const double *p = partial + (long long)blockIdx.x * nb;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += KT) acc += p[b];
    const double t = block_sum(acc, red);
    if (threadIdx.x != 0) return;
    const int i = blockIdx.x;
    d[i] = t;
    if (d[L.sc + GM_DONE] != 0.0) return;
    double *h = d + L.H + i + (m + 1) * j;
    *h = add ? *h + t : t;
}

// After dsc[0] = |w|^2: H[j+1, j] = |w|, the previous rotations and a new one on
// column j, g rotated, the residual estimate |g[j+1]|, the scale 1/|w| for w.
// The block stages column j and the rotations in shared memory (3 (m + 1)
// doubles, dynamic) so that the sequential rotation loop of thread 0 does not
// wait on global loads.
// |w|^2 is summed here from the nb block partials of k_mdot, in k_partial_sum's
// fixed order (KT threads).
__global__ void __launch_bounds__(KT) k_gm_step(const double *partial, int nb, double *d, int m, int j)
{
    extern __shared__ double gs[];
    __shared__ double red[KT / 32];
    const GmLayout L(m);
    double *sc = d + L.sc;
    {
        double acc = 0.0;
        for (int b = threadIdx.x; b < nb; b += KT) acc += partial[b];
        const double t = block_sum(acc, red);
        if (threadIdx.x == 0) d[0] = t;
        __syncthreads();
    }
    if (sc[GM_DONE] != 0.0) {
        if (threadIdx.x == 0) sc[GM_INVH] = 0.0;
        return;
    }
    double *hj = d + L.H + (m + 1) * j;
    double *hs = gs, *css = gs + (m + 1), *sns = gs + 2 * (m + 1);
    for (int i = threadIdx.x; i <= j; i += blockDim.x) hs[i] = hj[i];
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        css[i] = d[L.cs + i];
        sns[i] = d[L.sn + i];
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double hn = sqrt(d[0]);
    double *cs = d + L.cs, *sn = d + L.sn, *g = d + L.g;
    hs[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        const double t = css[i] * hs[i] + sns[i] * hs[i + 1];
        hs[i + 1] = -sns[i] * hs[i] + css[i] * hs[i + 1];
        hs[i] = t;
    }
    const double den = hypot(hs[j], hs[j + 1]);
    cs[j] = den > 0.0 ? hs[j] / den : 1.0;
    sn[j] = den > 0.0 ? hs[j + 1] / den : 0.0;
    hs[j] = den;
    hs[j + 1] = 0.0;
    for (int i = 0; i <= j + 1; ++i) hj[i] = hs[i];
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    sc[GM_K] = j + 1;
    sc[GM_ITERS] += 1.0;
    sc[GM_RES] = fabs(g[j + 1]);
    sc[GM_INVH] = hn > 0.0 ? 1.0 / hn : 0.0;
    if (sc[GM_RES] <= sc[GM_TARGET] || hn == 0.0) sc[GM_DONE] = 1.0;
}

// y = H(0:k, 0:k)^-1 g(0:k), back substitution
__global__ void k_gm_solve(double *d, int m)
{
    const GmLayout L(m);
    const int k = (int)d[L.sc + GM_K];
    const double *H = d + L.H, *g = d + L.g;
    double *y = d + L.y;
    for (int i = k - 1; i >= 0; --i) {
        double t = g[i];
        for (int l = i + 1; l < k; ++l) t -= H[i + (m + 1) * l] * y[l];
        const double dd = H[i + (m + 1) * i];
        y[i] = dd != 0.0 ? t / dd : 0.0;
    }
}

// y *= d[idx]
__global__ void k_scale_dev(const double *d, int idx, double *y, long long n)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    y[e] = d[idx] * y[e];
}

// Restarted GMRES with classical Gram-Schmidt applied twice (CGS2) and Givens
// rotations: solve A x = b from x = 0 until ||b - A x|| <= rtol ||b||. With a
// preconditioner M it is right-preconditioned (Arnoldi on A M^-1, x += M^-1 V y),
// so the residual it monitors is the one of A x = b.
int krylov_gmres(const KrylovOp &op, const double *b, double *x, long long n, int restart, int maxit, double rtol,
                 KrylovWork &wk, KrylovStats *stats, cudaStream_t st)
{
    KrylovCtx c{n, st, wk.partial, wk.dsc, {}};
    const int m = restart;
    const GmLayout L(m);
    double *V = wk.basis;                    // (m + 1) vectors of n
    double *w = wk.tmp;
    double *zt = wk.aux, *ty = wk.aux + n;   // M^-1 v_j; V y before M^-1
    const bool pc = op.precond != nullptr;
    const unsigned nbk = (unsigned)((n + 255) / 256);
    PD_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    double bnorm = 0.0;
    int rc = norm2(c, b, &bnorm);
    if (rc != PD_OK) return rc;
    stats->res0 = bnorm;
    stats->iters = 0;
    stats->res = bnorm;
    stats->converged = 0;
    if (bnorm == 0.0) {
        stats->converged = 1;
        return PD_OK;
    }
    const double target = rtol * bnorm;
    // one Arnoldi step j of the cycle, enqueued on stream s without a host synchronisation
    auto arnoldi = [&](int j, cudaStream_t s) -> int {
        KrylovCtx cs{n, s, wk.partial, wk.dsc, {}};
        double *vj1 = V + (long long)(j + 1) * n;
        const double *src = V + (long long)j * n;
        int e = PD_OK;
        if (pc) {
            if ((e = op.precond(op.ctx, src, zt, s)) != PD_OK) return e;
            src = zt;
        }
        if ((e = op.apply(op.ctx, src, vj1, s)) != PD_OK) return e;
        const int nb = kblocks(n);
        // CGS2: h = V^T w, w -= V h; twice. (Fusing each pass's update with the
        // next products into one launch, every block summing the previous
        // products itself, measured slower on the 200^2 plate: 0.0975 -> 0.122 ms
        // per Arnoldi step; the per-thread loops over the basis vectors have far
        // less parallelism than k_mdot's (chunk, vector) grid. Each pass's products
        // and their sums in one launch, the block that finishes last summing the
        // partials one warp per dot, measured 0.1005 against 0.098 ms: inside a
        // captured graph the second launch costs no more than the atomic, the
        // fence and the last block's serial tail.)
        for (int pass = 0; pass < 2; ++pass) {
            k_mdot<<<dim3(nb, j + 1), KT, 0, s>>>(V, n, vj1, n, cs.partial);
            k_partial_sum_hcol<<<j + 1, KT, 0, s>>>(cs.partial, nb, cs.dsc, m, j, pass);
            if ((e = lincomb_dev(cs, vj1, 1.0, V, n, j + 1, -1.0)) != PD_OK) return e;
        }
        k_mdot<<<dim3(nb, 1), KT, 0, s>>>(vj1, 0, vj1, n, cs.partial);
        k_gm_step<<<1, KT, 3 * (m + 1) * sizeof(double), s>>>(cs.partial, nb, cs.dsc, m, j);
        k_scale_dev<<<nbk, 256, 0, s>>>(cs.dsc, L.sc + GM_INVH, vj1, n);
        PD_CUDA(cudaGetLastError());
        return PD_OK;
    };
    // The chunk of steps [j0, j0 + GM_CHUNK) as a CUDA graph, captured on first use
    // (launch gaps dominate at small n); null if the capture does not succeed, and
    // the chunk is then launched step by step.
    struct Graphs {
        std::vector<cudaGraphExec_t> g;
        ~Graphs()
        {
            for (cudaGraphExec_t e : g)
                if (e) cudaGraphExecDestroy(e);
        }
    } graphs;
    graphs.g.assign((m + GM_CHUNK - 1) / GM_CHUNK, nullptr);
    std::vector<char> tried(graphs.g.size(), 0);
    auto chunk_graph = [&](int j0) -> cudaGraphExec_t {
        const int ci = j0 / GM_CHUNK;
        if (!wk.cap || tried[ci]) return graphs.g[ci];
        tried[ci] = 1;
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(wk.cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            int crc = PD_OK;
            for (int j = j0; j < std::min(m, j0 + GM_CHUNK) && crc == PD_OK; ++j) crc = arnoldi(j, wk.cap);
            const cudaError_t e = cudaStreamEndCapture(wk.cap, &graph);
            if (crc != PD_OK || e != cudaSuccess || !graph ||
                cudaGraphInstantiate(&graphs.g[ci], graph, 0) != cudaSuccess)
                graphs.g[ci] = nullptr;
            if (graph) cudaGraphDestroy(graph);
        }
        cudaGetLastError();
        return graphs.g[ci];
    };
    std::vector<double> init(L.size(), 0.0);
    double back[8];
    bool first = true;
    while (true) {
        // r = b - A x  (x = 0 on the first cycle)
        double beta;
        if (first) {
            PD_CUDA(cudaMemcpyAsync(V, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
            beta = bnorm;
        } else {
            if ((rc = op.apply(op.ctx, x, w, st)) != PD_OK) return rc;
            if ((rc = axpby(c, 1.0, b, -1.0, w)) != PD_OK) return rc;    // w = b - A x
            PD_CUDA(cudaMemcpyAsync(V, w, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
            if ((rc = norm2(c, V, &beta)) != PD_OK) return rc;
        }
        first = false;
        stats->res = beta;
        if (beta <= target) {
            stats->converged = 1;
            return PD_OK;
        }
        if (stats->iters >= maxit) return PD_OK;
        if ((rc = axpby(c, 0.0, V, 1.0 / beta, V)) != PD_OK) return rc;   // V_0 = r / beta
        std::fill(init.begin(), init.end(), 0.0);
        init[L.g] = beta;
        init[L.sc + GM_TARGET] = target;
        PD_CUDA(cudaMemcpyAsync(c.dsc, init.data(), sizeof(double) * init.size(), cudaMemcpyHostToDevice, st));
        const int steps = std::min(m, maxit - stats->iters);
        int k = 0;
        bool done = false;
        for (int j0 = 0; j0 < steps && !done; j0 += GM_CHUNK) {
            const int j1 = std::min(steps, j0 + GM_CHUNK);
            cudaGraphExec_t ge = j1 == std::min(m, j0 + GM_CHUNK) ? chunk_graph(j0) : nullptr;
            if (ge) {
                PD_CUDA(cudaGraphLaunch(ge, st));
            } else {
                for (int j = j0; j < j1; ++j)
                    if ((rc = arnoldi(j, st)) != PD_OK) return rc;
            }
            PD_CUDA(cudaMemcpyAsync(back, c.dsc + L.sc, sizeof(back), cudaMemcpyDeviceToHost, st));
            PD_CUDA(cudaStreamSynchronize(st));
            done = back[GM_DONE] != 0.0;
            k = (int)back[GM_K];
        }
        stats->iters += (int)back[GM_ITERS];
        stats->res = back[GM_RES];
        // y = H(0:k, 0:k)^-1 g(0:k); x += V(:, 0:k) y
        if (k > 0) {
            k_gm_solve<<<1, 1, 0, st>>>(c.dsc, m);
            if (!pc) {
                k_lincomb<<<nbk, 256, 0, st>>>(x, 1.0, V, n, k, c.dsc + L.y, 1.0, n);
            } else {
                k_lincomb<<<nbk, 256, 0, st>>>(ty, 0.0, V, n, k, c.dsc + L.y, 1.0, n);
                if ((rc = op.precond(op.ctx, ty, zt, st)) != PD_OK) return rc;
                if ((rc = axpby(c, 1.0, zt, 1.0, x)) != PD_OK) return rc;
            }
            PD_CUDA(cudaGetLastError());
        }
    }
}

// ------------------------------------------------------------------------ CG

// CG's scalars live on the device, after the dot results in dsc[0..]: the host
// enqueues CG_CHUNK iterations at a time and reads back once per chunk, instead
// of waiting for p.Ap and r.r in every iteration. An iteration that finds the
// residual below the target sets DONE; the later iterations of the chunk then
// change neither x nor r (alpha = 0, p kept), so x is the iterate at which the
// host loop would have stopped.
// CG_BAD holds the offending p.Ap and CG_BADFLAG marks that one was met (a p.Ap
// of exactly 0 would not show in CG_BAD alone).
enum { CG_RZ = 8, CG_ALPHA, CG_BETA, CG_RR, CG_TARGET, CG_DONE, CG_ITERS, CG_BAD, CG_BADFLAG };
static_assert(CG_BADFLAG < (int)KRYLOV_DSC_MIN, "CG scalars exceed the device scalar block");
constexpr int CG_CHUNK = 32;

// after dsc[0] = p.Ap: alpha = (r.z) / (p.Ap), or a non-positive curvature flag
__device__ __forceinline__ void cg_alpha(double *s)
{
    if (s[CG_DONE] != 0.0) {
        s[CG_ALPHA] = 0.0;
        return;
    }
    const double pq = s[0];
    if (!(pq > 0.0)) {
        s[CG_BAD] = pq == pq ? pq : -1.0;     // the offending p.Ap (NaN reported as -1)
        s[CG_BADFLAG] = 1.0;
        s[CG_DONE] = 1.0;
        s[CG_ALPHA] = 0.0;
        return;
    }
    s[CG_ALPHA] = s[CG_RZ] / pq;
}

// after dsc[0] = r.r: count the iteration, test ||r|| <= target
__device__ __forceinline__ void cg_check(double *s)
{
    if (s[CG_DONE] != 0.0) return;
    const double rr1 = s[0];
    s[CG_ITERS] += 1.0;
    s[CG_RR] = rr1;
    if (sqrt(rr1) <= s[CG_TARGET]) s[CG_DONE] = 1.0;
}

// beta = (r.z)_new / (r.z)_old with (r.z)_new in dsc[0] (PCG) or r.r (CG)
__device__ __forceinline__ void cg_beta(double *s, int precond)
{
    if (s[CG_DONE] != 0.0) return;
    const double rz1 = precond ? s[0] : s[CG_RR];
    s[CG_BETA] = rz1 / s[CG_RZ];
    s[CG_RZ] = rz1;
}

// dsc[0] = the dot product from k_mdot's nb block partials (k_partial_sum's fixed
// order), then the scalar step `what` of the iteration: CG_STEP_ALPHA; CG_STEP_CHECK
// (and, without a preconditioner, beta, which needs only r.r); CG_STEP_BETA (PCG,
// after r.z). One block of KT threads; the scalars run on thread 0.
enum { CG_STEP_ALPHA = 0, CG_STEP_CHECK, CG_STEP_BETA };
__global__ void __launch_bounds__(KT) k_cg_sum_step(const double *partial, int nb, double *s, int what,
                                                  int precond)
{
    __shared__ double red[KT / 32];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += KT) acc += partial[b];
    const double t = block_sum(acc, red);
    if (threadIdx.x != 0) return;
    s[0] = t;
    if (what == CG_STEP_ALPHA) {
        cg_alpha(s);
    } else if (what == CG_STEP_CHECK) {
        cg_check(s);
        if (!precond) cg_beta(s, 0);
    } else {
        cg_beta(s, 1);
    }
}

// x += alpha p and r -= alpha q, alpha from the device
__global__ void k_cg_update(const double *s, const double *p, double *x, const double *q, double *r, long long n)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double alpha = s[CG_ALPHA];
    x[e] = (1.0 * alpha) * p[e] + 1.0 * x[e];
    r[e] = (-1.0 * alpha) * q[e] + 1.0 * r[e];
}

__global__ void k_cg_p(const double *s, const double *z, double *p, long long n)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n || s[CG_DONE] != 0.0) return;
    const double beta = s[CG_BETA];
    p[e] = 1.0 * z[e] + (beta == 0.0 ? 0.0 : beta * p[e]);
}

// Conjugate gradients for symmetric positive definite A: x = 0 start, stop when
// ||b - A x|| <= rtol ||b|| (recursive residual) or after maxit iterations. With
// a symmetric positive definite preconditioner M it is PCG (p from z = M^-1 r).
int krylov_cg(const KrylovOp &op, const double *b, double *x, long long n, int maxit, double rtol, KrylovWork &wk,
              KrylovStats *stats, cudaStream_t st)
{
    KrylovCtx c{n, st, wk.partial, wk.dsc, {}};
    double *r = wk.basis, *p = wk.basis + n, *q = wk.basis + 2 * n;
    double *z = op.precond ? wk.aux : r;       // without M, z is r itself
    const unsigned nbk = (unsigned)((n + 255) / 256);
    PD_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    PD_CUDA(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    int rc = PD_OK;
    if (op.precond && (rc = op.precond(op.ctx, r, z, st)) != PD_OK) return rc;
    PD_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    double rr = 0.0, rz = 0.0;
    if ((rc = dots(c, r, 0, 1, r, &rr)) != PD_OK) return rc;
    rz = rr;
    if (op.precond && (rc = dots(c, r, 0, 1, z, &rz)) != PD_OK) return rc;
    stats->res0 = sqrt(rr);
    stats->res = stats->res0;
    stats->iters = 0;
    stats->converged = rr == 0.0;
    if (stats->converged) return PD_OK;
    double init[CG_BADFLAG + 1] = {0.0};
    init[CG_RZ] = rz;
    init[CG_RR] = rr;
    init[CG_TARGET] = rtol * stats->res0;
    PD_CUDA(cudaMemcpyAsync(c.dsc, init, sizeof(init), cudaMemcpyHostToDevice, st));
    // one iteration, enqueued on stream s (no host synchronisation)
    auto iteration = [&](cudaStream_t s) -> int {
        KrylovCtx cs{n, s, wk.partial, wk.dsc, {}};
        const int nb = kblocks(n), pre = op.precond ? 1 : 0;
        int e = op.apply(op.ctx, p, q, s);
        if (e != PD_OK) return e;
        k_mdot<<<dim3(nb, 1), KT, 0, s>>>(p, 0, q, n, cs.partial);
        k_cg_sum_step<<<1, KT, 0, s>>>(cs.partial, nb, cs.dsc, CG_STEP_ALPHA, pre);
        k_cg_update<<<nbk, 256, 0, s>>>(cs.dsc, p, x, q, r, n);
        k_mdot<<<dim3(nb, 1), KT, 0, s>>>(r, 0, r, n, cs.partial);
        k_cg_sum_step<<<1, KT, 0, s>>>(cs.partial, nb, cs.dsc, CG_STEP_CHECK, pre);
        if (op.precond) {
            if ((e = op.precond(op.ctx, r, z, s)) != PD_OK) return e;
            k_mdot<<<dim3(nb, 1), KT, 0, s>>>(r, 0, z, n, cs.partial);
            k_cg_sum_step<<<1, KT, 0, s>>>(cs.partial, nb, cs.dsc, CG_STEP_BETA, pre);
        }
        k_cg_p<<<nbk, 256, 0, s>>>(cs.dsc, z, p, n);
        PD_CUDA(cudaGetLastError());
        return PD_OK;
    };
    // a full chunk as one CUDA graph (its launch gaps, not its kernels, dominate at
    // small n); if the capture does not succeed the chunks are launched one by one
    cudaGraphExec_t exec = nullptr;
    if (wk.cap && maxit >= CG_CHUNK) {
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(wk.cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            int crc = PD_OK;
            for (int k = 0; k < CG_CHUNK && crc == PD_OK; ++k) crc = iteration(wk.cap);
            const cudaError_t e = cudaStreamEndCapture(wk.cap, &graph);
            if (crc != PD_OK || e != cudaSuccess || !graph || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
                exec = nullptr;
            if (graph) cudaGraphDestroy(graph);
        }
        cudaGetLastError();
    }
    int launched = 0;
    double back[CG_BADFLAG + 1];
    while (launched < maxit) {
        const int chunk = std::min(CG_CHUNK, maxit - launched);
        if (exec && chunk == CG_CHUNK) {
            const cudaError_t e = cudaGraphLaunch(exec, st);
            if (e != cudaSuccess) {
                cudaGraphExecDestroy(exec);
                return cuda_fail(e, "cudaGraphLaunch (CG chunk)");
            }
        } else {
            for (int k = 0; k < chunk; ++k)
                if ((rc = iteration(st)) != PD_OK) {
                    if (exec) cudaGraphExecDestroy(exec);
                    return rc;
                }
        }
        launched += chunk;
        cudaError_t e = cudaMemcpyAsync(back, c.dsc, sizeof(back), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            if (exec) cudaGraphExecDestroy(exec);
            return cuda_fail(e, "CG scalars");
        }
        stats->iters = (int)back[CG_ITERS];
        stats->res = sqrt(back[CG_RR]);
        if (back[CG_BADFLAG] != 0.0) {
            if (exec) cudaGraphExecDestroy(exec);
            set_error("CG: the operator is not positive definite (p.Ap = %g)", back[CG_BAD]);
            return PD_EINVAL;
        }
        if (back[CG_DONE] != 0.0) {
            stats->converged = 1;
            break;
        }
    }
    if (exec) cudaGraphExecDestroy(exec);
    return PD_OK;
}

size_t krylov_partial_doubles(long long n, int kmax) { return (size_t)kblocks(n) * (kmax + 1); }

int krylov_norm(const double *x, long long n, KrylovWork &wk, double *out, cudaStream_t st)
{
    KrylovCtx c{n, st, wk.partial, wk.dsc, {}};
    return norm2(c, x, out);
}

}  // namespace pdk
