// pd_krylov.cu -- Krylov solvers of the matrix-free Newton step that replaces the
// assembled-stiffness Newton iteration of Sec. 5 (Eq. (6), Algorithm 3): the
// tangent is applied by the JVP kernel (pd_jvp.cu), never assembled.
//
// Vectors are FP64, component-major over slots: v[c * nslots + s], c < dim;
// slots without a point hold 0 and every operation keeps them 0. All sums are
// deterministic: a fixed block partition, a fixed in-block tree, and a fixed
// final tree over the block partials. GMRES's few scalars per iteration (the
// Hessenberg column, the Givens rotations) are FP64 host arithmetic on values
// read back from the device; CG keeps alpha and beta on the device.
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

// partial[i * nb + b] = sum over block b of V_i . w, for i < k (V_i = V + i * ldv).
__global__ void __launch_bounds__(KT) k_mdot(const double *V, long long ldv, int k, const double *w, long long n,
                                             double *partial)
{
    __shared__ double red[KT / 32];
    const long long base = (long long)blockIdx.x * KCHUNK + threadIdx.x;
    double wq[KPER];
#pragma unroll
    for (int q = 0; q < KPER; ++q) {
        const long long e = base + (long long)q * KT;
        wq[q] = e < n ? w[e] : 0.0;
    }
    for (int i = 0; i < k; ++i) {
        const double *vi = V + (long long)i * ldv;
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < KPER; ++q) {
            const long long e = base + (long long)q * KT;
            if (e < n) acc = fma(vi[e], wq[q], acc);
        }
        const double t = block_sum(acc, red);
        if (threadIdx.x == 0) partial[(long long)i * gridDim.x + blockIdx.x] = t;
    }
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
    k_mdot<<<nb, KT, 0, c.st>>>(V, ldv, k, w, c.n, c.partial);
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

static int lincomb_host(KrylovCtx &c, double *y, double alpha, const double *V, long long ldv, int k,
                        const double *coef)
{
    PD_CUDA(cudaMemcpyAsync(c.dsc, coef, sizeof(double) * k, cudaMemcpyHostToDevice, c.st));
    return lincomb_dev(c, y, alpha, V, ldv, k, 1.0);
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

// Restarted GMRES with classical Gram-Schmidt applied twice (CGS2) and Givens
// rotations: solve A x = b from x = 0 until ||b - A x|| <= rtol ||b||. With a
// preconditioner M it is right-preconditioned (Arnoldi on A M^-1, x += M^-1 V y),
// so the residual it monitors is the one of A x = b.
int krylov_gmres(const KrylovOp &op, const double *b, double *x, long long n, int restart, int maxit, double rtol,
                 KrylovWork &wk, KrylovStats *stats, cudaStream_t st)
{
    KrylovCtx c{n, st, wk.partial, wk.dsc, {}};
    const int m = restart;
    double *V = wk.basis;                    // (m + 1) vectors of n
    double *w = wk.tmp;
    double *zt = wk.aux, *ty = wk.aux + n;   // M^-1 v_j; V y before M^-1
    const bool pc = op.precond != nullptr;
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
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), hcol(m + 2);
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
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < m && stats->iters < maxit; ++j) {
            double *vj1 = V + (long long)(j + 1) * n;
            const double *src = V + (long long)j * n;
            if (pc) {
                if ((rc = op.precond(op.ctx, src, zt, st)) != PD_OK) return rc;
                src = zt;
            }
            if ((rc = op.apply(op.ctx, src, vj1, st)) != PD_OK) return rc;
            // CGS2: h = V^T w, w -= V h; twice
            if ((rc = dots(c, V, n, j + 1, vj1, nullptr)) != PD_OK) return rc;
            if ((rc = lincomb_dev(c, vj1, 1.0, V, n, j + 1, -1.0)) != PD_OK) return rc;
            PD_CUDA(cudaMemcpyAsync(hcol.data(), c.dsc, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, st));
            if ((rc = dots(c, V, n, j + 1, vj1, nullptr)) != PD_OK) return rc;
            if ((rc = lincomb_dev(c, vj1, 1.0, V, n, j + 1, -1.0)) != PD_OK) return rc;
            std::vector<double> h2(j + 1);
            PD_CUDA(cudaMemcpyAsync(h2.data(), c.dsc, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, st));
            double hn = 0.0;
            if ((rc = norm2(c, vj1, &hn)) != PD_OK) return rc;     // synchronises the stream
            for (int i = 0; i <= j; ++i) H[i + (size_t)(m + 1) * j] = hcol[i] + h2[i];
            H[j + 1 + (size_t)(m + 1) * j] = hn;
            if (hn > 0.0 && (rc = axpby(c, 0.0, vj1, 1.0 / hn, vj1)) != PD_OK) return rc;
            // apply the previous rotations to column j, then a new one
            double *hj = &H[(size_t)(m + 1) * j];
            for (int i = 0; i < j; ++i) {
                const double t = cs[i] * hj[i] + sn[i] * hj[i + 1];
                hj[i + 1] = -sn[i] * hj[i] + cs[i] * hj[i + 1];
                hj[i] = t;
            }
            const double den = hypot(hj[j], hj[j + 1]);
            cs[j] = den > 0.0 ? hj[j] / den : 1.0;
            sn[j] = den > 0.0 ? hj[j + 1] / den : 0.0;
            hj[j] = den;
            hj[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++stats->iters;
            k = j + 1;
            stats->res = fabs(g[j + 1]);
            if (stats->res <= target || hn == 0.0) break;
        }
        // y = H(0:k, 0:k)^-1 g(0:k); x += V(:, 0:k) y
        for (int i = k - 1; i >= 0; --i) {
            double t = g[i];
            for (int l = i + 1; l < k; ++l) t -= H[i + (size_t)(m + 1) * l] * y[l];
            const double d = H[i + (size_t)(m + 1) * i];
            y[i] = d != 0.0 ? t / d : 0.0;
        }
        if (k > 0 && !pc && (rc = lincomb_host(c, x, 1.0, V, n, k, y.data())) != PD_OK) return rc;
        if (k > 0 && pc) {
            // x += M^-1 (V y)
            if ((rc = lincomb_host(c, ty, 0.0, V, n, k, y.data())) != PD_OK) return rc;
            if ((rc = op.precond(op.ctx, ty, zt, st)) != PD_OK) return rc;
            if ((rc = axpby(c, 1.0, zt, 1.0, x)) != PD_OK) return rc;
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
enum { CG_RZ = 8, CG_ALPHA, CG_BETA, CG_RR, CG_TARGET, CG_DONE, CG_ITERS, CG_BAD };
static_assert(CG_BAD < (int)KRYLOV_DSC_MIN, "CG scalars exceed the device scalar block");
constexpr int CG_CHUNK = 32;

// after dsc[0] = p.Ap: alpha = (r.z) / (p.Ap), or a non-positive curvature flag
__global__ void k_cg_alpha(double *s)
{
    if (s[CG_DONE] != 0.0) {
        s[CG_ALPHA] = 0.0;
        return;
    }
    const double pq = s[0];
    if (!(pq > 0.0)) {
        s[CG_BAD] = pq == pq ? pq : -1.0;     // the offending p.Ap (NaN reported as -1)
        s[CG_DONE] = 1.0;
        s[CG_ALPHA] = 0.0;
        return;
    }
    s[CG_ALPHA] = s[CG_RZ] / pq;
}

// y = (sign alpha) x + y, alpha from the device
__global__ void k_cg_axpy(const double *s, double sign, const double *x, double *y, long long n)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    y[e] = (sign * s[CG_ALPHA]) * x[e] + 1.0 * y[e];
}

// after dsc[0] = r.r: count the iteration, test ||r|| <= target
__global__ void k_cg_check(double *s)
{
    if (s[CG_DONE] != 0.0) return;
    const double rr1 = s[0];
    s[CG_ITERS] += 1.0;
    s[CG_RR] = rr1;
    if (sqrt(rr1) <= s[CG_TARGET]) s[CG_DONE] = 1.0;
}

// beta = (r.z)_new / (r.z)_old with (r.z)_new in dsc[0] (PCG) or r.r (CG)
__global__ void k_cg_beta(double *s, int precond)
{
    if (s[CG_DONE] != 0.0) return;
    const double rz1 = precond ? s[0] : s[CG_RR];
    s[CG_BETA] = rz1 / s[CG_RZ];
    s[CG_RZ] = rz1;
}

// p = z + beta p, unless done
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
    double init[CG_BAD + 1] = {0.0};
    init[CG_RZ] = rz;
    init[CG_RR] = rr;
    init[CG_TARGET] = rtol * stats->res0;
    PD_CUDA(cudaMemcpyAsync(c.dsc, init, sizeof(init), cudaMemcpyHostToDevice, st));
    // one iteration, enqueued on stream s (no host synchronisation)
    auto iteration = [&](cudaStream_t s) -> int {
        KrylovCtx cs{n, s, wk.partial, wk.dsc, {}};
        int e = op.apply(op.ctx, p, q, s);
        if (e == PD_OK) e = dots(cs, p, 0, 1, q, nullptr);
        if (e != PD_OK) return e;
        k_cg_alpha<<<1, 1, 0, s>>>(cs.dsc);
        k_cg_axpy<<<nbk, 256, 0, s>>>(cs.dsc, 1.0, p, x, n);
        k_cg_axpy<<<nbk, 256, 0, s>>>(cs.dsc, -1.0, q, r, n);
        if ((e = dots(cs, r, 0, 1, r, nullptr)) != PD_OK) return e;
        k_cg_check<<<1, 1, 0, s>>>(cs.dsc);
        if (op.precond) {
            if ((e = op.precond(op.ctx, r, z, s)) != PD_OK) return e;
            if ((e = dots(cs, r, 0, 1, z, nullptr)) != PD_OK) return e;
        }
        k_cg_beta<<<1, 1, 0, s>>>(cs.dsc, op.precond ? 1 : 0);
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
    double back[CG_BAD + 1];
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
        if (back[CG_BAD] != 0.0) {
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
