/*
 * pd.h -- C ABI of libpd, the GB300 (sm_103a) peridynamics hot path.
 *
 * The library evaluates the nonlocal internal force of peridynamics on a uniform
 * lattice (the EMU nodal discretization of Sec. 3.1 of Diehl et al., "An
 * asynchronous and task-based implementation of peridynamics utilizing HPX"):
 *   - the bond-based prototype micro-elastic brittle (PMB) model with bond
 *     breaking at a critical stretch (Eq. (3), Algorithm 1's loop structure);
 *   - the state-based linear peridynamic solid (LPS): a dilatation pass, then a
 *     force pass (Eq. (4), Algorithm 2);
 *   - the explicit central-difference / velocity-Verlet update (Eqs. (7)-(10),
 *     Algorithm 4);
 *   - the tangent Jacobian-vector product and its adjoint, the matrix-free
 *     form of the stiffness of Eq. (6) / Algorithm 3.
 *
 * Conventions for every call:
 *   - Return value: PD_OK (0) or a negative PD_E* code; pd_last_error() gives
 *     the message of the last failure on the calling thread. On failure no
 *     output is written unless the call says otherwise, and the simulation keeps
 *     its previous state.
 *   - Points are in user order at this boundary: i = x + nx*(y + ny*z), reference
 *     position X_i = origin + h*(x, y, z). Vectors are AoS (npoints, dim) FP64.
 *     The library keeps its own (Morton, tile-major) order internally.
 *   - Every array argument may be a host pointer or a device pointer of the
 *     current device (the library copies with cudaMemcpyDefault). Host arrays
 *     are read or written before the call returns only for calls marked
 *     "synchronous"; for the others a host array must stay valid until the
 *     stream has reached the call (as with cudaMemcpyAsync).
 *   - Caller-owned arrays are borrowed for the duration of the call; the library
 *     owns every buffer it allocates and frees them in pd_destroy(). Library
 *     buffers come from one stream-ordered memory pool per device that keeps
 *     released memory for reuse (allocation never synchronises the device).
 *   - stream: a cudaStream_t passed as void*; NULL selects the simulation's own
 *     stream. Work is ordered on that stream.
 *   - A pd_sim is not thread-safe: calls on one simulation must not overlap.
 */
#ifndef PD_H
#define PD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define PD_OK 0
#define PD_EINVAL (-1)     /* bad argument or unsupported configuration */
#define PD_ENOMEM (-2)     /* device or host allocation failed */
#define PD_ECUDA (-3)      /* a CUDA runtime call failed */
#define PD_ETIMEOUT (-4)   /* a bounded wait ran out */
#define PD_EBUSY (-5)      /* the resource is in use */
#define PD_ENOTREADY (-6)  /* result not available yet */
#define PD_ESTATE (-7)     /* call out of order (e.g. force before neighbours) */

/* ------------------------------------------------------------------- constants */
#define PD_MODEL_PMB 0     /* bond-based prototype micro-elastic brittle */
#define PD_MODEL_LPS 1     /* state-based linear peridynamic solid (3D only) */
#define PD_MODEL_NP 2      /* bond-based nonlinear law of Algorithm 1 (linearised bond
                              strain, potential psi(r) = C (1 - exp(-beta r))) */
#define PD_MODEL_LP 3      /* its linearisation: psi'(0) = C beta in place of psi' */

#define PD_FP32C 0         /* FP32 bond arithmetic on per-tile reference-frame
                              displacements; integrator state per pd_run.state */
#define PD_FP64 1          /* all-FP64 bond arithmetic and state */

/* Integrator state of a PD_FP32C simulation (pd_run.state). */
#define PD_STATE_F64 0     /* u and v in FP64: the velocity kicks and the drift are
                              FP64 additions / FMAs; the kernels stage u as an FP32
                              hi + lo pair (~47 bits) split from the FP64 value */
#define PD_STATE_DF 1      /* u and v as double-float numbers (FP32 hi + lo, ~48
                              bits) updated in FP32 arithmetic (two-sum, Dekker
                              product): no FP64 instruction on the step path */

#define PD_BC_FREE 0
#define PD_BC_VELOCITY 1       /* prescribed velocity on this DOF */
#define PD_BC_DISPLACEMENT 2   /* prescribed displacement, velocity held at 0 */

#define PD_FORCE_UPDATE_BREAKING 1u   /* pd_force: break bonds with s > s_c */

#define PD_JVP_MASK_DIRICHLET 1u      /* pd_jvp/pd_vjp: identity on prescribed-
                                         displacement DOFs, zero coupling to them */

/* ---------------------------------------------------------------- descriptions */

/* Uniform lattice: npoints = n[0]*n[1]*n[2] (n[2] = 1 in 2D), spacing h,
 * horizon delta = m*h. B_delta(X_i) = { X_j : j != i, |X_j - X_i| <= delta }
 * (Sec. 3.1), decided on integer offsets: a^2 + b^2 + c^2 <= m^2. */
typedef struct {
    int32_t dim;        /* 2 or 3 */
    int32_t n[3];       /* points per axis, each >= 1 */
    int32_t m;          /* horizon factor, 1 <= m <= 24 */
    int32_t reserved;   /* must be 0 */
    double h;           /* lattice spacing (m), > 0 */
    double origin[3];
} pd_grid;

/* Material. PMB micromodulus (the paper does not give it; literature values):
 * 3D c = 18 K'/(pi delta^4) with K' = E/(3(1-2nu)), nu = 1/4; 2D plane stress
 * c = 9E/(pi t delta^3) with nodal volume h^2 t. LPS uses K and mu
 * (Algorithm 2) and is 3D only. Influence function omega = 1. NP / LP
 * (Algorithm 1; Sec. 5.2.2): S = eta . xi / |xi|^2, f_i = 4 / (delta |B_delta|)
 * sum_j J psi'(|xi| S^2) S xi/|xi| V_j with |B_delta| the ball measure (pi
 * delta^2 in 2D, 4 pi delta^3 / 3 in 3D), J = 1 for |xi| < delta and 0 on the
 * horizon boundary; no bond breaking (s_c must be 0). */
typedef struct {
    int32_t model;      /* PD_MODEL_PMB, PD_MODEL_LPS, PD_MODEL_NP or PD_MODEL_LP */
    int32_t vol_corr;   /* 1: partial volume V_ij = (delta + h/2 - |xi|)/h for
                           |xi| > delta - h/2 (Remark of Sec. 3.1), else 1 */
    double E;           /* Young's modulus (PMB), Pa */
    double rho;         /* mass density, kg/m^3, > 0 */
    double K;           /* bulk modulus (LPS), Pa */
    double mu;          /* shear modulus (LPS), Pa */
    double s_c;         /* critical stretch (PMB); 0 disables breaking */
    double thickness;   /* 2D plate thickness t (m); ignored in 3D */
    double psi_c;       /* NP / LP potential scale C, > 0 for those models */
    double psi_beta;    /* NP / LP potential rate beta, > 0 for those models */
} pd_material;

/* Explicit integrators (Sec. 4.2.4 and its flow chart). Both give the same
 * trajectory in exact arithmetic; they round differently.
 * VERLET: v^{k+1/2} = v^k + dt/2 a^k, u^{k+1} = u^k + dt v^{k+1/2},
 *         v^{k+1} = v^{k+1/2} + dt/2 a^{k+1}          (Eqs. (7)-(9))
 * CD:     u^{k+1} = 2 u^k - u^{k-1} + dt^2 a^k          (Eq. (10))
 * with a = (f + b) / rho. CD starts, and restarts after pd_set_state,
 * pd_set_dt, pd_solve_static or pd_build_neighbors, with one velocity-Verlet
 * step (the Taylor start u^1 = u^0 + dt v^0 + dt^2/2 a^0). Under CD the library
 * still advances v by the two half-kicks, so pd_get_state and pd_energy report
 * the same velocity as under VERLET; a prescribed velocity advances u by dt
 * times its value and a prescribed displacement sets u, as under VERLET. */
#define PD_INTEGRATOR_VERLET 0
#define PD_INTEGRATOR_CD     1

/* Run parameters. */
typedef struct {
    double dt;          /* time step; 0 selects dt_factor * dt_crit with the
                           Silling-Askari bound dt_crit = min_i sqrt(2 rho /
                           sum_j c V_j V_ij / |xi_ij|) (PMB c of the same E for LPS) */
    double dt_factor;   /* used when dt == 0; 0 means 0.5 */
    int32_t precision;  /* PD_FP32C or PD_FP64 */
    int32_t tile_log2;  /* points per tile = 2^tile_log2 (a Morton brick);
                           0 selects 9, or less when the halo box of a large
                           horizon would not fit in shared memory; 6..9 */
    int32_t integrator; /* PD_INTEGRATOR_VERLET (0) or PD_INTEGRATOR_CD */
    int32_t state;      /* PD_FP32C: PD_STATE_F64 (0) or PD_STATE_DF; must be 0
                           for PD_FP64 */
    int32_t pair_threads; /* PD_FP32C PMB: threads that share a point pair's
                           stencil words (1, 2 or 4, at most the stencil's
                           32-bond words; their partial sums are added in a fixed
                           order); 0 lets the library choose (the most resident
                           threads per SM) */
    int32_t reserved;   /* must be 0 */
} pd_run;

typedef struct pd_sim pd_sim;

/* ------------------------------------------------------------------- lifecycle */

/* Validate the descriptions and allocate the simulation's device buffers on the
 * current device. *out receives an opaque handle owned by the caller until
 * pd_destroy(). Initial state: u = v = 0, all DOFs free, no body force.
 * Errors: PD_EINVAL (bad description, LPS in 2D, LPS with s_c > 0),
 * PD_ENOMEM, PD_ECUDA. Synchronous. */
int pd_create(pd_sim **out, const pd_grid *grid, const pd_material *mat, const pd_run *run);

/* Free every buffer, graph and stream of the simulation. NULL is accepted.
 * Waits for the simulation's own stream; work that uses the simulation on a
 * stream the caller passed must have completed (the buffers return, ordered on
 * the simulation's stream, to the library's device memory pool, which keeps
 * them for reuse instead of synchronising the device). */
int pd_destroy(pd_sim *sim);

/* Copy the message of the last failure on this thread into buf (NUL-terminated,
 * truncated to len). Returns the length of the full message. */
int pd_last_error(char *buf, size_t len);

/* ------------------------------------------------------------------ neighbours */

/* Build B_delta(X_i) for every point (Sec. 3.1; computed and stored once in the
 * reference configuration, Sec. 4.2.1) on the device: a cell list with cell edge
 * m h, a Morton permutation of the points, and a CSR bond list in Morton
 * numbering with each row ascending. The CSR is then encoded as one stencil
 * bit per (point, lattice offset) -- the bond-intact mask the force kernels
 * read -- and, for LPS, the weighted volume m_i = sum_j |xi|^2 V_j V_ij of
 * Algorithm 2's first loop. Also fixes dt when pd_run.dt was 0.
 * Synchronous. Errors: PD_ENOMEM, PD_ECUDA. Calling it again rebuilds and
 * resets every bond to intact. */
int pd_build_neighbors(pd_sim *sim, void *stream);

/* Number of directed bonds (CSR entries). Errors: PD_ESTATE before the build. */
int pd_bond_count(const pd_sim *sim, int64_t *nbonds);

/* Copy the CSR in Morton numbering: row_ptr[npoints+1] (int64), col[nbonds]
 * (int32, Morton ranks, rows ascending) and perm[npoints] (int64, perm[rank] =
 * user index). Any of the three may be NULL. Synchronous. */
int pd_get_neighbors(pd_sim *sim, int64_t *row_ptr, int32_t *col, int64_t *perm, void *stream);

/* One byte per CSR entry of pd_get_neighbors (1 = broken, 0 = intact).
 * Synchronous. */
int pd_get_broken(pd_sim *sim, uint8_t *broken, void *stream);

/* Pre-notch: every bond whose segment crosses the planar rectangle
 * { x[axis] = pos, lo[b] <= x[b] <= hi[b] for the other axes b } (lattice units,
 * multiples of h from the origin) is marked broken. *nbroken (may be NULL)
 * receives the number of directed bonds marked by this call. Synchronous. */
int pd_break_bonds(pd_sim *sim, int axis, double pos, const double lo[3], const double hi[3],
                   int64_t *nbroken, void *stream);

/* -------------------------------------------------------------------- state */

/* Set displacement u and/or velocity v (npoints x dim, FP64, user order) at the
 * current time; a NULL pointer leaves that field unchanged (a kept v that the
 * last step left at a half step is first completed, as in pd_get_state).
 * Initial conditions u0, v0 of Eqs. (1)-(2). Stream-ordered. */
int pd_set_state(pd_sim *sim, const double *u, const double *v, void *stream);

/* Read u and/or v (npoints x dim, FP64, user order) at the current integer time
 * step; a NULL pointer skips that field. If v is requested and the last step
 * left the velocity at a half step, this evaluates the force at the current u
 * to complete it (Eq. (9)); the trajectory is unchanged. Synchronous. */
int pd_get_state(pd_sim *sim, double *u, double *v, void *stream);

/* Pipelined forms for host arrays (device arrays behave as in pd_set_state and
 * pd_get_state, stream-ordered). pd_set_state_async copies the host arrays
 * without first waiting for the work already queued on `stream` (only for the
 * library's staging buffer), so the upload of the next state can run while the
 * current step computes: the caller guarantees that the arrays hold their values
 * when the call is made and keeps them unchanged until pd_io_sync returns.
 * pd_get_state_async queues the read on `stream` and the copies to the caller's
 * arrays, and returns at once: the arrays hold the result after pd_io_sync has
 * returned; until then the caller neither reads nor writes them nor passes them
 * to pd_set_state(_async) (a later pd_get_state_async into the same arrays is
 * ordered after this one). Uploads and
 * downloads use separate staging buffers and copy streams, so one step's
 * download, the next step's upload and the compute between them overlap. */
int pd_set_state_async(pd_sim *sim, const double *u, const double *v, void *stream);
int pd_get_state_async(pd_sim *sim, double *u, double *v, void *stream);
/* Block until every host-array copy of pd_set_state(_async) and
 * pd_get_state(_async) issued so far has completed. */
int pd_io_sync(pd_sim *sim);

/* Boundary conditions on a collar Omega_c (Sec. 3; Sec. 5.2.2): kind and value
 * per DOF (npoints x dim; uint8 PD_BC_*, FP64). PD_BC_VELOCITY holds v = value
 * and advances u by dt*value; PD_BC_DISPLACEMENT holds u = value, v = 0.
 * kind == NULL frees every DOF. Stream-ordered. */
int pd_set_bc(pd_sim *sim, const uint8_t *kind, const double *value, void *stream);

/* External force density b (npoints x dim, FP64, user order) of Eq. (3);
 * NULL removes it. Stream-ordered. */
int pd_set_body_force(pd_sim *sim, const double *b, void *stream);

int pd_get_dt(const pd_sim *sim, double *dt);
/* Set dt (> 0). Stream-ordered with respect to later steps. */
int pd_set_dt(pd_sim *sim, double dt);
/* Number of explicit steps taken so far. */
int pd_get_step(const pd_sim *sim, int64_t *step);

/* --------------------------------------------------------------------- force */

/* One internal-force evaluation f_i = sum_{j in B(i)} f(eta, xi) V_j V_ij
 * (PMB, Eq. (3)) or sum_j (T_i<xi> - T_j<-xi>) V_j V_ij (LPS, Eq. (4), after the
 * dilatation pass of Algorithm 2) at displacement u (npoints x dim FP64, user
 * order) or, if u == NULL, at the current state. f_out: npoints x dim FP64,
 * user order, force per unit volume (N/m^3). With PD_FORCE_UPDATE_BREAKING a
 * bond whose stretch exceeds s_c breaks for good before it contributes.
 * Stream-ordered. */
int pd_force(pd_sim *sim, const double *u, double *f_out, unsigned flags, void *stream);

/* LPS dilatation theta_i = (3/m_i) sum_j |xi| e V_j V_ij (Algorithm 2, second
 * loop) at u (or the current state if NULL), npoints FP64, user order.
 * PD_EINVAL for PMB. Stream-ordered. */
int pd_dilatation(pd_sim *sim, const double *u, double *theta_out, void *stream);

/* ------------------------------------------------------------------ explicit */

/* Advance nsteps >= 0 explicit steps, velocity-Verlet form of the central
 * difference scheme (Eqs. (7)-(10), Algorithm 4): kick with f^k, drift,
 * boundary conditions, force at the new u (bonds break here), kick. One fused
 * force + update kernel per step (two for LPS), replayed as CUDA graphs.
 * Stream-ordered. */
int pd_step_explicit(pd_sim *sim, int64_t nsteps, void *stream);

/* The same steps as pd_step_explicit, for measurement: launched one kernel at
 * a time (no graph) with a CUDA event on `stream` before and after each
 * launch, the host waiting for every step. pass_ms[0] receives the summed
 * device time of the first launch of each step (PMB, NP, LP: the fused force +
 * update kernel; LPS: the dilatation pass), pass_ms[1] that of the LPS force +
 * update pass (0 for the bond-based laws). The trajectory is the one
 * pd_step_explicit gives. Synchronous. Errors: PD_EINVAL for nsteps < 0 or a
 * null pass_ms. */
int pd_step_explicit_timed(pd_sim *sim, int64_t nsteps, double pass_ms[2], void *stream);

/* Measured tile choice. For each tile size 2^9, 2^8, 2^7, 2^6 that the
 * description admits (the halo box of each kernel fits in shared memory),
 * create the simulation with run->tile_log2 set to it, build its neighbours,
 * take two untimed explicit steps from rest (u = v = 0, every DOF free, no
 * breaking reached), then time `steps` more three times with CUDA events on
 * `stream` (0 = each simulation's own stream) and keep the best; *tile_log2
 * receives the fastest, a smaller tile
 * only when it is at least 1 % faster than the best larger one. The trial
 * simulations are destroyed before return. The tile size changes the
 * per-tile reference of the FP32C staging, so results at different tiles agree
 * to the FP32C tolerance, not bit for bit. grid, mat, run: as for pd_create
 * (run->tile_log2 is ignored); steps >= 1. Errors: PD_EINVAL for a null
 * pointer or steps < 1, else the error of the last tile tried when none could
 * be built. Synchronous. */
int pd_tune_tile(const pd_grid *grid, const pd_material *mat, const pd_run *run, int32_t steps,
                 int32_t *tile_log2, void *stream);

/* Measured tile and threads-per-pair choice: as pd_tune_tile, over every
 * admissible tile size and, for the FP32C PMB kernel, every pd_run.pair_threads
 * of 1, 2 and 4 up to the stencil's 32-bond words (a larger count, like a
 * smaller tile, only when at least 1 % faster). *pair_threads receives the
 * choice (0 where the kernel has no such choice: other models and
 * precisions); pair_threads == NULL measures tiles only (pd_tune_tile).
 * Synchronous. */
int pd_tune(const pd_grid *grid, const pd_material *mat, const pd_run *run, int32_t steps, int32_t *tile_log2,
            int32_t *pair_threads, void *stream);

/* ------------------------------------------------------------------- tangent */

/* Tangent Jacobian-vector product out = K w with K = df/du at u_lin (npoints x
 * dim FP64, user order; NULL = current state), the matrix-free form of Eq. (6)
 * and Algorithm 3 for the PMB model:
 *   (K w)_i = sum_j D_ij (w_j - w_i) V_j V_ij,
 *   D_ij = c [ n n^T / |xi| + s (I - n n^T) / |xi + eta| ],  n = (xi+eta)/|xi+eta|,
 * over intact bonds. K is symmetric; -K is positive semi-definite near the
 * reference configuration. With PD_JVP_MASK_DIRICHLET, prescribed-displacement
 * DOFs give out = w and do not couple to the others. PD_EINVAL for LPS.
 * Stream-ordered. */
int pd_jvp(pd_sim *sim, const double *u_lin, const double *w, double *out,
           unsigned flags, void *stream);

/* Adjoint (vector-Jacobian) product out = K^T v, computed by its own kernel in
 * the transposed gather form (K^T v)_i = sum_j D_ij (V_i v_j - V_j v_i) V_ij.
 * Same arguments and errors as pd_jvp. */
int pd_vjp(pd_sim *sim, const double *u_lin, const double *v, double *out,
           unsigned flags, void *stream);

/* ------------------------------------------------------------------ implicit */

/* Static equilibrium by matrix-free Newton-Krylov: the implicit scheme of Sec. 5
 * (Newton on the residual, Eq. (6)) with the stiffness applied by the JVP kernel
 * instead of being assembled by central differences (Algorithm 3). */

#define PD_KRYLOV_GMRES 0    /* restarted GMRES(restart), CGS2 orthogonalisation */
#define PD_KRYLOV_CG 1       /* conjugate gradients (the operator is SPD) */

#define PD_TANGENT_CACHED 0  /* D_ij of every bond evaluated once per Newton iteration
                                and kept (3 or 6 values per bond in the simulation's
                                precision plus the neighbour index); each product
                                streams it */
#define PD_TANGENT_JVP 1     /* the JVP kernel of pd_jvp for every product (no cache) */

#define PD_PRECOND_NONE 0
#define PD_PRECOND_BLOCK_JACOBI 1   /* M = the d x d diagonal blocks sum_j D_ij of A (from
                                       the cached tangent; CG becomes PCG, GMRES is
                                       right-preconditioned) */

typedef struct {
    int32_t krylov;           /* PD_KRYLOV_GMRES or PD_KRYLOV_CG */
    int32_t restart;          /* GMRES restart length, 1..500 (50) */
    int32_t max_linear_iters; /* per linear solve, >= 1 */
    int32_t max_newton_iters; /* >= 1 */
    int32_t tangent;          /* PD_TANGENT_CACHED or PD_TANGENT_JVP */
    int32_t precond;          /* PD_PRECOND_NONE or PD_PRECOND_BLOCK_JACOBI (cached tangent) */
    double linear_rtol;       /* each solve: ||r - A du|| <= linear_rtol ||r|| */
    double newton_rtol;       /* stop when ||r|| <= newton_rtol ||r_0|| + newton_atol */
    double newton_atol;       /* N/m^3 */
} pd_newton_opts;

typedef struct {
    int32_t newton_iters;     /* linear solves done */
    int32_t linear_iters;     /* Krylov iterations, summed over the solves */
    int32_t converged;        /* 1 if the Newton test was met */
    int32_t linear_failures;  /* solves that stopped at max_linear_iters */
    double res0;              /* ||r_0||: residual at the start, after the BCs (N/m^3) */
    double res;               /* ||r|| at the last iterate */
} pd_newton_stats;

/* Solve f(u) + b = 0 (Eq. (3) with the inertia term dropped) for u on every DOF
 * without PD_BC_DISPLACEMENT; those DOFs are set to their prescribed values
 * first and stay there. r = f(u) + b on the free DOFs (0 on prescribed ones),
 * ||.|| the Euclidean norm over free DOFs. Newton from the current u: solve
 * A du = r, A = -K on free DOFs and the identity on prescribed ones (K = df/du
 * of pd_jvp, so A is symmetric and positive definite once the prescribed DOFs
 * remove the rigid modes), then u += du. The JVP is FP64 for PD_FP64 and FP32
 * for PD_FP32C simulations (inexact Newton; the residual is FP64 in both). Bonds
 * do not break during the solve. On return u is the last iterate and v = 0.
 * PMB only (PD_EINVAL for LPS). opts == NULL takes the defaults in brackets and
 * GMRES, 20000 linear iterations, 20 Newton iterations, the cached tangent, no
 * preconditioner, linear_rtol 1e-8, newton_rtol 1e-8, newton_atol 0. Returns PD_OK whether or not the test was met
 * (see stats->converged; stats may be NULL); PD_EINVAL if CG meets a
 * non-positive curvature. Work buffers are allocated on the first call and
 * kept until pd_destroy. Synchronous. */
int pd_solve_static(pd_sim *sim, const pd_newton_opts *opts, pd_newton_stats *stats, void *stream);

/* ------------------------------------------------------------------- serving */

/* A request server: independent simulations submitted at any time, run
 * concurrently on one GPU and collected through tickets (the futures of the
 * paper's task model, Sec. 2, applied to whole simulations). A worker thread of
 * the library admits queued requests in submission order while their device
 * memory (bond list, bond mask and per-point state, estimated before creation)
 * fits the budget and fewer than max_active run; each admitted request gets its
 * own simulation and advances in quanta of up to quantum_steps explicit steps,
 * and a finished request frees its memory for the next in the queue between
 * quanta (continuous batching).
 *
 * PD_SERVE_PACKED (default): FP32C PMB requests without breaking and FP32C LPS
 * requests without partial volume and of horizon m <= 3 (on 2^9-point tiles,
 * with the pair_threads the server sets: 2 where the stencil has two or more
 * 32-bond words, else 1; up to pack_max_tiles tiles when that is set) are
 * stepped together by one packed kernel: per explicit step one launch of a
 * persistent grid whose CTAs take (request, pass, tile) work items of every
 * such request from a device-side list (the LPS force items after the
 * dilatation items they need, with a bounded wait on completion flags), the
 * steps of a quantum replayed from a captured CUDA graph. Other requests run
 * on their own streams, as every request does under PD_SERVE_STREAMS.
 *
 * A request's result does not depend on what else runs: it equals the same
 * simulation run alone with the tile_log2 and pair_threads reported in
 * pd_result. */

typedef struct pd_server pd_server;

#define PD_SERVE_PACKED 0
#define PD_SERVE_STREAMS 1

typedef struct {
    int64_t device_bytes;     /* admission budget; 0 = half the free device memory */
    int32_t max_active;       /* simulations stepping at once, 1..256 (16) */
    int32_t quantum_steps;    /* steps per scheduling quantum, 1..4096 (64) */
    int32_t mode;             /* PD_SERVE_PACKED (0) or PD_SERVE_STREAMS */
    int32_t wait_limit_ms;    /* limit of one device-side wait of the packed kernel;
                                 0 = 2000 ms. A wait that runs out ends the quantum's
                                 launch, and every request of that quantum fails
                                 with PD_ETIMEOUT */
    int32_t test_stall;       /* tests only, else 0: in the server's first packed
                                 quantum the first LPS force item waits for a flag
                                 that nothing sets, so that its wait runs out */
    int32_t pack_max_tiles;   /* PD_SERVE_PACKED: a request of more than this many
                                 512-point tiles runs on its own stream with the
                                 simulation's own kernels, the smaller ones are
                                 packed; 0 = no limit (every eligible request is
                                 packed), >= 0 */
    int32_t max_queued;       /* back-pressure: while this many requests wait for
                                 admission, pd_submit refuses the next with PD_EBUSY
                                 (admitted and running requests do not count);
                                 0 = no limit, >= 0 */
    int32_t reserved;         /* must be 0 */
} pd_server_opts;

typedef struct {
    pd_grid grid;
    pd_material material;
    pd_run run;               /* run.tile_log2 = 0 lets the server choose */
    int64_t nsteps;           /* explicit steps, >= 0 */
    const double *u0, *v0;    /* host, npoints x dim, user order; NULL = 0; copied by pd_submit */
    const uint8_t *bc_kind;   /* host, npoints x dim, or NULL (no collar); copied */
    const double *bc_val;     /* host, with bc_kind; copied */
    double *u_out, *v_out;    /* host, npoints x dim, caller-owned; written when the
                                 request completes (NULL = not wanted); must stay
                                 valid until the ticket is done or cancelled */
} pd_request;

#define PD_REQ_QUEUED 0
#define PD_REQ_RUNNING 1
#define PD_REQ_DONE 2
#define PD_REQ_CANCELLED 3
#define PD_REQ_FAILED 4

typedef struct {
    int32_t state;            /* PD_REQ_* */
    int32_t error;            /* PD_OK, or the status that failed the request */
    int32_t tile_log2;        /* tile size the request runs with (0 before admission) */
    int32_t pair_threads;     /* pd_run.pair_threads it runs with (0: the library's choice) */
    int64_t steps_done;
    int64_t bonds;            /* directed bonds (0 before admission) */
    double submit_s, start_s, end_s;   /* server clock (s since pd_server_create); 0 if not yet */
    char message[160];        /* error text of a failed request */
} pd_result;

/* Start a server on the current device (its worker thread uses that device). */
int pd_server_create(pd_server **out, const pd_server_opts *opts);
/* Cancel what is queued or running (running requests stop after their current
 * quantum), join the worker, free everything. */
int pd_server_destroy(pd_server *srv);
/* Validate and copy a request and queue it; *ticket identifies it (> 0).
 * PD_EINVAL for an invalid description or one whose memory estimate exceeds the
 * budget on its own; PD_EBUSY (nothing queued) while max_queued requests wait. */
int pd_submit(pd_server *srv, const pd_request *req, uint64_t *ticket);
/* Current state of a ticket, without blocking. PD_EINVAL for an unknown ticket. */
int pd_poll(pd_server *srv, uint64_t ticket, pd_result *out);
/* Block until the ticket is done, cancelled or failed, at most timeout_s
 * seconds: PD_OK, or PD_ETIMEOUT with out holding the current state. */
int pd_wait(pd_server *srv, uint64_t ticket, double timeout_s, pd_result *out);
/* Cancel a queued or running request (a running one stops after its current
 * quantum; its outputs are not written). PD_OK also if it had already ended. */
int pd_cancel(pd_server *srv, uint64_t ticket);

/* -------------------------------------------------------------------- energy */

/* Kinetic energy sum_i rho |v_i|^2 V_i / 2 and strain energy sum_i V_i W_i
 * (PMB: W_i = 1/2 sum_j c s^2 |xi| / 2 V_j V_ij; LPS: W_i = K theta_i^2 / 2 +
 * 15 mu / (2 m_i) sum_j (e^d)^2 V_j V_ij) at the current integer step, reduced
 * in FP64 in a fixed order (bit-reproducible). Either pointer may be NULL.
 * Synchronous. */
int pd_energy(pd_sim *sim, double *kinetic, double *strain, void *stream);

/* ------------------------------------------------------------ no allocation */

/* Largest n pd_sum_noalloc accepts: its scratch holds 1024 partial sums of
 * 4096 values each. */
#define PD_SUM_NOALLOC_MAX_VALUES 4194304

/* out[0] = scale * (x[0] + ... + x[n-1]) in FP64, summed in the same fixed
 * order as the reductions of pd_energy, by the same two kernels, but with the
 * partial sums in a static device array of the library instead of a buffer
 * allocated by pd_create. The paper has no counterpart: this entry point is for
 * callers that may not allocate device memory at all, e.g. a host framework
 * that owns every device allocation through its own pool or budget, or a loop
 * where the implicit synchronisation of cudaMalloc/cudaFree is not allowed.
 * It calls no cudaMalloc, cudaFree or other allocating routine.
 *   x, out: device pointers of the current device (x may be NULL if n == 0).
 *   n: 0 <= n <= PD_SUM_NOALLOC_MAX_VALUES, else PD_EINVAL with a message.
 *   stream: cudaStream_t or NULL for the legacy default stream; stream-ordered.
 * The first call on a device looks up the device address of the static array
 * (cudaGetSymbolAddress) and keeps it for the rest of the process; make that
 * first call before any stream capture. The kept address belongs to the
 * device's current context: after cudaDeviceReset on that device, do not call
 * this entry point again in the same process. The
 * array (8 KiB per device, held until the process exits) is shared by every
 * call: each call overwrites every partial it reads, so nothing needs
 * clearing, but calls that overlap on the GPU (different streams, no ordering)
 * race on it and may return wrong sums. */
int pd_sum_noalloc(const double *x, int64_t n, double scale, double *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PD_H */
