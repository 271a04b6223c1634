/*
 * pd_oracle.c -- plain FP64 CPU oracle of the peridynamic hot path.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load this library. The CUDA library never calls it, and the
 * two share no code, header, table or helper.
 *
 * What it computes, each function citing the passage it follows
 * (Diehl, Jha, Kaiser, Lipton, Levesque, "An asynchronous and task-based
 * implementation of peridynamics utilizing HPX"):
 *   - discrete neighbourhoods B_delta(X_i)              Sec. 3.1
 *   - bond-based force (PMB law, breaking)              Eq. (3), Algorithm 1
 *   - bond-based NP law and its linearisation LP        Algorithm 1, Sec. 5.2.2
 *   - state-based LPS: weighted volume, dilatation,
 *     force (gather form and Algorithm 2's scatter)     Eq. (4), Algorithm 2
 *   - velocity-Verlet and central-difference updates    Eqs. (7)-(10), Algorithm 4
 *   - tangent stiffness by central differences          Eq. (6), Algorithm 3
 *   - strain and kinetic energy, stable time step       (literature, see below)
 *
 * Conventions restated here (not shared with the CUDA library's headers):
 *   - points in user order, i = x + nx*(y + ny*z), X_i = origin + h*(x, y, z);
 *   - vectors are AoS (n, dim) FP64;
 *   - neighbour lists are CSR in user numbering, each row ascending;
 *   - bond state is one byte per CSR entry (1 = broken).
 *
 * Every force loop is an outer loop over points i and an inner sequential loop
 * over j in B_delta(X_i) in ascending j, as in Algorithms 1 and 2. The outer
 * loop runs under OpenMP (the paper's parallel for_loop), writes only row i's
 * data, and is therefore deterministic for any thread count.
 *
 * Readings of the paper (where it is silent or garbled):
 *   - the neighbour predicate |X_j - X_i| <= delta is decided on integer
 *     lattice offsets, a^2 + b^2 + c^2 <= m^2 (points at exactly delta are in);
 *   - PMB micromodulus (not given in the paper): 3D c = 18 K' / (pi delta^4)
 *     with K' = E / (3 (1 - 2 nu)), nu = 1/4; 2D plane stress
 *     c = 9 E / (pi t delta^3) with nodal volume h^2 t;
 *   - PMB stretch s = (|xi + eta| - |xi|) / |xi|, force c s (xi+eta)/|xi+eta|;
 *     a bond breaks for good when s > s_c (s_c > 0), tested before its
 *     contribution is added;
 *   - influence function omega = J = 1;
 *   - PMB strain energy: pair potential w = c s^2 |xi| / 2 per unit volume^2,
 *     W = 1/2 sum_i V_i sum_j w V_j; LPS strain energy (Silling 2007):
 *     W_i = K theta_i^2 / 2 + 15 mu / (2 m_i) sum_j (e^d)^2 V_j;
 *   - stable step bound (Silling-Askari 2005):
 *     dt_crit = min_i sqrt(2 rho / sum_j c V_j / |xi_ij|);
 *   - optional partial volume V_ij = (delta + h/2 - |xi|) / h for
 *     |xi| > delta - h/2, else 1;
 *   - NP / LP (Algorithm 1 and the 2D study of Sec. 5.2.2): bond strain
 *     S = (eta . xi) / |xi|^2, direction xi/|xi| (reference configuration),
 *     psi(r) = C (1 - exp(-beta r)), LP uses psi'(0) = C beta in place of
 *     psi'(|xi| S^2) and psi(r) = C beta r; influence function J = 1 for
 *     |xi| < delta and 0 otherwise (on integer offsets a^2 + b^2 + c^2 < m^2);
 *     |B_delta(0)| is the ball measure pi delta^2 (2D) or 4 pi delta^3 / 3
 *     (3D); stable-step bound with the bond stiffness 4 C beta / (delta |B|)
 *     in place of the PMB micromodulus.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t dim;      /* 2 or 3 */
    int32_t nx, ny, nz;
    int32_t m;        /* horizon factor, delta = m h */
    int32_t pad_;
    double h;
    double ox, oy, oz;
} or_grid;

typedef struct {
    int32_t model;    /* 0 PMB, 1 LPS, 2 NP, 3 LP */
    int32_t vol_corr; /* partial-volume correction on/off */
    double E, rho, K, mu, s_c, thickness;
    double psi_c, psi_beta;   /* NP / LP potential psi(r) = C (1 - exp(-beta r)) */
} or_material;

enum { OR_PMB = 0, OR_LPS = 1, OR_NP = 2, OR_LP = 3 };
enum { OR_BC_FREE = 0, OR_BC_VELOCITY = 1, OR_BC_DISPLACEMENT = 2 };

static const double OR_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------ lattice */

static int64_t npoints(const or_grid *g) { return (int64_t)g->nx * g->ny * g->nz; }

static void lattice_coord(const or_grid *g, int64_t i, int64_t c[3])
{
    c[0] = i % g->nx;
    c[1] = (i / g->nx) % g->ny;
    c[2] = i / ((int64_t)g->nx * g->ny);
}

static void position(const or_grid *g, int64_t i, double X[3])
{
    int64_t c[3];
    lattice_coord(g, i, c);
    X[0] = g->ox + g->h * (double)c[0];
    X[1] = g->oy + g->h * (double)c[1];
    X[2] = g->dim == 3 ? g->oz + g->h * (double)c[2] : 0.0;
}

static double horizon(const or_grid *g) { return g->m * g->h; }

/* Nodal volume V_i (Sec. 3.1): h^3 in 3D, h^2 t for a plate of thickness t. */
static double nodal_volume(const or_grid *g, const or_material *mat)
{
    return g->dim == 3 ? g->h * g->h * g->h : g->h * g->h * mat->thickness;
}

/* Partial-volume factor V_ij (Remark in Sec. 3.1; linear reading). */
static double volume_factor(const or_grid *g, const or_material *mat, double xi_len)
{
    double delta = horizon(g);
    if (!mat->vol_corr) return 1.0;
    if (xi_len > delta - 0.5 * g->h) return (delta + 0.5 * g->h - xi_len) / g->h;
    return 1.0;
}

/* PMB micromodulus (literature calibration; the paper does not give it). */
double or_pmb_micromodulus(const or_grid *g, const or_material *mat)
{
    double delta = horizon(g);
    if (g->dim == 3) {
        double nu = 0.25;
        double Kb = mat->E / (3.0 * (1.0 - 2.0 * nu));
        return 18.0 * Kb / (OR_PI * pow(delta, 4));
    }
    return 9.0 * mat->E / (OR_PI * mat->thickness * pow(delta, 3));
}

/* |B_delta(0)|: the measure of the horizon ball. */
static double ball_measure(const or_grid *g)
{
    double delta = horizon(g);
    return g->dim == 3 ? 4.0 * OR_PI * delta * delta * delta / 3.0 : OR_PI * delta * delta;
}

/* Bond stiffness of the NP / LP laws at zero strain, 4 C beta / (delta |B|):
 * their force is this times S xi/|xi| V_j for small S. */
static double np_stiffness(const or_grid *g, const or_material *mat)
{
    return 4.0 * mat->psi_c * mat->psi_beta / (horizon(g) * ball_measure(g));
}

/* Young's modulus implied by K and mu (used for the LPS stable-step bound). */
static double lps_young(const or_material *mat)
{
    return 9.0 * mat->K * mat->mu / (3.0 * mat->K + mat->mu);
}

static int in_horizon(const or_grid *g, int64_t i, int64_t j)
{
    int64_t a[3], b[3];
    lattice_coord(g, i, a);
    lattice_coord(g, j, b);
    int64_t d0 = b[0] - a[0], d1 = b[1] - a[1], d2 = b[2] - a[2];
    return d0 * d0 + d1 * d1 + d2 * d2 <= (int64_t)g->m * g->m;
}

/* ----------------------------------------------------------- neighbourhoods */

/* B_delta(X_i) = { X_j : j != i, |X_j - X_i| <= delta } (Sec. 3.1), by testing
 * every pair. With col == NULL only row_ptr is filled; returns the bond count. */
int64_t or_neighbors_brute(const or_grid *g, int64_t *row_ptr, int32_t *col)
{
    int64_t n = npoints(g);
    if (col == NULL) {
        #pragma omp parallel for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            int64_t cnt = 0;
            for (int64_t j = 0; j < n; ++j)
                if (j != i && in_horizon(g, i, j)) ++cnt;
            row_ptr[i + 1] = cnt;
        }
        row_ptr[0] = 0;
        for (int64_t i = 0; i < n; ++i) row_ptr[i + 1] += row_ptr[i];
        return row_ptr[n];
    }
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = row_ptr[i];
        for (int64_t j = 0; j < n; ++j)
            if (j != i && in_horizon(g, i, j)) col[k++] = (int32_t)j;
    }
    return row_ptr[n];
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* The same sets through a cell list with cell edge m lattice spacings (>= delta):
 * only the 3^d cells around X_i hold candidates. Rows are sorted ascending. */
int64_t or_neighbors_cells(const or_grid *g, int64_t *row_ptr, int32_t *col)
{
    int64_t n = npoints(g);
    int m = g->m;
    int64_t cx = (g->nx + m - 1) / m, cy = (g->ny + m - 1) / m, cz = (g->nz + m - 1) / m;
    int64_t ncell = cx * cy * cz;
    int64_t *cstart = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    int64_t *cfill = (int64_t *)calloc((size_t)ncell, sizeof(int64_t));
    int64_t *cpts = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!cstart || !cfill || !cpts) { free(cstart); free(cfill); free(cpts); return -1; }
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3];
        lattice_coord(g, i, c);
        int64_t cell = c[0] / m + cx * (c[1] / m + cy * (c[2] / m));
        cstart[cell + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3];
        lattice_coord(g, i, c);
        int64_t cell = c[0] / m + cx * (c[1] / m + cy * (c[2] / m));
        cpts[cstart[cell] + cfill[cell]++] = i;
    }
    int pass_fill = col != NULL;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3];
        lattice_coord(g, i, c);
        int64_t ci = c[0] / m, cj = c[1] / m, ck = c[2] / m;
        int64_t cnt = 0, k0 = pass_fill ? row_ptr[i] : 0;
        for (int64_t dk = -1; dk <= 1; ++dk)
            for (int64_t dj = -1; dj <= 1; ++dj)
                for (int64_t di = -1; di <= 1; ++di) {
                    int64_t a = ci + di, b = cj + dj, e = ck + dk;
                    if (a < 0 || b < 0 || e < 0 || a >= cx || b >= cy || e >= cz) continue;
                    int64_t cell = a + cx * (b + cy * e);
                    for (int64_t p = cstart[cell]; p < cstart[cell + 1]; ++p) {
                        int64_t j = cpts[p];
                        if (j == i || !in_horizon(g, i, j)) continue;
                        if (pass_fill) col[k0 + cnt] = (int32_t)j;
                        ++cnt;
                    }
                }
        if (pass_fill)
            qsort(col + k0, (size_t)cnt, sizeof(int32_t), cmp_i32);
        else
            row_ptr[i + 1] = cnt;
    }
    if (!pass_fill) {
        row_ptr[0] = 0;
        for (int64_t i = 0; i < n; ++i) row_ptr[i + 1] += row_ptr[i];
    }
    free(cstart); free(cfill); free(cpts);
    return row_ptr[n];
}

/* Morton (Z-order) code: bit b of x, y, z goes to bit d*b, d*b+1, d*b+2. */
static uint64_t morton_code(const or_grid *g, int64_t i)
{
    int64_t c[3];
    lattice_coord(g, i, c);
    uint64_t code = 0;
    for (int b = 0; b < 21; ++b)
        for (int a = 0; a < g->dim; ++a)
            code |= (uint64_t)((c[a] >> b) & 1) << (g->dim * b + a);
    return code;
}

typedef struct { uint64_t code; int64_t idx; } code_idx;

static int cmp_code(const void *a, const void *b)
{
    const code_idx *x = (const code_idx *)a, *y = (const code_idx *)b;
    if (x->code != y->code) return x->code < y->code ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* perm[rank] = user index of the point with the rank-th smallest Morton code. */
int or_morton_perm(const or_grid *g, int64_t *perm)
{
    int64_t n = npoints(g);
    code_idx *t = (code_idx *)malloc((size_t)n * sizeof(code_idx));
    if (!t) return -1;
    for (int64_t i = 0; i < n; ++i) { t[i].code = morton_code(g, i); t[i].idx = i; }
    qsort(t, (size_t)n, sizeof(code_idx), cmp_code);
    for (int64_t r = 0; r < n; ++r) perm[r] = t[r].idx;
    free(t);
    return 0;
}

/* Pre-notch: bond (i, j) starts broken when its segment crosses the planar
 * rectangle {x[axis] = pos, lo[b] <= x[b] <= hi[b] for the other axes b},
 * all in lattice units. Returns the number of CSR entries marked. */
int64_t or_break_notch(const or_grid *g, const int64_t *row_ptr, const int32_t *col,
                       int axis, double pos, const double *lo, const double *hi,
                       uint8_t *broken)
{
    int64_t n = npoints(g), marked = 0;
    #pragma omp parallel for reduction(+:marked) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t ci[3];
        lattice_coord(g, i, ci);
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t cj[3];
            lattice_coord(g, col[k], cj);
            double di = (double)ci[axis] - pos, dj = (double)cj[axis] - pos;
            if (!(di * dj < 0.0)) continue;
            double t = (pos - (double)ci[axis]) / (double)(cj[axis] - ci[axis]);
            int inside = 1;
            for (int b = 0; b < g->dim; ++b) {
                if (b == axis) continue;
                double p = (double)ci[b] + t * (double)(cj[b] - ci[b]);
                if (p < lo[b] || p > hi[b]) inside = 0;
            }
            if (inside) { broken[k] = 1; ++marked; }
        }
    }
    return marked;
}

/* ------------------------------------------------------------ bond geometry */

static void bond_vectors(const or_grid *g, int64_t i, int64_t j, const double *u,
                         double xi[3], double eta[3])
{
    double Xi[3], Xj[3];
    position(g, i, Xi);
    position(g, j, Xj);
    int d = g->dim;
    for (int a = 0; a < 3; ++a) { xi[a] = 0.0; eta[a] = 0.0; }
    for (int a = 0; a < d; ++a) {
        xi[a] = Xj[a] - Xi[a];
        eta[a] = u[j * d + a] - u[i * d + a];
    }
}

static double norm3(const double v[3]) { return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

/* ---------------------------------------------------------------- PMB force */

/* Per-bond record of a run (diagnostics for the tests, no arithmetic of the
 * method): for every directed bond, the largest stretch it was evaluated at
 * while intact (including the evaluation that broke it) and the step at which
 * it broke (-1: never). */
typedef struct {
    double *s_max;       /* [nbonds], or NULL */
    int32_t *brk_step;   /* [nbonds], or NULL */
    int64_t step;        /* step number of the current force evaluation */
} or_track;

static void pmb_force_tracked(const or_grid *g, const or_material *mat,
                              const int64_t *row_ptr, const int32_t *col,
                              const double *u, uint8_t *broken, int update_breaking, double *f,
                              const or_track *tr);

/* Internal force density of the bond-based model, Eq. (3) with Algorithm 1's
 * loop structure and the PMB pair force f = c s (xi + eta)/|xi + eta|:
 *   f_i = sum_{j in B(i), intact} c s_ij M_ij V_j V_ij.
 * With update_breaking, a bond whose stretch exceeds s_c is marked broken in
 * this call before it would contribute. */
void or_pmb_force(const or_grid *g, const or_material *mat,
                  const int64_t *row_ptr, const int32_t *col,
                  const double *u, uint8_t *broken, int update_breaking, double *f)
{
    pmb_force_tracked(g, mat, row_ptr, col, u, broken, update_breaking, f, NULL);
}

/* Stretch s = (|xi + eta| - |xi|) / |xi| of every directed bond at u (the same
 * expression as the force), into s_out[nbonds]. */
void or_bond_stretch(const or_grid *g, const int64_t *row_ptr, const int32_t *col,
                     const double *u, double *s_out)
{
    int64_t n = npoints(g);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            double xi[3], eta[3], y[3];
            bond_vectors(g, i, col[k], u, xi, eta);
            for (int a = 0; a < 3; ++a) y[a] = xi[a] + eta[a];
            double r0 = norm3(xi), r = norm3(y);
            s_out[k] = (r - r0) / r0;
        }
    }
}

static void pmb_force_tracked(const or_grid *g, const or_material *mat,
                              const int64_t *row_ptr, const int32_t *col,
                              const double *u, uint8_t *broken, int update_breaking, double *f,
                              const or_track *tr)
{
    int64_t n = npoints(g);
    int d = g->dim;
    double c = or_pmb_micromodulus(g, mat), V = nodal_volume(g, mat);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double fi[3] = {0.0, 0.0, 0.0};
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            if (broken && broken[k]) continue;
            int64_t j = col[k];
            double xi[3], eta[3], y[3];
            bond_vectors(g, i, j, u, xi, eta);
            for (int a = 0; a < 3; ++a) y[a] = xi[a] + eta[a];
            double r0 = norm3(xi), r = norm3(y);
            double s = (r - r0) / r0;
            if (tr && tr->s_max && s > tr->s_max[k]) tr->s_max[k] = s;
            if (update_breaking && mat->s_c > 0.0 && s > mat->s_c) {
                broken[k] = 1;
                if (tr && tr->brk_step) tr->brk_step[k] = (int32_t)tr->step;
                continue;
            }
            double w = c * s * V * volume_factor(g, mat, r0) / r;
            for (int a = 0; a < 3; ++a) fi[a] += w * y[a];
        }
        for (int a = 0; a < d; ++a) f[i * d + a] = fi[a];
    }
}

/* ---------------------------------------------------------- NP / LP force */

/* J(|xi|) of the NP / LP laws: 1 inside the open horizon ball, 0 on its
 * boundary (Sec. 5.2.2), decided on the lattice offset of the bond. */
static double np_influence(const or_grid *g, int64_t i, int64_t j)
{
    int64_t ci[3], cj[3];
    lattice_coord(g, i, ci);
    lattice_coord(g, j, cj);
    int64_t a = cj[0] - ci[0], b = cj[1] - ci[1], c = cj[2] - ci[2];
    return a * a + b * b + c * c < (int64_t)g->m * g->m ? 1.0 : 0.0;
}

/* Algorithm 1: for every i, over j in B_delta(X_i) in ascending order,
 *   S = (u_j - u_i) . xi / |xi|^2,
 *   f_i += 4 / (delta |B_delta(0)|) J(|xi|) psi'(|xi| S^2) S xi/|xi| V_j (V_ij),
 * with psi'(r) = C beta exp(-beta r) (NP) or C beta (LP, linear). */
void or_np_force(const or_grid *g, const or_material *mat,
                 const int64_t *row_ptr, const int32_t *col, const uint8_t *broken,
                 const double *u, double *f)
{
    int64_t n = npoints(g);
    int d = g->dim;
    double k0 = 4.0 / (horizon(g) * ball_measure(g)), V = nodal_volume(g, mat);
    double C = mat->psi_c, beta = mat->psi_beta;
    int linear = mat->model == OR_LP;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double fi[3] = {0.0, 0.0, 0.0};
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            if (broken && broken[k]) continue;
            int64_t j = col[k];
            double xi[3], eta[3];
            bond_vectors(g, i, j, u, xi, eta);
            double r0 = norm3(xi);
            double S = (eta[0] * xi[0] + eta[1] * xi[1] + eta[2] * xi[2]) / (r0 * r0);
            double dpsi = linear ? C * beta : C * beta * exp(-beta * r0 * S * S);
            double w = k0 * np_influence(g, i, j) * dpsi * S * V * volume_factor(g, mat, r0) / r0;
            for (int a = 0; a < 3; ++a) fi[a] += w * xi[a];
        }
        for (int a = 0; a < d; ++a) f[i * d + a] = fi[a];
    }
}

/* ---------------------------------------------------------------- LPS model */

/* Algorithm 2, first loop: weighted volume m_i = sum_j |xi|^2 V_j (omega = 1),
 * over all bonds of the reference configuration. */
void or_lps_weighted_volume(const or_grid *g, const or_material *mat,
                            const int64_t *row_ptr, const int32_t *col, double *mvol)
{
    int64_t n = npoints(g);
    double V = nodal_volume(g, mat);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double Xi[3], Xj[3], mi = 0.0;
        position(g, i, Xi);
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            position(g, col[k], Xj);
            double xi[3] = {Xj[0] - Xi[0], Xj[1] - Xi[1], Xj[2] - Xi[2]};
            double r0 = norm3(xi);
            mi += r0 * r0 * V * volume_factor(g, mat, r0);
        }
        mvol[i] = mi;
    }
}

/* Algorithm 2, second loop: dilatation theta_i = sum_j (3/m_i) |xi| e V_j with
 * extension e = |xi + eta| - |xi|. Broken bonds are skipped. */
void or_lps_dilatation(const or_grid *g, const or_material *mat,
                       const int64_t *row_ptr, const int32_t *col, const uint8_t *broken,
                       const double *mvol, const double *u, double *theta)
{
    int64_t n = npoints(g);
    double V = nodal_volume(g, mat);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double th = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            if (broken && broken[k]) continue;
            double xi[3], eta[3], y[3];
            bond_vectors(g, i, col[k], u, xi, eta);
            for (int a = 0; a < 3; ++a) y[a] = xi[a] + eta[a];
            double r0 = norm3(xi), e = norm3(y) - r0;
            th += 3.0 / mvol[i] * r0 * e * V * volume_factor(g, mat, r0);
        }
        theta[i] = th;
    }
}

/* Scalar force state of Algorithm 2, third loop, for the owner p of the bond:
 *   t = (3 K theta_p / m_p) |xi| + (15 mu / m_p) e^d,  e^d = e - theta_p |xi| / 3. */
static double lps_scalar_state(const or_material *mat, double theta_p, double m_p,
                               double r0, double e)
{
    double ed = e - theta_p * r0 / 3.0;
    return 3.0 * mat->K * theta_p / m_p * r0 + 15.0 * mat->mu / m_p * ed;
}

/* Eq. (4) in gather form: f_i = sum_j (t_i<xi> + t_j<-xi>) M_ij V_j, where the
 * second term is what Algorithm 2's "f_j -= t M V_i" deposits on i from row j
 * (e is symmetric and M_ji = -M_ij). Equal to the scatter form below. */
void or_lps_force(const or_grid *g, const or_material *mat,
                  const int64_t *row_ptr, const int32_t *col, const uint8_t *broken,
                  const double *mvol, const double *theta, const double *u, double *f)
{
    int64_t n = npoints(g);
    int d = g->dim;
    double V = nodal_volume(g, mat);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double fi[3] = {0.0, 0.0, 0.0};
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            if (broken && broken[k]) continue;
            int64_t j = col[k];
            double xi[3], eta[3], y[3];
            bond_vectors(g, i, j, u, xi, eta);
            for (int a = 0; a < 3; ++a) y[a] = xi[a] + eta[a];
            double r0 = norm3(xi), r = norm3(y), e = r - r0;
            double t = lps_scalar_state(mat, theta[i], mvol[i], r0, e)
                     + lps_scalar_state(mat, theta[j], mvol[j], r0, e);
            double w = t * V * volume_factor(g, mat, r0) / r;
            for (int a = 0; a < 3; ++a) fi[a] += w * y[a];
        }
        for (int a = 0; a < d; ++a) f[i * d + a] = fi[a];
    }
}

/* Algorithm 2's third loop as printed: f_i += t M V_j; f_j -= t M V_i.
 * Serial, because the scatter writes other points' entries. Cross-check only. */
void or_lps_force_scatter(const or_grid *g, const or_material *mat,
                          const int64_t *row_ptr, const int32_t *col, const uint8_t *broken,
                          const double *mvol, const double *theta, const double *u, double *f)
{
    int64_t n = npoints(g);
    int d = g->dim;
    double V = nodal_volume(g, mat);
    memset(f, 0, (size_t)n * d * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            if (broken && broken[k]) continue;
            int64_t j = col[k];
            double xi[3], eta[3], y[3];
            bond_vectors(g, i, j, u, xi, eta);
            for (int a = 0; a < 3; ++a) y[a] = xi[a] + eta[a];
            double r0 = norm3(xi), r = norm3(y), e = r - r0;
            double t = lps_scalar_state(mat, theta[i], mvol[i], r0, e);
            double vf = volume_factor(g, mat, r0);
            for (int a = 0; a < d; ++a) {
                double M = y[a] / r;
                f[i * d + a] += t * M * V * vf;
                f[j * d + a] -= t * M * V * vf;
            }
        }
    }
}

/* ------------------------------------------------------------ model dispatch */

static void internal_force_tracked(const or_grid *g, const or_material *mat,
                                   const int64_t *row_ptr, const int32_t *col, uint8_t *broken,
                                   int update_breaking, const double *mvol, double *theta,
                                   const double *u, double *f, const or_track *tr)
{
    if (mat->model == OR_PMB) {
        pmb_force_tracked(g, mat, row_ptr, col, u, broken, update_breaking, f, tr);
    } else if (mat->model == OR_NP || mat->model == OR_LP) {
        or_np_force(g, mat, row_ptr, col, broken, u, f);
    } else {
        or_lps_dilatation(g, mat, row_ptr, col, broken, mvol, u, theta);
        or_lps_force(g, mat, row_ptr, col, broken, mvol, theta, u, f);
    }
}

static void internal_force(const or_grid *g, const or_material *mat,
                           const int64_t *row_ptr, const int32_t *col, uint8_t *broken,
                           int update_breaking, const double *mvol, double *theta,
                           const double *u, double *f)
{
    internal_force_tracked(g, mat, row_ptr, col, broken, update_breaking, mvol, theta, u, f, NULL);
}

/* Internal force of either model at u (no breaking update). theta may be NULL
 * for PMB; for LPS it receives the dilatation. */
void or_internal_force(const or_grid *g, const or_material *mat,
                       const int64_t *row_ptr, const int32_t *col, const uint8_t *broken,
                       const double *mvol, double *theta, const double *u, double *f)
{
    internal_force(g, mat, row_ptr, col, (uint8_t *)broken, 0, mvol, theta, u, f);
}

/* ------------------------------------------------------------------ energy */

/* Strain energy sum_i V_i W_i (readings above); W per point into W_point if given. */
double or_strain_energy(const or_grid *g, const or_material *mat,
                        const int64_t *row_ptr, const int32_t *col, const uint8_t *broken,
                        const double *mvol, const double *theta, const double *u,
                        double *W_point)
{
    int64_t n = npoints(g);
    double V = nodal_volume(g, mat), total = 0.0;
    double c = mat->model == OR_PMB ? or_pmb_micromodulus(g, mat) : 0.0;
    #pragma omp parallel for reduction(+:total) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double Wi = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            if (broken && broken[k]) continue;
            double xi[3], eta[3], y[3];
            bond_vectors(g, i, col[k], u, xi, eta);
            for (int a = 0; a < 3; ++a) y[a] = xi[a] + eta[a];
            double r0 = norm3(xi), r = norm3(y), vf = volume_factor(g, mat, r0);
            if (mat->model == OR_PMB) {
                double s = (r - r0) / r0;
                Wi += 0.5 * (0.5 * c * s * s * r0) * V * vf;
            } else if (mat->model == OR_NP || mat->model == OR_LP) {
                /* Algorithm 1: U_i += J psi(|xi| S^2) V_j / (delta |B_delta(0)|) */
                double S = (eta[0] * xi[0] + eta[1] * xi[1] + eta[2] * xi[2]) / (r0 * r0);
                double arg = r0 * S * S;
                double psi = mat->model == OR_LP ? mat->psi_c * mat->psi_beta * arg
                                                 : mat->psi_c * (1.0 - exp(-mat->psi_beta * arg));
                Wi += np_influence(g, i, col[k]) * psi * V * vf / (horizon(g) * ball_measure(g));
            } else {
                double ed = (r - r0) - theta[i] * r0 / 3.0;
                Wi += 15.0 * mat->mu / (2.0 * mvol[i]) * ed * ed * V * vf;
            }
        }
        if (mat->model == OR_LPS) Wi += 0.5 * mat->K * theta[i] * theta[i];
        if (W_point) W_point[i] = Wi;
        total += V * Wi;
    }
    return total;
}

double or_kinetic_energy(const or_grid *g, const or_material *mat, const double *v)
{
    int64_t n = npoints(g);
    int d = g->dim;
    double V = nodal_volume(g, mat), total = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double v2 = 0.0;
        for (int a = 0; a < d; ++a) v2 += v[i * d + a] * v[i * d + a];
        total += 0.5 * mat->rho * v2 * V;
    }
    return total;
}

/* --------------------------------------------------------------- time step */

/* Stable step bound dt_crit = min_i sqrt(2 rho / sum_j c V_j V_ij / |xi_ij|).
 * For LPS the PMB micromodulus of the same Young's modulus is used; for NP / LP
 * the bond stiffness 4 C beta / (delta |B|). */
double or_stable_dt(const or_grid *g, const or_material *mat,
                    const int64_t *row_ptr, const int32_t *col)
{
    int64_t n = npoints(g);
    or_material pm = *mat;
    if (mat->model == OR_LPS) pm.E = lps_young(mat);
    double c = (mat->model == OR_NP || mat->model == OR_LP) ? np_stiffness(g, mat) : or_pmb_micromodulus(g, &pm);
    double V = nodal_volume(g, mat);
    double best = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        double Xi[3], Xj[3], sum = 0.0;
        position(g, i, Xi);
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            position(g, col[k], Xj);
            double xi[3] = {Xj[0] - Xi[0], Xj[1] - Xi[1], Xj[2] - Xi[2]};
            double r0 = norm3(xi);
            sum += c * V * volume_factor(g, mat, r0) / r0;
        }
        if (sum > 0.0) {
            double dt = sqrt(2.0 * mat->rho / sum);
            if (dt < best) best = dt;
        }
    }
    return best;
}

/* ---------------------------------------------------------- explicit steps */

static void apply_bc(int64_t n, int d, const uint8_t *bc_kind, const double *bc_val,
                     double *u_prev, double *u, double *v, double dt)
{
    if (!bc_kind) return;
    for (int64_t q = 0; q < n * d; ++q) {
        if (bc_kind[q] == OR_BC_VELOCITY) {
            v[q] = bc_val[q];
            u[q] = u_prev[q] + dt * bc_val[q];
        } else if (bc_kind[q] == OR_BC_DISPLACEMENT) {
            v[q] = 0.0;
            u[q] = bc_val[q];
        }
    }
}

static void hold_bc_velocity(int64_t n, int d, const uint8_t *bc_kind, const double *bc_val,
                             double *v)
{
    if (!bc_kind) return;
    for (int64_t q = 0; q < n * d; ++q) {
        if (bc_kind[q] == OR_BC_VELOCITY) v[q] = bc_val[q];
        else if (bc_kind[q] == OR_BC_DISPLACEMENT) v[q] = 0.0;
    }
}

/* Velocity-Verlet, Eqs. (7)-(9) and Algorithm 4 (with the 1/rho of the
 * equations; Algorithm 4 as printed drops it):
 *   v^{k+1/2} = v^k + dt/(2 rho) (b + f^k)
 *   u^{k+1}   = u^k + dt v^{k+1/2}
 *   boundary conditions at t^{k+1}
 *   f^{k+1}   = F(u^{k+1})   (bonds break here)
 *   v^{k+1}   = v^{k+1/2} + dt/(2 rho) (b + f^{k+1})
 * Prescribed-velocity DOFs hold v = value and advance u by dt*value;
 * prescribed-displacement DOFs hold u = value, v = 0. The force f^{k+1} of one
 * step is the f^k of the next. f (n*dim) holds f^0 on entry when f_valid != 0
 * and the last force on exit; theta (n) is work space for LPS. */
int or_run_verlet_tracked(const or_grid *g, const or_material *mat,
                          const int64_t *row_ptr, const int32_t *col, uint8_t *broken,
                          const double *mvol, double *u, double *v, const double *b,
                          const uint8_t *bc_kind, const double *bc_val,
                          double dt, int64_t nsteps, double *f, int f_valid, double *theta,
                          double *s_max, int32_t *brk_step, int64_t step0)
{
    int64_t n = npoints(g);
    int d = g->dim;
    or_track tr = {s_max, brk_step, step0};
    double *u_prev = (double *)malloc((size_t)n * d * sizeof(double));
    if (!u_prev) return -1;
    if (!f_valid)
        internal_force_tracked(g, mat, row_ptr, col, broken, 1, mvol, theta, u, f, &tr);
    double kick = 0.5 * dt / mat->rho;
    for (int64_t k = 0; k < nsteps; ++k) {
        tr.step = step0 + k + 1;
        memcpy(u_prev, u, (size_t)n * d * sizeof(double));
        for (int64_t q = 0; q < n * d; ++q) {
            v[q] = v[q] + kick * ((b ? b[q] : 0.0) + f[q]);
            u[q] = u[q] + dt * v[q];
        }
        apply_bc(n, d, bc_kind, bc_val, u_prev, u, v, dt);
        internal_force_tracked(g, mat, row_ptr, col, broken, 1, mvol, theta, u, f, &tr);
        for (int64_t q = 0; q < n * d; ++q)
            v[q] = v[q] + kick * ((b ? b[q] : 0.0) + f[q]);
        hold_bc_velocity(n, d, bc_kind, bc_val, v);
    }
    free(u_prev);
    return 0;
}

int or_run_verlet(const or_grid *g, const or_material *mat,
                  const int64_t *row_ptr, const int32_t *col, uint8_t *broken,
                  const double *mvol, double *u, double *v, const double *b,
                  const uint8_t *bc_kind, const double *bc_val,
                  double dt, int64_t nsteps, double *f, int f_valid, double *theta)
{
    return or_run_verlet_tracked(g, mat, row_ptr, col, broken, mvol, u, v, b, bc_kind, bc_val, dt, nsteps,
                                 f, f_valid, theta, NULL, NULL, 0);
}

/* Central difference, Eq. (10): u^{k+1} = 2u^k - u^{k-1} + dt^2/rho (b + f^k),
 * started with u^1 = u^0 + dt v^0 + dt^2/(2 rho)(b + f^0) (the Taylor start that
 * makes it the same trajectory as velocity-Verlet). Free boundary, no breaking.
 * On exit u holds u^nsteps. */
int or_run_central_difference(const or_grid *g, const or_material *mat,
                              const int64_t *row_ptr, const int32_t *col, const uint8_t *broken,
                              const double *mvol, double *u, const double *v0, const double *b,
                              double dt, int64_t nsteps, double *theta)
{
    int64_t n = npoints(g);
    int d = g->dim;
    size_t bytes = (size_t)n * d * sizeof(double);
    double *u_old = (double *)malloc(bytes), *f = (double *)malloc(bytes);
    if (!u_old || !f) { free(u_old); free(f); return -1; }
    if (nsteps <= 0) { free(u_old); free(f); return 0; }
    internal_force(g, mat, row_ptr, col, (uint8_t *)broken, 0, mvol, theta, u, f);
    memcpy(u_old, u, bytes);
    for (int64_t q = 0; q < n * d; ++q)
        u[q] = u_old[q] + dt * v0[q] + 0.5 * dt * dt / mat->rho * ((b ? b[q] : 0.0) + f[q]);
    for (int64_t k = 1; k < nsteps; ++k) {
        internal_force(g, mat, row_ptr, col, (uint8_t *)broken, 0, mvol, theta, u, f);
        for (int64_t q = 0; q < n * d; ++q) {
            double un = 2.0 * u[q] - u_old[q] + dt * dt / mat->rho * ((b ? b[q] : 0.0) + f[q]);
            u_old[q] = u[q];
            u[q] = un;
        }
    }
    free(u_old); free(f);
    return 0;
}

/* ------------------------------------------------------------------ tangent */

/* Tangent stiffness by central differences, Eq. (6) and Algorithm 3:
 *   K[:, r] = (f(u + eps e_r) - f(u - eps e_r)) / (2 eps)
 * for every displacement degree of freedom r, as a dense (n d) x (n d)
 * row-major matrix. No breaking update. For small grids only. */
int or_tangent_fd(const or_grid *g, const or_material *mat,
                  const int64_t *row_ptr, const int32_t *col, const uint8_t *broken,
                  const double *mvol, const double *u, double eps, double *K)
{
    int64_t n = npoints(g);
    int d = g->dim;
    int64_t N = n * d;
    size_t bytes = (size_t)N * sizeof(double);
    double *up = (double *)malloc(bytes), *fp = (double *)malloc(bytes);
    double *fm = (double *)malloc(bytes), *th = (double *)malloc((size_t)n * sizeof(double));
    if (!up || !fp || !fm || !th) { free(up); free(fp); free(fm); free(th); return -1; }
    memcpy(up, u, bytes);
    for (int64_t r = 0; r < N; ++r) {
        up[r] = u[r] + eps;
        internal_force(g, mat, row_ptr, col, (uint8_t *)broken, 0, mvol, th, up, fp);
        up[r] = u[r] - eps;
        internal_force(g, mat, row_ptr, col, (uint8_t *)broken, 0, mvol, th, up, fm);
        up[r] = u[r];
        for (int64_t s = 0; s < N; ++s) K[s * N + r] = (fp[s] - fm[s]) / (2.0 * eps);
    }
    free(up); free(fp); free(fm); free(th);
    return 0;
}

/* Directional central difference (f(u + eps w) - f(u - eps w)) / (2 eps). */
int or_jvp_fd(const or_grid *g, const or_material *mat,
              const int64_t *row_ptr, const int32_t *col, const uint8_t *broken,
              const double *mvol, const double *u, const double *w, double eps, double *out)
{
    int64_t n = npoints(g);
    int d = g->dim;
    int64_t N = n * d;
    size_t bytes = (size_t)N * sizeof(double);
    double *up = (double *)malloc(bytes), *fm = (double *)malloc(bytes);
    double *th = (double *)malloc((size_t)n * sizeof(double));
    if (!up || !fm || !th) { free(up); free(fm); free(th); return -1; }
    for (int64_t q = 0; q < N; ++q) up[q] = u[q] + eps * w[q];
    internal_force(g, mat, row_ptr, col, (uint8_t *)broken, 0, mvol, th, up, out);
    for (int64_t q = 0; q < N; ++q) up[q] = u[q] - eps * w[q];
    internal_force(g, mat, row_ptr, col, (uint8_t *)broken, 0, mvol, th, up, fm);
    for (int64_t q = 0; q < N; ++q) out[q] = (out[q] - fm[q]) / (2.0 * eps);
    free(up); free(fm); free(th);
    return 0;
}

/* ------------------------------------------------------------------- misc */

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
