/* abi_smoke.c -- a plain C client of libpd (include/pd.h), no Python: build the
 * neighbours of a 2D plate, run explicit steps from a Gaussian displacement
 * (computed here, or read from the file named by the second argument),
 * read the state and the energies back, and print them. The test suite compiles
 * and links it on any machine and runs it on a GPU, comparing the printout with
 * the same simulation driven through the Python binding. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "pd.h"

static int check(int rc, const char *what)
{
    if (rc != PD_OK) {
        char msg[256];
        pd_last_error(msg, sizeof(msg));
        fprintf(stderr, "%s failed (%d): %s\n", what, rc, msg);
        exit(1);
    }
    return rc;
}

int main(int argc, char **argv)
{
    const int nx = 24, ny = 17, steps = argc > 1 ? atoi(argv[1]) : 50;
    pd_grid g = {0};
    g.dim = 2;
    g.n[0] = nx;
    g.n[1] = ny;
    g.n[2] = 1;
    g.m = 3;
    g.h = 0.02;
    pd_material m = {0};
    m.model = PD_MODEL_PMB;
    m.E = 72e9;
    m.rho = 2440.0;
    m.thickness = 1.0;
    pd_run r = {0};
    r.precision = PD_FP64;
    pd_sim *s = NULL;
    check(pd_create(&s, &g, &m, &r), "pd_create");
    check(pd_build_neighbors(s, NULL), "pd_build_neighbors");
    int64_t nb = 0;
    check(pd_bond_count(s, &nb), "pd_bond_count");
    const size_t n = (size_t)nx * ny;
    double *u = calloc(2 * n, sizeof(double)), *v = calloc(2 * n, sizeof(double));
    if (!u || !v) return 1;
    if (argc > 2) {
        /* the initial displacement as raw FP64, n x 2, user order */
        FILE *f = fopen(argv[2], "rb");
        if (!f || fread(u, sizeof(double), 2 * n, f) != 2 * n) {
            fprintf(stderr, "cannot read %s\n", argv[2]);
            return 1;
        }
        fclose(f);
    } else {
        for (size_t i = 0; i < n; ++i) {
            const double x = (double)(i % nx) * g.h, y = (double)(i / nx) * g.h;
            const double r2 = (x - 0.23) * (x - 0.23) + (y - 0.17) * (y - 0.17);
            u[2 * i] = 1e-5 * exp(-r2 / 0.002);
            u[2 * i + 1] = 0.5e-5 * exp(-r2 / 0.002);
        }
    }
    check(pd_set_state(s, u, v, NULL), "pd_set_state");
    double kin0 = 0.0, str0 = 0.0;
    check(pd_energy(s, &kin0, &str0, NULL), "pd_energy");
    check(pd_step_explicit(s, steps, NULL), "pd_step_explicit");
    check(pd_get_state(s, u, v, NULL), "pd_get_state");
    double kin = 0.0, str = 0.0, dt = 0.0;
    check(pd_energy(s, &kin, &str, NULL), "pd_energy");
    check(pd_get_dt(s, &dt), "pd_get_dt");
    printf("bonds %lld\n", (long long)nb);
    printf("dt %.17g\n", dt);
    printf("energy0 %.17g %.17g\n", kin0, str0);
    printf("energy %.17g %.17g\n", kin, str);
    printf("u %.17g %.17g %.17g\n", u[0], u[2 * (n / 2)], u[2 * n - 1]);
    check(pd_destroy(s), "pd_destroy");
    free(u);
    free(v);
    return 0;
}
