/* Host sanitizer run of the FP64 oracle (test infrastructure): every entry
 * point on small systems under AddressSanitizer and UndefinedBehaviorSanitizer.
 * Built and run by tests/test_oracle_sanitizers.py; exits non-zero on a
 * failed check (the sanitizers abort by themselves on an error). */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "../oracle/aap_oracle.h"

static int check(int ok, const char *what)
{
    if (!ok) fprintf(stderr, "check failed: %s\n", what);
    return ok ? 0 : 1;
}

int main(void)
{
    int bad = 0;
    orc_params p;
    memset(&p, 0, sizeof(p));
    p.n = 300; p.lx = 12.0; p.ly = 10.0; p.r = 1.0; p.v = 0.3; p.eta = 0.4; p.omega = 0.1;
    p.gamma = 1.2; p.dt = 0.05; p.seed = 77; p.order = 1; p.self_image = 1;
    const int64_t n = p.n;
    double *x = malloc(n * sizeof(double)), *y = malloc(n * sizeof(double)), *th = malloc(n * sizeof(double));
    double *xo = malloc(n * sizeof(double)), *yo = malloc(n * sizeof(double)), *to = malloc(n * sizeof(double));
    double *sm = malloc(n * sizeof(double)), phi[6];
    int32_t *nb = malloc(n * sizeof(int32_t)), *amb = malloc(n * sizeof(int32_t)), *c1 = malloc(n * sizeof(int32_t));
    int32_t *c2 = malloc(n * sizeof(int32_t));
    int64_t idx[3] = {0, 17, 299}, jj[64];
    int32_t img[64];
    double dd[64];
    orc_init_state(&p, x, y, th);
    for (int model = 0; model < 3; ++model)
        for (int b = 0; b < 4; ++b)
            for (int kn = 0; kn <= 7; kn += 7) {
                p.model = model; p.bx = b & 1; p.by = b >> 1; p.kn = kn;
                p.order = model == 1 ? 2 : 1;
                bad += check(orc_step_subset(&p, x, y, th, 3, NULL, n, xo, yo, to, nb, sm, amb, 1e-5) == 0, "step");
                bad += check(orc_step_subset(&p, x, y, th, 3, idx, 3, xo, yo, to, nb, sm, amb, 1e-5) == 0, "subset");
                for (int64_t i = 0; i < n; ++i) bad += check(isfinite(to[i]) || i >= 3, "finite");
            }
    p.kn = 0; p.model = 0; p.bx = 1; p.by = 0;
    orc_counts_brute(&p, x, y, c1);
    bad += check(orc_counts_cell(&p, x, y, c2) == 0, "counts_cell");
    for (int64_t i = 0; i < n; ++i) bad += check(c1[i] == c2[i], "cell == brute");
    bad += check(orc_neighbours_brute(&p, x, y, 5, jj, img, 64) >= 0, "neighbours");
    bad += check(orc_knn(&p, x, y, 5, 64, jj, img, dd) == 64, "knn");
    p.nspecies = 3; p.species_n[0] = 100; p.species_n[1] = 50; p.species_n[2] = 150;
    for (int s = 0; s < 3; ++s) {
        p.species_v[s] = 0.1 * (s + 1); p.species_eta[s] = 0.2; p.species_omega[s] = 0.05 * s;
        for (int t = 0; t < 3; ++t) p.species_gamma[8 * s + t] = 0.5 + s - t;
    }
    p.model = 1; p.weight_len = 3; p.weight_table[0] = 1.0; p.weight_table[1] = 0.6; p.weight_table[2] = 0.4;
    bad += check(orc_run(&p, x, y, th, 0, 5, phi, 2) == 0, "run");
    bad += check(phi[5] >= 0.0 && phi[5] <= 1.0, "phi range");
    bad += check(orc_species_of(&p, 120) == 1 && orc_species_of(&p, 299) == 2, "species");
    free(x); free(y); free(th); free(xo); free(yo); free(to); free(sm); free(nb); free(amb); free(c1); free(c2);
    printf("sanitized oracle run: %d failed checks\n", bad);
    return bad ? 1 : 0;
}
