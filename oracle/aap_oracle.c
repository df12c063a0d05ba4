/*
 * aap_oracle.c -- FP64 CPU oracle for the aligning-active-particles update.
 *
 * TEST INFRASTRUCTURE ONLY: the plain, slow, obviously correct reference the
 * CUDA library is checked against.  Only tests/, __graft_entry__.smoke() and
 * bench.py's CPU-baseline leg may load it; the product path never does.
 * Nothing here is shared with paper_2211_15630_gb300/.
 *
 * Every routine follows the model statement of Kuersten, "Aligning Active
 * Particles Py Package" (CPC); the section or equation is cited at each one.
 * Readings taken where the paper is silent:
 *   - a particle's own mirror image at a reflecting wall is a neighbour when
 *     it lies within R (self_image = 1; Sec. 2.4 gives every real particle
 *     image particles that interact "in the same way");
 *   - the Langevin noise xi is unit white noise, so the Euler-Maruyama
 *     increment is eta * sqrt(dt) * g with g ~ N(0,1) (Eq. Langevin_dynamics);
 *   - Euler-Maruyama moves positions with the orientation at time t;
 *   - a reflecting y wall maps theta -> -theta (the paper states x only);
 *   - periodic re-entry maps x >= L to x - L; reflecting re-entry maps
 *     x < 0 to -x and x > L to 2L - x (x = L stays);
 *   - orientations are stored wrapped into [-pi, pi).
 *
 * Parity: pinned by tests/test_oracle.py (cuRAND's host Philox generator,
 * scipy's k-d tree neighbour search, closed-form VM/Langevin cases, the
 * reflecting-wall mirror extension, translation invariance, mean neighbour
 * number of uniform states, free rotational diffusion).
 */
#include "aap_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n > 0 ? n : 1; }

int orc_get_threads(void)
{
#ifdef _OPENMP
    return g_threads;
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon et al., SC'11): ten rounds of the 4x32 S-box with
 * multipliers 0xD2511F53, 0xCD9E8D57 and Weyl key increments 0x9E3779B9,
 * 0xBB67AE85.  Replaces the paper's Mersenne twister (Sec. 3.1).
 * ---------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform on (0,1) from the top 23 bits: u = (2k+1) 2^-24 with 2k+1 < 2^24,
 * so u and 2u - 1 are exactly representable in FP32 and FP64 alike. */
double orc_u01(uint32_t w)
{
    return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Counter (id, step_lo, step_hi, tag), key (seed_lo, seed_hi). */
void orc_draw(const orc_params *p, uint32_t id, uint64_t step, uint32_t tag, uint32_t out[4])
{
    uint32_t ctr[4] = { id, (uint32_t)step, (uint32_t)(step >> 32), tag };
    uint32_t key[2] = { (uint32_t)p->seed, (uint32_t)(p->seed >> 32) };
    orc_philox4x32_10(ctr, key, out);
}

/* Uniform, isotropic random initial state (Fig. runtime caption, Sec. 4.2). */
void orc_init_state(const orc_params *p, double *x, double *y, double *th)
{
    for (int64_t i = 0; i < p->n; ++i) {
        uint32_t w[4];
        orc_draw(p, (uint32_t)i, 0, 1, w);
        x[i]  = p->lx * orc_u01(w[0]);
        y[i]  = p->ly * orc_u01(w[1]);
        th[i] = ORC_PI * (2.0 * orc_u01(w[2]) - 1.0);
    }
}

/* Cell geometry (Sec. 3.2): side L / floor(L/R), a little larger than R. */
int orc_geometry(const orc_params *p, int32_t *ncx, int32_t *ncy, double *csx, double *csy)
{
    double fx = floor(p->lx / p->r), fy = floor(p->ly / p->r);
    if (!(fx >= 3.0) || !(fy >= 3.0)) return -1;
    *ncx = (int32_t)fx;
    *ncy = (int32_t)fy;
    *csx = p->lx / fx;
    *csy = p->ly / fy;
    return 0;
}

/* ------------------------------------------------------------------------
 * Image particles (Sec. 2.4).  code -1 / +1 is the image on the low / high
 * side: periodic shifts by -L / +L; reflecting mirrors at 0 (x -> -x) or at
 * L (x -> 2L - x) and maps theta -> pi - theta (x) or theta -> -theta (y).
 * ---------------------------------------------------------------------- */
static double image_coord(double c, int code, double L, int reflecting)
{
    if (code == 0) return c;
    if (!reflecting) return code < 0 ? c - L : c + L;
    return code < 0 ? -c : 2.0 * L - c;
}

static double image_theta(double th, int ix, int iy, const orc_params *p)
{
    if (ix != 0 && p->bx) th = ORC_PI - th;
    if (iy != 0 && p->by) th = -th;
    return th;
}

int64_t orc_neighbours_brute(const orc_params *p, const double *x, const double *y,
                             int64_t i, int64_t *j_out, int32_t *img_out, int64_t cap)
{
    /* Eq. (metric_neighborhood) over every particle and every image of it. */
    const double r2 = p->r * p->r;
    int64_t count = 0;
    for (int64_t j = 0; j < p->n; ++j) {
        for (int iy = -1; iy <= 1; ++iy) {
            for (int ix = -1; ix <= 1; ++ix) {
                int self = (j == i);
                if (self && ix == 0 && iy == 0) continue;     /* j != i */
                if (self && !p->self_image) continue;
                double xj = image_coord(x[j], ix, p->lx, p->bx);
                double yj = image_coord(y[j], iy, p->ly, p->by);
                double dx = x[i] - xj, dy = y[i] - yj;
                if (dx * dx + dy * dy <= r2) {
                    if (count < cap) {
                        if (j_out) j_out[count] = j;
                        if (img_out) img_out[count] = (ix + 1) + 3 * (iy + 1);
                    }
                    ++count;
                }
            }
        }
    }
    return count;
}

void orc_counts_brute(const orc_params *p, const double *x, const double *y, int32_t *cnt)
{
    for (int64_t i = 0; i < p->n; ++i)
        cnt[i] = (int32_t)orc_neighbours_brute(p, x, y, i, NULL, NULL, 0);
}

/* ------------------------------------------------------------------------
 * Cell lists (Sec. 3.2): every step, a list of the particles in each cell;
 * the neighbours of i are searched in its cell and the eight around it.
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t ncx, ncy;
    double  csx, csy;
    int64_t *start;   /* ncx*ncy + 1 */
    int64_t *order;   /* particle indices grouped by cell */
} cell_list;

static int cell_of(double c, double cs, int32_t nc)
{
    int k = (int)floor(c / cs);
    if (k < 0) k = 0;
    if (k > nc - 1) k = nc - 1;
    return k;
}

static int build_cells(const orc_params *p, const double *x, const double *y, cell_list *cl)
{
    if (orc_geometry(p, &cl->ncx, &cl->ncy, &cl->csx, &cl->csy) != 0) return -1;
    int64_t ncell = (int64_t)cl->ncx * cl->ncy;
    cl->start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    cl->order = (int64_t *)malloc((size_t)(p->n > 0 ? p->n : 1) * sizeof(int64_t));
    int64_t *fill = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    if (!cl->start || !cl->order || !fill) {
        free(cl->start); free(cl->order); free(fill);
        return -2;
    }
    for (int64_t i = 0; i < p->n; ++i) {
        int64_t c = (int64_t)cell_of(y[i], cl->csy, cl->ncy) * cl->ncx + cell_of(x[i], cl->csx, cl->ncx);
        cl->start[c + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) cl->start[c + 1] += cl->start[c];
    for (int64_t i = 0; i < p->n; ++i) {
        int64_t c = (int64_t)cell_of(y[i], cl->csy, cl->ncy) * cl->ncx + cell_of(x[i], cl->csx, cl->ncx);
        cl->order[cl->start[c] + fill[c]++] = i;
    }
    free(fill);
    return 0;
}

static void free_cells(cell_list *cl)
{
    free(cl->start);
    free(cl->order);
}

/* Neighbour cell c along one axis: the real cell, or the cell whose images
 * (code -1 / +1) fill it in when c lies outside the box. */
static void resolve_cell(int c, int32_t nc, int reflecting, int *src, int *code)
{
    if (c >= 0 && c < nc) { *src = c; *code = 0; return; }
    if (!reflecting) {
        if (c < 0) { *src = c + nc; *code = -1; }
        else       { *src = c - nc; *code = +1; }
    } else {
        if (c < 0) { *src = 0;      *code = -1; }
        else       { *src = nc - 1; *code = +1; }
    }
}

typedef struct {
    int64_t n;          /* |Omega_i| */
    double  sx, sy;     /* VM / NVM sum S_i, including e^{i theta_i}          */
    double  t;          /* Langevin sum of sin(o (theta_j - theta_i))         */
    int     amb;        /* a candidate within `band` of R                      */
} accum;

/* ------------------------------------------------------------------------
 * Species (Sec. 2.5): each species has its own v, eta, omega, and the
 * Langevin coupling of i to a neighbour j is Gamma_{s_i s_j}.  Species are
 * consecutive blocks of particle ids.
 * ---------------------------------------------------------------------- */
int orc_species_of(const orc_params *p, int64_t id)
{
    if (p->nspecies <= 1) return 0;
    int64_t end = 0;
    for (int s = 0; s < p->nspecies; ++s) {
        end += p->species_n[s];
        if (id < end) return s;
    }
    return p->nspecies - 1;
}

static double sp_v(const orc_params *p, int s) { return p->nspecies > 1 ? p->species_v[s] : p->v; }
static double sp_eta(const orc_params *p, int s) { return p->nspecies > 1 ? p->species_eta[s] : p->eta; }
static double sp_omega(const orc_params *p, int s) { return p->nspecies > 1 ? p->species_omega[s] : p->omega; }
static double sp_gamma(const orc_params *p, int a, int b)
{
    return p->nspecies > 1 ? p->species_gamma[a * 8 + b] : p->gamma;
}

/* One neighbour with (image) orientation tj and coupling g (Langevin)
 * joins the sums of particle i. */
static void add_neighbour(const orc_params *p, double ti, double tj, double g, accum *a)
{
    a->n++;
    if (p->model == 0) {                 /* Eq. (collision_VM) */
        a->sx += cos(tj);
        a->sy += sin(tj);
    } else if (p->model == 2) {          /* Eq. (collision_NVM), sign(0) = +1 */
        double sgn = cos(ti - tj) >= 0.0 ? 1.0 : -1.0;
        double tn = tj + 0.5 * ORC_PI * (1.0 - sgn);
        a->sx += cos(tn);
        a->sy += sin(tn);
    } else {                             /* Eq. (Langevin_dynamics), Gamma inside the sum */
        a->t += g * sin((double)p->order * (tj - ti));
    }
}

/* ------------------------------------------------------------------------
 * Metric-free neighbourhoods (Sec. 2.3): the k nearest particles.  This is
 * the definition written out by brute force over every particle and image;
 * the cell rings the paper describes (Sec. 3.3) only make it faster.
 * ---------------------------------------------------------------------- */
typedef struct {
    double  d2;
    int64_t j;
    int32_t img;
} knn_cand;

static int cand_less(double d2, int64_t j, int32_t img, const knn_cand *b)
{
    if (d2 != b->d2) return d2 < b->d2;
    if (j != b->j) return j < b->j;
    return img < b->img;
}

/* Image codes of particle j along one axis: the nearest periodic copy, or
 * all three copies at a reflecting axis. */
static int axis_codes(double ci, double cj, double L, int reflecting, int codes[3])
{
    if (reflecting) {
        codes[0] = -1; codes[1] = 0; codes[2] = 1;
        return 3;
    }
    int best = 0;
    double bd = fabs(ci - cj);
    if (fabs(ci - (cj - L)) < bd) { best = -1; bd = fabs(ci - (cj - L)); }
    if (fabs(ci - (cj + L)) < bd) { best = 1; }
    codes[0] = best;
    return 1;
}

static int64_t knn_collect(const orc_params *p, const double *x, const double *y, int64_t i,
                           int64_t m, knn_cand *out)
{
    int64_t cnt = 0;
    if (m <= 0) return 0;
    for (int64_t j = 0; j < p->n; ++j) {
        int cx[3], cy[3];
        int nx = axis_codes(x[i], x[j], p->lx, p->bx, cx);
        int ny = axis_codes(y[i], y[j], p->ly, p->by, cy);
        for (int b = 0; b < ny; ++b) {
            for (int a = 0; a < nx; ++a) {
                int ix = cx[a], iy = cy[b];
                if (j == i && ix == 0 && iy == 0) continue;
                if (j == i && !p->self_image) continue;
                double dx = x[i] - image_coord(x[j], ix, p->lx, p->bx);
                double dy = y[i] - image_coord(y[j], iy, p->ly, p->by);
                double d2 = dx * dx + dy * dy;
                int32_t img = (ix + 1) + 3 * (iy + 1);
                if (cnt == m && !cand_less(d2, j, img, &out[m - 1])) continue;
                int64_t s = cnt < m ? cnt++ : m - 1;
                while (s > 0 && cand_less(d2, j, img, &out[s - 1])) {
                    out[s] = out[s - 1];
                    --s;
                }
                out[s].d2 = d2;
                out[s].j = j;
                out[s].img = img;
            }
        }
    }
    return cnt;
}

int64_t orc_knn(const orc_params *p, const double *x, const double *y, int64_t i, int64_t m,
                int64_t *j_out, int32_t *img_out, double *d_out)
{
    if (m <= 0) return 0;
    knn_cand *c = (knn_cand *)malloc((size_t)m * sizeof(knn_cand));
    if (!c) return -1;
    int64_t cnt = knn_collect(p, x, y, i, m, c);
    for (int64_t s = 0; s < cnt; ++s) {
        if (j_out) j_out[s] = c[s].j;
        if (img_out) img_out[s] = c[s].img;
        if (d_out) d_out[s] = sqrt(c[s].d2);
    }
    free(c);
    return cnt;
}

/* Sums over the k nearest (h = 1 is applied by the caller, Sec. 2.3). */
static void gather_knn(const orc_params *p, const double *x, const double *y, const double *th,
                       int64_t i, double band, accum *a)
{
    const double ti = th[i];
    a->n = 0;
    a->sx = cos(ti);
    a->sy = sin(ti);
    a->t = 0.0;
    a->amb = 0;
    const int64_t k = p->kn;
    knn_cand *c = (knn_cand *)malloc((size_t)(k + 1) * sizeof(knn_cand));
    if (!c) { a->amb = 1; return; }
    int64_t cnt = knn_collect(p, x, y, i, k + 1, c);
    if (cnt > k && sqrt(c[k].d2) - sqrt(c[k - 1].d2) < band) a->amb = 1;
    for (int64_t s = 0; s < cnt && s < k; ++s) {
        int ix = c[s].img % 3 - 1, iy = c[s].img / 3 - 1;
        add_neighbour(p, ti, image_theta(th[c[s].j], ix, iy, p),
                      sp_gamma(p, orc_species_of(p, i), orc_species_of(p, c[s].j)), a);
    }
    free(c);
}

static void gather(const orc_params *p, const cell_list *cl, const double *x, const double *y,
                   const double *th, int64_t i, double band, accum *a)
{
    const double r2 = p->r * p->r;
    const double xi = x[i], yi = y[i], ti = th[i];
    int cx = cell_of(xi, cl->csx, cl->ncx), cy = cell_of(yi, cl->csy, cl->ncy);
    a->n = 0;
    a->sx = cos(ti);
    a->sy = sin(ti);
    a->t = 0.0;
    a->amb = 0;
    for (int dcy = -1; dcy <= 1; ++dcy) {
        int sy, iy;
        resolve_cell(cy + dcy, cl->ncy, p->by, &sy, &iy);
        for (int dcx = -1; dcx <= 1; ++dcx) {
            int sx, ix;
            resolve_cell(cx + dcx, cl->ncx, p->bx, &sx, &ix);
            int64_t c = (int64_t)sy * cl->ncx + sx;
            for (int64_t k = cl->start[c]; k < cl->start[c + 1]; ++k) {
                int64_t j = cl->order[k];
                int self = (j == i);
                if (self && ix == 0 && iy == 0) continue;
                if (self && !p->self_image) continue;
                double xj = image_coord(x[j], ix, p->lx, p->bx);
                double yj = image_coord(y[j], iy, p->ly, p->by);
                double dx = xi - xj, dy = yi - yj;
                double d2 = dx * dx + dy * dy;
                if (fabs(sqrt(d2) - p->r) < band) a->amb = 1;
                if (d2 > r2) continue;
                add_neighbour(p, ti, image_theta(th[j], ix, iy, p),
                              sp_gamma(p, orc_species_of(p, i), orc_species_of(p, j)), a);
            }
        }
    }
}

int orc_counts_cell(const orc_params *p, const double *x, const double *y, int32_t *cnt)
{
    cell_list cl;
    int rc = build_cells(p, x, y, &cl);
    if (rc) return rc;
    double *th0 = (double *)calloc((size_t)(p->n > 0 ? p->n : 1), sizeof(double));
    if (!th0) { free_cells(&cl); return -2; }
    for (int64_t i = 0; i < p->n; ++i) {
        accum a;
        gather(p, &cl, x, y, th0, i, 0.0, &a);
        cnt[i] = (int32_t)a.n;
    }
    free(th0);
    free_cells(&cl);
    return 0;
}

static double wrap_angle(double t)
{
    return t - 2.0 * ORC_PI * floor((t + ORC_PI) / (2.0 * ORC_PI));
}

/* One particle's update t -> t+1 (Sec. 2.1 collision then streaming, or the
 * Euler-Maruyama step of Sec. 2.2), then the boundary rule of Sec. 2.4. */
static void update_one(const orc_params *p, const cell_list *cl, const double *x, const double *y,
                       const double *th, uint64_t step, int64_t i, double band,
                       double *xo, double *yo, double *to, int32_t *nb, double *smag, int32_t *amb)
{
    accum a;
    if (p->kn > 0) gather_knn(p, x, y, th, i, band, &a);
    else gather(p, cl, x, y, th, i, band, &a);
    uint32_t w[4];
    orc_draw(p, (uint32_t)i, step, 0, w);
    double u0 = orc_u01(w[0]), u1 = orc_u01(w[1]);
    const int si = orc_species_of(p, i);
    const double v = sp_v(p, si), eta = sp_eta(p, si), omega = sp_omega(p, si);
    double tn, xn, yn;
    if (p->model == 0 || p->model == 2) {
        /* Eq. (collision): f + eta * xi with xi uniform on [-pi, pi]. */
        tn = atan2(a.sy, a.sx) + omega + eta * ORC_PI * (2.0 * u0 - 1.0);
        /* Eq. (streaming) uses the new orientation. */
        xn = x[i] + v * cos(tn);
        yn = y[i] + v * sin(tn);
    } else {
        /* metric-free: h = 1 (Sec. 2.3, the weight is absorbed in Gamma); a
         * tabulated h(n) uses its last entry beyond its length (Sec. 4) */
        double h = (p->weight == 0 && p->kn == 0) ? 1.0 / (1.0 + (double)a.n) : 1.0;
        if (p->kn == 0 && p->weight_len > 0)
            h = p->weight_table[a.n < p->weight_len ? a.n : p->weight_len - 1];
        /* Box-Muller Gaussian (Sec. 3.1). */
        double g = sqrt(-2.0 * log(u0)) * cos(2.0 * ORC_PI * u1);
        tn = th[i] + p->dt * (h * a.t + omega) + eta * sqrt(p->dt) * g;
        xn = x[i] + v * p->dt * cos(th[i]);
        yn = y[i] + v * p->dt * sin(th[i]);
    }
    if (!p->bx) {
        if (xn < 0.0) xn += p->lx;
        else if (xn >= p->lx) xn -= p->lx;
    } else {
        if (xn < 0.0)        { xn = -xn;              tn = ORC_PI - tn; }
        else if (xn > p->lx) { xn = 2.0 * p->lx - xn; tn = ORC_PI - tn; }
    }
    if (!p->by) {
        if (yn < 0.0) yn += p->ly;
        else if (yn >= p->ly) yn -= p->ly;
    } else {
        if (yn < 0.0)        { yn = -yn;              tn = -tn; }
        else if (yn > p->ly) { yn = 2.0 * p->ly - yn; tn = -tn; }
    }
    *xo = xn;
    *yo = yn;
    *to = wrap_angle(tn);
    if (nb) *nb = (int32_t)a.n;
    if (smag) *smag = (p->model == 1) ? 0.0 : sqrt(a.sx * a.sx + a.sy * a.sy);
    if (amb) *amb = a.amb;
}

int orc_step_subset(const orc_params *p, const double *x, const double *y, const double *th,
                    uint64_t step, const int64_t *idx, int64_t m,
                    double *x_out, double *y_out, double *th_out,
                    int32_t *nb, double *smag, int32_t *amb, double band)
{
    cell_list cl = {0, 0, 0.0, 0.0, NULL, NULL};
    if (p->kn < 0) return -1;
    if (p->kn == 0) {
        int rc = build_cells(p, x, y, &cl);
        if (rc) return rc;
    }
    if (!idx && m != p->n) { free_cells(&cl); return -1; }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(g_threads)
#endif
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = idx ? idx[k] : k;
        update_one(p, &cl, x, y, th, step, i, band, &x_out[k], &y_out[k], &th_out[k],
                   nb ? &nb[k] : NULL, smag ? &smag[k] : NULL, amb ? &amb[k] : NULL);
    }
    free_cells(&cl);
    return 0;
}

int orc_run(const orc_params *p, double *x, double *y, double *th,
            uint64_t step0, int64_t nsteps, double *phi, int nthreads)
{
    int saved = g_threads;
    if (nthreads > 0) g_threads = nthreads;
    size_t sz = (size_t)(p->n > 0 ? p->n : 1) * sizeof(double);
    double *xn = (double *)malloc(sz), *yn = (double *)malloc(sz), *tn = (double *)malloc(sz);
    int rc = (xn && yn && tn) ? 0 : -2;
    for (int64_t t = 0; rc == 0 && t < nsteps; ++t) {
        if (phi) phi[t] = orc_polar(p->n, th);
        rc = orc_step_subset(p, x, y, th, step0 + (uint64_t)t, NULL, p->n, xn, yn, tn,
                             NULL, NULL, NULL, 0.0);
        if (rc == 0) {
            memcpy(x, xn, (size_t)p->n * sizeof(double));
            memcpy(y, yn, (size_t)p->n * sizeof(double));
            memcpy(th, tn, (size_t)p->n * sizeof(double));
        }
    }
    if (rc == 0 && phi) phi[nsteps] = orc_polar(p->n, th);
    free(xn); free(yn); free(tn);
    g_threads = saved;
    return rc;
}

/* Polar order parameter p = |(1/N) sum e^{i theta_j}| (Sec. 3.4). */
double orc_polar(int64_t n, const double *th)
{
    double c = 0.0, s = 0.0;
    for (int64_t i = 0; i < n; ++i) { c += cos(th[i]); s += sin(th[i]); }
    return n > 0 ? sqrt(c * c + s * s) / (double)n : 0.0;
}

/* Nematic order parameter q = |(1/N) sum e^{2 i theta_j}| (Sec. 3.4). */
double orc_nematic(int64_t n, const double *th)
{
    double c = 0.0, s = 0.0;
    for (int64_t i = 0; i < n; ++i) { c += cos(2.0 * th[i]); s += sin(2.0 * th[i]); }
    return n > 0 ? sqrt(c * c + s * s) / (double)n : 0.0;
}
