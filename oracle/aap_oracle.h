/*
 * aap_oracle.h -- FP64 CPU oracle for the aligning-active-particles update.
 *
 * TEST INFRASTRUCTURE ONLY.  This header and aap_oracle.c are the plain,
 * slow, obviously correct reference that the CUDA path is checked against.
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load it.  It shares no code, header, table or helper with the CUDA library
 * in paper_2211_15630_gb300/.
 *
 * Model (Kuersten, "Aligning Active Particles Py Package", CPC):
 *   state      (x_i, y_i, theta_i), x in [0,Lx], y in [0,Ly]          Sec. 2
 *   VM         theta_i(t+1) = arg[e^{i theta_i} + sum_{j in Omega_i} e^{i theta_j}]
 *                             + omega + eta * xi,  xi ~ U[-pi,pi]     Eq. (collision), (collision_VM)
 *   NVM        as VM with theta_j -> theta_j + pi/2 (1 - sign(cos(theta_i - theta_j)))
 *                                                                      Eq. (collision_NVM)
 *   streaming  x += v cos theta(t+1), y += v sin theta(t+1)            Eq. (streaming)
 *   Langevin   dtheta = [Gamma h(|Omega_i|) sum sin(o (theta_j - theta_i)) + omega] dt
 *                       + eta dW,  dx = v cos theta dt  (Euler-Maruyama)  Eq. (Langevin_dynamics), Sec. 2.2
 *   Omega_i    { j != i : |r_i - r_j| <= R }                           Eq. (metric_neighborhood)
 *              or the k nearest j != i (metric-free, h = 1)            Sec. 2.3
 *   boundaries periodic or reflecting per axis, with image particles   Sec. 2.4
 *   cell lists side L/floor(L/R)                                        Sec. 3.2
 *   species    per-species v, eta, omega and a coupling matrix Gamma_ab  Sec. 2.5
 *   polar order p = |sum e^{i theta}| / N                               Sec. 3.4
 *
 * Random numbers: counter-based Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 * SC'11), written here from its published definition; the paper's own
 * program used a Mersenne twister (Sec. 3.1), which is not reproduced.
 */
#ifndef AAP_ORACLE_H
#define AAP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Field order: 8-byte members first so the layout has no interior padding. */
typedef struct {
    int64_t  n;          /* particle number N                                  */
    double   lx, ly;     /* box Lx, Ly                                         */
    double   r;          /* interaction radius R                               */
    double   v;          /* speed v                                            */
    double   eta;        /* noise strength eta                                 */
    double   omega;      /* chirality omega                                    */
    double   gamma;      /* coupling Gamma (Langevin)                          */
    double   dt;         /* Euler-Maruyama step (Langevin)                     */
    uint64_t seed;       /* Philox key                                         */
    int32_t  model;      /* 0 VM, 1 Langevin, 2 NVM                            */
    int32_t  order;      /* interaction order o (Langevin)                     */
    int32_t  weight;     /* 0: h(n) = 1/(1+n), 1: h(n) = 1                     */
    int32_t  bx, by;     /* 0 periodic, nonzero reflecting                     */
    int32_t  self_image; /* 1: a particle's own mirror image is a neighbour    */
    int32_t  kn;         /* 0: metric neighbourhood (radius R); k > 0: the k
                            nearest particles (metric-free, Sec. 2.3)          */
    /* Particle species (Sec. 2.5): with nspecies >= 2, particles
     * 0 .. species_n[0]-1 are species 0, the next species_n[1] species 1, ...;
     * particle i then uses v, eta, omega of its species s_i and, in the
     * Langevin sum, Gamma_{s_i s_j} = species_gamma[s_i * 8 + s_j] for each
     * neighbour j.  nspecies 0 or 1: the scalar parameters above. */
    int32_t  nspecies;
    int32_t  pad_;
    int64_t  species_n[8];
    double   species_v[8];
    double   species_eta[8];
    double   species_omega[8];
    double   species_gamma[64];
    /* Tabulated weight function (Sec. 4, weight_function / weight_vector_length):
     * with weight_len > 0 the Langevin weight is h(n) = weight_table[min(n, weight_len-1)]
     * (metric neighbourhoods only; metric-free models use h = 1, Sec. 2.3). */
    int32_t  weight_len;
    int32_t  pad2_;
    double   weight_table[128];
} orc_params;

/* Species of particle `id` (0 with a single species). */
int      orc_species_of(const orc_params *p, int64_t id);

/* OpenMP threads used by orc_step_subset / orc_run (1 without OpenMP). */
void     orc_set_threads(int n);
int      orc_get_threads(void);

/* ---- random numbers ---------------------------------------------------- */
void     orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double   orc_u01(uint32_t w);
/* draws for particle `id` at step `step`; tag 0 = dynamics, 1 = initial state */
void     orc_draw(const orc_params *p, uint32_t id, uint64_t step, uint32_t tag, uint32_t out[4]);
void     orc_init_state(const orc_params *p, double *x, double *y, double *th);

/* ---- neighbourhoods ----------------------------------------------------- */
int      orc_geometry(const orc_params *p, int32_t *ncx, int32_t *ncy, double *csx, double *csy);
/* Neighbour list of particle i by brute force over all particles and images.
 * Writes up to `cap` (j, image) pairs, image = (ix+1) + 3 (iy+1) with ix, iy in
 * {-1,0,1}; returns the number of neighbours (may exceed cap). */
int64_t  orc_neighbours_brute(const orc_params *p, const double *x, const double *y,
                              int64_t i, int64_t *j_out, int32_t *img_out, int64_t cap);
/* Neighbour counts of all particles: brute force and cell list. */
void     orc_counts_brute(const orc_params *p, const double *x, const double *y, int32_t *cnt);
int      orc_counts_cell(const orc_params *p, const double *x, const double *y, int32_t *cnt);

/* Metric-free neighbourhood of particle i (Sec. 2.3): the m nearest
 * candidates in ascending (distance, j, image) order.  Candidates are all
 * particles j with their nearest copy along a periodic axis and all three
 * copies (itself, mirror at 0, mirror at L) along a reflecting axis; the
 * untransformed particle i is excluded, its mirror images are not (self_image).
 * Returns the number stored (< m only when there are fewer candidates). */
int64_t  orc_knn(const orc_params *p, const double *x, const double *y, int64_t i, int64_t m,
                 int64_t *j_out, int32_t *img_out, double *d_out);

/* ---- dynamics ----------------------------------------------------------- */
/* One update t -> t+1 of particles idx[0..m) (all particles if idx == NULL,
 * then m must be N) from the state (x, y, th) at step `step`.  Outputs are
 * indexed like idx.  nb: |Omega_i|; smag: |S_i| of the VM/NVM sum (0 for
 * Langevin); amb: 1 if some candidate lies within `band` of the radius R, or,
 * metric-free, if the k-th and (k+1)-th nearest lie within `band` of each other. */
int      orc_step_subset(const orc_params *p, const double *x, const double *y, const double *th,
                         uint64_t step, const int64_t *idx, int64_t m,
                         double *x_out, double *y_out, double *th_out,
                         int32_t *nb, double *smag, int32_t *amb, double band);
/* nsteps full updates in place; phi[0..nsteps] = p(t) before and after each. */
int      orc_run(const orc_params *p, double *x, double *y, double *th,
                 uint64_t step0, int64_t nsteps, double *phi, int nthreads);

/* ---- measurements ------------------------------------------------------- */
double   orc_polar(int64_t n, const double *th);
double   orc_nematic(int64_t n, const double *th);

#ifdef __cplusplus
}
#endif
#endif
