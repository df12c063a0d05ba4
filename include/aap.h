/*
 * aap.h -- C ABI of the GB300 (sm_103a) aligning-active-particles library.
 *
 * The library advances N self-propelled particles in a 2-D box with the
 * alignment rules of Kuersten, "Aligning Active Particles Py Package" (CPC):
 * the Vicsek collision and streaming rule (Sec. 2.1, Eq. collision_VM and
 * Eq. streaming), its nematic variant (Eq. collision_NVM), and the overdamped
 * Langevin alignment dynamics integrated by Euler-Maruyama (Sec. 2.2,
 * Eq. Langevin_dynamics), with the metric neighbourhood
 * Omega_i = { j != i : |r_i - r_j| <= R } (Eq. metric_neighborhood) found
 * through cell lists (Sec. 3.2) and periodic or reflecting boundaries per axis
 * (Sec. 2.4).  Every step runs in the library's own CUDA kernels on the
 * caller's stream.
 *
 * Conventions shared by every entry point:
 *  - Every function returns an int status: AAP_OK (0) or a negative AAP_E*
 *    code.  aap_last_error() returns a message for the calling thread's last
 *    failure.  On failure no output argument is written except where stated.
 *  - Handles are opaque.  The library owns all device memory it allocates and
 *    frees it in the matching *_destroy.  Host buffers passed in are owned by
 *    the caller and are only read or written during the call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  All device work of a handle is ordered on that stream.
 *  - Calls that return data to host memory (aap_observe, aap_phi_trace,
 *    aap_get_state, aap_step_neighbours, aap_ens_phi_mean, aap_ens_get_state)
 *    synchronise the stream; aap_step and aap_ens_step only enqueue work.
 *  - A handle is not thread-safe; different handles may be used from
 *    different threads.
 *  - Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by the seed,
 *    counter (particle id, step low word, step high word, 0) for the dynamics
 *    and (id, 0, 0, 1) for the initial state; uniforms are
 *    ((w >> 9) + 1/2) 2^-23.  The paper's own program used a Mersenne
 *    twister (Sec. 3.1); trajectories are therefore not comparable to it.
 */
#ifndef AAP_H
#define AAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define AAP_OK          0
#define AAP_EINVAL    (-1)   /* invalid argument or parameter set            */
#define AAP_ENOMEM    (-2)   /* device or host allocation failed             */
#define AAP_ECUDA     (-3)   /* a CUDA runtime call failed                   */
#define AAP_ETIMEOUT  (-4)   /* a bounded device wait gave up                */
#define AAP_ENAN      (-5)   /* a non-finite value reached the state         */
#define AAP_ESTATE    (-6)   /* handle in an unusable state (after a fault)  */
#define AAP_EOVERFLOW (-7)   /* more particles in a tile than it can hold    */
#define AAP_EIO       (-8)   /* a saved-state file could not be written/read */

/* ---- models (Sec. 2) ----------------------------------------------------- */
#define AAP_VM        0      /* Vicsek model, Eq. (collision_VM)              */
#define AAP_LANGEVIN  1      /* overdamped Langevin, Eq. (Langevin_dynamics)  */
#define AAP_NVM       2      /* nematic Vicsek model, Eq. (collision_NVM)     */

/* weight function h of Eq. (Langevin_dynamics), Sec. 2.2 */
#define AAP_H_INV_1PN 0      /* h(n) = 1/(1+n): "nonadditiveL" (the default)  */
#define AAP_H_ONE     1      /* h(n) = 1:       "additiveL"                   */

/* Observation flags (aap_obs.flags). */
#define AAP_FLAG_SPILLED  1  /* some tile region overflowed into the spill list
                                (results stay exact; the layout was enlarged) */

/*
 * Model parameters, named as in the paper's parameter list (Sec. 4).
 * Positions live in [0,Lx] x [0,Ly]; orientations in [-pi, pi).
 * Constraints checked by aap_create (AAP_EINVAL otherwise):
 *   n >= 0, n < 2^31; lx, ly, r > 0 and finite; floor(L/R) >= 3 on both axes
 *   (a 3x3 cell stencil must not see a cell twice); v >= 0 and the per-step
 *   displacement v (VM, NVM) or v*dt (Langevin) at most one cell side;
 *   eta >= 0 (eta <= 1 is the paper's range for the VM but not enforced);
 *   dt > 0 for the Langevin model; order >= 1; model, weight as defined above.
 */
typedef struct aap_params {
    int64_t  n;          /* particle number N                                   */
    double   lx, ly;     /* box size Lx, Ly                                     */
    double   r;          /* interaction radius R                                */
    double   v;          /* speed v                                             */
    double   eta;        /* noise strength eta                                  */
    double   omega;      /* chirality omega                                     */
    double   gamma;      /* coupling Gamma (Langevin)                           */
    double   dt;         /* Euler-Maruyama step (Langevin; ignored by VM/NVM)   */
    uint64_t seed;       /* Philox key                                          */
    int32_t  model;      /* AAP_VM, AAP_LANGEVIN or AAP_NVM                     */
    int32_t  order;      /* interaction order o (Langevin), 1 = polar           */
    int32_t  weight;     /* AAP_H_INV_1PN or AAP_H_ONE (Langevin)               */
    int32_t  bx, by;     /* 0 periodic, nonzero reflecting (per axis)           */
    int32_t  tile_w;     /* cells per tile along x; 0 = automatic               */
    int32_t  tile_h;     /* cells per tile along y; 0 = automatic               */
    int32_t  threads;    /* threads per block of the step kernel: 0 (automatic),
                            256 or 512 (whole-block tile kernel), 1024 (the
                            pipelined kernel: one block per SM with copy, sort
                            and update warps; one species per system).
                            Automatic picks 1024 where it applies, else 512;
                            an ensemble follows its first replica's value   */
    double   capacity;   /* tile-region capacity over the mean occupancy;
                            0 = automatic (4)                                   */
    int32_t  binnum_theta;      /* bins of the orientation histogram over
                                   [-pi, pi) (Sec. 3.4); 0 = 100, at most 512     */
    int32_t  binnum_neighbors;  /* bins 0..binnum_neighbors-1 of the neighbour-
                                   number histogram, the last collecting all
                                   larger |Omega_i|; 0 = 100, at most 512         */
    int32_t  kn;         /* [kn] 0: metric neighbourhood of radius r; k in
                            [1, 32]: metric-free, Omega_i = the k nearest other
                            particles (mfVM / mfNVM / mfL, Sec. 2.3, with h = 1
                            whatever `weight` says; r is then unused)          */
    /* Species (Sec. 2.5; the paper lets v, eta, omega, N and gamma be lists).
     * nspecies 0 or 1: one species with the scalars above.  2..8: particles
     * 0 .. species_n[0]-1 are species 0, the next species_n[1] species 1, and
     * so on (the counts must add up to n); particle i moves with
     * species_v[s_i], takes noise species_eta[s_i] and chirality
     * species_omega[s_i], and its Langevin sum weighs neighbour j by
     * species_gamma[8 * s_i + s_j] (the scalar gamma is then unused).        */
    int32_t  nspecies;
    int64_t  species_n[8];
    double   species_v[8];
    double   species_eta[8];
    double   species_omega[8];
    double   species_gamma[64];
    /* [weight_function, weight_vector_length] (Sec. 4): weight_len in [0, 128];
     * with weight_len > 0 the Langevin weight is h(n) = weight_table[min(n,
     * weight_len - 1)] for |Omega_i| = n (the paper evaluates the function once
     * for n = 0 .. weight_vector_length - 1 and uses the last value beyond);
     * 0: `weight` decides.  Metric-free models always use h = 1 (Sec. 2.3).   */
    int32_t  weight_len;
    double   weight_table[128];
} aap_params;

/* Observables of the current state (Sec. 3.4). */
typedef struct aap_obs {
    double  phi;              /* polar order p = |sum e^{i theta}| / N          */
    double  q;                /* nematic order q = |sum e^{2 i theta}| / N      */
    double  mean_neighbours;  /* mean |Omega_i| measured by the last step
                                 (NaN before the first step)                    */
    int64_t step;             /* number of steps taken                          */
    int32_t flags;            /* AAP_FLAG_* bits                                */
    int32_t reserved;
} aap_obs;

/* Geometry and memory layout chosen for a handle (for tests and tools). */
typedef struct aap_layout {
    int32_t ncx, ncy;         /* cells per axis, floor(L/R) (Sec. 3.2)          */
    int32_t ntx, nty;         /* tiles per axis                                 */
    int32_t tile_w, tile_h;   /* largest tile in cells                          */
    int32_t fix_bits_x;       /* fixed-point bits per cell side, x              */
    int32_t fix_bits_y;       /* fixed-point bits per cell side, y              */
    int32_t threads;          /* threads per block of the step kernel           */
    int32_t stage_cap;        /* particles a block stages in shared memory      */
    int64_t tile_slots;       /* particle slots per tile                        */
    int64_t device_bytes;     /* device memory held by the handle               */
    double  cell_x, cell_y;   /* cell sides L/floor(L/R)                        */
} aap_layout;

/* On-the-fly measurements (Sec. 3.4): moments k = 1..4 of the polar order
 * p, the nematic order q and the mean neighbour number nbar, over the states
 * t = t0 .. t0+n-1 of n measured steps (the last state is not used). */
typedef struct aap_results {
    int64_t samples;          /* number of measured states                      */
    double  p[4];             /* <p>, <p^2>, <p^3>, <p^4>                        */
    double  q[4];             /* <q^k>                                           */
    double  nbar[4];          /* <nbar^k> of the ensemble-averaged neighbour number */
    double  binder;           /* U = 1 - <p^4> / (3 <p^2>^2) (Fig. mfL caption)  */
} aap_results;

typedef struct aap_handle aap_handle;
typedef struct aap_ens aap_ens;

/* Message of the calling thread's last failure ("" if none).  The pointer
 * stays valid until the next call from the same thread. */
const char *aap_last_error(void);

/* ABI version of this header (bumped on any incompatible change). */
int32_t aap_abi_version(void);   /* 2 */

/* Fill *p with this library's defaults: N = 1000, Lx = Ly = 32, R = 1, v = 0.5,
 * eta = 0.4, omega = 0, Gamma = 1, dt = 0.01, seed = 1, VM, order 1,
 * h(n) = 1/(1+n) (the paper's default weight, Sec. 4), periodic on both axes,
 * automatic tiling.  Never fails. */
void aap_params_default(aap_params *p);

/* Create a system: validate *p, allocate device memory, draw the uniform
 * isotropic initial state (positions U(0,L), angles U(-pi,pi); the initial
 * condition of Fig. runtime) from Philox with tag 1, and build the cell lists.
 * Mirrors aappp_init (Sec. 4).  On success *out is a new handle, step = 0.
 * Errors: AAP_EINVAL (parameters, NULL out), AAP_ENOMEM, AAP_ECUDA. */
int aap_create(const aap_params *p, void *stream, aap_handle **out);

/* Free every resource of h (NULL is accepted).  Synchronises h's stream. */
int aap_destroy(aap_handle *h);

/* Advance nsteps >= 0 time steps: for the VM and NVM one collision followed by
 * streaming (Sec. 2.1); for the Langevin model one Euler-Maruyama step of
 * length dt (Sec. 2.2); then the boundary rule of Sec. 2.4.  Every step also
 * measures p and the mean neighbour number on the fly.  Enqueues work; every
 * 128 steps (counted across calls) the device error word is copied, and the
 * call waits for the copy taken 128 steps before, so that tile regions
 * overflowed by growing clusters are enlarged in time (the state is kept bit
 * for bit) while the GPU keeps at least 128 steps queued.
 * Mirrors <model>_update_timesteps (Sec. 4). */
int aap_step(aap_handle *h, int64_t nsteps);

/* Record p(t) for the current state and after each of nsteps steps:
 * phi_out[0..nsteps] (nsteps + 1 host doubles, caller-owned).  Like
 * <model>_measurement_timesteps (Sec. 4), which uses states t = 0..n-1 of the
 * n+1 visited (Sec. 3.4); here all n+1 values are returned. */
int aap_phi_trace(aap_handle *h, int64_t nsteps, double *phi_out);

/* Observables of the current state (Sec. 3.4): p, q, the mean neighbour number
 * measured by the last step, the step count and flags.  Synchronises.
 * Errors: AAP_EOVERFLOW if particles were lost to an overflow, AAP_ENAN if an
 * orientation became non-finite. */
int aap_observe(aap_handle *h, aap_obs *out);

/* Copy the state to host buffers indexed by particle id: x[i], y[i] (FP64,
 * the exact value of the device's fixed-point position) and theta[i] (FP32,
 * in [-pi, pi)).  n must equal N.  Synchronises. */
int aap_get_state(aap_handle *h, double *x, double *y, float *theta, int64_t n);

/* Replace the state by host arrays indexed by particle id (x in [0,Lx],
 * y in [0,Ly], finite theta; n must equal N) and set the step counter, which
 * keys the noise of the next step.  Positions are rounded to the fixed-point
 * grid (2^-fix_bits of a cell side).  Synchronises.  Errors: AAP_EINVAL for
 * positions outside the box or non-finite values (the state is unchanged). */
int aap_set_state(aap_handle *h, const double *x, const double *y, const float *theta,
                  int64_t n, int64_t step);

/* Take one step and write |Omega_i| of the state before it to nbr_out[i]
 * (host, N int32, by particle id).  Synchronises. */
int aap_step_neighbours(aap_handle *h, int32_t *nbr_out, int64_t n);

/* Block until all work enqueued on h has finished; report device-side errors
 * (AAP_EOVERFLOW, AAP_ENAN, AAP_ECUDA). */
int aap_sync(aap_handle *h);

/* Geometry and memory layout of h. */
int aap_get_layout(aap_handle *h, aap_layout *out);

/* Advance nsteps steps measuring on the fly (like
 * <model>_measurement_timesteps, Sec. 4): the states t0 .. t0+nsteps-1 are
 * added to the running sums read by aap_get_results.  Queues and waits like
 * aap_step. */
int aap_measure(aap_handle *h, int64_t nsteps);

/* Normalised measurement results accumulated since creation or the last
 * aap_clear_results (like aappp_get_results, Sec. 4).  Synchronises. */
int aap_get_results(aap_handle *h, aap_results *out);

/* Fault injection for tests: the allocation after n more successful device
 * allocations of any handle fails with AAP_ENOMEM (the library must then
 * release everything it holds); n < 0 switches it off.  Not thread-safe with
 * respect to which call sees the failure. */
int aap_test_fail_alloc_after(int32_t n);

/* Fault injection for tests of the pipelined step kernel's bounded waits
 * (its hand-offs between the copy, sort and update warps are mbarrier waits
 * that give up after a bound; the kernel then sets AAP_ETIMEOUT in the
 * handle's error word, every later step of that handle returns at once, and
 * the handle reports AAP_ETIMEOUT at its next synchronising call).
 * wait_cycles: the bound in SM clock cycles for kernels launched from now on
 * (<= 0: the default, about 2 s).  stall: 1 makes the copy warp of every
 * block withhold the first tile it claims (no copies, no arrival), so that
 * the waits behind it run out; 0 switches it off.  Process-wide; call only
 * while no step kernel is running.  The GPU context stays usable. */
int aap_test_pipe_wait(int64_t wait_cycles, int32_t stall);

/* Forget the accumulated measurements (moments and histograms). */
int aap_clear_results(aap_handle *h);

/* Normalised histograms of the measured states (Sec. 3.4): theta_hist[k] is the
 * fraction of (particle, state) samples with theta in bin k of [-pi, pi)
 * (nt must equal binnum_theta); nbr_hist[k] the fraction with |Omega_i| = k
 * (the last bin: >= nn-1; nn must equal binnum_neighbors).  Either pointer may
 * be NULL.  Synchronises. */
int aap_get_histograms(aap_handle *h, double *theta_hist, int32_t nt, double *nbr_hist, int32_t nn);

/* Save the system to a binary file (Sec. 4: the paper's program can save a
 * simulation and load it later): parameters, step counter, state by particle
 * id and the accumulated measurements (moments and histograms).  Little-endian
 * layout: "AAPSAVE1", u32 version 1, u32 sizeof(aap_params), aap_params,
 * i64 step, i64 N, x[N] f64, y[N] f64, theta[N] f32, 16 f64 sums, i32 bins
 * theta, i32 bins |Omega|, u64 counts.  Synchronises.  AAP_EIO when the file
 * cannot be written. */
int aap_save(aap_handle *h, const char *path);

/* Create a handle from a file written by aap_save, on `stream`: continuing it
 * reproduces the trajectory of the saved handle bit for bit, and aap_get_results
 * / aap_get_histograms keep the saved measurements.  AAP_EIO for a missing,
 * foreign or truncated file; no handle is returned on error. */
int aap_load(const char *path, void *stream, aap_handle **out);

/* Coarse-grained fields of the current state into a caller-owned DEVICE
 * buffer dev_out of 3 * nbx * nby floats (e.g. a torch tensor's data_ptr()):
 * plane 0 the particle density, planes 1 and 2 the polarisation density
 * sum cos theta, sum sin theta, each per unit area of the nbx x nby bins of
 * the box (row-major, x fastest).  Sums are exact 64-bit integer sums, so the
 * fields are reproducible bit for bit.  Runs on h's stream without syncing.
 * The binned density integrates to N and the binned polarisation to
 * sum e^{i theta}, so p (Sec. 3.4) follows from the fields.  nbx, nby >= 1. */
int aap_coarse_grain(aap_handle *h, int32_t nbx, int32_t nby, float *dev_out);

/* Coarse-graining without any device allocation, for callers that cannot
 * allocate: code whose device memory all belongs to a pool or arena, callers
 * that must not call cudaMalloc (it may synchronise the device and is not
 * allowed during stream capture), fixed-budget embedded users.  The paper has
 * no counterpart; this is a library convenience.
 * Same fields as aap_coarse_grain, from caller-owned DEVICE arrays x, y
 * (FP64, in [0,lx] x [0,ly]) and theta (FP32) of n particles, into the
 * caller-owned DEVICE buffer dev_out (3 * nbx * nby floats), on `stream`.
 * Positions are not checked: a coordinate below 0 or NaN is counted in the
 * first bin of its axis, one beyond the box in the last; a non-finite theta
 * adds to the density but not to the polarisation.  lx and ly must be finite
 * and positive (AAP_EINVAL otherwise).
 * The integer sums live in a fixed file-scope device array of 3 x 65,536
 * 64-bit words (1.5 MiB, held by every device that loads the library until
 * the process exits): nbx * nby must not exceed 65,536 (AAP_EINVAL
 * otherwise).  The first call on a device looks up that array's address
 * (cudaGetSymbolAddress), so make it before any stream capture; that address
 * is kept until the process exits and does not survive cudaDeviceReset, after
 * which the entry point must not be called on that device.  All calls
 * share the array, which keeps the last call's sums and is cleared at the
 * start of each call: calls whose work overlaps on the GPU (other streams or
 * threads) race; calls ordered on one stream are safe.  Calls no cudaMalloc
 * or cudaFree.  Messages: aap_noalloc_last_error(). */
int aap_coarse_grain_noalloc(const double *x, const double *y, const float *theta, int64_t n, double lx, double ly,
                             int32_t nbx, int32_t nby, float *dev_out, void *stream);
const char *aap_noalloc_last_error(void);

/* Per-kernel timing (tracing aid).  enable != 0: every step enqueued by
 * aap_step / aap_phi_trace / aap_step_neighbours records CUDA events on h's
 * stream around its two kernels (the tile step and the step finish); the
 * accumulated times restart from zero at each call. */
int aap_set_timing(aap_handle *h, int32_t enable);

/* Milliseconds and launch counts accumulated since aap_set_timing:
 * index 0 the tile step kernel, 1 the finish kernel, 2 reserved (0)
 * (ms[3], launches[3], caller-owned host arrays).  Synchronises. */
int aap_get_timing(aap_handle *h, double *ms, int64_t *launches);

/* ---- batched ensembles ---------------------------------------------------
 * Independent replicas (a phase-diagram sweep) advanced together: every step
 * of all replicas is one launch of the tile kernel over a shared work list of
 * (replica, tile) plus one finish launch, replayed from a captured CUDA graph.
 * Each replica follows exactly the trajectory a standalone handle with the
 * same parameters (and the same tile shape) would: the results are bit for
 * bit identical.  All replicas must use the same model. */

/* Create count >= 1 replicas from params[0..count-1] on `stream`; tile shapes
 * left at 0 follow the ensemble's tiling policy (aap_ens_autotune).
 * Errors: AAP_EINVAL (any invalid replica, mixed models), AAP_ENOMEM,
 * AAP_ECUDA. */
int aap_ens_create(const aap_params *params, int32_t count, void *stream, aap_ens **out);

/* Advance every replica by nsteps steps.  Enqueues work only. */
int aap_ens_step(aap_ens *e, int64_t nsteps);

/* Advance nsteps steps measuring p, q and nbar on the fly for every replica
 * (the window convention of aap_measure).  Enqueues work only. */
int aap_ens_measure(aap_ens *e, int64_t nsteps);

/* Time-averaged polar order <p> of every replica over its measured states
 * (out: count host doubles).  Synchronises. */
int aap_ens_phi_mean(aap_ens *e, double *out);

/* Full measurement results of replica r.  Synchronises. */
int aap_ens_results(aap_ens *e, int32_t r, aap_results *out);

/* State of replica r, as aap_get_state.  Synchronises. */
int aap_ens_get_state(aap_ens *e, int32_t r, double *x, double *y, float *theta, int64_t n);

/* Coarse-grained fields of replica r into a caller-owned DEVICE buffer, as
 * aap_coarse_grain (enqueued on the ensemble's stream, no sync). */
int aap_ens_coarse_grain(aap_ens *e, int32_t r, int32_t nbx, int32_t nby, float *dev_out);

/* Layout of replica r (its tile shape reproduces the replica standalone). */
int aap_ens_get_layout(aap_ens *e, int32_t r, aap_layout *out);

/* Autotuner of block and tile shapes: time trial_steps steps of the whole
 * ensemble under each candidate policy (nominal tile; threads per block for
 * the whole-block kernel),
 * keep the fastest and re-create every replica in its initial state with it.
 * Only allowed before the first step.  *policy_out (may be NULL) receives the
 * chosen policy index; *ms_out (may be NULL, 8 doubles) the trial times in
 * milliseconds per step (0 for policies not tried).  Synchronises. */
int aap_ens_autotune(aap_ens *e, int32_t trial_steps, int32_t *policy_out, double *ms_out);

/* Number of replicas and the current step. */
int aap_ens_info(aap_ens *e, int32_t *count, int64_t *step);

/* Free the ensemble (NULL accepted).  Synchronises its stream. */
int aap_ens_destroy(aap_ens *e);

#ifdef __cplusplus
}
#endif
#endif /* AAP_H */
