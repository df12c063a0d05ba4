// aap_api.cu -- the C ABI declared in include/aap.h.
//
// Host side of one simulated system: parameter checks, geometry and memory
// layout, device allocations, the step loop (optionally replayed from a
// captured CUDA graph), and the transfers in and out of host memory.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/aap.h"
#include "aap_internal.cuh"
#include "aap_kernels.cuh"

using aapk::Ctl;
using aapk::LaunchCfg;
using aapk::Sys;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

// NVTX range around an entry point (tracing; free unless a tool is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

// Test hook: the allocation after g_fail_after more successful ones fails
// (negative: never).  Set through aap_test_fail_alloc_after.
std::atomic<int> g_fail_after{-1};

#define AAP_CK(call)                                                                    \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(AAP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
    return n;
}

}  // namespace

struct aap_handle {
    aap_params p{};
    cudaStream_t stream = nullptr;
    Sys hs{};                       // host copy of the device descriptor
    Sys *d_sys = nullptr;
    int *d_tile_base = nullptr;
    Ctl *d_ctl = nullptr;
    int *d_x0tab = nullptr, *d_y0tab = nullptr;
    unsigned char *d_scratch = nullptr;
    int *d_dense = nullptr;             // pipelined step: tiles left to the whole-block routine
    unsigned long long *d_obs = nullptr;
    int *d_seen = nullptr;
    unsigned long long *d_bad = nullptr;     // [2] first invalid position / orientation of aap_set_state
    double *d_trace = nullptr, *d_trace_nbar = nullptr;
    long long trace_alloc = 0;
    int *d_nbr = nullptr;
    double *d_x = nullptr, *d_y = nullptr;
    float *d_th = nullptr;
    LaunchCfg L{};
    long long step = 0;
    int flags = 0;
    bool broken = false;
    size_t bytes = 0;
    std::vector<void *> allocs;
    int ncx = 0, ncy = 0;
    double csx = 0, csy = 0;
    // captured step graph
    cudaGraphExec_t gexec = nullptr;
    int gsteps = 0;
    // per-kernel timing (aap_set_timing)
    bool timing = false;
    std::vector<cudaEvent_t> events;
    size_t ev_used = 0;
    double ms[3] = {0, 0, 0};
    long long launches[3] = {0, 0, 0};
    // capacity management
    double factor = 4.0;            // region slots over the mean occupancy
    int *pinned_err = nullptr;      // [3]: error word copied after each aap_step; two batch slots
    cudaEvent_t err_event = nullptr;
    cudaEvent_t batch_ev[2] = {nullptr, nullptr};   // error words taken every kAdaptSteps steps
    int batch_prev = -1;            // slot of the newest copy not yet read (-1: none)
    int batch_slot = 0;             // slot of the next copy
    long long since_copy = 0;       // steps queued since the last copy
    bool err_pending = false;
    int relayouts = 0;
    // ensemble membership: steps are launched by the ensemble for all members
    bool member = false;
    int nom_tw = 0, nom_th = 0;     // nominal tile shape actually used
    // coarse-graining accumulator (3 * bins 64-bit sums)
    unsigned long long *d_cg = nullptr;
    long long cg_bins = 0;
    cudaStream_t cap_stream = nullptr;   // private stream for graph capture
};

namespace {

template <typename T>
int dev_alloc(aap_handle *h, T **ptr, size_t bytes)
{
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    int left = g_fail_after.load();
    while (left >= 0 && !g_fail_after.compare_exchange_weak(left, left - 1)) {
    }
    if (left == 0) return fail(AAP_ENOMEM, "injected allocation failure (aap_test_fail_alloc_after)");
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(AAP_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    }
    h->allocs.push_back(p);
    h->bytes += bytes;
    *ptr = static_cast<T *>(p);
    return AAP_OK;
}

void free_all(aap_handle *h)
{
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    h->events.clear();
    if (h->err_event) cudaEventDestroy(h->err_event);
    h->err_event = nullptr;
    for (cudaEvent_t &e : h->batch_ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    if (h->pinned_err) cudaFreeHost(h->pinned_err);
    h->pinned_err = nullptr;
    for (void *p : h->allocs) cudaFree(p);
    h->allocs.clear();
}

bool finite(double v) { return std::isfinite(v); }

int check_params(const aap_params *p)
{
    if (!p) return fail(AAP_EINVAL, "params is NULL");
    if (p->n < 0 || p->n >= (1ll << 31)) return fail(AAP_EINVAL, "n must be in [0, 2^31)");
    if (p->kn < 0 || p->kn > aapk::kMaxKnn) return fail(AAP_EINVAL, "kn must be in [0, 32]");
    if (!finite(p->lx) || !finite(p->ly) || !(p->lx > 0) || !(p->ly > 0))
        return fail(AAP_EINVAL, "lx and ly must be finite and positive");
    if (p->kn > 0) {
        // metric-free (Sec. 2.3): R is not used and may be anything
        if (p->n >= (1ll << 28)) return fail(AAP_EINVAL, "metric-free systems need n < 2^28");
    } else {
        if (!finite(p->r) || !(p->r > 0)) return fail(AAP_EINVAL, "r must be finite and positive");
        if (std::floor(p->lx / p->r) < 3 || std::floor(p->ly / p->r) < 3)
            return fail(AAP_EINVAL, "the box must hold at least 3 cells of side >= R per axis (L >= 3R)");
        if (std::floor(p->lx / p->r) > (1 << 26) || std::floor(p->ly / p->r) > (1 << 26))
            return fail(AAP_EINVAL, "more than 2^26 cells per axis");
    }
    if (!finite(p->v) || p->v < 0) return fail(AAP_EINVAL, "v must be finite and >= 0");
    if (!finite(p->eta) || p->eta < 0) return fail(AAP_EINVAL, "eta must be finite and >= 0");
    if (!finite(p->omega) || !finite(p->gamma)) return fail(AAP_EINVAL, "omega and gamma must be finite");
    if (p->model != AAP_VM && p->model != AAP_LANGEVIN && p->model != AAP_NVM)
        return fail(AAP_EINVAL, "model must be AAP_VM, AAP_LANGEVIN or AAP_NVM");
    if (p->model == AAP_LANGEVIN && (!finite(p->dt) || !(p->dt > 0)))
        return fail(AAP_EINVAL, "dt must be finite and positive for the Langevin model");
    if (p->order < 1 || p->order > 64) return fail(AAP_EINVAL, "order must be in [1, 64]");
    if (p->weight != AAP_H_INV_1PN && p->weight != AAP_H_ONE)
        return fail(AAP_EINVAL, "weight must be AAP_H_INV_1PN or AAP_H_ONE");
    double vmax = p->v;
    if (p->nspecies < 0 || p->nspecies > aapk::kMaxSpecies) return fail(AAP_EINVAL, "nspecies must be in [0, 8]");
    if (p->nspecies > 1) {
        long long tot = 0;
        vmax = 0.0;
        for (int a = 0; a < p->nspecies; ++a) {
            if (p->species_n[a] < 0) return fail(AAP_EINVAL, "species_n must be >= 0");
            tot += p->species_n[a];
            if (!finite(p->species_v[a]) || p->species_v[a] < 0 || !finite(p->species_eta[a]) ||
                p->species_eta[a] < 0 || !finite(p->species_omega[a]))
                return fail(AAP_EINVAL, "species_v and species_eta must be finite and >= 0, species_omega finite");
            for (int b = 0; b < p->nspecies; ++b)
                if (!finite(p->species_gamma[8 * a + b])) return fail(AAP_EINVAL, "species_gamma must be finite");
            vmax = std::max(vmax, p->species_v[a]);
        }
        if (tot != p->n) return fail(AAP_EINVAL, "species_n must add up to n");
    }
    const double disp = p->model == AAP_LANGEVIN ? vmax * p->dt : vmax;
    if (p->kn > 0) {
        if (disp > 0.25 * std::min(p->lx, p->ly))
            return fail(AAP_EINVAL, "the displacement per step (v, or v*dt) must not exceed a quarter of the box");
    } else {
        const double cs = std::min(p->lx / std::floor(p->lx / p->r), p->ly / std::floor(p->ly / p->r));
        if (disp > cs)
            return fail(AAP_EINVAL, "the displacement per step (v, or v*dt) must not exceed one cell side");
    }
    if (p->tile_w < 0 || p->tile_h < 0 || p->tile_w > aapk::kMaxTile || p->tile_h > aapk::kMaxTile)
        return fail(AAP_EINVAL, "tile_w and tile_h must be 0 (automatic) or in [6, 64]");
    if ((p->tile_w && p->tile_w < 6) || (p->tile_h && p->tile_h < 6))
        return fail(AAP_EINVAL, "tile_w and tile_h must be 0 (automatic) or in [6, 64]");
    if (p->threads != 0 && p->threads != 256 && p->threads != 512 && p->threads != 1024)
        return fail(AAP_EINVAL, "threads must be 0, 256, 512 or 1024");
    if (p->threads == 1024 && (p->nspecies > 1 || p->kn > 0))
        return fail(AAP_EINVAL, "threads = 1024 (the pipelined step) needs one species and a metric neighbourhood");
    if (!finite(p->capacity) || p->capacity < 0 || (p->capacity > 0 && p->capacity < 1))
        return fail(AAP_EINVAL, "capacity must be 0 (automatic) or >= 1");
    if (p->weight_len < 0 || p->weight_len > 128) return fail(AAP_EINVAL, "weight_len must be in [0, 128]");
    for (int k = 0; k < p->weight_len; ++k)
        if (!finite(p->weight_table[k])) return fail(AAP_EINVAL, "weight_table must be finite");
    if (p->binnum_theta < 0 || p->binnum_theta > aapk::kMaxBins || p->binnum_neighbors < 0 ||
        p->binnum_neighbors > aapk::kMaxBins)
        return fail(AAP_EINVAL, "binnum_theta and binnum_neighbors must be in [0, 512]");
    return AAP_OK;
}

int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

int fix_bits(int wmax)
{
    int s = 0;
    while (((long long)(wmax + 2) << (s + 1)) <= 2147483647ll && s < 28) ++s;
    return s;
}

// Region capacities and the per-tile layout.
void layout_regions(Sys &S, double mu, double factor)
{
    const int wi = std::max(S.twmax - 2, 1), hi = std::max(S.thmax - 2, 1);
    int cells[aapk::kRegions];
    for (int ry = 0; ry < 3; ++ry)
        for (int rx = 0; rx < 3; ++rx) {
            const int cw = rx == 1 ? wi : 1, ch = ry == 1 ? hi : 1;
            cells[ry * 3 + rx] = cw * ch;
        }
    int off = 0;
    for (int r = 0; r < aapk::kRegions; ++r) {
        const double want = factor * mu * cells[r] + 4.0 * std::sqrt(mu * cells[r] + 1.0) + 24.0;
        const int cap = aapk::round_up((int)std::ceil(want), 4);
        S.cap[r] = cap;
        S.off[r] = off;
        off += cap;
    }
    S.tile_slots = aapk::round_up(off, 4);
}

// Whether regions sized by `factor` keep a tile's staged set (own slots, the
// facing halo regions, the spill matches) within the 16-bit staged indices.
bool capacity_fits(const aap_handle *h, double factor)
{
    if (h->p.kn > 0) return true;
    Sys S = h->hs;
    layout_regions(S, (double)h->p.n / ((double)S.ncx * S.ncy), factor);
    const long long spill_cap = std::max<long long>(4096, h->p.n / 8);
    const long long own = S.tile_slots;
    const long long halo = 2 * (2 * S.cap[0] + S.cap[1]) + 2 * (2 * S.cap[0] + S.cap[3]) + 4 * S.cap[0];
    return own + halo + std::min<long long>(16384, 4 * spill_cap) <= 65472;
}

// Region capacities, spill list, staging capacities and launch shapes for a
// capacity factor (slots per region over the mean occupancy).
// Metric-free layout: one tile over the box, every record in region 0.
int set_capacity_mf(aap_handle *h)
{
    const aap_params &p = h->p;
    Sys &S = h->hs;
    S.cap[0] = aapk::round_up((int)std::max<long long>(p.n, 1), 4);
    S.off[0] = 0;
    for (int r = 1; r < aapk::kRegions; ++r) {
        S.cap[r] = 0;
        S.off[r] = S.cap[0];
    }
    S.tile_slots = S.cap[0];
    S.spill_cap = 64;
    LaunchCfg &L = h->L;
    L.spill_list_cap = 0;
    L.scratch_cap = 0;
    L.scratch_per_block = 0;
    L.threads = 256;
    L.pipe = 0;
    L.model = p.model;
    L.stage_cap = 0;
    L.nce_max = 0;
    L.hist_words = (p.binnum_theta ? p.binnum_theta : 100) + (p.binnum_neighbors ? p.binnum_neighbors : 100);
    L.grid_step = 0;
    L.grid_finish = 1;
    L.nsys = 1;
    L.knn = p.kn;
    L.mf_n = p.n;
    L.mf_ncell = (long long)S.ncx * S.ncy;
    AAP_CK(aapk::configure_mf_kernels(p.model, p.kn, L.hist_words, sm_count(), &L.mf_grid));
    return AAP_OK;
}

// Shared buffers of the pipelined step: the largest staging capacity (a
// multiple of 64, at most kPipeMaxStage) whose two raw and two sorted buffers,
// with own lists sized for 7/8 of it, fit the block's shared memory.
int set_pipe_launch(LaunchCfg &L, int twmax, int thmax, int total_tiles)
{
    int dev = 0, optin = 0;
    AAP_CK(cudaGetDevice(&dev));
    AAP_CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    size_t stat = 0;
    AAP_CK(aapk::pipe_static_smem(L.model, &stat));
    int cap = aapk::kPipeMaxStage;
    auto own_of = [](int c) { return aapk::round_up(c * 7 / 8, 64); };
    L.pipe_nceh = (2 * twmax + 4) * (thmax + 2);
    while (cap >= 256 && aapk::pipe_smem_bytes(cap, own_of(cap), L.pipe_nceh, L.hist_words) + stat > (size_t)optin)
        cap -= 64;
    if (cap < 256) return AAP_OK;
    // the whole-block routine for oversized tiles reuses the same shared memory
    if (aapk::step_smem_bytes(256, L.nce_max, L.hist_words) >
        aapk::pipe_smem_bytes(cap, own_of(cap), L.pipe_nceh, L.hist_words))
        return AAP_OK;
    L.pipe_cap = cap;
    L.pipe_cap_own = own_of(cap);
    L.pipe_grid = std::max(1, std::min(total_tiles, sm_count()));
    AAP_CK(aapk::configure_pipe_kernel(L.model, aapk::pipe_smem_bytes(L.pipe_cap, L.pipe_cap_own, L.pipe_nceh,
                                                                      L.hist_words)));
    L.pipe = 1;
    L.threads = 1024;
    return AAP_OK;
}

int set_pipe(aap_handle *h) { return set_pipe_launch(h->L, h->hs.twmax, h->hs.thmax, h->hs.ntiles); }

int set_capacity(aap_handle *h, double factor)
{
    if (h->p.kn > 0) return set_capacity_mf(h);
    const aap_params &p = h->p;
    Sys &S = h->hs;
    const int nsm = sm_count();
    const double mu = (double)p.n / ((double)S.ncx * S.ncy);
    layout_regions(S, mu, factor);
    // every particle beyond its region's slots goes to the spill list; it is
    // sized for an eighth of the particles so that a step never loses one
    S.spill_cap = (int)std::max<long long>(4096, p.n / 8);
    // shared-memory staging capacity: about twice the mean tile + ring load
    const int nce = (S.twmax + 2) * (S.thmax + 2);
    const double mean_stage = mu * nce;
    int scap = aapk::round_up((int)std::ceil(1.85 * mean_stage + 128.0), 64);
    scap = std::min(scap, 4096);
    const int own = S.tile_slots;
    const int halo = 2 * (2 * S.cap[0] + S.cap[1]) + 2 * (2 * S.cap[0] + S.cap[3]) + 4 * S.cap[0];
    LaunchCfg &L = h->L;
    L.spill_list_cap = (int)std::min<long long>(16384, 4ll * S.spill_cap);
    if ((long long)own + halo + L.spill_list_cap > 65472)
        return fail(AAP_EINVAL, "tile capacity too large (reduce tile size or capacity)");
    L.scratch_cap = aapk::round_up(own + halo + L.spill_list_cap, 64);
    L.threads = p.threads == 1024 ? 512 : (p.threads ? p.threads : 512);
    L.model = p.model;
    L.stage_cap = scap;
    L.nce_max = nce;
    L.hist_words = (p.binnum_theta ? p.binnum_theta : 100) + (p.binnum_neighbors ? p.binnum_neighbors : 100);
    const size_t smem = aapk::step_smem_bytes(scap, nce, L.hist_words);
    int bps = 0;
    AAP_CK(aapk::configure_step_kernel(L.model, L.threads, smem, &bps));
    if (bps < 1) return fail(AAP_EINVAL, "step kernel does not fit on an SM with this tiling");
    L.grid_step = std::max(1, std::min(S.ntiles, bps * nsm));
    L.grid_finish = std::max(1, std::min(64, ceil_div((long long)S.ntiles * (aapk::kCntStride / 4), 1024)));
    L.scratch_per_block = aapk::stage_bytes(L.scratch_cap) + aapk::spill_list_bytes(L.spill_list_cap);
    L.scratch_per_block = (L.scratch_per_block + 255) / 256 * 256;
    L.nsys = 1;
    // the pipelined step: one system, one species (ensemble members use the
    // whole-block kernel, which batches systems)
    L.pipe = 0;
    if (!h->member && p.nspecies <= 1 && (p.threads == 0 || p.threads == 1024)) {
        int rc = set_pipe(h);
        if (rc) return rc;
        if (!L.pipe && p.threads == 1024) return fail(AAP_EINVAL, "the pipelined step kernel does not fit this tiling");
    }
    return AAP_OK;
}

void set_model(Sys &S, const aap_params &p)
{
    S.model = p.model;
    S.order = p.model == AAP_LANGEVIN ? p.order : 1;
    S.weight = p.kn > 0 ? AAP_H_ONE : p.weight;       // metric-free: h = 1 (Sec. 2.3)
    S.bx = p.bx != 0;
    S.by = p.by != 0;
    S.eta_pi = (float)(p.eta * M_PI);
    S.omega_step = (float)(p.model == AAP_LANGEVIN ? p.omega * p.dt : p.omega);
    S.gamma_dt = (float)(p.gamma * p.dt);
    S.noise_amp = (float)(p.eta * std::sqrt(p.dt));
    S.seed_lo = (uint32_t)p.seed;
    S.seed_hi = (uint32_t)(p.seed >> 32);
    S.n = p.n;
    // tabulated weight (Sec. 4); metric-free models use h = 1 (Sec. 2.3)
    S.wlen = p.kn > 0 ? 0 : p.weight_len;
    for (int k = 0; k < 128; ++k) S.wtab[k] = k < S.wlen ? (float)p.weight_table[k] : 0.f;
    // species (Sec. 2.5); entry 0 repeats the scalars with a single species
    const bool multi = p.nspecies > 1;
    S.nsp = multi ? p.nspecies : 1;
    long long end = 0;
    for (int a = 0; a < aapk::kMaxSpecies; ++a) {
        end += (multi && a < p.nspecies) ? p.species_n[a] : 0;
        S.sp_end[a] = multi ? end : p.n;
        const double eta = multi ? p.species_eta[a] : p.eta, om = multi ? p.species_omega[a] : p.omega;
        S.sp_eta_pi[a] = (float)(eta * M_PI);
        S.sp_omega_step[a] = (float)(p.model == AAP_LANGEVIN ? om * p.dt : om);
        S.sp_noise_amp[a] = (float)(eta * std::sqrt(p.dt));
        for (int b = 0; b < aapk::kMaxSpecies; ++b)
            S.sp_gamma_dt[a * aapk::kMaxSpecies + b] = (float)((multi ? p.species_gamma[8 * a + b] : p.gamma) * p.dt);
    }
    if (!multi) {
        S.sp_eta_pi[0] = S.eta_pi;
        S.sp_omega_step[0] = S.omega_step;
        S.sp_noise_amp[0] = S.noise_amp;
    }
}

// Displacement per step of each species in fixed-point units (after the
// geometry is known); entry 0 repeats kx, ky with a single species.
void set_species_kinematics(Sys &S, const aap_params &p)
{
    for (int a = 0; a < aapk::kMaxSpecies; ++a) {
        const double v = p.nspecies > 1 ? p.species_v[a] : p.v;
        const double disp = p.model == AAP_LANGEVIN ? v * p.dt : v;
        S.sp_kx[a] = (float)(disp / S.csx_d * (double)(1ll << S.sx));
        S.sp_ky[a] = (float)(disp / S.csy_d * (double)(1ll << S.sy));
    }
    if (p.nspecies <= 1) {
        S.sp_kx[0] = S.kx;
        S.sp_ky[0] = S.ky;
    }
}

// Cell side of the metric-free search over R_eff.  The result does not
// depend on it (the search is exact for any cell size); it only trades the
// number of rings against the particles per cell.
#ifndef AAP_MF_CELL_FACTOR
#define AAP_MF_CELL_FACTOR 1.0
#endif

// Metric-free geometry (Sec. 3.3): cells of side about
// R_eff = sqrt(Lx Ly k / (N pi)) (Eq. effective_radius), one flat tile.
int build_layout_mf(aap_handle *h)
{
    const aap_params &p = h->p;
    Sys &S = h->hs;
    const double reff = AAP_MF_CELL_FACTOR *
                        (p.n > 0 ? std::sqrt(p.lx * p.ly * p.kn / ((double)p.n * M_PI)) : std::max(p.lx, p.ly));
    h->ncx = (int)std::max(1.0, std::min(std::floor(p.lx / reff), (double)(1 << 24)));
    h->ncy = (int)std::max(1.0, std::min(std::floor(p.ly / reff), (double)(1 << 24)));
    if ((long long)h->ncx * h->ncy >= (1ll << 30)) return fail(AAP_EINVAL, "too many metric-free cells");
    h->csx = p.lx / h->ncx;
    h->csy = p.ly / h->ncy;
    S.ncx = h->ncx;
    S.ncy = h->ncy;
    S.ntx = S.nty = 1;
    S.twmax = S.ncx;
    S.thmax = S.ncy;
    S.ntiles = 1;
    S.sx = fix_bits(2 * S.ncx);      // twice the box fits int32: exact image coordinates
    S.sy = fix_bits(2 * S.ncy);
    S.lx = p.lx;
    S.ly = p.ly;
    S.csx_d = h->csx;
    S.csy_d = h->csy;
    S.ux = (float)(h->csx / (double)(1ll << S.sx));
    S.uy = (float)(h->csy / (double)(1ll << S.sy));
    const double disp = p.model == AAP_LANGEVIN ? p.v * p.dt : p.v;
    S.kx = (float)(disp / h->csx * (double)(1ll << S.sx));
    S.ky = (float)(disp / h->csy * (double)(1ll << S.sy));
    S.r2 = 0.f;
    set_model(S, p);
    set_species_kinematics(S, p);
    S.flat = 1;
    S.knn = p.kn;
    h->factor = 1.0;
    return set_capacity_mf(h);
}

int build_layout(aap_handle *h)
{
    if (h->p.kn > 0) return build_layout_mf(h);
    const aap_params &p = h->p;
    Sys &S = h->hs;
    h->ncx = (int)std::floor(p.lx / p.r);
    h->ncy = (int)std::floor(p.ly / p.r);
    h->csx = p.lx / h->ncx;
    h->csy = p.ly / h->ncy;
    S.ncx = h->ncx;
    S.ncy = h->ncy;
    const int nsm = sm_count();
    int tw = p.tile_w ? p.tile_w : (h->nom_tw ? h->nom_tw : 32);
    int th = p.tile_h ? p.tile_h : (h->nom_th ? h->nom_th : 16);
    if (!p.tile_w && !p.tile_h && !h->member) {
        // small systems: shrink tiles until there are a few per SM
        while ((long long)ceil_div(S.ncx, tw) * ceil_div(S.ncy, th) < 2ll * nsm && (tw > 8 || th > 8)) {
            if (tw >= th && tw > 8) tw /= 2; else if (th > 8) th /= 2; else break;
        }
    }
    h->nom_tw = tw;
    h->nom_th = th;
    S.ntx = ceil_div(S.ncx, std::min(tw, S.ncx));
    S.nty = ceil_div(S.ncy, std::min(th, S.ncy));
    S.twmax = ceil_div(S.ncx, S.ntx);
    S.thmax = ceil_div(S.ncy, S.nty);
    if (S.twmax > aapk::kMaxTile || S.thmax > aapk::kMaxTile)
        return fail(AAP_EINVAL, "tile larger than 64 cells");
    if ((long long)S.ntx * S.nty >= (1ll << 27)) return fail(AAP_EINVAL, "too many tiles");
    S.ntiles = S.ntx * S.nty;
    S.sx = fix_bits(S.twmax);
    S.sy = fix_bits(S.thmax);
    S.lx = p.lx;
    S.ly = p.ly;
    S.csx_d = h->csx;
    S.csy_d = h->csy;
    S.ux = (float)(h->csx / (double)(1ll << S.sx));
    S.uy = (float)(h->csy / (double)(1ll << S.sy));
    const double disp = p.model == AAP_LANGEVIN ? p.v * p.dt : p.v;
    S.kx = (float)(disp / h->csx * (double)(1ll << S.sx));
    S.ky = (float)(disp / h->csy * (double)(1ll << S.sy));
    S.r2 = (float)(p.r * p.r);
    set_model(S, p);
    set_species_kinematics(S, p);
    h->factor = p.capacity > 0 ? p.capacity : 4.0;
    return set_capacity(h, h->factor);
}

int push_sys(aap_handle *h)
{
    AAP_CK(cudaMemcpyAsync(h->d_sys, &h->hs, sizeof(Sys), cudaMemcpyHostToDevice, h->stream));
    return AAP_OK;
}

int dev_free(aap_handle *h, void *p, size_t bytes)
{
    if (!p) return AAP_OK;
    for (size_t i = 0; i < h->allocs.size(); ++i)
        if (h->allocs[i] == p) {
            h->allocs.erase(h->allocs.begin() + (long)i);
            break;
        }
    h->bytes -= std::min(h->bytes, bytes);
    AAP_CK(cudaFree(p));
    return AAP_OK;
}

size_t region_bytes(const Sys &S) { return (size_t)S.ntiles * S.tile_slots * sizeof(int4); }
size_t spill_bits_bytes(const Sys &S) { return (size_t)(S.ntiles / 32 + 1) * sizeof(unsigned); }

// Buffers whose size depends on the capacity factor.
int alloc_regions(aap_handle *h)
{
    Sys &S = h->hs;
    int rc;
    for (int b = 0; b < 2; ++b) {
        if ((rc = dev_alloc(h, &S.rec[b], region_bytes(S)))) return rc;
        if ((rc = dev_alloc(h, &S.spill_rec[b], (size_t)S.spill_cap * sizeof(int4)))) return rc;
        if ((rc = dev_alloc(h, &S.spill_key[b], (size_t)S.spill_cap * sizeof(int)))) return rc;
    }
    if (!h->member) {
        if ((rc = dev_alloc(h, &h->d_scratch, h->L.scratch_per_block * h->L.grid_step))) return rc;
        h->L.scratch = h->d_scratch;
    }
    return AAP_OK;
}

int free_regions(aap_handle *h)
{
    Sys &S = h->hs;
    int rc;
    for (int b = 0; b < 2; ++b) {
        if ((rc = dev_free(h, S.rec[b], region_bytes(S)))) return rc;
        if ((rc = dev_free(h, S.spill_rec[b], (size_t)S.spill_cap * sizeof(int4)))) return rc;
        if ((rc = dev_free(h, S.spill_key[b], (size_t)S.spill_cap * sizeof(int)))) return rc;
        S.rec[b] = nullptr;
        S.spill_rec[b] = nullptr;
        S.spill_key[b] = nullptr;
    }
    if (h->member) return AAP_OK;
    rc = dev_free(h, h->d_scratch, h->L.scratch_per_block * h->L.grid_step);
    h->d_scratch = nullptr;
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    return rc;
}

// Clear both buffers' counters, the spill counts, the step sums and errors.
int clear_buffers(aap_handle *h)
{
    Sys &S = h->hs;
    h->batch_prev = -1;
    h->batch_slot = 0;
    h->since_copy = 0;
    for (int b = 0; b < 2; ++b)
        AAP_CK(cudaMemsetAsync(S.cnt[b], 0, (size_t)S.ntiles * aapk::kCntStride * sizeof(int), h->stream));
    AAP_CK(cudaMemsetAsync(S.spill_cnt, 0, 2 * sizeof(int), h->stream));
    for (int b = 0; b < 2; ++b)
        AAP_CK(cudaMemsetAsync(S.spill_bits[b], 0, spill_bits_bytes(S), h->stream));
    AAP_CK(cudaMemsetAsync(S.acc, 0, 2 * aapk::kAccSlots * aapk::kAccWords * sizeof(unsigned long long), h->stream));
    AAP_CK(cudaMemsetAsync(S.err, 0, sizeof(int), h->stream));
    return AAP_OK;
}

int alloc_all(aap_handle *h)
{
    Sys &S = h->hs;
    int rc;
    for (int b = 0; b < 2; ++b)
        if ((rc = dev_alloc(h, &S.cnt[b], (size_t)S.ntiles * aapk::kCntStride * sizeof(int)))) return rc;
    if ((rc = alloc_regions(h))) return rc;
    if ((rc = dev_alloc(h, &S.spill_cnt, 2 * sizeof(int)))) return rc;
    for (int b = 0; b < 2; ++b)
        if ((rc = dev_alloc(h, &S.spill_bits[b], spill_bits_bytes(S)))) return rc;
    if ((rc = dev_alloc(h, &S.acc, 2 * aapk::kAccSlots * aapk::kAccWords * sizeof(unsigned long long)))) return rc;
    if ((rc = dev_alloc(h, &S.last, 4 * sizeof(double)))) return rc;
    if ((rc = dev_alloc(h, &S.stats, 16 * sizeof(double)))) return rc;
    S.bins_theta = h->p.binnum_theta ? h->p.binnum_theta : 100;     // theta + |Omega| bins = L.hist_words
    S.bins_nbr = h->p.binnum_neighbors ? h->p.binnum_neighbors : 100;
    if ((rc = dev_alloc(h, &S.hist, (size_t)(S.bins_theta + S.bins_nbr) * sizeof(unsigned long long)))) return rc;
    if ((rc = dev_alloc(h, &S.err, sizeof(int)))) return rc;
    if (S.knn > 0) {
        const long long ncell = (long long)S.ncx * S.ncy;
        const long long nchunk = (ncell + 1 + aapk::kScanChunk - 1) / aapk::kScanChunk;
        const size_t n = (size_t)std::max<long long>(h->p.n, 1);
        if ((rc = dev_alloc(h, &S.mf_cnt, (size_t)ncell * sizeof(int)))) return rc;
        if ((rc = dev_alloc(h, &S.mf_start, (size_t)(ncell + 1) * sizeof(int)))) return rc;
        if ((rc = dev_alloc(h, &S.mf_blk, (size_t)(nchunk + 1) * sizeof(int)))) return rc;
        if ((rc = dev_alloc(h, &S.mf_cs, n * sizeof(int2)))) return rc;
        if ((rc = dev_alloc(h, &S.mf_sorted, n * sizeof(int4)))) return rc;
        if ((rc = dev_alloc(h, &S.mf_fix, n * sizeof(int2)))) return rc;
        if ((rc = dev_alloc(h, &S.mf_nfix, 2 * sizeof(int)))) return rc;
        AAP_CK(cudaMemsetAsync(S.mf_nfix, 0, 2 * sizeof(int), h->stream));
        AAP_CK(cudaMemsetAsync(S.mf_cnt, 0, (size_t)ncell * sizeof(int), h->stream));
    }
    if (!h->member) {
        if ((rc = dev_alloc(h, &h->d_sys, sizeof(Sys)))) return rc;
        if ((rc = dev_alloc(h, &h->d_tile_base, 2 * sizeof(int)))) return rc;
        if ((rc = dev_alloc(h, &h->d_ctl, sizeof(Ctl)))) return rc;
        if ((rc = dev_alloc(h, &h->d_dense, (size_t)std::max(S.ntiles, 1) * sizeof(int)))) return rc;
        AAP_CK(cudaMemsetAsync(h->d_dense, 0, (size_t)std::max(S.ntiles, 1) * sizeof(int), h->stream));
    }
    if ((rc = dev_alloc(h, &h->d_x0tab, (size_t)(S.ntx + 1) * sizeof(int)))) return rc;
    if ((rc = dev_alloc(h, &h->d_y0tab, (size_t)(S.nty + 1) * sizeof(int)))) return rc;
    {
        std::vector<int> xt(S.ntx + 1), yt(S.nty + 1);
        for (int t = 0; t <= S.ntx; ++t) xt[t] = (int)((long long)t * S.ncx / S.ntx);
        for (int t = 0; t <= S.nty; ++t) yt[t] = (int)((long long)t * S.ncy / S.nty);
        AAP_CK(cudaMemcpy(h->d_x0tab, xt.data(), xt.size() * sizeof(int), cudaMemcpyHostToDevice));
        AAP_CK(cudaMemcpy(h->d_y0tab, yt.data(), yt.size() * sizeof(int), cudaMemcpyHostToDevice));
        S.x0tab = h->d_x0tab;
        S.y0tab = h->d_y0tab;
    }
    if ((rc = dev_alloc(h, &h->d_obs, 8 * sizeof(unsigned long long)))) return rc;
    if ((rc = dev_alloc(h, &h->d_seen, sizeof(int)))) return rc;
    AAP_CK(cudaMallocHost(&h->pinned_err, 3 * sizeof(int)));
    AAP_CK(cudaEventCreateWithFlags(&h->err_event, cudaEventDisableTiming));
    for (cudaEvent_t &e : h->batch_ev) AAP_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if ((rc = clear_buffers(h))) return rc;
    AAP_CK(cudaMemsetAsync(S.last, 0, 4 * sizeof(double), h->stream));
    AAP_CK(cudaMemsetAsync(S.stats, 0, 16 * sizeof(double), h->stream));
    AAP_CK(cudaMemsetAsync(S.hist, 0, (size_t)(S.bins_theta + S.bins_nbr) * sizeof(unsigned long long), h->stream));
    S.meas_until = 0;
    if (!h->member) {
        AAP_CK(cudaMemsetAsync(h->d_ctl, 0, sizeof(Ctl), h->stream));
        int tb[2] = {0, S.ntiles};
        AAP_CK(cudaMemcpyAsync(h->d_tile_base, tb, sizeof(tb), cudaMemcpyHostToDevice, h->stream));
    }
    AAP_CK(cudaStreamSynchronize(h->stream));
    LaunchCfg &L = h->L;
    L.sys = h->d_sys;
    L.tile_base = h->d_tile_base;
    L.ctl = h->d_ctl;
    L.dense_list = h->d_dense;
    return push_sys(h);
}

// Read and clear nothing: map the sticky device error word to a status.
int read_errors(aap_handle *h)
{
    int err = 0;
    AAP_CK(cudaMemcpyAsync(&err, h->hs.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    AAP_CK(cudaStreamSynchronize(h->stream));
    if (err & aapk::ERR_SPILL) h->flags |= AAP_FLAG_SPILLED;
    if (err & (aapk::ERR_LOST | aapk::ERR_STAGE)) {
        h->broken = true;
        return fail(AAP_EOVERFLOW, "particles were lost: a tile overflowed its spill capacity "
                                   "(increase aap_params.capacity)");
    }
    if (err & aapk::ERR_BOUNDS) {
        h->broken = true;
        return fail(AAP_ESTATE, "a particle record decoded outside its tile (internal fault)");
    }
    if (err & aapk::ERR_TIMEOUT) {
        h->broken = true;
        return fail(AAP_ETIMEOUT, "a bounded wait of the pipelined step kernel ran out");
    }
    if (err & aapk::ERR_NAN) return fail(AAP_ENAN, "a non-finite orientation was produced");
    return AAP_OK;
}

// Fold the durations of recorded timing events into h->ms.
int resolve_timing(aap_handle *h)
{
    if (h->ev_used == 0) return AAP_OK;
    AAP_CK(cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i + 2 < h->ev_used; i += 3) {
        for (int k = 0; k < 2; ++k) {
            float t = 0.f;
            AAP_CK(cudaEventElapsedTime(&t, h->events[i + k], h->events[i + k + 1]));
            h->ms[k] += t;
            h->launches[k] += 1;
        }
    }
    h->ev_used = 0;
    return AAP_OK;
}

constexpr int kGraphSteps = 32;

// Capture kGraphSteps steps of L into an executable graph (on a private
// stream, so any caller stream works, the legacy default one included).
int capture_steps(const LaunchCfg &L, cudaStream_t &cap, cudaGraphExec_t &exec)
{
    if (!cap) AAP_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    AAP_CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < kGraphSteps && e == cudaSuccess; ++i) e = aapk::launch_step(L, cap);
    cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(AAP_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(AAP_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return AAP_OK;
}

// nsteps steps of L on stream st: whole chunks replay the captured graph (the
// step index and buffer parity live on the device, so one graph serves every
// chunk), the rest launch directly.
int launch_steps(const LaunchCfg &L, cudaStream_t st, long long nsteps, cudaStream_t &cap,
                 cudaGraphExec_t &exec)
{
    long long done = 0;
    if (nsteps >= kGraphSteps) {
        if (!exec) {
            int rc = capture_steps(L, cap, exec);
            if (rc) return rc;
        }
        for (; done + kGraphSteps <= nsteps; done += kGraphSteps) AAP_CK(cudaGraphLaunch(exec, st));
    }
    for (; done < nsteps; ++done) AAP_CK(aapk::launch_step(L, st));
    return AAP_OK;
}

int run_steps(aap_handle *h, long long nsteps);
int act_on_error(aap_handle *h, int err, bool *relaid);

// Steps between capacity checks inside one long call.
constexpr long long kAdaptSteps = 32;

// nsteps steps, with the device error word copied to the host after every
// kAdaptSteps steps (counted across calls).  When a copy is taken the host
// waits for the one before it (kAdaptSteps older, so the GPU still has that
// many steps queued) and reads it: regions overflowed by growing clusters are
// then re-laid out within a long call, or within a loop of short calls,
// before the spill list that absorbs the overflow fills up (and every tile
// scans it meanwhile).  A re-layout keeps the state bit for bit.
int run_steps_adaptive(aap_handle *h, long long nsteps)
{
    int rc;
    long long left = nsteps;
    while (left > 0) {
        const long long k = std::min(left, kAdaptSteps - h->since_copy);
        if ((rc = run_steps(h, k))) return rc;
        left -= k;
        h->since_copy += k;
        if (h->since_copy < kAdaptSteps) continue;
        h->since_copy = 0;
        const int slot = h->batch_slot;
        AAP_CK(cudaMemcpyAsync(h->pinned_err + 1 + slot, h->hs.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        AAP_CK(cudaEventRecord(h->batch_ev[slot], h->stream));
        h->batch_slot ^= 1;
        const int prev = h->batch_prev;
        h->batch_prev = slot;
        if (prev >= 0) {
            AAP_CK(cudaEventSynchronize(h->batch_ev[prev]));
            // a re-layout resets the copies (the newer one predates it)
            if ((rc = act_on_error(h, h->pinned_err[1 + prev], nullptr))) return rc;
        }
    }
    return AAP_OK;
}

int run_steps(aap_handle *h, long long nsteps)
{
    if (!h->timing) {
        int rc = launch_steps(h->L, h->stream, nsteps, h->cap_stream, h->gexec);
        if (rc) return rc;
        h->step += nsteps;
        return AAP_OK;
    }
    for (long long i = 0; i < nsteps; ++i) {
        cudaEvent_t *ev = nullptr;
        if (h->ev_used + 3 > 3072) {
            int rc = resolve_timing(h);
            if (rc) return rc;
        }
        while (h->events.size() < h->ev_used + 3) {
            cudaEvent_t e;
            AAP_CK(cudaEventCreate(&e));
            h->events.push_back(e);
        }
        ev = &h->events[h->ev_used];
        h->ev_used += 3;
        AAP_CK(aapk::launch_step(h->L, h->stream, ev));
    }
    h->step += nsteps;
    return AAP_OK;
}

int ensure_xfer(aap_handle *h)
{
    int rc;
    if (!h->d_x) {
        const size_t n = (size_t)std::max<long long>(h->p.n, 1);
        if ((rc = dev_alloc(h, &h->d_x, n * sizeof(double)))) return rc;
        if ((rc = dev_alloc(h, &h->d_y, n * sizeof(double)))) return rc;
        if ((rc = dev_alloc(h, &h->d_th, n * sizeof(float)))) return rc;
    }
    return AAP_OK;
}

// Put the particles back into freshly sized regions.  mode 0: from the flat
// device arrays d_x, d_y, d_th; mode 1: the Philox initial state.  With an
// automatic capacity the factor doubles until nothing spills; with an explicit
// one spilled particles are kept (exactly) in the spill list.
int reinsert(aap_handle *h, double factor, int mode)
{
    int rc;
    for (int attempt = 0; attempt < 12; ++attempt) {
        // new layout; the buffers are kept when their sizes do not change
        // (aap_set_state, aap_load at the same capacity), else replaced
        const Sys old_s = h->hs;
        const LaunchCfg old_l = h->L;
        if ((rc = set_capacity(h, factor))) {
            h->hs = old_s;
            h->L = old_l;
            return rc;
        }
        const bool same = old_s.rec[0] && region_bytes(old_s) == region_bytes(h->hs) &&
                          old_s.spill_cap == h->hs.spill_cap &&
                          (h->member || old_l.scratch_per_block * old_l.grid_step ==
                                            h->L.scratch_per_block * h->L.grid_step);
        if (h->gexec) {
            cudaGraphExecDestroy(h->gexec);
            h->gexec = nullptr;
        }
        if (!same) {
            Sys new_s = h->hs;
            LaunchCfg new_l = h->L;
            h->hs = old_s;
            h->L = old_l;
            if ((rc = free_regions(h))) return rc;      // the old buffers, with their sizes
            for (int b = 0; b < 2; ++b) {
                new_s.rec[b] = nullptr;
                new_s.spill_rec[b] = nullptr;
                new_s.spill_key[b] = nullptr;
            }
            h->hs = new_s;
            h->L = new_l;
            if ((rc = alloc_regions(h))) return rc;
        }
        if ((rc = clear_buffers(h))) return rc;
        if ((rc = push_sys(h))) return rc;
        AAP_CK(aapk::launch_insert(h->hs, (int)(h->step & 1), h->d_x, h->d_y, h->d_th, mode, h->stream));
        int err = 0;
        AAP_CK(cudaMemcpyAsync(&err, h->hs.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        AAP_CK(cudaStreamSynchronize(h->stream));
        const bool spilled = err & (aapk::ERR_SPILL | aapk::ERR_LOST);
        // spilled particles are kept exactly: accepted with an explicit
        // capacity, or when doubling the regions would exceed the staged indices
        if (!spilled || (!(err & aapk::ERR_LOST) && (h->p.capacity > 0 || !capacity_fits(h, factor * 2.0)))) {
            h->factor = factor;
            return AAP_OK;
        }
        if (h->p.capacity > 0) return fail(AAP_EOVERFLOW, "the particles do not fit the explicit capacity");
        factor *= 2.0;
    }
    return fail(AAP_EOVERFLOW, "could not size the tile regions for this state");
}

// Gather the current state and re-insert it with a larger capacity factor;
// the state is unchanged bit for bit (same tiles and fixed-point grid).
int relayout(aap_handle *h, double factor)
{
    int rc;
    if ((rc = ensure_xfer(h))) return rc;
    if (h->p.n > 0) {
        AAP_CK(cudaMemsetAsync(h->d_seen, 0, sizeof(int), h->stream));
        AAP_CK(aapk::launch_gather(h->hs, (int)(h->step & 1), h->d_x, h->d_y, h->d_th, h->d_seen, h->stream));
        int seen = 0;
        AAP_CK(cudaMemcpyAsync(&seen, h->d_seen, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        AAP_CK(cudaStreamSynchronize(h->stream));
        if (seen != h->p.n) {
            h->broken = true;
            return fail(AAP_EOVERFLOW, "stored particle count " + std::to_string(seen) + " != N");
        }
    }
    ++h->relayouts;
    return reinsert(h, factor, 0);
}

// React to an error word copied from the device: lost particles make the
// handle unusable; spilled ones (an automatic capacity) grow the regions, and
// *relaid (if given) reports that.
int act_on_error(aap_handle *h, int err, bool *relaid)
{
    if (err & aapk::ERR_SPILL) h->flags |= AAP_FLAG_SPILLED;
    if (err & (aapk::ERR_LOST | aapk::ERR_STAGE)) {
        h->broken = true;
        return fail(AAP_EOVERFLOW, "particles were lost: a tile overflowed its spill capacity");
    }
    if (err & aapk::ERR_TIMEOUT) {
        h->broken = true;
        return fail(AAP_ETIMEOUT, "a bounded wait of the pipelined step kernel ran out");
    }
    if ((err & aapk::ERR_SPILL) && h->p.capacity == 0) {
        // grow by 1.5, or by as much as the staged indices allow; at the limit
        // the overflow stays in the spill list (exact, only slower)
        double f = h->factor * 1.5;
        for (int k = 0; k < 8 && !capacity_fits(h, f); ++k) f = 0.5 * (f + h->factor);
        if (f < h->factor * 1.05 || !capacity_fits(h, f)) return AAP_OK;
        if (relaid) *relaid = true;
        return relayout(h, f);
    }
    return AAP_OK;
}

// At the start of aap_step: look at the error word copied after the previous
// batch (without waiting); grow the regions if particles spilled.
int poll_capacity(aap_handle *h)
{
    if (!h->err_pending) return AAP_OK;
    const cudaError_t q = cudaEventQuery(h->err_event);
    if (q == cudaErrorNotReady) return AAP_OK;
    if (q != cudaSuccess) return fail(AAP_ECUDA, std::string("error event: ") + cudaGetErrorString(q));
    h->err_pending = false;
    return act_on_error(h, *h->pinned_err, nullptr);
}


// Start a measurement window of nsteps steps at the current step: the
// current state's p and q seed last[0..1] (state t0 is the first sample).
int begin_measure(aap_handle *h, long long nsteps)
{
    aap_obs ob;
    const Sys &S = h->hs;
    AAP_CK(cudaMemsetAsync(h->d_obs, 0, 8 * sizeof(unsigned long long), h->stream));
    AAP_CK(aapk::launch_observe(S, (int)(h->step & 1), h->d_obs, h->stream));
    unsigned long long o[8];
    AAP_CK(cudaMemcpyAsync(o, h->d_obs, sizeof(o), cudaMemcpyDeviceToHost, h->stream));
    AAP_CK(cudaStreamSynchronize(h->stream));
    const double n = (double)h->p.n;
    const double c1 = (double)(long long)o[0] / aapk::kFix, s1 = (double)(long long)o[1] / aapk::kFix;
    const double c2 = (double)(long long)o[2] / aapk::kFix, s2 = (double)(long long)o[3] / aapk::kFix;
    double last[2] = {n > 0 ? std::sqrt(c1 * c1 + s1 * s1) / n : 0.0, n > 0 ? std::sqrt(c2 * c2 + s2 * s2) / n : 0.0};
    (void)ob;
    AAP_CK(cudaMemcpyAsync(h->hs.last, last, sizeof(last), cudaMemcpyHostToDevice, h->stream));
    h->hs.meas_until = h->step + nsteps;
    AAP_CK(cudaStreamSynchronize(h->stream));
    return push_sys(h);
}

int read_results(aap_handle *h, aap_results *out)
{
    double st[16];
    AAP_CK(cudaMemcpyAsync(st, h->hs.stats, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
    AAP_CK(cudaStreamSynchronize(h->stream));
    const double c = st[12];
    out->samples = (int64_t)c;
    for (int k = 0; k < 4; ++k) {
        out->p[k] = c > 0 ? st[k] / c : NAN;
        out->q[k] = c > 0 ? st[4 + k] / c : NAN;
        out->nbar[k] = c > 0 ? st[8 + k] / c : NAN;
    }
    out->binder = (c > 0 && out->p[1] > 0) ? 1.0 - out->p[3] / (3.0 * out->p[1] * out->p[1]) : NAN;
    return AAP_OK;
}


// ------------------------------------------------------------ ensembles --
// Candidate launch policies of the ensemble autotuner: threads per block and
// the nominal tile shape of every replica (clipped to the replica's box); a
// shape of 0 x 0 picks each replica's tile by its density (density_tile).
struct EnsPolicy {
    int threads, tw, th;
};
constexpr EnsPolicy kPolicies[8] = {{512, 32, 16}, {256, 32, 16}, {512, 16, 16}, {512, 0, 0},
                                    {512, 32, 32}, {256, 16, 8},  {512, 64, 16}, {512, 16, 8}};
constexpr int kNumPolicies = 8;

// A tile of about 1024 particles (the load that suits one block of 512
// threads at rho = 2 with 32 x 16 cells): fewer cells at high density, more
// at low density, so that the staging area (sized by the densest replica)
// still allows two blocks per SM.
void density_tile(const aap_params &p, int *tw, int *th)
{
    const double ncx = std::max(1.0, std::floor(p.lx / p.r)), ncy = std::max(1.0, std::floor(p.ly / p.r));
    const double mu = (double)p.n / (ncx * ncy);
    if (mu <= 1.25) { *tw = 32; *th = 32; }
    else if (mu <= 2.5) { *tw = 32; *th = 16; }
    else if (mu <= 5.0) { *tw = 16; *th = 16; }
    else { *tw = 16; *th = 8; }
}

}  // namespace

struct aap_ens {
    std::vector<aap_params> params;
    std::vector<aap_handle *> m;
    cudaStream_t stream = nullptr;
    Sys *d_sys = nullptr;
    int *d_tile_base = nullptr;
    Ctl *d_ctl = nullptr;
    unsigned char *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    int *d_dense = nullptr;             // pipelined step: tiles left to the whole-block routine
    size_t dense_tiles = 0;
    LaunchCfg L{};
    long long step = 0;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    int policy = 0;
    int *pinned_err = nullptr;      // [3][count]: after each aap_ens_step; two batch slots
    cudaEvent_t err_event = nullptr;
    cudaEvent_t batch_ev[2] = {nullptr, nullptr};   // error words taken every kAdaptSteps steps
    int batch_prev = -1;
    int batch_slot = 0;
    long long since_copy = 0;
    bool err_pending = false;
};

namespace {

void ens_free(aap_ens *e)
{
    for (aap_handle *h : e->m) {
        free_all(h);
        delete h;
    }
    e->m.clear();
    if (e->exec) cudaGraphExecDestroy(e->exec);
    e->exec = nullptr;
    if (e->d_sys) cudaFree(e->d_sys);
    if (e->d_tile_base) cudaFree(e->d_tile_base);
    if (e->d_ctl) cudaFree(e->d_ctl);
    if (e->d_scratch) cudaFree(e->d_scratch);
    if (e->d_dense) cudaFree(e->d_dense);
    e->d_sys = nullptr;
    e->d_tile_base = nullptr;
    e->d_ctl = nullptr;
    e->d_scratch = nullptr;
    e->d_dense = nullptr;
    e->dense_tiles = 0;
    e->scratch_bytes = 0;
}

// Combine the members' launch needs into the ensemble's launch: the largest
// staging capacities, a shared scratch, one grid over all tiles.
int ens_combine(aap_ens *e)
{
    LaunchCfg &L = e->L;
    const EnsPolicy &pol = kPolicies[e->policy];
    L.sys = e->d_sys;
    L.nsys = (int)e->m.size();
    L.model = e->params[0].model;
    L.tile_base = e->d_tile_base;
    L.ctl = e->d_ctl;
    L.threads = (e->params[0].threads && e->params[0].threads != 1024) ? e->params[0].threads : pol.threads;
    L.pipe = 0;
    L.stage_cap = 64;
    L.nce_max = 9;
    L.hist_words = 0;
    L.scratch_cap = 64;
    L.spill_list_cap = 16;
    long long total = 0;
    std::vector<int> tb(e->m.size() + 1, 0);
    for (size_t r = 0; r < e->m.size(); ++r) {
        const aap_handle *h = e->m[r];
        L.stage_cap = std::max(L.stage_cap, h->L.stage_cap);
        L.nce_max = std::max(L.nce_max, h->L.nce_max);
        L.hist_words = std::max(L.hist_words, h->L.hist_words);
        L.scratch_cap = std::max(L.scratch_cap, h->L.scratch_cap);
        L.spill_list_cap = std::max(L.spill_list_cap, h->L.spill_list_cap);
        total += h->hs.ntiles;
        tb[r + 1] = (int)total;
    }
    if (total >= (1ll << 30)) return fail(AAP_EINVAL, "too many tiles in the ensemble");
    AAP_CK(cudaMemcpy(e->d_tile_base, tb.data(), tb.size() * sizeof(int), cudaMemcpyHostToDevice));
    int bps = 0;
    {
        // a second block per SM is worth more than staging the densest
        // replicas' tiles in shared memory: lower the staging capacity while
        // that gains it (denser tiles then take the global-scratch path)
        int cap = L.stage_cap;
        for (;;) {
            AAP_CK(aapk::configure_step_kernel(L.model, L.threads,
                                               aapk::step_smem_bytes(cap, L.nce_max, L.hist_words), &bps));
            if (bps >= 2 || cap <= 1024) break;
            cap -= 64;
        }
        if (bps >= 2) {
            L.stage_cap = cap;
        } else {
            AAP_CK(aapk::configure_step_kernel(L.model, L.threads,
                                               aapk::step_smem_bytes(L.stage_cap, L.nce_max, L.hist_words), &bps));
        }
    }
    if (bps < 1) return fail(AAP_EINVAL, "step kernel does not fit on an SM for this ensemble");
    const int nsm = sm_count();
    L.grid_step = (int)std::max<long long>(1, std::min<long long>(total, (long long)bps * nsm));
    // one warp per replica for the sums, and about one counter word per thread
    L.grid_finish = (int)std::max<long long>(std::max<long long>(1, ((long long)e->m.size() + 7) / 8),
                                             std::min<long long>(256, (total * aapk::kCntStride + 255) / 256));
    L.scratch_per_block = aapk::stage_bytes(L.scratch_cap) + aapk::spill_list_bytes(L.spill_list_cap);
    L.scratch_per_block = (L.scratch_per_block + 255) / 256 * 256;
    const size_t need = L.scratch_per_block * L.grid_step;
    if (need > e->scratch_bytes) {
        if (e->d_scratch) cudaFree(e->d_scratch);
        e->d_scratch = nullptr;
        e->scratch_bytes = 0;
        if (cudaMalloc(&e->d_scratch, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(AAP_ENOMEM, "ensemble scratch allocation failed");
        }
        e->scratch_bytes = need;
    }
    L.scratch = e->d_scratch;
    // the pipelined kernel (threads 0 or 1024): one block per SM over all
    // replicas' tiles, tiles that do not fit listed for the whole-block routine
    bool one_species = true;
    for (const aap_params &q : e->params) one_species = one_species && q.nspecies <= 1;
    if (one_species && (e->params[0].threads == 0 || e->params[0].threads == 1024)) {
        int twmax = 1, thmax = 1;
        for (const aap_handle *h : e->m) {
            twmax = std::max(twmax, h->hs.twmax);
            thmax = std::max(thmax, h->hs.thmax);
        }
        if ((size_t)total > e->dense_tiles) {
            if (e->d_dense) cudaFree(e->d_dense);
            e->d_dense = nullptr;
            e->dense_tiles = 0;
            if (cudaMalloc(&e->d_dense, (size_t)total * sizeof(int)) != cudaSuccess) {
                cudaGetLastError();
                return fail(AAP_ENOMEM, "ensemble tile list allocation failed");
            }
            e->dense_tiles = (size_t)total;
        }
        AAP_CK(cudaMemset(e->d_dense, 0, (size_t)total * sizeof(int)));
        L.dense_list = e->d_dense;
        int rc = set_pipe_launch(L, twmax, thmax, (int)total);
        if (rc) return rc;
        if (!L.pipe && e->params[0].threads == 1024)
            return fail(AAP_EINVAL, "the pipelined step kernel does not fit this ensemble's tiling");
    }
    if (e->exec) cudaGraphExecDestroy(e->exec);
    e->exec = nullptr;
    return AAP_OK;
}

// Create every replica with policy `pol`, in its Philox initial state.
int ens_build(aap_ens *e, int pol)
{
    e->policy = pol;
    e->batch_prev = -1;
    e->batch_slot = 0;
    e->since_copy = 0;
    const int count = (int)e->params.size();
    if (cudaMalloc(&e->d_sys, (size_t)count * sizeof(Sys)) != cudaSuccess ||
        cudaMalloc(&e->d_tile_base, (size_t)(count + 1) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&e->d_ctl, sizeof(Ctl)) != cudaSuccess) {
        cudaGetLastError();
        return fail(AAP_ENOMEM, "ensemble descriptor allocation failed");
    }
    AAP_CK(cudaMemset(e->d_ctl, 0, sizeof(Ctl)));
    for (int r = 0; r < count; ++r) {
        aap_handle *h = new aap_handle();
        e->m.push_back(h);
        h->member = true;
        h->p = e->params[r];
        h->stream = e->stream;
        h->nom_tw = kPolicies[pol].tw;
        h->nom_th = kPolicies[pol].th;
        if (h->nom_tw == 0) density_tile(h->p, &h->nom_tw, &h->nom_th);
        if (!h->p.threads) h->p.threads = kPolicies[pol].threads;
        h->d_sys = e->d_sys + r;
        h->d_ctl = e->d_ctl;
        int rc;
        if ((rc = build_layout(h)) || (rc = alloc_all(h)) || (rc = reinsert(h, h->factor, 1)) ||
            (rc = read_errors(h))) {
            g_err = "replica " + std::to_string(r) + ": " + g_err;
            return rc;
        }
    }
    e->step = 0;
    return ens_combine(e);
}

// React to the replicas' error words: lost particles fail the call; spilled
// ones (an automatic capacity) grow that replica's regions (as far as the
// staged indices allow), after which the ensemble's launch is rebuilt.
int ens_act(aap_ens *e, const int *words)
{
    bool regrow = false;
    for (size_t r = 0; r < e->m.size(); ++r) {
        aap_handle *h = e->m[r];
        const int err = words[r];
        if (err & (aapk::ERR_LOST | aapk::ERR_STAGE))
            return fail(AAP_EOVERFLOW, "replica " + std::to_string(r) + " lost particles");
        bool relaid = false;
        int rc = act_on_error(h, err, &relaid);
        if (rc) return rc;
        regrow = regrow || relaid;
    }
    if (!regrow) return AAP_OK;
    e->batch_prev = -1;             // the copies in flight predate the re-layout
    e->batch_slot = 0;
    e->since_copy = 0;
    return ens_combine(e);
}

int ens_poll(aap_ens *e)
{
    if (!e->err_pending) return AAP_OK;
    const cudaError_t q = cudaEventQuery(e->err_event);
    if (q == cudaErrorNotReady) return AAP_OK;
    if (q != cudaSuccess) return fail(AAP_ECUDA, std::string("error event: ") + cudaGetErrorString(q));
    e->err_pending = false;
    return ens_act(e, e->pinned_err);
}

}  // namespace

#ifdef AAP_PHASE_TIMING
namespace aapk {
cudaError_t read_phase_times(unsigned long long *out16);
}
#endif
#ifdef AAP_PIPE_TIMING
namespace aapk {
cudaError_t read_pipe_times(unsigned long long *out16);
}
#endif

namespace {
constexpr char kSaveMagic[8] = {'A', 'A', 'P', 'S', 'A', 'V', 'E', '1'};
constexpr uint32_t kSaveVersion = 1;

struct FileCloser {
    FILE *f;
    ~FileCloser()
    {
        if (f) std::fclose(f);
    }
};

template <class T>
bool put(FILE *f, const T *v, size_t n)
{
    return n == 0 || std::fwrite(v, sizeof(T), n, f) == n;
}

template <class T>
bool get(FILE *f, T *v, size_t n)
{
    return n == 0 || std::fread(v, sizeof(T), n, f) == n;
}
}  // namespace

extern "C" {

const char *aap_last_error(void) { return g_err.c_str(); }

int aap_test_fail_alloc_after(int32_t n)
{
    g_fail_after.store(n < 0 ? -1 : n);
    return AAP_OK;
}

int aap_test_pipe_wait(int64_t wait_cycles, int32_t stall)
{
    if (stall != 0 && stall != 1) return fail(AAP_EINVAL, "stall must be 0 or 1");
    AAP_CK(aapk::set_pipe_test(wait_cycles, stall));
    return AAP_OK;
}

int32_t aap_abi_version(void) { return 2; }

void aap_params_default(aap_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->n = 1000;
    p->lx = p->ly = 32.0;
    p->r = 1.0;
    p->v = 0.5;
    p->eta = 0.4;
    p->omega = 0.0;
    p->gamma = 1.0;
    p->dt = 0.01;
    p->seed = 1;
    p->model = AAP_VM;
    p->order = 1;
    p->weight = AAP_H_INV_1PN;
}

int aap_create(const aap_params *p, void *stream, aap_handle **out)
{
    Range range_("aap_create");
    g_err.clear();
    if (!out) return fail(AAP_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = check_params(p);
    if (rc) return rc;
    aap_handle *h = new aap_handle();
    h->p = *p;
    h->stream = static_cast<cudaStream_t>(stream);
    if ((rc = build_layout(h)) || (rc = alloc_all(h))) {
        free_all(h);
        delete h;
        return rc;
    }
    if ((rc = reinsert(h, h->factor, 1)) || (rc = read_errors(h))) {
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return AAP_OK;
}

int aap_destroy(aap_handle *h)
{
    if (!h) return AAP_OK;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return AAP_OK;
}

int aap_step(aap_handle *h, int64_t nsteps)
{
    Range range_("aap_step");
    if (!h) return fail(AAP_EINVAL, "handle is NULL");
    if (nsteps < 0) return fail(AAP_EINVAL, "nsteps < 0");
    if (h->broken) return fail(AAP_ESTATE, "handle is unusable after an earlier fault");
    int rc = poll_capacity(h);
    if (rc) return rc;
    if ((rc = run_steps_adaptive(h, nsteps))) return rc;
    AAP_CK(cudaMemcpyAsync(h->pinned_err, h->hs.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    AAP_CK(cudaEventRecord(h->err_event, h->stream));
    h->err_pending = true;
    return AAP_OK;
}

int aap_sync(aap_handle *h)
{
    if (!h) return fail(AAP_EINVAL, "handle is NULL");
    AAP_CK(cudaStreamSynchronize(h->stream));
    return read_errors(h);
}

int aap_observe(aap_handle *h, aap_obs *out)
{
    if (!h || !out) return fail(AAP_EINVAL, "NULL argument");
    if (h->broken) return fail(AAP_ESTATE, "handle is unusable after an earlier fault");
    const Sys &S = h->hs;
    AAP_CK(cudaMemsetAsync(h->d_obs, 0, 8 * sizeof(unsigned long long), h->stream));
    AAP_CK(aapk::launch_observe(S, (int)(h->step & 1), h->d_obs, h->stream));
    unsigned long long o[8];
    double last[4];
    AAP_CK(cudaMemcpyAsync(o, h->d_obs, sizeof(o), cudaMemcpyDeviceToHost, h->stream));
    AAP_CK(cudaMemcpyAsync(last, S.last, sizeof(last), cudaMemcpyDeviceToHost, h->stream));
    AAP_CK(cudaStreamSynchronize(h->stream));
    int rc = read_errors(h);
    if (rc) return rc;
    if ((long long)o[4] != h->p.n) {
        h->broken = true;
        return fail(AAP_EOVERFLOW, "particle count changed: " + std::to_string((long long)o[4]) +
                                       " stored of " + std::to_string(h->p.n));
    }
    const double n = (double)h->p.n;
    const double c1 = (double)(long long)o[0] / aapk::kFix, s1 = (double)(long long)o[1] / aapk::kFix;
    const double c2 = (double)(long long)o[2] / aapk::kFix, s2 = (double)(long long)o[3] / aapk::kFix;
    out->phi = n > 0 ? std::sqrt(c1 * c1 + s1 * s1) / n : 0.0;
    out->q = n > 0 ? std::sqrt(c2 * c2 + s2 * s2) / n : 0.0;
    out->mean_neighbours = h->step > 0 ? last[2] : NAN;
    out->step = h->step;
    out->flags = h->flags;
    out->reserved = 0;
    return AAP_OK;
}

int aap_phi_trace(aap_handle *h, int64_t nsteps, double *phi_out)
{
    Range range_("aap_phi_trace");
    if (!h || !phi_out) return fail(AAP_EINVAL, "NULL argument");
    if (nsteps < 0) return fail(AAP_EINVAL, "nsteps < 0");
    aap_obs ob;
    int rc = aap_observe(h, &ob);
    if (rc) return rc;
    phi_out[0] = ob.phi;
    if (nsteps == 0) return AAP_OK;
    if (h->trace_alloc < nsteps + 1) {
        // replace the smaller buffers (a failed allocation leaves none)
        const size_t old = (size_t)h->trace_alloc * sizeof(double);
        if ((rc = dev_free(h, h->d_trace, old)) || (rc = dev_free(h, h->d_trace_nbar, old))) return rc;
        h->d_trace = h->d_trace_nbar = nullptr;
        h->trace_alloc = 0;
        if ((rc = dev_alloc(h, &h->d_trace, (size_t)(nsteps + 1) * sizeof(double)))) return rc;
        if ((rc = dev_alloc(h, &h->d_trace_nbar, (size_t)(nsteps + 1) * sizeof(double)))) return rc;
        h->trace_alloc = nsteps + 1;
    }
    h->hs.trace = h->d_trace;
    h->hs.trace_nbar = h->d_trace_nbar;
    h->hs.trace_base = h->step;
    h->hs.trace_cap = nsteps + 1;
    if ((rc = push_sys(h))) return rc;
    if ((rc = run_steps_adaptive(h, nsteps))) return rc;
    AAP_CK(cudaMemcpyAsync(phi_out + 1, h->d_trace + 1, (size_t)nsteps * sizeof(double),
                           cudaMemcpyDeviceToHost, h->stream));
    h->hs.trace = nullptr;
    h->hs.trace_nbar = nullptr;
    h->hs.trace_cap = 0;
    if ((rc = push_sys(h))) return rc;
    AAP_CK(cudaStreamSynchronize(h->stream));
    return read_errors(h);
}

int aap_get_state(aap_handle *h, double *x, double *y, float *theta, int64_t n)
{
    Range range_("aap_get_state");
    if (!h || !x || !y || !theta) return fail(AAP_EINVAL, "NULL argument");
    if (n != h->p.n) return fail(AAP_EINVAL, "n must equal the particle number");
    if (h->broken) return fail(AAP_ESTATE, "handle is unusable after an earlier fault");
    int rc = ensure_xfer(h);
    if (rc) return rc;
    if (n == 0) return AAP_OK;
    AAP_CK(cudaMemsetAsync(h->d_seen, 0, sizeof(int), h->stream));
    AAP_CK(aapk::launch_gather(h->hs, (int)(h->step & 1), h->d_x, h->d_y, h->d_th, h->d_seen, h->stream));
    int seen = 0;
    AAP_CK(cudaMemcpyAsync(x, h->d_x, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    AAP_CK(cudaMemcpyAsync(y, h->d_y, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    AAP_CK(cudaMemcpyAsync(theta, h->d_th, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    AAP_CK(cudaMemcpyAsync(&seen, h->d_seen, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    AAP_CK(cudaStreamSynchronize(h->stream));
    if ((rc = read_errors(h))) return rc;
    if (seen != n) {
        h->broken = true;
        return fail(AAP_EOVERFLOW, "stored particle count " + std::to_string(seen) + " != N");
    }
    return AAP_OK;
}

int aap_set_state(aap_handle *h, const double *x, const double *y, const float *theta, int64_t n,
                  int64_t step)
{
    Range range_("aap_set_state");
    if (!h || (n > 0 && (!x || !y || !theta))) return fail(AAP_EINVAL, "NULL argument");
    if (n != h->p.n) return fail(AAP_EINVAL, "n must equal the particle number");
    if (step < 0) return fail(AAP_EINVAL, "step < 0");
    int rc = ensure_xfer(h);
    if (rc) return rc;
    if (!h->d_bad && (rc = dev_alloc(h, &h->d_bad, 2 * sizeof(unsigned long long)))) return rc;
    AAP_CK(cudaStreamSynchronize(h->stream));
    h->err_pending = false;
    // copy in, then check every value on the device (the state and step are
    // untouched until the check has passed)
    if (n > 0) {
        AAP_CK(cudaMemcpyAsync(h->d_x, x, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        AAP_CK(cudaMemcpyAsync(h->d_y, y, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        AAP_CK(cudaMemcpyAsync(h->d_th, theta, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    }
    AAP_CK(aapk::launch_validate(h->d_x, h->d_y, h->d_th, n, h->p.lx, h->p.ly, h->d_bad, h->stream));
    unsigned long long bad[2];
    AAP_CK(cudaMemcpyAsync(bad, h->d_bad, sizeof(bad), cudaMemcpyDeviceToHost, h->stream));
    AAP_CK(cudaStreamSynchronize(h->stream));
    if (bad[0] != ~0ull && bad[0] <= bad[1])
        return fail(AAP_EINVAL, "position " + std::to_string(bad[0]) + " outside the box");
    if (bad[1] != ~0ull) return fail(AAP_EINVAL, "non-finite orientation " + std::to_string(bad[1]));
    Ctl c{};
    c.step = step;
    AAP_CK(cudaMemcpyAsync(h->d_ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, h->stream));
    h->step = step;
    h->flags = 0;
    h->broken = false;
    // an automatic capacity keeps the size it has grown to (a restored state
    // of the same system needs it again; the re-insert doubles it if not)
    if ((rc = reinsert(h, h->p.capacity > 0 ? h->p.capacity : h->factor, 0))) return rc;
    return read_errors(h);
}

int aap_step_neighbours(aap_handle *h, int32_t *nbr_out, int64_t n)
{
    Range range_("aap_step_neighbours");
    if (!h || (n > 0 && !nbr_out)) return fail(AAP_EINVAL, "NULL argument");
    if (n != h->p.n) return fail(AAP_EINVAL, "n must equal the particle number");
    if (h->broken) return fail(AAP_ESTATE, "handle is unusable after an earlier fault");
    int rc;
    if (!h->d_nbr && (rc = dev_alloc(h, &h->d_nbr, (size_t)std::max<long long>(n, 1) * sizeof(int))))
        return rc;
    h->hs.nbr_out = h->d_nbr;
    if ((rc = push_sys(h))) return rc;
    rc = run_steps(h, 1);
    h->hs.nbr_out = nullptr;
    int rc2 = push_sys(h);
    if (rc) return rc;
    if (rc2) return rc2;
    if (n > 0)
        AAP_CK(cudaMemcpyAsync(nbr_out, h->d_nbr, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    AAP_CK(cudaStreamSynchronize(h->stream));
    return read_errors(h);
}


int aap_measure(aap_handle *h, int64_t nsteps)
{
    Range range_("aap_measure");
    if (!h) return fail(AAP_EINVAL, "handle is NULL");
    if (nsteps < 0) return fail(AAP_EINVAL, "nsteps < 0");
    if (h->broken) return fail(AAP_ESTATE, "handle is unusable after an earlier fault");
    int rc = poll_capacity(h);
    if (rc) return rc;
    if ((rc = begin_measure(h, nsteps))) return rc;
    return aap_step(h, nsteps);
}

int aap_get_results(aap_handle *h, aap_results *out)
{
    if (!h || !out) return fail(AAP_EINVAL, "NULL argument");
    AAP_CK(cudaStreamSynchronize(h->stream));
    int rc = read_errors(h);
    if (rc) return rc;
    return read_results(h, out);
}

int aap_clear_results(aap_handle *h)
{
    if (!h) return fail(AAP_EINVAL, "handle is NULL");
    AAP_CK(cudaMemsetAsync(h->hs.stats, 0, 16 * sizeof(double), h->stream));
    AAP_CK(cudaMemsetAsync(h->hs.hist, 0, (size_t)(h->hs.bins_theta + h->hs.bins_nbr) * sizeof(unsigned long long),
                           h->stream));
    return AAP_OK;
}

int aap_get_histograms(aap_handle *h, double *theta_hist, int32_t nt, double *nbr_hist, int32_t nn)
{
    if (!h) return fail(AAP_EINVAL, "handle is NULL");
    const Sys &S = h->hs;
    if ((theta_hist && nt != S.bins_theta) || (nbr_hist && nn != S.bins_nbr))
        return fail(AAP_EINVAL, "bin counts must equal binnum_theta / binnum_neighbors");
    std::vector<unsigned long long> v((size_t)(S.bins_theta + S.bins_nbr));
    AAP_CK(cudaMemcpyAsync(v.data(), S.hist, v.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
    AAP_CK(cudaStreamSynchronize(h->stream));
    int rc = read_errors(h);
    if (rc) return rc;
    double tt = 0, tn = 0;
    for (int k = 0; k < S.bins_theta; ++k) tt += (double)v[k];
    for (int k = 0; k < S.bins_nbr; ++k) tn += (double)v[S.bins_theta + k];
    if (theta_hist)
        for (int k = 0; k < S.bins_theta; ++k) theta_hist[k] = tt > 0 ? (double)v[k] / tt : 0.0;
    if (nbr_hist)
        for (int k = 0; k < S.bins_nbr; ++k) nbr_hist[k] = tn > 0 ? (double)v[S.bins_theta + k] / tn : 0.0;
    return AAP_OK;
}

// Saved-state file (little-endian): "AAPSAVE1", u32 version, u32 sizeof(aap_params),
// aap_params, i64 step, i64 n, x[n] f64, y[n] f64, theta[n] f32, stats[16] f64,
// i32 bins_theta, i32 bins_nbr, hist[bins_theta + bins_nbr] u64.

int aap_save(aap_handle *h, const char *path)
{
    Range range_("aap_save");
    if (!h || !path) return fail(AAP_EINVAL, "NULL argument");
    if (h->broken) return fail(AAP_ESTATE, "handle is unusable after an earlier fault");
    const int64_t n = h->p.n;
    std::vector<double> x((size_t)n), y((size_t)n);
    std::vector<float> th((size_t)n);
    int rc = aap_get_state(h, x.data(), y.data(), th.data(), n);
    if (rc) return rc;
    const Sys &S = h->hs;
    double st[16];
    std::vector<unsigned long long> hist((size_t)(S.bins_theta + S.bins_nbr));
    AAP_CK(cudaMemcpyAsync(st, S.stats, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
    AAP_CK(cudaMemcpyAsync(hist.data(), S.hist, hist.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                           h->stream));
    AAP_CK(cudaStreamSynchronize(h->stream));
    FileCloser fc{std::fopen(path, "wb")};
    if (!fc.f) return fail(AAP_EIO, std::string("cannot open ") + path + " for writing");
    const uint32_t ver = kSaveVersion, psz = (uint32_t)sizeof(aap_params);
    const int64_t step = h->step;
    const int32_t bins[2] = {S.bins_theta, S.bins_nbr};
    bool ok = put(fc.f, kSaveMagic, 8) && put(fc.f, &ver, 1) && put(fc.f, &psz, 1) && put(fc.f, &h->p, 1) &&
              put(fc.f, &step, 1) && put(fc.f, &n, 1) && put(fc.f, x.data(), x.size()) &&
              put(fc.f, y.data(), y.size()) && put(fc.f, th.data(), th.size()) && put(fc.f, st, 16) &&
              put(fc.f, bins, 2) && put(fc.f, hist.data(), hist.size());
    ok = (std::fclose(fc.f) == 0) && ok;
    fc.f = nullptr;
    if (!ok) return fail(AAP_EIO, std::string("write to ") + path + " failed");
    return AAP_OK;
}

int aap_load(const char *path, void *stream, aap_handle **out)
{
    Range range_("aap_load");
    if (!path || !out) return fail(AAP_EINVAL, "NULL argument");
    *out = nullptr;
    FileCloser fc{std::fopen(path, "rb")};
    if (!fc.f) return fail(AAP_EIO, std::string("cannot open ") + path);
    char magic[8];
    uint32_t ver = 0, psz = 0;
    aap_params p;
    int64_t step = 0, n = 0;
    if (!get(fc.f, magic, 8) || std::memcmp(magic, kSaveMagic, 8) != 0)
        return fail(AAP_EIO, std::string(path) + " is not a saved state");
    if (!get(fc.f, &ver, 1) || ver != kSaveVersion || !get(fc.f, &psz, 1) || psz != sizeof(aap_params))
        return fail(AAP_EIO, std::string(path) + ": unsupported version or parameter layout");
    if (!get(fc.f, &p, 1) || !get(fc.f, &step, 1) || !get(fc.f, &n, 1) || n != p.n || n < 0 || step < 0)
        return fail(AAP_EIO, std::string(path) + ": truncated or inconsistent header");
    std::vector<double> x((size_t)n), y((size_t)n);
    std::vector<float> th((size_t)n);
    double st[16];
    int32_t bins[2];
    if (!get(fc.f, x.data(), x.size()) || !get(fc.f, y.data(), y.size()) || !get(fc.f, th.data(), th.size()) ||
        !get(fc.f, st, 16) || !get(fc.f, bins, 2))
        return fail(AAP_EIO, std::string(path) + ": truncated");
    if (bins[0] < 1 || bins[0] > aapk::kMaxBins || bins[1] < 1 || bins[1] > aapk::kMaxBins)
        return fail(AAP_EIO, std::string(path) + ": bad histogram size");
    std::vector<unsigned long long> hist((size_t)(bins[0] + bins[1]));
    if (!get(fc.f, hist.data(), hist.size())) return fail(AAP_EIO, std::string(path) + ": truncated");
    aap_handle *h = nullptr;
    int rc = aap_create(&p, stream, &h);
    if (rc) return rc;
    if (h->hs.bins_theta != bins[0] || h->hs.bins_nbr != bins[1]) {
        aap_destroy(h);
        return fail(AAP_EIO, std::string(path) + ": histogram size does not match its parameters");
    }
    if ((rc = aap_set_state(h, x.data(), y.data(), th.data(), n, step))) {
        aap_destroy(h);
        return rc;
    }
    cudaError_t e = cudaMemcpyAsync(h->hs.stats, st, sizeof(st), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->hs.hist, hist.data(), hist.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice,
                            h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        aap_destroy(h);
        return fail(AAP_ECUDA, std::string("restoring measurements: ") + cudaGetErrorString(e));
    }
    *out = h;
    return AAP_OK;
}

int aap_coarse_grain(aap_handle *h, int32_t nbx, int32_t nby, float *dev_out)
{
    Range range_("aap_coarse_grain");
    if (!h || !dev_out) return fail(AAP_EINVAL, "NULL argument");
    if (nbx < 1 || nby < 1 || (long long)nbx * nby > (1ll << 26))
        return fail(AAP_EINVAL, "nbx, nby must be >= 1 with nbx * nby <= 2^26");
    if (h->broken) return fail(AAP_ESTATE, "handle is unusable after an earlier fault");
    const long long bins = (long long)nbx * nby;
    if (h->cg_bins < bins) {
        int rc;
        if (h->d_cg && (rc = dev_free(h, h->d_cg, (size_t)h->cg_bins * 3 * sizeof(unsigned long long)))) return rc;
        h->d_cg = nullptr;
        if ((rc = dev_alloc(h, &h->d_cg, (size_t)bins * 3 * sizeof(unsigned long long)))) return rc;
        h->cg_bins = bins;
    }
    AAP_CK(aapk::launch_coarse(h->hs, (int)(h->step & 1), nbx, nby, h->d_cg, dev_out, h->stream));
    return AAP_OK;
}


int aap_ens_create(const aap_params *params, int32_t count, void *stream, aap_ens **out)
{
    Range range_("aap_ens_create");
    g_err.clear();
    if (!out || !params) return fail(AAP_EINVAL, "NULL argument");
    *out = nullptr;
    if (count < 1) return fail(AAP_EINVAL, "count must be >= 1");
    for (int r = 0; r < count; ++r) {
        int rc = check_params(&params[r]);
        if (rc) {
            g_err = "replica " + std::to_string(r) + ": " + g_err;
            return rc;
        }
        if (params[r].kn > 0) return fail(AAP_EINVAL, "metric-free systems (kn > 0) are not batched; use aap_create");
        if (params[r].model != params[0].model) return fail(AAP_EINVAL, "all replicas must use the same model");
        if (params[r].threads != params[0].threads) return fail(AAP_EINVAL, "all replicas must use the same threads");
        if (params[r].nspecies > 1 && params[r].threads == 1024)
            return fail(AAP_EINVAL, "an ensemble of multi-species replicas needs threads = 0, 256 or 512");
    }
    aap_ens *e = new aap_ens();
    e->params.assign(params, params + count);
    e->stream = static_cast<cudaStream_t>(stream);
    int rc = ens_build(e, 0);
    if (rc == AAP_OK) {
        if (cudaMallocHost(&e->pinned_err, (size_t)3 * count * sizeof(int)) != cudaSuccess ||
            cudaEventCreateWithFlags(&e->err_event, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&e->batch_ev[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&e->batch_ev[1], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            rc = fail(AAP_ECUDA, "ensemble host buffers");
        }
    }
    if (rc) {
        ens_free(e);
        if (e->pinned_err) cudaFreeHost(e->pinned_err);
        for (cudaEvent_t ev : e->batch_ev)
            if (ev) cudaEventDestroy(ev);
        if (e->err_event) cudaEventDestroy(e->err_event);
        delete e;
        return rc;
    }
    *out = e;
    return AAP_OK;
}

int aap_ens_destroy(aap_ens *e)
{
    if (!e) return AAP_OK;
    cudaStreamSynchronize(e->stream);
    ens_free(e);
    if (e->cap) cudaStreamDestroy(e->cap);
    if (e->err_event) cudaEventDestroy(e->err_event);
    for (cudaEvent_t ev : e->batch_ev)
        if (ev) cudaEventDestroy(ev);
    if (e->pinned_err) cudaFreeHost(e->pinned_err);
    delete e;
    return AAP_OK;
}

int aap_ens_step(aap_ens *e, int64_t nsteps)
{
    Range range_("aap_ens_step");
    if (!e) return fail(AAP_EINVAL, "ensemble is NULL");
    if (nsteps < 0) return fail(AAP_EINVAL, "nsteps < 0");
    int rc = ens_poll(e);
    if (rc) return rc;
    // in pieces, with every replica's error word copied every kAdaptSteps
    // steps and the copy before it read (as run_steps_adaptive does)
    const size_t count = e->m.size();
    long long left = nsteps;
    while (left > 0) {
        const long long k = std::min(left, kAdaptSteps - e->since_copy);
        if ((rc = launch_steps(e->L, e->stream, k, e->cap, e->exec))) return rc;
        e->step += k;
        for (aap_handle *h : e->m) h->step += k;
        left -= k;
        e->since_copy += k;
        if (e->since_copy < kAdaptSteps) continue;
        e->since_copy = 0;
        const int slot = e->batch_slot;
        for (size_t r = 0; r < count; ++r)
            AAP_CK(cudaMemcpyAsync(e->pinned_err + (1 + slot) * count + r, e->m[r]->hs.err, sizeof(int),
                                   cudaMemcpyDeviceToHost, e->stream));
        AAP_CK(cudaEventRecord(e->batch_ev[slot], e->stream));
        e->batch_slot ^= 1;
        const int prev = e->batch_prev;
        e->batch_prev = slot;
        if (prev >= 0) {
            AAP_CK(cudaEventSynchronize(e->batch_ev[prev]));
            if ((rc = ens_act(e, e->pinned_err + (1 + prev) * count))) return rc;
        }
    }
    for (size_t r = 0; r < e->m.size(); ++r)
        AAP_CK(cudaMemcpyAsync(e->pinned_err + r, e->m[r]->hs.err, sizeof(int), cudaMemcpyDeviceToHost, e->stream));
    AAP_CK(cudaEventRecord(e->err_event, e->stream));
    e->err_pending = true;
    return AAP_OK;
}

int aap_ens_measure(aap_ens *e, int64_t nsteps)
{
    Range range_("aap_ens_measure");
    if (!e) return fail(AAP_EINVAL, "ensemble is NULL");
    if (nsteps < 0) return fail(AAP_EINVAL, "nsteps < 0");
    int rc = ens_poll(e);
    if (rc) return rc;
    for (aap_handle *h : e->m)
        if ((rc = begin_measure(h, nsteps))) return rc;
    return aap_ens_step(e, nsteps);
}

int aap_ens_phi_mean(aap_ens *e, double *out)
{
    if (!e || !out) return fail(AAP_EINVAL, "NULL argument");
    AAP_CK(cudaStreamSynchronize(e->stream));
    for (size_t r = 0; r < e->m.size(); ++r) {
        aap_results res;
        int rc = read_errors(e->m[r]);
        if (rc) return rc;
        if ((rc = read_results(e->m[r], &res))) return rc;
        out[r] = res.p[0];
    }
    return AAP_OK;
}

int aap_ens_results(aap_ens *e, int32_t r, aap_results *out)
{
    if (!e || !out) return fail(AAP_EINVAL, "NULL argument");
    if (r < 0 || r >= (int)e->m.size()) return fail(AAP_EINVAL, "replica index out of range");
    return aap_get_results(e->m[r], out);
}

int aap_ens_get_state(aap_ens *e, int32_t r, double *x, double *y, float *theta, int64_t n)
{
    if (!e) return fail(AAP_EINVAL, "ensemble is NULL");
    if (r < 0 || r >= (int)e->m.size()) return fail(AAP_EINVAL, "replica index out of range");
    AAP_CK(cudaStreamSynchronize(e->stream));
    return aap_get_state(e->m[r], x, y, theta, n);
}

int aap_ens_coarse_grain(aap_ens *e, int32_t r, int32_t nbx, int32_t nby, float *dev_out)
{
    if (!e) return fail(AAP_EINVAL, "ensemble is NULL");
    if (r < 0 || r >= (int)e->m.size()) return fail(AAP_EINVAL, "replica index out of range");
    return aap_coarse_grain(e->m[r], nbx, nby, dev_out);
}

int aap_ens_get_layout(aap_ens *e, int32_t r, aap_layout *out)
{
    if (!e) return fail(AAP_EINVAL, "ensemble is NULL");
    if (r < 0 || r >= (int)e->m.size()) return fail(AAP_EINVAL, "replica index out of range");
    int rc = aap_get_layout(e->m[r], out);
    if (rc == AAP_OK) {
        out->threads = e->L.threads;
        out->stage_cap = e->L.pipe ? e->L.pipe_cap : e->L.stage_cap;
        out->tile_w = e->m[r]->nom_tw;
        out->tile_h = e->m[r]->nom_th;
    }
    return rc;
}

int aap_ens_info(aap_ens *e, int32_t *count, int64_t *step)
{
    if (!e) return fail(AAP_EINVAL, "ensemble is NULL");
    if (count) *count = (int32_t)e->m.size();
    if (step) *step = e->step;
    return AAP_OK;
}

int aap_ens_autotune(aap_ens *e, int32_t trial_steps, int32_t *policy_out, double *ms_out)
{
    Range range_("aap_ens_autotune");
    if (!e) return fail(AAP_EINVAL, "ensemble is NULL");
    if (e->step != 0) return fail(AAP_EINVAL, "autotune is only allowed before the first step");
    if (trial_steps < 1) return fail(AAP_EINVAL, "trial_steps must be >= 1");
    double ms[kNumPolicies];
    for (int k = 0; k < kNumPolicies; ++k) ms[k] = 0.0;
    int best = -1;
    cudaEvent_t t0, t1;
    AAP_CK(cudaEventCreate(&t0));
    AAP_CK(cudaEventCreate(&t1));
    int rc = AAP_OK;
    for (int k = 0; k < kNumPolicies && rc == AAP_OK; ++k) {
        AAP_CK(cudaStreamSynchronize(e->stream));
        ens_free(e);
        if ((rc = ens_build(e, k)) != AAP_OK) {
            if (rc == AAP_EINVAL) {     // this shape does not fit: skip it
                g_err.clear();
                ens_free(e);
                rc = AAP_OK;
            }
            continue;
        }
        // warm up (captures the graph), then time
        if ((rc = launch_steps(e->L, e->stream, 2 + 32, e->cap, e->exec))) break;
        AAP_CK(cudaEventRecord(t0, e->stream));
        if ((rc = launch_steps(e->L, e->stream, trial_steps, e->cap, e->exec))) break;
        AAP_CK(cudaEventRecord(t1, e->stream));
        AAP_CK(cudaEventSynchronize(t1));
        float t = 0.f;
        AAP_CK(cudaEventElapsedTime(&t, t0, t1));
        ms[k] = t / trial_steps;
        if (best < 0 || ms[k] < ms[best]) best = k;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    AAP_CK(cudaStreamSynchronize(e->stream));
    ens_free(e);
    if (rc != AAP_OK) return rc;
    if (best < 0) return fail(AAP_EINVAL, "no launch policy fits this ensemble");
    if ((rc = ens_build(e, best))) return rc;
    if (policy_out) *policy_out = best;
    if (ms_out)
        for (int k = 0; k < kNumPolicies; ++k) ms_out[k] = ms[k];
    return AAP_OK;
}

int aap_set_timing(aap_handle *h, int32_t enable)
{
    if (!h) return fail(AAP_EINVAL, "handle is NULL");
    int rc = resolve_timing(h);
    if (rc) return rc;
    h->timing = enable != 0;
    for (int k = 0; k < 3; ++k) {
        h->ms[k] = 0;
        h->launches[k] = 0;
    }
    return AAP_OK;
}

int aap_get_timing(aap_handle *h, double *ms, int64_t *launches)
{
    if (!h || !ms || !launches) return fail(AAP_EINVAL, "NULL argument");
    int rc = resolve_timing(h);
    if (rc) return rc;
    for (int k = 0; k < 3; ++k) {
        ms[k] = h->ms[k];
        launches[k] = h->launches[k];
    }
    return AAP_OK;
}

int aap_get_layout(aap_handle *h, aap_layout *out)
{
    if (!h || !out) return fail(AAP_EINVAL, "NULL argument");
    const Sys &S = h->hs;
    out->ncx = S.ncx;
    out->ncy = S.ncy;
    out->ntx = S.ntx;
    out->nty = S.nty;
    out->tile_w = S.twmax;
    out->tile_h = S.thmax;
    out->fix_bits_x = S.sx;
    out->fix_bits_y = S.sy;
    out->threads = h->L.threads;
    out->stage_cap = h->L.pipe ? h->L.pipe_cap : h->L.stage_cap;
    out->tile_slots = S.tile_slots;
    out->device_bytes = (int64_t)h->bytes;
    out->cell_x = h->csx;
    out->cell_y = h->csy;
    return AAP_OK;
}

#ifdef AAP_PIPE_TIMING
// Instrumented builds only: cycles per role of the pipelined step kernel.
int aap_debug_pipe_times(unsigned long long *out16)
{
    AAP_CK(aapk::read_pipe_times(out16));
    return AAP_OK;
}
#endif

#ifdef AAP_PHASE_TIMING
// Instrumented builds only: cycles per step-kernel phase summed over blocks.
int aap_debug_phase_times(unsigned long long *out16)
{
    AAP_CK(aapk::read_phase_times(out16));
    return AAP_OK;
}
#endif

}  // extern "C"
