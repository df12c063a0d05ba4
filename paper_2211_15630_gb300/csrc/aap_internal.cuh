// aap_internal.cuh -- device-side data layout of the GB300 particle library.
//
// State layout in HBM (one system):
//   The Lx x Ly box is cut into ncx x ncy cells of side L/floor(L/R)
//   (Sec. 3.2 of the paper), and the cells into ntx x nty tiles (balanced
//   partition, every tile >= 3 cells per axis).  Each tile owns a fixed block
//   of `tile_slots` particle records split into 9 regions by cell class:
//   interior, four edges, four corners (region = ry*3 + rx with
//   rx = 0 for the first column, 2 for the last, 1 otherwise).  A block that
//   updates one tile can therefore read exactly its one-cell halo: the facing
//   edge and corner regions of the 8 neighbour tiles.
//   A record is 16 bytes {X, Y, theta, id}: X, Y are fixed-point positions
//   relative to the tile's lower-left corner with 2^s units per cell side, so
//   the cell of a particle is X >> s and every wrap or mirror is exact integer
//   arithmetic.  Regions are filled through warp-aggregated atomic counters;
//   records inside a region are unordered (the step kernel groups them by
//   cell in shared memory and sums neighbours in exact integers, so every
//   result is deterministic whatever the order).
//   Particles that do not fit their region go to a spill list.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace aapk {

constexpr int kRegions = 9;
constexpr int kCntStride = 16;      // counters per tile (9 used): one 64-byte line
constexpr int kAccSlots = 64;       // spread of the per-step integer accumulators
constexpr int kAccWords = 8;        // sum cos, sin, |Omega|, cos 2theta, sin 2theta; 3 unused
constexpr double kFix = 4294967296.0;     // 2^32: scale of the observation sums
constexpr float kFixStepF = 1073741824.0f;  // 2^30: scale of the per-step sums
constexpr double kFixStep = 1073741824.0;
constexpr float kFixNbF = 4194304.0f;       // 2^22: staged cos / sin as exact integers
constexpr int kSegs = 25;           // 9 own regions + 16 halo regions
constexpr int kMaxTile = 64;        // largest tile side in cells
constexpr int kMaxBins = 512;       // histogram bins (each of theta and |Omega|)

// error bits (Sys::err)
enum : int {
    ERR_SPILL = 1,    // a region overflowed into the spill list (still exact)
    ERR_LOST = 2,     // the spill list overflowed: particles were dropped
    ERR_BOUNDS = 4,   // a record decoded outside its tile (internal fault)
    ERR_NAN = 8,      // a non-finite orientation was produced
    ERR_STAGE = 16,   // a tile exceeded the scratch staging capacity
    ERR_TIMEOUT = 32, // a bounded wait of the pipelined step kernel ran out
};

constexpr int kPipeMaxStage = 4096;     // staged particles per tile in the pipelined step
constexpr int kPipeMaxSpill = 256;      // spilled records one pipelined tile may take
constexpr int kPipeSpillScan = 256;     // longest spill list the pipelined copy warp scans itself

struct Sys {
    // geometry
    int ncx, ncy, ntx, nty;
    const int *x0tab, *y0tab;   // first cell of every tile column / row, [ntx+1], [nty+1]
    int sx, sy;                 // fixed-point bits per cell side
    int twmax, thmax;           // largest tile in cells
    double lx, ly, csx_d, csy_d;
    float ux, uy;               // length of one fixed-point unit, cs * 2^-s
    float kx, ky;               // displacement per step in units, times cos / sin
    float r2;                   // R^2
    // model (Sec. 2)
    int model, order, weight, bx, by;
    float eta_pi;               // VM / NVM: eta * pi (noise amplitude)
    float omega_step;           // omega (VM / NVM) or omega * dt (Langevin)
    float gamma_dt;             // Gamma * dt (Langevin)
    float noise_amp;            // eta * sqrt(dt) (Langevin)
    uint32_t seed_lo, seed_hi;
    long long n;
    // layout
    int ntiles;
    int tile_slots;
    int cap[kRegions];
    int off[kRegions];
    int spill_cap;
    int4 *rec[2];
    int *cnt[2];                // [ntiles * kCntStride]
    int4 *spill_rec[2];
    int *spill_key[2];          // tile * kCntStride + region
    int *spill_cnt;             // [2]
    unsigned *spill_bits[2];    // [ntiles / 32 + 1]: bit t set when a record bound for tile t spilled
    unsigned long long *acc;    // [2][kAccSlots][kAccWords]
    // measurement outputs
    double *trace;              // p(t) for t = trace_base .. trace_base + trace_cap - 1
    double *trace_nbar;         // mean |Omega| of state t
    long long trace_base, trace_cap;
    double *last;               // [4]: p, q of the current state; mean |Omega| of the
                                //      state before it; step
    double *stats;              // [16]: sums of p^k, q^k, nbar^k (k = 1..4), count
    long long meas_until;       // steps t < meas_until add state t to stats
    unsigned long long *hist;   // [bins_theta + bins_nbr] measured histograms
    int bins_theta, bins_nbr;
    int *nbr_out;               // optional |Omega_i| by particle id
    int *err;
    // metric-free neighbourhoods (Sec. 2.3): one tile over the whole box whose
    // records all sit in region 0 (flat), re-sorted by cell every step
    int flat;                   // 1: every record goes to region 0 of tile 0
    int knn;                    // k nearest neighbours (0: metric, radius R)
    int *mf_cnt;                // [ncx * ncy] records per cell (zero between steps)
    int *mf_start;              // [ncx * ncy + 1] chunk-local exclusive prefix of mf_cnt
    int *mf_blk;                // [chunks + 1] exclusive prefix of the chunk totals
    int2 *mf_cs;                // [n] cell and arrival rank of each record
    int4 *mf_sorted;            // [n] records in cell order
    int2 *mf_fix;               // [n] particles left to the exact pass: sorted index, rings or -1
    int *mf_nfix;               // [2]: queue length, next warp task of the update
    // species (Sec. 2.5): ids in [sp_end[s-1], sp_end[s]) are species s; with
    // one species, entry 0 repeats the scalar parameters above
    int nsp;
    long long sp_end[8];
    float sp_eta_pi[8], sp_omega_step[8], sp_noise_amp[8], sp_kx[8], sp_ky[8];
    float sp_gamma_dt[64];      // Gamma_{s_i s_j} dt, row s_i
    int wlen;                   // tabulated Langevin weight h(n), n < wlen (0: none)
    float wtab[128];
};

constexpr int kMaxSpecies = 8;

__host__ __device__ inline int species_of(const Sys &S, unsigned id)
{
    int s = 0;
    for (int k = 0; k < S.nsp - 1; ++k) s += (long long)id >= S.sp_end[k];
    return s;
}

constexpr int kScanChunk = 4096;    // cells per block of the metric-free cell scan
constexpr int kMaxKnn = 32;         // largest metric-free k

struct Ctl {
    long long step;             // steps taken; parity selects the current buffer
    int tile_next;              // dynamic tile fetch of the step kernel
    int finish_ticket;
    int dense_count;            // pipelined step: tiles listed for the whole-block routine
    int dense_next;             // ... and taken
    int pad[2];
};

// Segment: one region of one (possibly the same) tile mapped into the
// extended (tile + one-cell ring) frame of the tile being updated.
struct Seg {
    const int4 *base;
    long long bx, by;           // position map X_ext = ax * X + bx
    int count;
    int ax, ay;                 // +1 or -1 (mirror)
    int cx, cy;                 // cell map: ext = a * l + c (before the +1 ring offset)
    int flip;                   // bit0: mirrored in x, bit1: mirrored in y
    int tile, region;
};

// Per-particle staging arrays of one block: shared memory for ordinary tiles,
// the block's slice of global scratch for tiles that do not fit.
struct Stage {
    float4 *P;                  // in cell order: x, y rel. tile centre, then cos, sin as int32 in units of 2^-22
    int4 *R;                    // staged record: X, Y in the tile's extended frame (fixed
                                // point), orientation bits, id
    unsigned short *cell;       // extended cell | flip << 14
    unsigned short *slot;       // rank of arrival in the cell
    unsigned short *gidx;       // species by sorted position (several species only)
    unsigned short *sk;         // cell order -> staged index
    unsigned char *segc;        // segment of staged index 32 i
    int cap;
};

__host__ __device__ inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

__host__ __device__ inline size_t stage_bytes(int cap)
{
    return (size_t)cap * (16 + 4 * 4 + 4 * 2) + (size_t)round_up(cap / 32 + 2, 16);
}

__host__ __device__ inline void carve_stage(Stage &st, unsigned char *p, int cap)
{
    st.cap = cap;
    st.P = (float4 *)p;               p += (size_t)cap * 16;
    st.R = (int4 *)p;                 p += (size_t)cap * 16;
    st.cell = (unsigned short *)p;    p += (size_t)cap * 2;
    st.slot = (unsigned short *)p;    p += (size_t)cap * 2;
    st.gidx = (unsigned short *)p;    p += (size_t)cap * 2;
    st.sk = (unsigned short *)p;      p += (size_t)cap * 2;
    st.segc = p;
}

// Per-tile tables held in shared memory.
struct Tables {
    int *hist;                  // [nce]
    int *cstart;                // [nce + 1]
    int *rowpre;                // [kMaxTile + 1]
    int *mhist;                 // [bins_theta + bins_nbr] measured theta / |Omega| counts of the tile
};

// hist_words: bins_theta + bins_nbr of the widest system run by the launch.
__host__ __device__ inline size_t table_bytes(int nce, int hist_words)
{
    return (size_t)round_up(nce, 4) * 4 + (size_t)round_up(nce + 1, 4) * 4 + (kMaxTile + 4) * 4 +
           (size_t)round_up(hist_words, 4) * 4;
}

__host__ __device__ inline void carve_tables(Tables &t, unsigned char *p, int nce)
{
    t.hist = (int *)p;   p += (size_t)round_up(nce, 4) * 4;
    t.cstart = (int *)p; p += (size_t)round_up(nce + 1, 4) * 4;
    t.rowpre = (int *)p; p += (kMaxTile + 4) * 4;
    t.mhist = (int *)p;
}

// Spill-match list (entry, segment) kept in the block's global scratch.
__host__ __device__ inline size_t spill_list_bytes(int cap) { return (size_t)round_up(cap * 5 + 16, 256); }

}  // namespace aapk
