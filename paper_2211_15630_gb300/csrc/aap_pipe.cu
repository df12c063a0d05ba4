// aap_pipe.cu -- the pipelined tile step of one system or an ensemble of
// systems with one species each (sm_103a).
//
// One time step (Sec. 2 of Kuersten, "Aligning Active Particles Py
// Package") with the arithmetic of the whole-block tile routine of
// aap_tile.cuh, but the 32 warps of a persistent block (one per SM) split into
// three roles that hand tiles to each other through mbarriers instead of
// block-wide barriers:
//
//   copy warp (warp 0)     claims tiles, computes each tile's geometry and its
//                          25 source segments (own regions, facing halo
//                          regions with periodic shifts or mirror maps,
//                          Sec. 2.4; the cell lists of Sec. 3.2) and copies
//                          them global -> shared with one cp.async.bulk per
//                          segment into one of three raw record buffers
//                          (a tile keeps its buffer until its update is
//                          done), completing on that buffer's mbarrier;
//   sort warps (NSORT)     map each staged record into the tile's extended
//                          frame, histogram it by half cell (a cell split in
//                          two along x), prefix-scan the histogram and place
//                          the records in half-cell order (x, y and cos, sin
//                          as exact integers) into one of two output buffers,
//                          with the tile's own particles listed in that order
//                          (their sorted positions and raw records);
//   update warps (rest)    take chunks of 32 own particles from the ready
//                          output buffer, sum over three rows of five half
//                          cells (every point within R of a half cell lies in
//                          that block, which covers 15/18 of the 3x3 cells;
//                          Eq. collision_VM / collision_NVM, or the Langevin
//                          coupling sum of Eq. Langevin_dynamics) in exact
//                          integers, so the result is the 3x3 kernel's bit for
//                          bit, draw
//                          Philox noise, stream, apply the boundary rule and
//                          scatter the new records into the next step's
//                          regions.
//
// Tile i+1 is copied and sorted while the update warps work on tile i, and an
// update warp that is done with tile i starts on tile i+1 without waiting for
// the slowest warp.  Tiles whose staged set does not fit the shared buffers
// go to a list and are done at the end by the whole block with the tile
// routine of aap_tile.cuh (shared staging area or global scratch).  Every
// mbarrier wait is bounded (about two seconds of SM clock); a wait that runs
// out sets ERR_TIMEOUT in the error word and the block winds down.
#include <algorithm>
#include <atomic>
#include <cstdint>

#include <cuda_runtime.h>

#include "aap_device.cuh"
#include "aap_internal.cuh"
#include "aap_kernels.cuh"
#include "aap_tile.cuh"

namespace aapk {

namespace {

constexpr int kPipeThreads = 1024;
constexpr int kPipeWarps = kPipeThreads / 32;
constexpr int kPipeMaxChunks = 2 * kPipeMaxStage / 32 + 1;   // a wide tile spans two raw buffers
// raw buffers: a tile's holds its staged records from the copy until its
// update is done (the update reads its own particles' records there)
#ifndef AAP_PIPE_RAW_BUFFERS
#define AAP_PIPE_RAW_BUFFERS 3
#endif
constexpr int kNR = AAP_PIPE_RAW_BUFFERS;
constexpr long long kPipeWaitCycles = 4000000000ll;    // about 2 s at 2 GHz

// test hooks (aap_test_pipe_wait): the wait bound (<= 0: kPipeWaitCycles) and
// whether every block's copy warp withholds the first tile it claims
__constant__ long long c_pipe_wait_cycles;
__constant__ int c_pipe_stall;

}  // namespace

// Optional per-role timing (tracing aid, compiled out unless AAP_PIPE_TIMING
// is defined): SM cycles each role spends waiting and working, summed over
// warps and blocks.  Slots: 0 copy total, 1 copy waiting, 2 copy setup,
// 3 sort waiting for records, 4 sort waiting for a free buffer, 5 sort map,
// 6 sort order, 7 update waiting, 8 update working, 9 copy issuing the bulk copies,
// 10 tiles through the pipeline, 11 whole-block tiles, 12 kernel per block,
// 13 copy waiting for its next tile index, 14 copy planning, 15 copy spill
// records and proxy fence.
#ifdef AAP_PIPE_TIMING
__device__ unsigned long long g_pipe_t[16];
#define PT_NOW() clock64()
#define PT_ADD(i, v) atomicAdd(&g_pipe_t[i], (unsigned long long)(v))
cudaError_t read_pipe_times(unsigned long long *out16)
{
    return cudaMemcpyFromSymbol(out16, g_pipe_t, sizeof(unsigned long long) * 16);
}
#else
#define PT_NOW() 0ll
#define PT_ADD(i, v) do { } while (0)
#endif

namespace {

// Segment maps and counts of one staged tile, written by the copy warp.
struct RawMeta {
    int tile;                   // tile index, -1: no more tiles, -2: the second half of the wide tile in the
                                // buffer before (released with it), -3: empty (released at once)
    int m, m_seg, n_spill, n_own;
    int wide;                   // 1: the tile spans both raw buffers (staged from buffer 0's start)
    int si;                     // system of the tile (ensembles: its replica)
    int sx, sy, order;          // of that system: fixed-point bits per cell side, interaction order
    float ux, uy;               // length of one fixed-point unit
    int *err;                   // its error word
    int tx, ty, tw, th, twL, twR, thD, thU;
    int segpre[kSegs + 1];
    // map of segment s into the extended frame: x = offset of X (mod 2^32),
    // y = offset of Y, z = 2 e + (mirrored in x) with e the extended
    // half-cell column of source half-cell column 0, w = 2 (cy + 1) +
    // (mirrored in y); a mirrored axis negates the local index first
    int4 map[kSegs];
    unsigned char segc[kPipeMaxChunks];     // segment of staged index 32 i
    unsigned char spill_seg[kPipeMaxSpill]; // segment of staged spill record j
};

// What the update warps need of a sorted tile.
struct OutMeta {
    int tile;                   // -1: no more tiles, -2: skip (the buffer holds part of a wide tile)
    int rbuf, rwide;            // raw buffer of the tile's staged records, and whether it spans the next one too
    int n_own, tx, ty, tw, th, W2, twL, twR, thD, thU;   // W2: half cells per extended row, 2 tw + 4
    int wide;                   // a half cell holds enough particles for 512 candidates
    int dense;                  // more than 1.5 staged records per half cell on average
};

struct PipeShared {
    Sys os[2];                  // system of the tile in each output buffer (read by the update warps)
    int osys[2];                // its index, -1: none yet
    Sys cs;                     // the copy warp's current system
    RawMeta raw[kNR];
    OutMeta out[2];
    int chunk[2];               // next chunk of 32 own particles, per output buffer
    int flag;                   // a previous step's wait ran out
    int dense_tile;
    int warp_tot[kPipeWarps];
    long long red[5][kPipeWarps];
    __align__(8) unsigned long long bar_raw_full[kNR], bar_raw_empty[kNR], bar_full[2], bar_empty[2];
};

// Per-buffer shared arrays, carved from dynamic shared memory.  Buffer b of
// each kind is reached by pointer arithmetic (no arrays of pointers indexed at
// run time, which would live in local memory).
struct PipeBufs {
    int4 *raw0;                 // [kNR][cap] staged records as copied; mapped in place by the sort warps
    float4 *P0;                 // [2][cap] records in cell order: x, y from the tile centre, cos, sin (int32, 2^-22)
    unsigned short *cst0;       // [2][cst_stride] half-cell starts in P
    unsigned short *oq0;        // [2][oq_stride] position in P of own particle o
    unsigned short *or0;        // [2][oq_stride] its staged record in the tile's raw buffer(s)
    unsigned short *cellw;      // sort scratch: ey << 8 | ex (extended half cell) of staged record k
    unsigned short *slotw;      // flip << 14 | arrival rank in its half cell
    int *hist;                  // [nce] (half cells)
    int *rowoff;                // own index = position in P + rowoff[ey]
    int *mhist0;                // [2][mh_stride] measured theta / |Omega| counts of each output buffer's tile
    int cap, cap_own, cst_stride, oq_stride, mh_stride;
    __device__ __forceinline__ int *mhist(int b) const { return mhist0 + b * mh_stride; }
    __device__ __forceinline__ int4 *raw(int b) const { return raw0 + b * cap; }
    __device__ __forceinline__ float4 *P(int b) const { return P0 + b * cap; }
    __device__ __forceinline__ unsigned short *cstart(int b) const { return cst0 + b * cst_stride; }
    __device__ __forceinline__ unsigned short *ownq(int b) const { return oq0 + b * oq_stride; }
    __device__ __forceinline__ unsigned short *ownr(int b) const { return or0 + b * oq_stride; }
};

__device__ __forceinline__ void carve_pipe(PipeBufs &B, unsigned char *p, int cap, int cap_own, int nce, int hist_words)
{
    B.cap = cap;
    B.mh_stride = round_up(hist_words, 4);
    B.cap_own = cap_own;
    B.cst_stride = round_up(nce + 1, 8);
    B.oq_stride = round_up(cap_own, 8);
    B.raw0 = (int4 *)p;
    p += (size_t)kNR * cap * 16;
    B.P0 = (float4 *)p;
    p += (size_t)2 * cap * 16;
    B.cst0 = (unsigned short *)p;
    p += (size_t)2 * B.cst_stride * 2;
    B.oq0 = (unsigned short *)p;
    p += (size_t)2 * B.oq_stride * 2;
    B.or0 = (unsigned short *)p;
    p += (size_t)2 * B.oq_stride * 2;
    B.cellw = (unsigned short *)p;              // sized for a wide tile (two buffers)
    p += (size_t)round_up(2 * cap, 8) * 2;
    B.slotw = (unsigned short *)p;
    p += (size_t)round_up(2 * cap, 8) * 2;
    B.hist = (int *)p;
    p += (size_t)round_up(nce, 4) * 4;
    B.rowoff = (int *)p;
    p += (size_t)(kMaxTile + 4) * 4;
    B.mhist0 = (int *)p;
}

// ------------------------------------------------------------- mbarriers --
__device__ __forceinline__ uint32_t sa(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(sa(bar)) : "memory");
}

// count arrivals at once
__device__ __forceinline__ void mbar_arrive_cnt(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(sa(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(sa(bar)), "r"(bytes)
                 : "memory");
}

// Wait for the completion of the phase of the given parity, bounded in time.
// false: the bound ran out (ERR_TIMEOUT is set).
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, int *err)
{
    const long long t0 = clock64();
    const long long bound = c_pipe_wait_cycles > 0 ? c_pipe_wait_cycles : kPipeWaitCycles;
    for (;;) {
        unsigned done;
        // the hint lets the hardware suspend the warp (up to 0.1 ms) instead of
        // spinning on issue slots the working warps need
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done) : "r"(sa(bar)), "r"(parity), "r"(100000u) : "memory");
        if (done) return true;
        if (clock64() - t0 > bound) {
            atomicOr(err, ERR_TIMEOUT);
            return false;
        }
    }
}

// Every lane of the warp polls (one instruction for the warp), so that each
// lane itself acquires what the phase released; the outcome is made
// warp-uniform (a lane whose bound ran out makes the warp give up).
__device__ __forceinline__ bool warp_wait(unsigned long long *bar, unsigned parity, int *err)
{
    const bool ok = mbar_wait(bar, parity, err);
    return __all_sync(0xffffffffu, ok);
}

// Named barrier of the sort warps (id 1).
__device__ __forceinline__ void sort_sync(int nthreads)
{
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// The same barrier, returning whether every participating thread passed ok.
__device__ __forceinline__ bool sort_sync_and(int nthreads, bool ok)
{
    int r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
                 "bar.red.and.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
                 : "=r"(r) : "r"((int)ok), "r"(nthreads) : "memory");
    return r != 0;
}

// One bulk copy global -> shared of `bytes` (a multiple of 16, both addresses
// 16-byte aligned) that completes on bar's transaction count.
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(sa(dst)), "l"(src), "r"(bytes), "r"(sa(bar)) : "memory");
}

// -------------------------------------------------------------- copy warp --
// What the copy warp learns of a tile before it needs a raw buffer: the
// geometry and, in lane s < 25, source segment s with its record count and
// the inclusive prefix of the counts.
struct CopyPlan {
    TileGeo G;
    Seg sg;
    int c, incl, m_seg, own_seg;
};

// Geometry and the 25 segments of tile g (all lanes of the copy warp; global
// loads of the region counts, no shared-memory writes).
__device__ __forceinline__ void copy_plan(const Sys &S, int g, int cur, CopyPlan &pl)
{
    const int lane = threadIdx.x & 31;
    pl.G = tile_geo(S, g);
    if (lane < kSegs) pl.sg = make_seg(S, pl.G, lane, cur);
    pl.c = lane < kSegs ? pl.sg.count : 0;
    pl.incl = warp_incl_scan(pl.c);
    pl.m_seg = __shfl_sync(0xffffffffu, pl.incl, kSegs - 1);
    pl.own_seg = __shfl_sync(0xffffffffu, pl.incl, 8);
}

// The planned tile's spill matches (nsp spilled records): spill_e / spill_s
// (the copy warp's global scratch) receive the spill entry and the segment of
// staged spill record j; n_spill and the own count follow.  Only a tile whose
// source tiles received spilled records (their bits in spill_bits) looks at
// the list, and only a short list is scanned here: false (warp-uniform) when
// the tile must go to the whole-block routine, which scans with all threads.
__device__ __forceinline__ bool copy_spills(const Sys &S, const CopyPlan &pl, int cur, int nsp, int *spill_e,
                                            unsigned char *spill_s, int &n_spill, int &n_own)
{
    const int lane = threadIdx.x & 31;
    int ns = 0, nos = 0;
    bool near = false;
    if (nsp > 0) {
        const bool b = lane < kSegs && ((S.spill_bits[cur][pl.sg.tile >> 5] >> (pl.sg.tile & 31)) & 1u);
        near = __any_sync(0xffffffffu, b);
    }
    if (near && nsp > kPipeSpillScan) return false;
    if (near) {
        const int mt = lane < kSegs ? pl.sg.tile : -1, mr = lane < kSegs ? pl.sg.region : -1;
        for (int e0 = 0; e0 < nsp; e0 += 32) {
            const int e = e0 + lane;
            const int key = e < nsp ? S.spill_key[cur][e] : -1;
            const int et = key >= 0 ? key / kCntStride : -2, er = key >= 0 ? key % kCntStride : -2;
            for (int s = 0; s < kSegs; ++s) {
                const int st = __shfl_sync(0xffffffffu, mt, s), sr = __shfl_sync(0xffffffffu, mr, s);
                const bool hit = et == st && er == sr;
                const unsigned bal = __ballot_sync(0xffffffffu, hit);
                const int j = ns + __popc(bal & ((1u << lane) - 1u));
                if (hit && j < kPipeMaxSpill) {
                    spill_s[j] = (unsigned char)s;
                    spill_e[j] = e;
                }
                ns += __popc(bal);
                if (s < 9) nos += __popc(bal);
            }
        }
    }
    __syncwarp();
    n_spill = ns;
    n_own = pl.own_seg + nos;
    return true;
}

// The planned tile's meta into raw buffer meta M (the raw buffer, or both for
// a wide tile, must be free).
__device__ __forceinline__ void copy_commit(const CopyPlan &pl, const Sys &S, int si, int g, RawMeta &M, int n_spill,
                                            int n_own, int wide, const unsigned char *spill_s)
{
    const int lane = threadIdx.x & 31;
    const Seg &sg = pl.sg;
    const int m_seg = pl.m_seg;
    const int start = pl.incl - pl.c;                   // segment start (lanes < 25)
    if (lane < kSegs) {
        M.segpre[lane] = start;
        // the mapped coordinate fits int32, so its offset is kept mod 2^32;
        // extended half-cell column of local half cell h: a h + 2 cx + (mirrored) + 2
        const int mxr = sg.ax < 0;
        M.map[lane] = make_int4((int)(unsigned)(unsigned long long)sg.bx, (int)(unsigned)(unsigned long long)sg.by,
                                2 * (2 * sg.cx + mxr + 2) + mxr, 2 * (sg.cy + 1) + (sg.ay < 0));
    }
    for (int j = lane; j < n_spill; j += 32) M.spill_seg[j] = spill_s[j];
    if (lane == 0) {
        M.segpre[kSegs] = m_seg;
        M.tile = g;
        M.m = m_seg + n_spill;
        M.m_seg = m_seg;
        M.n_spill = n_spill;
        M.n_own = n_own;
        M.wide = wide;
        M.si = si;
        M.sx = S.sx;
        M.sy = S.sy;
        M.order = S.order;
        M.ux = S.ux;
        M.uy = S.uy;
        M.err = S.err;
        M.tx = pl.G.tx; M.ty = pl.G.ty; M.tw = pl.G.tw; M.th = pl.G.th;
        M.twL = pl.G.twL; M.twR = pl.G.twR; M.thD = pl.G.thD; M.thU = pl.G.thU;
    }
    // segment of every 32nd staged index: the last segment starting at or
    // before it (segment starts taken from the lanes, no shared-memory reads)
    const int sp = lane < kSegs ? start : 0x7fffffff;
    for (int i0 = 0; i0 * 32 < m_seg; i0 += 32) {
        const int k = (i0 + lane) * 32;
        // binary search over the non-decreasing starts: the last segment s
        // with start <= k (segment 0 starts at 0)
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int v = __shfl_sync(0xffffffffu, sp, min(lo + step, 31));
            if (lo + step < kSegs && v <= k) lo += step;
        }
        if (k < m_seg) M.segc[i0 + lane] = (unsigned char)lo;
    }
    __syncwarp();
}

// ------------------------------------------------------------- sort warps --
// Map every staged record of raw buffer r into the tile's extended frame (in
// place) and histogram it by cell.  tid: index among the NS sort threads.
__device__ __forceinline__ void sort_map(PipeShared &sh, const PipeBufs &B, int r, int tid, int NS)
{
    const RawMeta &M = sh.raw[r];
    const int m = M.m, m_seg = M.m_seg;
    const int W2 = 2 * M.tw + 4, H2 = M.th + 2;       // half cells per extended row, rows
    int4 *R = B.raw(r);
    for (int k = tid; k < m; k += NS) {
        int s;
        if (k < m_seg) {
            s = M.segc[k >> 5];
            while (M.segpre[s + 1] <= k) ++s;
        } else {
            s = M.spill_seg[k - m_seg];
        }
        const int4 rr = R[k];
        const int4 g = M.map[s];
        const int mx = -(g.z & 1), my = -(g.w & 1);       // all ones where the axis is mirrored
        const int lx = rr.x >> (M.sx - 1), ly = rr.y >> M.sy;
        int ex = ((lx ^ mx) - mx) + (g.z >> 1), ey = ((ly ^ my) - my) + (g.w >> 1);
        if ((unsigned)ex >= (unsigned)W2 || (unsigned)ey >= (unsigned)H2) {
            atomicOr(M.err, ERR_BOUNDS);
            ex = min(max(ex, 0), W2 - 1);
            ey = min(max(ey, 0), H2 - 1);
        }
        // X_ext = a X + b in 32-bit wrapping arithmetic (the result fits int32)
        const unsigned Xe = ((unsigned)rr.x ^ (unsigned)mx) - (unsigned)mx + (unsigned)g.x;
        const unsigned Ye = ((unsigned)rr.y ^ (unsigned)my) - (unsigned)my + (unsigned)g.y;
        R[k] = make_int4((int)Xe, (int)Ye, rr.z, rr.w);
        B.cellw[k] = (unsigned short)((ey << 8) | ex);
        B.slotw[k] = (unsigned short)((((g.z & 1) | ((g.w & 1) << 1)) << 14) | atomicAdd(&B.hist[ey * W2 + ex], 1));
    }
}

// Scan the histogram into output buffer b's cell starts (clearing the
// histogram), the own-row offsets and the tile's output meta, then place the
// records in cell order.  The output buffer must be free.
template <int MODEL>
__device__ __forceinline__ void sort_order(PipeShared &sh, const PipeBufs &B, int r, int b, int tid, int NS,
                                           int cap_own)
{
    const RawMeta &M = sh.raw[r];
    const int m = M.m, tw = M.tw, th = M.th;
    const int W2 = 2 * tw + 4, nce = W2 * (th + 2);     // half cells of the extended tile
    unsigned short *cst = B.cstart(b);
    const int lane = tid & 31, w = tid >> 5, nw = NS >> 5;
    int maxc = 0;
    {
        const int per = (nce + NS - 1) / NS;
        const int b0 = min(tid * per, nce), e0 = min(b0 + per, nce);
        int sum = 0;
        for (int i = b0; i < e0; ++i) {
            const int h = B.hist[i];
            sum += h;
            maxc = max(maxc, h);
        }
        const int incl = warp_incl_scan(sum);
        if (lane == 31) sh.warp_tot[w] = incl;
        sort_sync(NS);
        if (w == 0) {
            const int v = lane < nw ? sh.warp_tot[lane] : 0;
            const int wi = warp_incl_scan(v);
            if (lane < nw) sh.warp_tot[lane] = wi - v;
            if (lane == nw - 1) cst[nce] = (unsigned short)wi;
        }
        sort_sync(NS);
        int run = incl - sum + sh.warp_tot[w];
        for (int i = b0; i < e0; ++i) {
            cst[i] = (unsigned short)run;
            run += B.hist[i];
            B.hist[i] = 0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxc = max(maxc, __shfl_xor_sync(0xffffffffu, maxc, o));
    sort_sync(NS);                            // every warp has read its scan offset
    if (lane == 0) sh.warp_tot[w] = maxc;
    sort_sync(NS);
    // own rows: index offsets; the tile's output meta
    if (w == 0) {
        int carry = 0;
        for (int r0 = 0; r0 < th; r0 += 32) {
            const int rw = r0 + lane;
            int len = 0, first = 0;
            if (rw < th) {               // own half cells 2 .. 2 tw + 1 of row rw + 1
                first = cst[(rw + 1) * W2 + 2];
                len = cst[(rw + 1) * W2 + 2 * tw + 2] - first;
            }
            const int incl = warp_incl_scan(len);
            if (rw < th) B.rowoff[rw + 1] = carry + incl - len - first;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        int mx = lane < nw ? sh.warp_tot[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) {
            OutMeta &O = sh.out[b];
            O.tile = M.tile;
            O.rbuf = r;
            O.rwide = M.wide;
            O.n_own = min(carry, cap_own);
            O.tx = M.tx; O.ty = M.ty; O.tw = tw; O.th = th; O.W2 = W2;
            O.twL = M.twL; O.twR = M.twR; O.thD = M.thD; O.thU = M.thU;
            O.wide = 15 * mx >= 512;
            O.dense = 2 * m > 3 * nce;
            sh.chunk[b] = 0;
            if (carry != M.n_own) atomicOr(M.err, ERR_BOUNDS);
        }
    }
    sort_sync(NS);
    // records into cell order (arrival order inside a cell: the sums are
    // exact integers, so this order does not matter); own particles listed
    const int xc = tw << (M.sx - 1), yc = th << (M.sy - 1);
    const int4 *R = B.raw(r);
    float4 *P = B.P(b);
    unsigned short *OR = B.ownr(b);
    unsigned short *OQ = B.ownq(b);
    for (int k = tid; k < m; k += NS) {
        const unsigned cf = B.cellw[k], sl = B.slotw[k];
        const int ex = cf & 255, ey = cf >> 8;
        const int q = cst[ey * W2 + ex] + (sl & 0x3fff);
        const int4 rk = R[k];
        float thv = __int_as_float(rk.z);
        float sn, cs;
        if (MODEL == 1 && M.order != 1) {
            thv *= (float)M.order;
            sincosf(thv, &sn, &cs);
        } else {
            // |theta| <= pi: the hardware sine/cosine is within 2^-21.4 absolute
            __sincosf(thv, &sn, &cs);
        }
        const int flip = sl >> 14;
        if (flip & 1) {
            if (MODEL != 1 || (M.order & 1)) cs = -cs; else sn = -sn;
        }
        if (flip & 2) sn = -sn;
        P[q] = make_float4((float)(rk.x - xc) * M.ux, (float)(rk.y - yc) * M.uy,
                           __int_as_float(__float2int_rn(cs * kFixNbF)), __int_as_float(__float2int_rn(sn * kFixNbF)));
        if (ex >= 2 && ex < 2 * tw + 2 && ey >= 1 && ey <= th) {
            const int o = q + B.rowoff[ey];
            if (o < cap_own) {
                OR[o] = (unsigned short)k;      // the update reads the record in the raw buffer
                OQ[o] = (unsigned short)q;
            }
        }
    }
}

// ----------------------------------------------------------- update warps --
// The neighbour sum of one particle over three rows of five half cells,
// each row contiguous in the half-cell order.  The particle itself is
// included (it adds e^{i theta_i} to the VM/NVM sum and sin 0 to the
// Langevin sum; cnt counts it).  The staged (cos, sin) are integers in units
// of 2^-22, so the sums are exact and order-free; ACC is int below 512
// candidates and long long beyond.
template <int MODEL, typename ACC, int UNR>
__device__ __forceinline__ void neighbour_sum_h(const float4 *__restrict__ P, const unsigned short *cstart, int ec,
                                                int W2, float4 pi, float r2, ACC &sc, ACC &ss, int &cnt)
{
    sc = 0;
    ss = 0;
    cnt = 0;
    const float pcf = (float)__float_as_int(pi.z), psf = (float)__float_as_int(pi.w);
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
        const int c0 = ec + dy * W2 - 2;
        const int a = cstart[c0], b = cstart[c0 + 5];
#pragma unroll UNR
        for (int j = a; j < b; ++j) {
            const float4 pj = P[j];
            const float dx = pj.x - pi.x, dyy = pj.y - pi.y;
            const float d2 = fmaf(dx, dx, dyy * dyy);
            if (d2 <= r2) {
                int cj = __float_as_int(pj.z), sj = __float_as_int(pj.w);
                if (MODEL == 2 && fmaf(pcf, (float)cj, psf * (float)sj) < 0.f) {
                    cj = -cj;                         // Eq. (collision_NVM): the reversed direction
                    sj = -sj;
                }
                sc += cj;
                ss += sj;
                ++cnt;
            }
        }
    }
}

struct Acc {
    long long c, s, n, c2, s2;
};

// One particle per lane (own index o, inactive when o >= n_own); every lane
// of the warp must call (the scatter is warp-aggregated).
template <int MODEL>
__device__ __forceinline__ void update_one(const Sys &S, const OutMeta &O, const float4 *__restrict__ P,
                                           const unsigned short *cstart, const int4 *RB, const unsigned short *OR,
                                           const unsigned short *OQ,
                                           int o, long long step, bool measure, int *mhist, Acc &acc)
{
    const int nxt = (int)(step & 1) ^ 1;
    const bool act = o < O.n_own;
    int4 rec = make_int4(0, 0, 0, 0);
    int dtile = 0, region = 0;
    if (act) {
        const int tw = O.tw, th = O.th, W2 = O.W2;
        const int4 rk = RB[OR[o]];                // own regions map to themselves (no shift, no mirror)
        const int X = rk.x, Y = rk.y;
        const float thi = __int_as_float(rk.z);
        const unsigned id = (unsigned)rk.w;
        const int ec = ((Y >> S.sy) + 1) * W2 + (X >> (S.sx - 1)) + 2;      // extended half cell
        const float4 pi = P[OQ[o]];
        float sc, ss;                    // neighbour sums in units of 2^-22
        int cnt;
        bool narrow = !O.wide;
        if (!narrow) {
            const int ncand = cstart[ec - W2 + 3] - cstart[ec - W2 - 2] + cstart[ec + 3] - cstart[ec - 2] +
                              cstart[ec + W2 + 3] - cstart[ec + W2 - 2];
            narrow = ncand < 512;
        }
        if (narrow) {
            // short candidate rows run faster unrolled twice, long ones
            // (dense tiles) four times
            int a, b;
            if (O.dense) neighbour_sum_h<MODEL, int, 4>(P, cstart, ec, W2, pi, S.r2, a, b, cnt);
            else neighbour_sum_h<MODEL, int, 2>(P, cstart, ec, W2, pi, S.r2, a, b, cnt);
            sc = (float)a;
            ss = (float)b;
        } else {
            long long a, b;
            neighbour_sum_h<MODEL, long long, 4>(P, cstart, ec, W2, pi, S.r2, a, b, cnt);
            sc = (float)a;
            ss = (float)b;
        }
        const int nb = cnt - 1;          // the particle itself was counted
        if (measure) {
            int bt = (int)floorf((thi + AAP_PI_F) * ((float)S.bins_theta * (1.0f / AAP_2PI_F)));
            bt = min(max(bt, 0), S.bins_theta - 1);
            atomicAdd(&mhist[bt], 1);
            atomicAdd(&mhist[S.bins_theta + min(nb, S.bins_nbr - 1)], 1);
        }
        uint32_t c4[4] = {id, (uint32_t)step, (uint32_t)((unsigned long long)step >> 32), 0u};
        philox4x32_10(c4, S.seed_lo, S.seed_hi);
        const float u0 = u01f(c4[0]);
        float thn, cn, sn;
        int dX, dY;
        if (MODEL != 1) {
            // Eq. (collision_VM) / (collision_NVM) + noise; Eq. (streaming)
            thn = arg2(ss, sc) + S.omega_step + S.eta_pi * (2.0f * u0 - 1.0f);
            __sincosf(thn, &sn, &cn);
            dX = __float2int_rn(S.kx * cn);
            dY = __float2int_rn(S.ky * sn);
        } else {
            // Eq. (Langevin_dynamics), one Euler-Maruyama step
            const float u1 = u01f(c4[1]);
            const float h = S.wlen > 0 ? S.wtab[min(nb, S.wlen - 1)]
                                       : (S.weight ? 1.0f : 1.0f / (1.0f + (float)nb));
            // sum_j sin(o (theta_j - theta_i)) from the exact sums (units 2^-22 x 2^-22)
            const float tsum = ((float)__float_as_int(pi.z) * ss - (float)__float_as_int(pi.w) * sc) *
                               (1.0f / (kFixNbF * kFixNbF));
            const float gz = sqrtf(-2.0f * logf(u0)) * cospif(2.0f * u1);
            thn = thi + S.gamma_dt * h * tsum + S.omega_step + S.noise_amp * gz;
            float co, so;
            __sincosf(thi, &so, &co);    // streaming direction theta(t), |theta| <= pi
            dX = __float2int_rn(S.kx * co);
            dY = __float2int_rn(S.ky * so);
            cn = 0.f;
            sn = 0.f;
        }
        // boundary rule (Sec. 2.4) in exact fixed point
        const int TWs = tw << S.sx, THs = th << S.sy;
        int Xn = X + dX, Yn = Y + dY;
        int dtx = O.tx, dty = O.ty, twd = tw, thd = th;
        bool fx = false, fy = false;
        if (Xn < 0) {
            if (S.bx && O.tx == 0) { Xn = -Xn; fx = true; }
            else { dtx = O.tx > 0 ? O.tx - 1 : S.ntx - 1; twd = O.twL; Xn += O.twL << S.sx; }
        } else if (Xn >= TWs) {
            if (S.bx && O.tx == S.ntx - 1) {
                if (Xn == TWs) Xn = TWs - 1; else { Xn = TWs - (Xn - TWs); fx = true; }
            } else { dtx = O.tx < S.ntx - 1 ? O.tx + 1 : 0; twd = O.twR; Xn -= TWs; }
        }
        if (Yn < 0) {
            if (S.by && O.ty == 0) { Yn = -Yn; fy = true; }
            else { dty = O.ty > 0 ? O.ty - 1 : S.nty - 1; thd = O.thD; Yn += O.thD << S.sy; }
        } else if (Yn >= THs) {
            if (S.by && O.ty == S.nty - 1) {
                if (Yn == THs) Yn = THs - 1; else { Yn = THs - (Yn - THs); fy = true; }
            } else { dty = O.ty < S.nty - 1 ? O.ty + 1 : 0; thd = O.thU; Yn -= THs; }
        }
        if (fx) { thn = AAP_PI_F - thn; cn = -cn; }
        if (fy) { thn = -thn; sn = -sn; }
        if (thn >= AAP_PI_F || thn < -AAP_PI_F)
            thn -= AAP_2PI_F * floorf((thn + AAP_PI_F) * (1.0f / AAP_2PI_F));
        if (MODEL == 1) __sincosf(thn, &sn, &cn);
        if (!isfinite(thn)) atomicOr(S.err, ERR_NAN);
        dtile = dty * S.ntx + dtx;
        region = region_of(Xn >> S.sx, Yn >> S.sy, twd, thd);
        rec = make_int4(Xn, Yn, __float_as_int(thn), (int)id);
        acc.c += __float2int_rn(cn * kFixStepF);
        acc.s += __float2int_rn(sn * kFixStepF);
        acc.c2 += __float2int_rn(fmaf(cn, cn, -sn * sn) * kFixStepF);
        acc.s2 += __float2int_rn(2.0f * cn * sn * kFixStepF);
        acc.n += nb;
        if (S.nbr_out && id < (unsigned long long)S.n) S.nbr_out[id] = nb;
    }
    warp_insert(S, nxt, act, dtile, region, rec);
}

}  // namespace

// nceh: half cells of the largest extended tile, (2 tw + 4)(th + 2).
__host__ __device__ size_t pipe_smem_bytes(int cap, int cap_own, int nceh, int hist_words)
{
    return (size_t)(kNR + 2) * cap * 16 + 2 * (size_t)round_up(nceh + 1, 8) * 2 +
           4 * (size_t)round_up(cap_own, 8) * 2 + 2 * (size_t)round_up(2 * cap, 8) * 2 +
           (size_t)round_up(nceh, 4) * 4 + (size_t)(kMaxTile + 4) * 4 + 2 * (size_t)round_up(hist_words, 4) * 4;
}

// Flush output buffer b's measured histograms into the system of the tile it
// held, and clear them.  tid, nt: the calling threads.
__device__ __forceinline__ void flush_hist(PipeShared &sh, const PipeBufs &B, int b, long long step, int tid, int nt)
{
    if (sh.osys[b] < 0) return;
    const Sys &S = sh.os[b];
    if (step < S.meas_until) {
        int *mh = B.mhist(b);
        for (int i = tid; i < S.bins_theta + S.bins_nbr; i += nt)
            if (mh[i]) {
                atomicAdd(S.hist + i, (unsigned long long)mh[i]);
                mh[i] = 0;
            }
    }
}

// A warp's integer sums of one system (exact, so order-free) into that
// system's step accumulators.
__device__ __forceinline__ void flush_acc(const Acc &acc, unsigned long long *sys_acc, int cur)
{
    const long long a[5] = {acc.c, acc.s, acc.n, acc.c2, acc.s2};
    const int lane = threadIdx.x & 31;
    unsigned long long *slot =
        sys_acc + ((size_t)cur * kAccSlots + ((blockIdx.x * 32 + (threadIdx.x >> 5)) & (kAccSlots - 1))) * kAccWords;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const long long v = warp_sum_ll(a[k]);
        if (lane == 0 && v) atomicAdd(slot + k, (unsigned long long)v);
    }
}

// The pipelined step of one or more systems with one species each (any
// model; the systems of one launch share it): one block of kPipeThreads
// threads per SM.  tile_base[nsys + 1] is the prefix of the systems' tiles.
template <int MODEL, int NSORT>
__global__ void __launch_bounds__(kPipeThreads, 1)
k_step_pipe(const Sys *__restrict__ sys, int nsys, const int *__restrict__ tile_base, Ctl *ctl, int cap, int cap_own,
            int nceh_max, int nce_max, int hist_words, int *dense_list, unsigned char *scratch,
            size_t scratch_per_block, int scratch_cap, int spill_list_cap)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ PipeShared sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long tk0 = PT_NOW();
    (void)tk0;
    constexpr int NS = NSORT * 32;                          // sort threads
    constexpr int NU = kPipeWarps - 1 - NSORT;              // update warps
    PipeBufs B;
    carve_pipe(B, smem, cap, cap_own, nceh_max, hist_words);
    if (tid == 0) {
        for (int b = 0; b < kNR; ++b) {
            mbar_init(&sh.bar_raw_full[b], 1);
            mbar_init(&sh.bar_raw_empty[b], NU);    // released by the update warps (or a token by the sort)
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sh.bar_full[b], 1);
            mbar_init(&sh.bar_empty[b], NU);
            sh.osys[b] = -1;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < nceh_max; i += kPipeThreads) B.hist[i] = 0;
    for (int i = tid; i < 2 * B.mh_stride; i += kPipeThreads) B.mhist0[i] = 0;
    // pipeline waits that run out are reported in the first system's error word
    int *const err0 = sys[0].err;
    if (tid == 0) sh.flag = *((volatile int *)err0) & ERR_TIMEOUT;
    __syncthreads();
    // after a wait has run out the handle is unusable: later steps do nothing
    // (so that a queue of steps cannot each wait out their bounds)
    if (sh.flag) return;
    const long long step = ctl->step;
    const int cur = (int)(step & 1);
    const int total = tile_base[nsys];
    unsigned char *mine = scratch + scratch_per_block * blockIdx.x;

    if (warp == 0) {
        // ---------------------------------------------------- copy warp --
        // Each tile is planned (its system, geometry, segments, counts: global
        // loads) while the sort warps still hold the raw buffer it will go to;
        // only writing its meta and issuing its copies wait for that buffer.
        // A tile with up to twice the staging capacity goes as one wide tile
        // over both raw buffers (from buffer 0's start; the other buffer gets
        // a skip token), so that it stays in the pipeline; larger ones go to
        // the list for the whole-block routine.
        int *spill_e = reinterpret_cast<int *>(mine);
        unsigned char *spill_s = reinterpret_cast<unsigned char *>(spill_e + kPipeMaxSpill);
        unsigned kpar = 0, used = 0;       // per raw buffer: parity of its fills, filled before
        int r = 0;
        int g = 0;
        if (lane == 0) g = atomicAdd(&ctl->tile_next, 1);
        g = __shfl_sync(0xffffffffu, g, 0);
        // the planned tile: its system, local index and the system's spill
        // list length (final during this step), re-read when the system changes
        int si = -1, lt = 0, nsp = 0;
        CopyPlan pl;
        const Sys &Sc = sh.cs;
        auto plan = [&](int gg) {
            const int s2 = nsys > 1 ? sys_of_tile(tile_base, nsys, gg) : 0;
            if (s2 != si) {
                si = s2;
                const int words = (int)(sizeof(Sys) / 4);
                const int *src = reinterpret_cast<const int *>(sys + si);
                int *dst = reinterpret_cast<int *>(&sh.cs);
                for (int i = lane; i < words; i += 32) dst[i] = src[i];
                __syncwarp();
                nsp = min(*((volatile int *)&Sc.spill_cnt[cur]), Sc.spill_cap);
            }
            lt = gg - (nsys > 1 ? tile_base[si] : 0);
            copy_plan(Sc, lt, cur, pl);
        };
        const long long tc0 = PT_NOW();
        if (g < total) plan(g);
        bool ok = true;
        bool withhold = c_pipe_stall != 0;
        for (;;) {
            // the following tile, claimed now so that its round trip overlaps this one's copies
            int gn = 0;
            if (g < total && lane == 0) gn = atomicAdd(&ctl->tile_next, 1);
            int n_spill = 0, n_own = 0, mode = 0;               // 0: whole-block list, 1: normal, 2: wide
            if (g < total) {
                const bool scanned = copy_spills(Sc, pl, cur, nsp, spill_e, spill_s, n_spill, n_own);
                const int m = pl.m_seg + n_spill;
                if (scanned && n_spill <= kPipeMaxSpill) {
                    if (m <= cap && n_own <= cap_own) mode = 1;
                    else if (m <= 2 * cap && n_own <= 2 * cap_own) mode = 2;
                }
                if (mode == 0) {
                    // done by the whole block after the pipeline
                    if (lane == 0) {
                        const int j = atomicAdd(&ctl->dense_count, 1);
                        dense_list[j] = g + 1;
                    }
                    g = __shfl_sync(0xffffffffu, gn, 0);
                    if (g < total) plan(g);
                    continue;
                }
                if (mode == 2 && r == kNR - 1) {
                    // a wide tile needs two adjacent buffers: the last one
                    // passes an empty token first and the tile starts at 0
                    if (((used >> r) & 1u) && !warp_wait(&sh.bar_raw_empty[r], ((kpar >> r) & 1u) ^ 1u, err0)) {
                        ok = false;
                        break;
                    }
                    if (lane == 0) {
                        sh.raw[r].tile = -3;
                        mbar_arrive(&sh.bar_raw_full[r]);
                    }
                    kpar ^= 1u << r;
                    used |= 1u << r;
                    r = 0;
                }
            }
            // the raw buffer (both for a wide tile) must be free (its previous tile updated)
            const long long tw0 = PT_NOW();
            if (((used >> r) & 1u) && !warp_wait(&sh.bar_raw_empty[r], ((kpar >> r) & 1u) ^ 1u, err0)) {
                ok = false;
                break;
            }
            if (mode == 2 && ((used >> (r + 1)) & 1u) &&
                !warp_wait(&sh.bar_raw_empty[r + 1], ((kpar >> (r + 1)) & 1u) ^ 1u, err0)) {
                ok = false;
                break;
            }
            if (lane == 0) PT_ADD(1, PT_NOW() - tw0);
            RawMeta &M = sh.raw[r];
            if (g >= total) {
                if (lane == 0) {
                    M.tile = -1;
                    mbar_arrive(&sh.bar_raw_full[r]);
                }
                break;
            }
            const Sys &Sg = Sc;
            const long long ts0 = PT_NOW();
            copy_commit(pl, Sg, si, lt, M, n_spill, n_own, mode == 2, spill_s);
            if (lane == 0) PT_ADD(2, PT_NOW() - ts0);
            const long long ti0 = PT_NOW();
            int4 *R = B.raw(r);
            // spilled records by plain loads, after the segments
            for (int j = lane; j < n_spill; j += 32) R[pl.m_seg + j] = Sg.spill_rec[cur][spill_e[j]];
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            const long long ti1 = PT_NOW();
            if (withhold) {
                // test hook: this fill never arrives, so the waits behind it run out
                withhold = false;
            } else {
                if (lane == 0) mbar_arrive_tx(&sh.bar_raw_full[r], (unsigned)pl.m_seg * 16u);
                __syncwarp();
                if (lane < kSegs && pl.c > 0)
                    bulk_copy(R + (pl.incl - pl.c), pl.sg.base, (unsigned)pl.c * 16u, &sh.bar_raw_full[r]);
            }
            __syncwarp();
            if (lane == 0) {
                PT_ADD(15, ti1 - ti0);
                PT_ADD(9, PT_NOW() - ti1);
            }
            kpar ^= 1u << r;
            used |= 1u << r;
            if (mode == 2) {
                // the wide tile's second buffer: a token (no copies into it;
                // released together with the tile by the update warps)
                if (lane == 0) {
                    sh.raw[r + 1].tile = -2;
                    mbar_arrive(&sh.bar_raw_full[r + 1]);
                }
                kpar ^= 2u << r;
                used |= 2u << r;
                r = (r + 2) % kNR;
            } else {
                r = (r + 1) % kNR;
            }
            const long long tq0 = PT_NOW();
            g = __shfl_sync(0xffffffffu, gn, 0);
            const long long tq1 = PT_NOW();
            if (g < total) plan(g);
            if (lane == 0) {
                PT_ADD(13, tq1 - tq0);
                PT_ADD(14, PT_NOW() - tq1);
            }
        }
        if (!ok) {
            // given up: before the block may exit, the bulk copies of the last
            // fill of each raw buffer must have landed.  Those fills were
            // issued at least one wait bound ago and nothing has filled the
            // buffers since, so the phase of each last fill is the barrier's
            // latest and the bounded wait returns at once.
            for (int b = 0; b < kNR; ++b)
                if ((used >> b) & 1u) warp_wait(&sh.bar_raw_full[b], ((kpar >> b) & 1u) ^ 1u, err0);
        }
        if (lane == 0) PT_ADD(0, PT_NOW() - tc0);
    } else if (warp <= NSORT) {
        // --------------------------------------------------- sort warps --
        const int st = tid - 32;
        unsigned rpar = 0, opar = 0, oused = 0;
        int r = 0, b = 0;
        for (;;) {
            long long t0 = PT_NOW();
            bool ok = mbar_wait(&sh.bar_raw_full[r], (rpar >> r) & 1u, err0);
            if (!sort_sync_and(NS, ok)) break;
            if (st == 0) PT_ADD(3, PT_NOW() - t0);
            rpar ^= 1u << r;
            const int tile = sh.raw[r].tile;
            if (tile == -2 || tile == -3) {
                // a token: the second half of the wide tile just sorted (the
                // update warps release it with the tile), or an empty buffer
                // (released here, for all the update warps)
                if (tile == -3 && st == 0) mbar_arrive_cnt(&sh.bar_raw_empty[r], (unsigned)NU);
                r = (r + 1) % kNR;
                continue;
            }
            const bool end = tile < 0;
            const bool wide = !end && sh.raw[r].wide;
            if (wide && b == 1) {
                // a wide tile fills output buffers 0 and 1: buffer 1 passes a skip token first
                ok = !((oused >> 1) & 1u) || mbar_wait(&sh.bar_empty[1], ((opar >> 1) & 1u) ^ 1u, err0);
                if (!sort_sync_and(NS, ok)) break;
                if (st == 0) {
                    sh.out[1].tile = -2;
                    mbar_arrive(&sh.bar_full[1]);
                }
                opar ^= 2u;
                oused |= 2u;
                b = 0;
            }
            t0 = PT_NOW();
            if (!end) sort_map(sh, B, r, st, NS);
            if (st == 0) PT_ADD(5, PT_NOW() - t0);
            // the output buffer (both for a wide tile) must be free (its previous tile updated)
            t0 = PT_NOW();
            ok = !((oused >> b) & 1u) || mbar_wait(&sh.bar_empty[b], ((opar >> b) & 1u) ^ 1u, err0);
            if (wide) ok = ok && (!((oused >> 1) & 1u) || mbar_wait(&sh.bar_empty[1], ((opar >> 1) & 1u) ^ 1u, err0));
            if (!sort_sync_and(NS, ok)) break;
            if (st == 0) PT_ADD(4, PT_NOW() - t0);
            if (end) {
                if (st == 0) {
                    sh.out[b].tile = -1;
                    mbar_arrive(&sh.bar_full[b]);
                }
                break;
            }
            t0 = PT_NOW();
            // the buffer's histograms go to the system of its previous tile (when
            // measuring); the buffer takes this tile's system
            const int si = sh.raw[r].si;
            const int oi = sh.osys[b];
            if (oi >= 0 && step < sh.os[b].meas_until) {
                flush_hist(sh, B, b, step, st, NS);
                sort_sync(NS);
            }
            if (oi != si) {
                const int words = (int)(sizeof(Sys) / 4);
                const int *src = reinterpret_cast<const int *>(sys + si);
                int *dst = reinterpret_cast<int *>(&sh.os[b]);
                for (int i = st; i < words; i += NS) dst[i] = src[i];
                if (st == 0) sh.osys[b] = si;
            }
            sort_order<MODEL>(sh, B, r, b, st, NS, wide ? 2 * cap_own : cap_own);
            sort_sync(NS);
            if (st == 0) {
                PT_ADD(6, PT_NOW() - t0);
                PT_ADD(10, 1);
                mbar_arrive(&sh.bar_full[b]);
                if (wide) {
                    sh.out[1].tile = -2;
                    mbar_arrive(&sh.bar_full[1]);
                }
            }
            opar ^= 1u << b;
            oused |= 1u << b;
            if (wide) {
                opar ^= 2u;
                oused |= 2u;
                b = 0;
            } else {
                b ^= 1;
            }
            r = (r + 1) % kNR;
        }
    } else {
        // ------------------------------------------------- update warps --
        // Each warp sums its particles' contributions in registers and hands
        // them to the system's accumulators when it moves to another system
        // (a single system: once, at the end).
        unsigned fpar = 0;
        int b = 0;
        Acc acc = {0, 0, 0, 0, 0};
        unsigned long long *acc_sys = nullptr;
        for (;;) {
            const long long t0 = PT_NOW();
            if (!warp_wait(&sh.bar_full[b], (fpar >> b) & 1u, err0)) break;
            const long long t1 = PT_NOW();
            if (lane == 0) PT_ADD(7, t1 - t0);
            fpar ^= 1u << b;
            const OutMeta &O = sh.out[b];
            if (O.tile == -2) {
                // skip token: this buffer holds part of the wide tile just updated
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh.bar_empty[b]);
                b ^= 1;
                continue;
            }
            if (O.tile < 0) break;
            const Sys &S = sh.os[b];
            const bool measure = step < S.meas_until;
            if (S.acc != acc_sys) {
                if (acc_sys) flush_acc(acc, acc_sys, cur);
                acc = {0, 0, 0, 0, 0};
                acc_sys = S.acc;
            }
            const float4 *P = B.P(b);
            const unsigned short *cst = B.cstart(b);
            const int rb = O.rbuf, rwide = O.rwide;
            const int4 *RB = B.raw(rb);
            const unsigned short *OR = B.ownr(b);
            const unsigned short *OQ = B.ownq(b);
            for (;;) {
                int c = 0;
                if (lane == 0) c = atomicAdd(&sh.chunk[b], 1);
                c = __shfl_sync(0xffffffffu, c, 0);
                const int o0 = c * 32;
                if (o0 >= O.n_own) break;
                update_one<MODEL>(S, O, P, cst, RB, OR, OQ, o0 + lane, step, measure, B.mhist(b), acc);
            }
            __syncwarp();
            if (lane == 0) {
                // the tile's output buffer and its raw buffer(s) are free
                mbar_arrive(&sh.bar_empty[b]);
                mbar_arrive(&sh.bar_raw_empty[rb]);
                if (rwide) mbar_arrive(&sh.bar_raw_empty[rb + 1]);
                PT_ADD(8, PT_NOW() - t1);
            }
            b ^= 1;
        }
        if (acc_sys) flush_acc(acc, acc_sys, cur);
    }
    __syncthreads();
    // --- the last tiles' histograms -> their systems -----------------------
    flush_hist(sh, B, 0, step, tid, kPipeThreads);
    flush_hist(sh, B, 1, step, tid, kPipeThreads);
    __syncthreads();

    // --- tiles too large for the pipeline's buffers: the whole block, with
    //     the shared staging area or the block's global scratch ------------
    __shared__ TileCtx T;
    const size_t tbytes = table_bytes(nce_max, hist_words);
    const size_t dyn = pipe_smem_bytes(cap, cap_own, nceh_max, hist_words);
    // stage_bytes(a) <= 41 a + 18: the staging area and the tables fit in dyn
    const int as_cap = (int)(((dyn - tbytes - 256) / 41) & ~63);
    Stage As;
    carve_stage(As, smem, as_cap);
    Tables tb;
    carve_tables(tb, smem + stage_bytes(as_cap), nce_max);
    Stage Ag;
    carve_stage(Ag, mine, scratch_cap);
    int *spill_e = (int *)(mine + stage_bytes(scratch_cap));
    unsigned char *spill_s = (unsigned char *)(spill_e + spill_list_cap);
    bool first = true;
    const long long td0 = PT_NOW();
    for (;;) {
        if (tid == 0) {
            int got = -1;
            int d = *((volatile int *)&ctl->dense_next);
            while (d < *((volatile int *)&ctl->dense_count)) {
                const int prev = atomicCAS(&ctl->dense_next, d, d + 1);
                if (prev == d) {
                    // the entry is written right after its index was taken
                    const long long t0 = clock64();
                    int v;
                    const long long bound = c_pipe_wait_cycles > 0 ? c_pipe_wait_cycles : kPipeWaitCycles;
                    while ((v = *((volatile int *)&dense_list[d])) == 0) {
                        if (clock64() - t0 > bound) {
                            atomicOr(err0, ERR_TIMEOUT);
                            break;
                        }
                    }
                    dense_list[d] = 0;
                    got = v - 1;
                    break;
                }
                d = prev;
            }
            sh.dense_tile = got;
        }
        __syncthreads();
        const int g = sh.dense_tile;
        if (g < 0) break;
        const int si = nsys > 1 ? sys_of_tile(tile_base, nsys, g) : 0;
        if (first || si != T.sysi) {
            __syncthreads();                // every thread is done with the previous system
            const int words = (int)(sizeof(Sys) / 4);
            const int *src = reinterpret_cast<const int *>(sys + si);
            int *dst = reinterpret_cast<int *>(&T.S);
            for (int i = tid; i < words; i += kPipeThreads) dst[i] = src[i];
            first = false;
        }
        __syncthreads();
        if (tid == 0) {
            T.sysi = si;
            T.tile = g - tile_base[si];
            T.pf_tile = -1;
            T.total = total;
            T.nsys = nsys;
            T.tile_base = tile_base;
            T.next = total;
        }
        __syncthreads();
        tile_setup<kPipeThreads>(T, tb, cur, nce_max, spill_e, spill_s, spill_list_cap);
        if (T.m <= as_cap) {
            tile_body<kPipeThreads, MODEL>(T, As, tb, step, spill_e, spill_s, total);
        } else if (T.m <= scratch_cap) {
            Stage Ah = Ag;
            if ((size_t)T.m * sizeof(float4) <= stage_bytes(as_cap)) Ah.P = reinterpret_cast<float4 *>(smem);
            tile_body<kPipeThreads, MODEL>(T, Ah, tb, step, spill_e, spill_s, total);
        } else if (tid == 0) {
            atomicOr(T.S.err, ERR_STAGE | ERR_LOST);
        }
        if (tid == 0) PT_ADD(11, 1);
        __syncthreads();
    }
    if (tid == 0) PT_ADD(12, PT_NOW() - tk0);
    (void)td0;
}

#ifndef AAP_PIPE_SORT_WARPS
#define AAP_PIPE_SORT_WARPS 8
#endif


template <int MODEL>
static cudaError_t static_pipe_t(size_t *bytes)
{
    cudaFuncAttributes a;
    const cudaError_t e = cudaFuncGetAttributes(&a, k_step_pipe<MODEL, AAP_PIPE_SORT_WARPS>);
    if (e == cudaSuccess) *bytes = a.sharedSizeBytes;
    return e;
}

cudaError_t pipe_static_smem(int model, size_t *bytes)
{
    switch (model) {
    case 0: return static_pipe_t<0>(bytes);
    case 1: return static_pipe_t<1>(bytes);
    case 2: return static_pipe_t<2>(bytes);
    default: return cudaErrorInvalidValue;
    }
}

template <int MODEL>
static cudaError_t config_pipe_t(size_t smem)
{
    // The limit belongs to the kernel, not to a handle: keep the largest size
    // any handle of this process asked for, so that a handle with smaller
    // buffers never breaks the launches of one with larger buffers.
    static std::atomic<int> limit{0};
    int want = (int)smem, prev = limit.load();
    while (want > prev && !limit.compare_exchange_weak(prev, want)) {
    }
    return cudaFuncSetAttribute(k_step_pipe<MODEL, AAP_PIPE_SORT_WARPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                std::max(want, limit.load()));
}

cudaError_t set_pipe_test(long long wait_cycles, int stall)
{
    cudaError_t e = cudaMemcpyToSymbol(c_pipe_wait_cycles, &wait_cycles, sizeof(wait_cycles));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_pipe_stall, &stall, sizeof(stall));
}

cudaError_t configure_pipe_kernel(int model, size_t smem)
{
    switch (model) {
    case 0: return config_pipe_t<0>(smem);
    case 1: return config_pipe_t<1>(smem);
    case 2: return config_pipe_t<2>(smem);
    default: return cudaErrorInvalidValue;
    }
}

template <int MODEL>
static cudaError_t launch_pipe_t(const LaunchCfg &L, cudaStream_t st)
{
    const size_t smem = pipe_smem_bytes(L.pipe_cap, L.pipe_cap_own, L.pipe_nceh, L.hist_words);
    k_step_pipe<MODEL, AAP_PIPE_SORT_WARPS><<<L.pipe_grid, kPipeThreads, smem, st>>>(
        L.sys, L.nsys, L.tile_base, L.ctl, L.pipe_cap, L.pipe_cap_own, L.pipe_nceh, L.nce_max, L.hist_words,
        L.dense_list, L.scratch, L.scratch_per_block, L.scratch_cap, L.spill_list_cap);
    return cudaGetLastError();
}

cudaError_t launch_step_pipe(const LaunchCfg &L, cudaStream_t st)
{
    switch (L.model) {
    case 0: return launch_pipe_t<0>(L, st);
    case 1: return launch_pipe_t<1>(L, st);
    case 2: return launch_pipe_t<2>(L, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace aapk
