// aap_mf.cu -- the metric-free (k nearest neighbour) step: mfVM, mfNVM and
// mfL of Sec. 2.3 of Kuersten, "Aligning Active Particles Py Package".
//
// Omega_i is the set of the k particles other than i that lie closest to it
// (images at periodic and reflecting boundaries included as in Sec. 2.4; a
// particle's own mirror image counts like any other image).  The paper finds
// them with cell lists of side R_eff = sqrt(Lx Ly k / (N pi))
// (Eq. effective_radius): the particle's own cell first, then the ring of 8
// cells around it, then the ring of 16, and so on, until no unvisited cell can
// hold a particle closer than the k-th found (Sec. 3.3).
//
// A metric-free system is kept flat: one tile covers the whole box and all
// records sit in region 0 in any order, so the insert, gather, observe and
// coarse-graining kernels of the metric path serve it unchanged.  One step is
//   k_mf_count     cell of each record and its arrival rank in the cell
//   k_mf_scan      chunk-local exclusive prefix of the cell counts (and clears
//                  the counts for the next step)
//   k_mf_scan_top  exclusive prefix of the chunk totals
//   k_mf_scatter   records into cell order
//   k_mf_update    one thread per record, in cell order so that a warp shares
//                  its rings: ring search for the k-th smallest distance tau
//                  (a register list kept by min/max passes), a second pass
//                  over the same cells that sums the neighbours (distance
//                  below tau, or at tau) in 2^32 fixed point, then the VM /
//                  NVM / Langevin update with h = 1 (Sec. 2.3), streaming,
//                  boundary rule, the new record, and exact integer sums for
//                  p, q and the histograms
//   k_mf_exact     the few particles the first kernel queued: several
//                  candidates at exactly tau (the tie is broken by id and
//                  image), or a periodic window too small to certify the list
//                  (an exhaustive scan)
// followed by the k_finish of the metric path.
//
// Determinism: the neighbour set is fixed by (distance, id, image) and the
// sums are integers, so nothing depends on the arrival order in a cell.
// Fixed point: positions carry 2^s units per cell with s chosen so that twice
// the box still fits int32; every image coordinate and displacement below is
// then an exact int32.
#include <algorithm>

#include <cuda_runtime.h>

#include "aap_device.cuh"
#include "aap_internal.cuh"
#include "aap_kernels.cuh"

namespace aapk {

namespace {

constexpr int kMfThreads = 256;
constexpr float kFix32F = 4294967296.0f;    // 2^32: order-free weighted sums (several species)

// x in units of 2^-22, rounded to the nearest integer (ties to even), as the
// bits of x 2^22 + 1.5 2^23: one FFMA whose single rounding lands on an
// integer because the float spacing there is 1.  For |x| <= 1 the integer is
// the bits minus 0x4B400000, so a sum of n such words minus n 0x4B400000
// (mod 2^32) is the exact integer sum as long as it fits int32 -- here at
// most 32 terms of |x| <= 1, below 2^28.  No float-to-int conversion
// instruction is needed.
__device__ __forceinline__ unsigned fix22_word(float x)
{
    return __float_as_uint(fmaf(x, 4194304.0f, 12582912.0f));
}
constexpr unsigned kFix22Bias = 0x4B400000u;

__global__ void k_mf_count(const Sys *__restrict__ sys, const Ctl *__restrict__ ctl)
{
    const Sys &S = *sys;
    const int cur = (int)(ctl->step & 1);
    const int ncx = S.ncx, ncy = S.ncy, sx = S.sx, sy = S.sy;
    const int4 *__restrict__ rec = S.rec[cur];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        S.mf_nfix[0] = 0;       // queue of k_mf_exact
        S.mf_nfix[1] = 0;       // next warp task of k_mf_update
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S.n;
         i += (long long)gridDim.x * blockDim.x) {
        const int4 r = rec[i];
        int cx = r.x >> sx, cy = r.y >> sy;
        if ((unsigned)cx >= (unsigned)ncx || (unsigned)cy >= (unsigned)ncy) {
            atomicOr(S.err, ERR_BOUNDS);
            cx = min(max(cx, 0), ncx - 1);
            cy = min(max(cy, 0), ncy - 1);
        }
        const int c = cy * ncx + cx;
        S.mf_cs[i] = make_int2(c, atomicAdd(&S.mf_cnt[c], 1));
    }
}

// Exclusive prefix of the counts inside each chunk of kScanChunk cells; the
// entry at index ncell (one past the last cell) is included with count 0.
__global__ void __launch_bounds__(1024) k_mf_scan(const Sys *__restrict__ sys, long long ncell)
{
    __shared__ int s_w[32];
    const Sys &S = *sys;
    const long long c0 = (long long)blockIdx.x * kScanChunk + threadIdx.x * 4;
    int v[4], sum = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const long long c = c0 + k;
        v[k] = c < ncell ? S.mf_cnt[c] : 0;
        if (c < ncell) S.mf_cnt[c] = 0;
        sum += v[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int incl = warp_incl_scan(sum);
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) s_w[lane] = warp_incl_scan(s_w[lane]);
    __syncthreads();
    int run = incl - sum + (warp > 0 ? s_w[warp - 1] : 0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const long long c = c0 + k;
        if (c <= ncell) S.mf_start[c] = run;
        run += v[k];
    }
    if (threadIdx.x == 1023) S.mf_blk[blockIdx.x] = run;
}

// Exclusive prefix of the nchunk chunk totals, in place; mf_blk[nchunk] = N.
__global__ void __launch_bounds__(1024) k_mf_scan_top(const Sys *__restrict__ sys, int nchunk)
{
    __shared__ int s_w[32];
    __shared__ int s_carry;
    const Sys &S = *sys;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nchunk; b0 += 1024) {
        const int b = b0 + threadIdx.x;
        const int v = b < nchunk ? S.mf_blk[b] : 0;
        const int incl = warp_incl_scan(v);
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        if (warp == 0) s_w[lane] = warp_incl_scan(s_w[lane]);
        __syncthreads();
        const int carry = s_carry;
        const int excl = carry + incl - v + (warp > 0 ? s_w[warp - 1] : 0);
        if (b < nchunk) S.mf_blk[b] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) S.mf_blk[nchunk] = s_carry;
}

__device__ __forceinline__ int cell_begin(const int *__restrict__ st, const int *__restrict__ blk, int c)
{
    return st[c] + blk[c / kScanChunk];
}

__global__ void k_mf_scatter(const Sys *__restrict__ sys, const Ctl *__restrict__ ctl)
{
    const Sys &S = *sys;
    const int cur = (int)(ctl->step & 1);
    const int4 *__restrict__ rec = S.rec[cur];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S.n;
         i += (long long)gridDim.x * blockDim.x) {
        const int2 cs = S.mf_cs[i];
        const long long q = (long long)cell_begin(S.mf_start, S.mf_blk, cs.x) + cs.y;
        if ((unsigned long long)q >= (unsigned long long)S.n) {
            atomicOr(S.err, ERR_BOUNDS);
            continue;
        }
        S.mf_sorted[q] = rec[i];
    }
}

// Virtual cell v along an axis of nc cells (W = nc << s units): the real cell,
// and the image coordinate relative to the particle as a * X_j + off.  code is
// -1 / 0 / +1 for the image on the low side / none / the high side; at a
// reflecting axis a nonzero code is a mirror image (a = -1).
struct AxisMap {
    int real, a, off, code;
};

__device__ __forceinline__ bool map_axis(int v, int nc, int W, bool refl, int Xi, AxisMap &m)
{
    if (v >= 0 && v < nc) {
        m.real = v; m.a = 1; m.off = -Xi; m.code = 0;
        return true;
    }
    if (!refl) {
        // periodic: the window never wraps onto itself, so v is in (-nc, 2nc)
        m.a = 1;
        if (v < 0) { m.real = v + nc; m.off = -W - Xi; m.code = -1; }
        else       { m.real = v - nc; m.off = W - Xi;  m.code = 1; }
        return true;
    }
    if (v < -nc || v >= 2 * nc) return false;      // beyond every mirror image
    m.a = -1;
    if (v < 0) { m.real = -v - 1;         m.off = -Xi;        m.code = -1; }
    else       { m.real = 2 * nc - 1 - v; m.off = 2 * W - Xi; m.code = 1; }
    return true;
}

// Candidate (d2, key, ref) enters the ascending top-KMAX list if it precedes
// the last entry.  Entries 0 .. KMAX-k-1 hold d = -1 (never displaced), so the
// last entry is always the k-th nearest so far.
template <int KMAX>
__device__ __forceinline__ void topk_offer(float (&d)[KMAX], unsigned (&key)[KMAX], unsigned (&ref)[KMAX],
                                           float d2, unsigned k2, unsigned r2)
{
    if (!(d2 < d[KMAX - 1] || (d2 == d[KMAX - 1] && k2 < key[KMAX - 1]))) return;
    bool done = false;
#pragma unroll
    for (int s = KMAX - 1; s > 0; --s) {
        if (!done) {
            if (d2 < d[s - 1] || (d2 == d[s - 1] && k2 < key[s - 1])) {
                d[s] = d[s - 1];
                key[s] = key[s - 1];
                ref[s] = ref[s - 1];
            } else {
                d[s] = d2;
                key[s] = k2;
                ref[s] = r2;
                done = true;
            }
        }
    }
    if (!done) {
        d[0] = d2;
        key[0] = k2;
        ref[0] = r2;
    }
}

struct MfGeo {
    int ncx, ncy, W, H;
    float ux, uy;
    bool bx, by;
};

// Every candidate of virtual cell (vx, vy) for particle q (at X, Y):
// f(d2, record, sorted index, image code, mirror flips).  The untransformed
// particle itself is skipped (j != i); d2 is computed the same way for every
// pass, so passes over the same cells see bit-identical distances.
template <class F>
__device__ __forceinline__ void for_cell(const MfGeo &G, const int4 *__restrict__ srt, const int *__restrict__ st,
                                         const int *__restrict__ blk, int vx, int vy, int X, int Y, long long q,
                                         F &&f)
{
    AxisMap mx, my;
    if (!map_axis(vx, G.ncx, G.W, G.bx, X, mx) || !map_axis(vy, G.ncy, G.H, G.by, Y, my)) return;
    const int c = my.real * G.ncx + mx.real;
    const int b = cell_begin(st, blk, c), e = cell_begin(st, blk, c + 1);
    const bool untransformed = mx.code == 0 && my.code == 0;
    const unsigned code = (unsigned)((mx.code + 1) + 3 * (my.code + 1));
    const unsigned flips = (G.bx && mx.code ? 1u : 0u) | (G.by && my.code ? 2u : 0u);
#pragma unroll 1
    for (int j = b; j < e; ++j) {
        if (untransformed && j == q) continue;
        const int4 rj = srt[j];
        const float dx = (float)(mx.a * rj.x + mx.off) * G.ux;
        const float dy = (float)(my.a * rj.y + my.off) * G.uy;
        f(fmaf(dx, dx, dy * dy), rj, j, code, flips);
    }
}

// Every candidate in ring `ring` (the cells at Chebyshev distance ring from
// (cx, cy)) of a window capped at rmx, rmy cells per axis.
template <class F>
__device__ __forceinline__ void for_ring(const MfGeo &G, const int4 *__restrict__ srt, const int *__restrict__ st,
                                         const int *__restrict__ blk, int ring, int rmx, int rmy, int cx, int cy,
                                         int X, int Y, long long q, F &&f)
{
    const int rx = min(ring, rmx), ry = min(ring, rmy);
    for (int dy = -ry; dy <= ry; ++dy) {
        if (dy == -ring || dy == ring) {
            for (int dx = -rx; dx <= rx; ++dx) for_cell(G, srt, st, blk, cx + dx, cy + dy, X, Y, q, f);
        } else if (ring <= rmx) {
            for_cell(G, srt, st, blk, cx - ring, cy + dy, X, Y, q, f);
            for_cell(G, srt, st, blk, cx + ring, cy + dy, X, Y, q, f);
        }
    }
}

// Rings 0 .. kWin of a particle whose window of (2 kWin + 1)^2 cells lies
// inside the box (no image, no mirror) are visited by rows: cells x0 .. x1
// (offsets from the particle's cell) of one row are one contiguous range of
// the cell order, so a warp of particles from neighbouring cells walks a few
// ranges in step instead of one cell at a time.  d2 is formed exactly as
// for_cell forms it for an untransformed cell, so both see bit-identical
// distances.
constexpr int kWin = 2;

template <class F>
__device__ __forceinline__ void for_row(const MfGeo &G, const int4 *__restrict__ srt, const int *__restrict__ st,
                                        const int *__restrict__ blk, int c, int x0, int x1, int X, int Y,
                                        long long q, F &&f)
{
    if (x0 > x1) return;
    const int b = cell_begin(st, blk, c + x0), e = cell_begin(st, blk, c + x1 + 1);
#pragma unroll 2
    for (int j = b; j < e; ++j) {
        const int4 rj = srt[j];
        const float dx = (float)(rj.x - X) * G.ux;
        const float dy = (float)(rj.y - Y) * G.uy;
        if (j != q) f(fmaf(dx, dx, dy * dy), rj, j, 4u, 0u);
    }
}

// Cell offsets lo .. hi (clamped to the window) along one axis that a disc of
// squared radius tau around the coordinate X of cell cx can reach.  The disc is
// widened by 1e-4 relative and 2 units, so every candidate left out lies
// strictly farther than tau even after the rounding of d2; an infinite tau
// gives the whole window.
__device__ __forceinline__ void window_span(float tau, int X, int cx, int s, float u, int &lo, int &hi)
{
    const float r = sqrtf(tau) * 1.0001f / u + 2.0f;
    const int ru = r < (float)(3 << s) ? (int)r : (3 << s);
    lo = max(((X - ru) >> s) - cx, -kWin);
    hi = min(((X + ru) >> s) - cx, kWin);
}

__device__ __forceinline__ bool window_inside(const MfGeo &G, int cx, int cy)
{
    return cx >= kWin && cx < G.ncx - kWin && cy >= kWin && cy < G.ncy - kWin;
}

// The k-th smallest distance so far: an ascending list whose first KMAX - k
// entries hold -1.  Inserting x into the sorted list sets entry s to
// max(d[s-1], min(d[s], x)): every entry comes from the old list alone, so
// the KMAX updates are independent (no dependency chain, no indices).
template <int KMAX>
__device__ __forceinline__ void kth_offer(float (&d)[KMAX], float d2)
{
    if (d2 < d[KMAX - 1]) {
#pragma unroll
        for (int s = KMAX - 1; s > 0; --s) d[s] = fmaxf(d[s - 1], fminf(d[s], d2));
        d[0] = fminf(d[0], d2);
    }
}

// sin and cos of o theta for |theta| <= pi and an order o <= 64: Cody-Waite
// reduction (Cody and Waite, "Software Manual for the Elementary Functions",
// 1980) of o theta by 2 pi split into a float head and tail, then the hardware
// sine and cosine on [-pi, pi].
__device__ __forceinline__ void sincos_order(float t, int order, float &sn, float &cs)
{
    const float x = t * (float)order;
    const float m = rintf(x * 0.15915494309189535f);              // 1 / (2 pi)
    float r = fmaf(-m, 6.28318548202514648f, x);                  // 2 pi rounded to float
    r = fmaf(-m, -1.7484556025237907e-07f, r);                    // 2 pi minus that
    __sincosf(r, &sn, &cs);
}

// Orientation term of neighbour j: (cos, sin) of o theta_j for its image
// (mirrored in x: theta -> pi - theta; in y: theta -> -theta).
template <int MODEL>
__device__ __forceinline__ void image_cos_sin(float tj, unsigned flips, int order, float &cs, float &sn)
{
    if (MODEL == 1 && order != 1) sincos_order(tj, order, sn, cs);
    else __sincosf(tj, &sn, &cs);                // |theta| <= pi
    if (flips & 1u) {
        if (MODEL != 1 || (order & 1)) cs = -cs; else sn = -sn;
    }
    if (flips & 2u) sn = -sn;
}

// Neighbour sums over a finished list (ascending distance, id, image):
// VM / NVM add e^{i theta_j} (NVM reversed when more than pi/2 from theta_i,
// Eq. collision_NVM), Langevin adds sin(o (theta_j - theta_i)).  Returns |Omega_i|.
template <int MODEL, int KMAX>
__device__ __forceinline__ void list_sums(const float (&d)[KMAX], const unsigned (&ref)[KMAX],
                                          const int4 *__restrict__ srt, const Sys &S, const float *grow, int order,
                                          float ci, float si, float oci, float osi, float &sc, float &ss,
                                          float &tsum, int &nb)
{
#pragma unroll
    for (int s = 0; s < KMAX; ++s) {
        if (d[s] >= 0.0f && d[s] < __int_as_float(0x7f800000)) {
            const unsigned rf = ref[s];
            const int4 rj = srt[rf & 0x3fffffffu];
            float sn, cs;
            image_cos_sin<MODEL>(__int_as_float(rj.z), rf >> 30, order, cs, sn);
            ++nb;
            if (MODEL == 1) {
                const float t = oci * sn - osi * cs;             // sin(o (theta_j - theta_i))
                tsum = grow ? fmaf(grow[species_of(S, (unsigned)rj.w)], t, tsum) : tsum + t;
            } else {
                if (MODEL == 2 && fmaf(ci, cs, si * sn) < 0.f) {
                    cs = -cs;
                    sn = -sn;
                }
                sc += cs;
                ss += sn;
            }
        }
    }
}

// The k nearest by exhaustive scan of all n records (only for a periodic
// window that cannot certify the list, i.e. systems with about k particles or
// fewer across half the box).  out: sum cos, sum sin, Langevin sum; returns
// |Omega_i|.
template <int MODEL, int KMAX>
__device__ __forceinline__ int brute_sums(const MfGeo &G, const int4 *__restrict__ srt, const Sys &S, const float *grow,
                                       long long n, long long q, int X, int Y, int k, int order, float ci, float si,
                                       float oci, float osi, float *out)
{
    float d[KMAX];
    unsigned key[KMAX], ref[KMAX];
#pragma unroll
    for (int s = 0; s < KMAX; ++s) {
        const bool dummy = s < KMAX - k;
        d[s] = dummy ? -1.0f : __int_as_float(0x7f800000);
        key[s] = dummy ? 0u : 0xffffffffu;
        ref[s] = 0u;
    }
    for (long long j = 0; j < n; ++j) {
        const int4 rj = srt[j];
        int ox[3], cxs[3], ax[3], nx = 0, oy[3], cys[3], ay[3], ny = 0;
        if (!G.bx) {
            int dd = rj.x - X, c = 0;
            if (2 * dd > G.W) { dd -= G.W; c = -1; } else if (2 * dd < -G.W) { dd += G.W; c = 1; }
            ox[0] = dd; cxs[0] = c; ax[0] = 0; nx = 1;
        } else {
            ox[0] = rj.x - X;           cxs[0] = 0;  ax[0] = 0;
            ox[1] = -rj.x - X;          cxs[1] = -1; ax[1] = 1;
            ox[2] = 2 * G.W - rj.x - X; cxs[2] = 1;  ax[2] = 1;
            nx = 3;
        }
        if (!G.by) {
            int dd = rj.y - Y, c = 0;
            if (2 * dd > G.H) { dd -= G.H; c = -1; } else if (2 * dd < -G.H) { dd += G.H; c = 1; }
            oy[0] = dd; cys[0] = c; ay[0] = 0; ny = 1;
        } else {
            oy[0] = rj.y - Y;           cys[0] = 0;  ay[0] = 0;
            oy[1] = -rj.y - Y;          cys[1] = -1; ay[1] = 2;
            oy[2] = 2 * G.H - rj.y - Y; cys[2] = 1;  ay[2] = 2;
            ny = 3;
        }
        for (int b = 0; b < ny; ++b)
            for (int a = 0; a < nx; ++a) {
                if (j == q && cxs[a] == 0 && cys[b] == 0) continue;     // j != i
                const float dx = (float)ox[a] * G.ux, dy = (float)oy[b] * G.uy;
                const unsigned code = (unsigned)((cxs[a] + 1) + 3 * (cys[b] + 1));
                topk_offer<KMAX>(d, key, ref, fmaf(dx, dx, dy * dy), (unsigned)rj.w * 9u + code,
                                 (unsigned)j | ((unsigned)(ax[a] | ay[b]) << 30));
            }
    }
    float sc = 0.f, ss = 0.f, tsum = 0.f;
    int nb = 0;
    list_sums<MODEL, KMAX>(d, ref, srt, S, grow, order, ci, si, oci, osi, sc, ss, tsum, nb);
    out[0] = sc;
    out[1] = ss;
    out[2] = tsum;
    return nb;
}

// The k nearest over rings 0 .. rfin with the full (distance, id, image)
// order, for the rare particle whose k-th distance is shared by several
// candidates.  Same outputs as brute_sums.
template <int MODEL, int KMAX>
__device__ __forceinline__ int exact_sums(const MfGeo &G, const int4 *__restrict__ srt, const int *__restrict__ st,
                                       const int *__restrict__ blk, const Sys &S, const float *grow, int rfin,
                                       int rmx, int rmy, int cx, int cy, long long q, int X, int Y, int k,
                                       int order, float ci, float si, float oci, float osi, float *out)
{
    float d[KMAX];
    unsigned key[KMAX], ref[KMAX];
#pragma unroll
    for (int s = 0; s < KMAX; ++s) {
        const bool dummy = s < KMAX - k;
        d[s] = dummy ? -1.0f : __int_as_float(0x7f800000);
        key[s] = dummy ? 0u : 0xffffffffu;
        ref[s] = 0u;
    }
    for (int ring = 0; ring <= rfin; ++ring)
        for_ring(G, srt, st, blk, ring, rmx, rmy, cx, cy, X, Y, q,
                 [&](float d2, const int4 &rj, int j, unsigned code, unsigned flips) {
                     topk_offer<KMAX>(d, key, ref, d2, (unsigned)rj.w * 9u + code, (unsigned)j | (flips << 30));
                 });
    float sc = 0.f, ss = 0.f, tsum = 0.f;
    int nb = 0;
    list_sums<MODEL, KMAX>(d, ref, srt, S, grow, order, ci, si, oci, osi, sc, ss, tsum, nb);
    out[0] = sc;
    out[1] = ss;
    out[2] = tsum;
    return nb;
}

// Geometry of the flat system, read once per thread.
__device__ __forceinline__ MfGeo mf_geo(const Sys &S)
{
    MfGeo G;
    G.ncx = S.ncx;
    G.ncy = S.ncy;
    G.W = S.ncx << S.sx;
    G.H = S.ncy << S.sy;
    G.ux = S.ux;
    G.uy = S.uy;
    G.bx = S.bx != 0;
    G.by = S.by != 0;
    return G;
}

// One particle's own quantities and its search window.
struct MfSelf {
    int X, Y, cx, cy, rmx, rmy, sp;
    float thi, ci, si, oci, osi;     // theta, cos/sin theta, cos/sin of o theta
    unsigned id;
    const float *grow;               // Gamma_{s_i .} dt with several species (Langevin), else null
};

template <int MODEL>
__device__ __forceinline__ MfSelf mf_self(const Sys &S, const MfGeo &G, int4 r)
{
    MfSelf P;
    P.X = r.x;
    P.Y = r.y;
    P.thi = __int_as_float(r.z);
    P.id = (unsigned)r.w;
    P.cx = min(P.X >> S.sx, G.ncx - 1);
    P.cy = min(P.Y >> S.sy, G.ncy - 1);
    // a periodic window stops short of wrapping onto itself, a reflecting
    // one at the outermost mirror image
    P.rmx = G.bx ? max(P.cx + G.ncx, 2 * G.ncx - 1 - P.cx) : (G.ncx - 1) / 2;
    P.rmy = G.by ? max(P.cy + G.ncy, 2 * G.ncy - 1 - P.cy) : (G.ncy - 1) / 2;
    __sincosf(P.thi, &P.si, &P.ci);              // |theta| <= pi
    P.oci = P.ci;
    P.osi = P.si;
    if (MODEL == 1 && S.order != 1) sincos_order(P.thi, S.order, P.osi, P.oci);
    P.sp = S.nsp > 1 ? species_of(S, P.id) : 0;
    P.grow = (MODEL == 1 && S.nsp > 1) ? S.sp_gamma_dt + P.sp * kMaxSpecies : nullptr;
    return P;
}

// Integer contributions of one particle to the step's sums (p, q, |Omega|).
struct MfAcc {
    long long c, s, n, c2, s2;
};

// The update of particle q from its neighbour sums (sc, ss: VM / NVM sum S_i
// including e^{i theta_i}; tsum: Langevin sum, Gamma dt already inside with
// several species): noise, Eq. (collision) or the Euler-Maruyama step with
// h = 1 (Sec. 2.3), streaming, the boundary rule (Sec. 2.4) in fixed point,
// the new record, histograms and sums.
template <int MODEL>
__device__ __forceinline__ void mf_finish(const Sys &S, const MfGeo &G, const MfSelf &P, long long step, int nxt,
                                          long long q, float sc, float ss, float tsum, int nb, bool measure,
                                          int *s_hist, MfAcc &acc)
{
    if (measure) {
        int bt = (int)floorf((P.thi + AAP_PI_F) * ((float)S.bins_theta * (1.0f / AAP_2PI_F)));
        bt = min(max(bt, 0), S.bins_theta - 1);
        atomicAdd(&s_hist[bt], 1);
        atomicAdd(&s_hist[S.bins_theta + min(nb, S.bins_nbr - 1)], 1);
    }
    uint32_t c4[4] = {P.id, (uint32_t)step, (uint32_t)((unsigned long long)step >> 32), 0u};
    philox4x32_10(c4, S.seed_lo, S.seed_hi);
    const float u0 = u01f(c4[0]);
    const int sp = P.sp;
    float thn, cn = 0.f, sn = 0.f;
    int dX, dY;
    if (MODEL != 1) {
        // Eq. (collision_VM) / (collision_NVM) + noise; Eq. (streaming)
        thn = atan2f(ss, sc) + S.sp_omega_step[sp] + S.sp_eta_pi[sp] * (2.0f * u0 - 1.0f);
        __sincosf(thn, &sn, &cn);
        dX = __float2int_rn(S.sp_kx[sp] * cn);
        dY = __float2int_rn(S.sp_ky[sp] * sn);
    } else {
        // Eq. (Langevin_dynamics) with h = 1 (Sec. 2.3), one Euler-Maruyama step
        const float u1 = u01f(c4[1]);
        const float gz = sqrtf(-2.0f * logf(u0)) * cospif(2.0f * u1);
        thn = P.thi + (P.grow ? tsum : S.gamma_dt * tsum) + S.sp_omega_step[sp] + S.sp_noise_amp[sp] * gz;
        dX = __float2int_rn(S.sp_kx[sp] * P.ci);
        dY = __float2int_rn(S.sp_ky[sp] * P.si);
    }
    int Xn = P.X + dX, Yn = P.Y + dY;
    bool fx = false, fy = false;
    if (Xn < 0) {
        if (G.bx) { Xn = -Xn; fx = true; } else Xn += G.W;
    } else if (Xn >= G.W) {
        if (G.bx) {
            if (Xn == G.W) Xn = G.W - 1; else { Xn = 2 * G.W - Xn; fx = true; }
        } else Xn -= G.W;
    }
    if (Yn < 0) {
        if (G.by) { Yn = -Yn; fy = true; } else Yn += G.H;
    } else if (Yn >= G.H) {
        if (G.by) {
            if (Yn == G.H) Yn = G.H - 1; else { Yn = 2 * G.H - Yn; fy = true; }
        } else Yn -= G.H;
    }
    if (fx) { thn = AAP_PI_F - thn; cn = -cn; }
    if (fy) { thn = -thn; sn = -sn; }
    if (thn >= AAP_PI_F || thn < -AAP_PI_F)
        thn -= AAP_2PI_F * floorf((thn + AAP_PI_F) * (1.0f / AAP_2PI_F));
    if (MODEL == 1) __sincosf(thn, &sn, &cn);
    if (!isfinite(thn)) atomicOr(S.err, ERR_NAN);
    S.rec[nxt][q] = make_int4(Xn, Yn, __float_as_int(thn), (int)P.id);
    acc.c += __float2int_rn(cn * kFixStepF);
    acc.s += __float2int_rn(sn * kFixStepF);
    acc.c2 += __float2int_rn(fmaf(cn, cn, -sn * sn) * kFixStepF);
    acc.s2 += __float2int_rn(2.0f * cn * sn * kFixStepF);
    acc.n += nb;
    if (S.nbr_out && P.id < (unsigned long long)S.n) S.nbr_out[P.id] = nb;
}

// Block sums into the step's accumulators; the block's histogram counts.
template <int NT>
__device__ __forceinline__ void mf_flush(const Sys &S, int cur, MfAcc acc, long long (*s_red)[NT / 32],
                                         bool measure, const int *s_hist)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    acc.c = warp_sum_ll(acc.c);
    acc.s = warp_sum_ll(acc.s);
    acc.n = warp_sum_ll(acc.n);
    acc.c2 = warp_sum_ll(acc.c2);
    acc.s2 = warp_sum_ll(acc.s2);
    if (lane == 0) {
        s_red[0][warp] = acc.c;
        s_red[1][warp] = acc.s;
        s_red[2][warp] = acc.n;
        s_red[3][warp] = acc.c2;
        s_red[4][warp] = acc.s2;
    }
    __syncthreads();
    if (tid < 5) {
        long long v = 0;
        for (int w = 0; w < NT / 32; ++w) v += s_red[tid][w];
        unsigned long long *slot = S.acc + ((size_t)cur * kAccSlots + (blockIdx.x & (kAccSlots - 1))) * kAccWords;
        atomicAdd(slot + tid, (unsigned long long)v);
    }
    if (measure)
        for (int i = tid; i < S.bins_theta + S.bins_nbr; i += NT)
            if (s_hist[i]) atomicAdd(S.hist + i, (unsigned long long)s_hist[i]);
}

// One thread per record in cell order; each warp takes tasks of 32
// consecutive records from a counter until none are left (persistent blocks,
// so that no warp idles behind a slow one of its block).  Pass 1 finds the k-th smallest
// distance tau by the ring search (Sec. 3.3); pass 2 sums over the candidates
// below tau and at tau in 2^32 fixed point, so that the sums do not depend on
// the arrival order inside a cell.  Particles whose window cannot certify the
// list, or with several candidates at exactly tau, are queued for
// k_mf_exact and left to it.
template <int NT, int MODEL, int KMAX>
__global__ void __launch_bounds__(NT, KMAX > 16 ? 2 : 4) k_mf_update(const Sys *__restrict__ sys, const Ctl *__restrict__ ctl)
{
    extern __shared__ int s_hist[];                 // [bins_theta + bins_nbr] while measuring
    __shared__ long long s_red[5][NT / 32];
    const Sys &S = *sys;
    const long long step = ctl->step;
    const int cur = (int)(step & 1), nxt = cur ^ 1;
    const long long n = S.n;
    const int sx = S.sx, sy = S.sy, k = S.knn;
    const MfGeo G = mf_geo(S);
    const int4 *__restrict__ srt = S.mf_sorted;
    const int *__restrict__ st = S.mf_start;
    const int *__restrict__ blk = S.mf_blk;
    const bool measure = step < S.meas_until;       // on-the-fly histograms (Sec. 3.4)
    if (measure)
        for (int i = threadIdx.x; i < S.bins_theta + S.bins_nbr; i += NT) s_hist[i] = 0;
    __syncthreads();
    MfAcc acc = {0, 0, 0, 0, 0};
    const long long ntask = (n + 31) >> 5;
    for (;;) {
        int task = 0;
        if ((threadIdx.x & 31) == 0) task = atomicAdd(S.mf_nfix + 1, 1);
        task = __shfl_sync(0xffffffffu, task, 0);
        if (task >= ntask) break;
        const long long q = ((long long)task << 5) + (threadIdx.x & 31);
        if (q < n) {
            const MfSelf P = mf_self<MODEL>(S, G, srt[q]);
            float d[KMAX];
#pragma unroll
            for (int s = 0; s < KMAX; ++s) d[s] = s < KMAX - k ? -1.0f : __int_as_float(0x7f800000);
            bool certified = false;
            int rfin = 0;
            const bool win = window_inside(G, P.cx, P.cy);
            const int crow = P.cy * G.ncx + P.cx;       // cell index of the particle's cell
            for (int ring = win ? kWin : 0;; ++ring) {
                const auto offer = [&](float d2, const int4 &, int, unsigned, unsigned) { kth_offer<KMAX>(d, d2); };
                if (win && ring == kWin) {
                    // rings 0 and 1, then the cells of ring 2 that the k-th
                    // distance found so far still reaches (the others hold
                    // only candidates beyond it, which can never enter the list)
                    for (int dy = -1; dy <= 1; ++dy)
                        for_row(G, srt, st, blk, crow + dy * G.ncx, -1, 1, P.X, P.Y, q, offer);
                    int xl, xh, yl, yh;
                    window_span(d[KMAX - 1], P.X, P.cx, sx, G.ux, xl, xh);
                    window_span(d[KMAX - 1], P.Y, P.cy, sy, G.uy, yl, yh);
                    for (int dy = yl; dy <= yh; ++dy) {
                        const int c = crow + dy * G.ncx;
                        if (dy == -kWin || dy == kWin) {
                            for_row(G, srt, st, blk, c, xl, xh, P.X, P.Y, q, offer);
                        } else {
                            if (xl == -kWin) for_row(G, srt, st, blk, c, -kWin, -kWin, P.X, P.Y, q, offer);
                            if (xh == kWin) for_row(G, srt, st, blk, c, kWin, kWin, P.X, P.Y, q, offer);
                        }
                    }
                } else {
                    for_ring(G, srt, st, blk, ring, P.rmx, P.rmy, P.cx, P.cy, P.X, P.Y, q, offer);
                }
                // every unvisited candidate lies at least this far away
                const int rx = min(ring, P.rmx), ry = min(ring, P.rmy);
                float gx = __int_as_float(0x7f800000), gy = gx;
                const int lo = P.cx - rx, hi = P.cx + rx, lo2 = P.cy - ry, hi2 = P.cy + ry;
                if (!(G.bx && lo <= -G.ncx)) gx = (float)(P.X - lo * (1 << sx)) * G.ux;
                if (!(G.bx && hi >= 2 * G.ncx - 1)) gx = fminf(gx, (float)((hi + 1) * (1 << sx) - P.X) * G.ux);
                if (!(G.by && lo2 <= -G.ncy)) gy = (float)(P.Y - lo2 * (1 << sy)) * G.uy;
                if (!(G.by && hi2 >= 2 * G.ncy - 1)) gy = fminf(gy, (float)((hi2 + 1) * (1 << sy) - P.Y) * G.uy);
                const float g = fminf(gx, gy);
                if (d[KMAX - 1] <= g * g * 0.99999f) {
                    certified = true;
                    rfin = ring;
                    break;
                }
                if (ring >= P.rmx && ring >= P.rmy) break;
            }
            bool queued = !certified;
            if (certified) {
                const float tau = d[KMAX - 1];
                long long g0 = 0;                    // several species (weights beyond 1): 2^-32 units
                unsigned w0 = 0, w1 = 0;             // otherwise fix22 words, bias removed below
                int nlt = 0, neq = 0;
                const int order = S.order;
                const auto sum = [&](float d2, const int4 &rj, int, unsigned, unsigned flips) {
                    if (d2 > tau) return;
                    float cs, sn;
                    image_cos_sin<MODEL>(__int_as_float(rj.z), flips, order, cs, sn);
                    if (MODEL == 1) {
                        float t = P.osi * -cs + P.oci * sn;      // sin(o (theta_j - theta_i))
                        if (P.grow) g0 += __float2ll_rn(t * P.grow[species_of(S, (unsigned)rj.w)] * kFix32F);
                        else w0 += fix22_word(t);
                    } else {
                        if (MODEL == 2 && fmaf(P.ci, cs, P.si * sn) < 0.f) {   // Eq. (collision_NVM)
                            cs = -cs;
                            sn = -sn;
                        }
                        w0 += fix22_word(cs);
                        w1 += fix22_word(sn);
                    }
                    if (d2 < tau) ++nlt; else ++neq;
                };
                if (win) {
                    // the window's cells that a disc of squared radius tau reaches
                    int xl, xh, yl, yh;
                    window_span(tau, P.X, P.cx, sx, G.ux, xl, xh);
                    window_span(tau, P.Y, P.cy, sy, G.uy, yl, yh);
                    for (int dy = yl; dy <= yh; ++dy)
                        for_row(G, srt, st, blk, crow + dy * G.ncx, xl, xh, P.X, P.Y, q, sum);
                }
                for (int ring = win ? kWin + 1 : 0; ring <= rfin; ++ring)
                    for_ring(G, srt, st, blk, ring, P.rmx, P.rmy, P.cx, P.cy, P.X, P.Y, q, sum);
                if (nlt + neq <= k) {
                    const unsigned bias = kFix22Bias * (unsigned)(nlt + neq);
                    const float f0 = (MODEL == 1 && P.grow) ? (float)g0 * (1.0f / kFix32F)
                                                            : (float)(int)(w0 - bias) * (1.0f / kFixNbF);
                    const float f1 = (float)(int)(w1 - bias) * (1.0f / kFixNbF);
                    mf_finish<MODEL>(S, G, P, step, nxt, q, P.ci + f0, P.si + f1, f0, nlt + neq, measure, s_hist, acc);
                } else {
                    queued = true;                       // several candidates at exactly tau
                }
            }
            if (queued) {
                const int e = atomicAdd(S.mf_nfix, 1);
                S.mf_fix[e] = make_int2((int)q, certified ? rfin : -1);
            }
        }
    }
    mf_flush<NT>(S, cur, acc, s_red, measure, s_hist);
    if (blockIdx.x == 0 && threadIdx.x == 0) S.cnt[nxt][0] = (int)n;   // all records in region 0 of tile 0
}

// The queued particles: the k nearest with the full (distance, id, image)
// order, over the certified rings (ties at tau) or over every particle (a
// periodic window that cannot certify: systems of about k particles or fewer
// across half the box).
template <int NT, int MODEL, int KMAX>
__global__ void __launch_bounds__(NT) k_mf_exact(const Sys *__restrict__ sys, const Ctl *__restrict__ ctl)
{
    extern __shared__ int s_hist[];
    __shared__ long long s_red[5][NT / 32];
    const Sys &S = *sys;
    const long long step = ctl->step;
    const int cur = (int)(step & 1), nxt = cur ^ 1;
    const MfGeo G = mf_geo(S);
    const bool measure = step < S.meas_until;
    if (measure)
        for (int i = threadIdx.x; i < S.bins_theta + S.bins_nbr; i += NT) s_hist[i] = 0;
    __syncthreads();
    MfAcc acc = {0, 0, 0, 0, 0};
    const int nfix = *S.mf_nfix;
    for (int e = blockIdx.x * NT + threadIdx.x; e < nfix; e += gridDim.x * NT) {
        const int2 f = S.mf_fix[e];
        const long long q = f.x;
        const MfSelf P = mf_self<MODEL>(S, G, S.mf_sorted[q]);
        float out[3];
        int nb;
        if (f.y >= 0)
            nb = exact_sums<MODEL, KMAX>(G, S.mf_sorted, S.mf_start, S.mf_blk, S, P.grow, f.y, P.rmx, P.rmy, P.cx,
                                         P.cy, q, P.X, P.Y, S.knn, S.order, P.ci, P.si, P.oci, P.osi, out);
        else
            nb = brute_sums<MODEL, KMAX>(G, S.mf_sorted, S, P.grow, S.n, q, P.X, P.Y, S.knn, S.order, P.ci, P.si,
                                         P.oci, P.osi, out);
        const float sc = (MODEL == 1 ? 0.f : P.ci) + out[0], ss = (MODEL == 1 ? 0.f : P.si) + out[1];
        mf_finish<MODEL>(S, G, P, step, nxt, q, sc, ss, out[2], nb, measure, s_hist, acc);
    }
    mf_flush<NT>(S, cur, acc, s_red, measure, s_hist);
}

template <int MODEL, int KMAX>
cudaError_t launch_update(const LaunchCfg &L, cudaStream_t st)
{
    const long long blocks = std::min<long long>((L.mf_n + kMfThreads - 1) / kMfThreads, L.mf_grid);
    const size_t smem = (size_t)L.hist_words * sizeof(int);
    k_mf_update<kMfThreads, MODEL, KMAX><<<(unsigned)std::max<long long>(blocks, 1), kMfThreads, smem, st>>>(L.sys,
                                                                                                        L.ctl);
    k_mf_exact<64, MODEL, KMAX><<<(unsigned)std::min<long long>((L.mf_n + 63) / 64, 1024), 64, smem, st>>>(L.sys,
                                                                                                           L.ctl);
    return cudaGetLastError();
}

template <int MODEL>
cudaError_t launch_update_m(const LaunchCfg &L, cudaStream_t st)
{
    if (L.knn <= 6) return launch_update<MODEL, 6>(L, st);       // k = 6: the common metric-free choice
    if (L.knn <= 8) return launch_update<MODEL, 8>(L, st);
    if (L.knn <= 16) return launch_update<MODEL, 16>(L, st);
    return launch_update<MODEL, kMaxKnn>(L, st);
}

template <int MODEL, int KMAX>
cudaError_t update_blocks_per_sm(size_t smem, int *bps)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_mf_update<kMfThreads, MODEL, KMAX>, kMfThreads, smem);
}

template <int MODEL>
cudaError_t update_blocks_per_sm_m(int knn, size_t smem, int *bps)
{
    if (knn <= 6) return update_blocks_per_sm<MODEL, 6>(smem, bps);
    if (knn <= 8) return update_blocks_per_sm<MODEL, 8>(smem, bps);
    if (knn <= 16) return update_blocks_per_sm<MODEL, 16>(smem, bps);
    return update_blocks_per_sm<MODEL, kMaxKnn>(smem, bps);
}

}  // namespace

cudaError_t configure_mf_kernels(int model, int knn, int hist_words, int sm_count, int *grid)
{
    const size_t smem = (size_t)hist_words * sizeof(int);
    int bps = 0;
    cudaError_t e;
    switch (model) {
    case 0: e = update_blocks_per_sm_m<0>(knn, smem, &bps); break;
    case 1: e = update_blocks_per_sm_m<1>(knn, smem, &bps); break;
    case 2: e = update_blocks_per_sm_m<2>(knn, smem, &bps); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    *grid = std::max(1, bps) * std::max(1, sm_count);
    return cudaSuccess;
}

cudaError_t launch_mf_step(const LaunchCfg &L, cudaStream_t st, cudaEvent_t *ev)
{
    cudaError_t e;
    if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
    if (L.mf_n > 0) {
        if (L.knn < 1 || L.knn > kMaxKnn) return cudaErrorInvalidValue;
        const unsigned g = (unsigned)std::min<long long>((L.mf_n + 255) / 256, 1ll << 20);
        const long long nchunk = (L.mf_ncell + 1 + kScanChunk - 1) / kScanChunk;
        k_mf_count<<<g, 256, 0, st>>>(L.sys, L.ctl);
        k_mf_scan<<<(unsigned)nchunk, 1024, 0, st>>>(L.sys, L.mf_ncell);
        k_mf_scan_top<<<1, 1024, 0, st>>>(L.sys, (int)nchunk);
        k_mf_scatter<<<g, 256, 0, st>>>(L.sys, L.ctl);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        switch (L.model) {
        case 0: e = launch_update_m<0>(L, st); break;
        case 1: e = launch_update_m<1>(L, st); break;
        case 2: e = launch_update_m<2>(L, st); break;
        default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return e;
    return cudaSuccess;
}

}  // namespace aapk
