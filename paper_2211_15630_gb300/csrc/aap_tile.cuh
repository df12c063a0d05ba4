// aap_tile.cuh -- device code shared by the tile step kernels: tile geometry,
// the 25 source segments of a tile (its own 9 regions and the facing halo
// regions of its 8 neighbours, with periodic shifts or mirror maps, Sec. 2.4),
// warp-aggregated insertion into the next step's regions, the 3x3-cell
// neighbour sums (Eq. collision_VM / collision_NVM, the Langevin coupling
// sum), and the whole-block tile routine (stage, counting sort by cell,
// update, scatter) that serves tiles staged in global scratch.
#pragma once

#include <cuda_runtime.h>

#include "aap_device.cuh"
#include "aap_internal.cuh"

namespace aapk {

// Optional per-phase timing of the step kernel (tracing aid, compiled out
// unless AAP_PHASE_TIMING is defined): thread 0 of every block adds the clock
// cycles between phase marks to g_phase[].
#ifdef AAP_PHASE_TIMING
static __device__ unsigned long long g_phase[16];
#define PHASE_START() long long ph_t0_ = clock64()
#define PHASE_MARK(i)                                                         \
    do {                                                                      \
        if (threadIdx.x == 0) {                                               \
            const long long t_ = clock64();                                   \
            atomicAdd(&g_phase[i], (unsigned long long)(t_ - ph_t0_));        \
            ph_t0_ = t_;                                                      \
        }                                                                     \
    } while (0)
#else
#define PHASE_START() do { } while (0)
#define PHASE_MARK(i) do { } while (0)
#endif

// ------------------------------------------------------------ geometry ----
__device__ __forceinline__ int tile_x0(const Sys &S, int tx) { return S.x0tab[tx]; }
__device__ __forceinline__ int tile_y0(const Sys &S, int ty) { return S.y0tab[ty]; }
__device__ __forceinline__ int tile_of_x(const Sys &S, int cx)
{
    return (int)((((long long)cx + 1) * S.ntx - 1) / S.ncx);
}
__device__ __forceinline__ int tile_of_y(const Sys &S, int cy)
{
    return (int)((((long long)cy + 1) * S.nty - 1) / S.ncy);
}
__device__ __forceinline__ int region_of(int lx, int ly, int tw, int th)
{
    const int rx = lx == 0 ? 0 : (lx == tw - 1 ? 2 : 1);
    const int ry = ly == 0 ? 0 : (ly == th - 1 ? 2 : 1);
    return ry * 3 + rx;
}

// Append rec to region `region` of tile `dtile` in buffer b.  Every lane of
// the warp must call; lanes with act == false take part in the vote only.
// Lanes headed for the same region share one atomicAdd (warp aggregation).
__device__ __forceinline__ void warp_insert(const Sys &S, int b, bool act, int dtile, int region, int4 rec)
{
    const int lane = threadIdx.x & 31;
    const int key = act ? dtile * kCntStride + region : -1 - lane;
    // most warps send every lane to one region: skip the match in that case
    const bool same = __all_sync(0xffffffffu, key == __shfl_sync(0xffffffffu, key, 0));
    const unsigned peers = same ? 0xffffffffu : __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (act && lane == leader) base = atomicAdd(&S.cnt[b][key], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (act) {
        const int slot = base + __popc(peers & ((1u << lane) - 1u));
        if (slot < S.cap[region]) {
            S.rec[b][(long long)dtile * S.tile_slots + S.off[region] + slot] = rec;
        } else {
            const int e = atomicAdd(&S.spill_cnt[b], 1);
            if (e < S.spill_cap) {
                S.spill_rec[b][e] = rec;
                S.spill_key[b][e] = key;
                atomicOr(&S.spill_bits[b][dtile >> 5], 1u << (dtile & 31));
                atomicOr(S.err, ERR_SPILL);
            } else {
                atomicOr(S.err, ERR_LOST);
            }
        }
    }
}


// ---------------------------------------------------------- tile context --
// Geometry of one tile and its neighbours' sizes.
struct TileGeo {
    int tx, ty, tw, th;
    int twL, twR, thD, thU;     // widths / heights of the neighbour tiles
};

struct TileCtx {
    Sys S;
    int sysi, tile, tx, ty, tw, th, W2, H2, nce;
    int twL, twR, thD, thU;     // widths / heights of the neighbour tiles
    int m_seg, n_spill, m, n_own;
    int next;                   // index of the next tile this block takes
    int total, nsys;            // tiles and systems of the launch
    const int *tile_base;
    int pf_tile, pf_sys, pf_nsp;    // segments of the next tile, read ahead during this one
    TileGeo pf_geo;
    int segpre[kSegs + 1];
    int warp_tot[32];
    Seg seg[kSegs];
    Seg pf_seg[kSegs];
    long long red[5][32];
};

__device__ __forceinline__ int sys_of_tile(const int *tile_base, int nsys, int g)
{
    int lo = 0, hi = nsys;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tile_base[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

// Resolve the halo column (side -1: left, +1: right) of tile t into a source
// tile column, the region column class there, and the position / cell maps.
__device__ __forceinline__ void resolve_axis(int side, int t, int nt, int w, int wlo, int refl, int s,
                                             int &src, int &cls, int &a, int &c, long long &b, int &flip)
{
    if (side == 0) {
        src = t; a = 1; c = 0; b = 0; flip = 0; cls = -1;
        return;
    }
    if (side < 0) {
        if (t > 0 || !refl) {
            src = (t > 0) ? t - 1 : nt - 1;
            cls = 2; a = 1; c = -wlo; b = -((long long)wlo << s); flip = 0;
        } else {        // mirror at the wall x = 0: X -> -X, cell 0 -> -1
            src = t; cls = 0; a = -1; c = -1; b = 0; flip = 1;
        }
    } else {
        if (t < nt - 1 || !refl) {
            src = (t < nt - 1) ? t + 1 : 0;
            cls = 0; a = 1; c = w; b = (long long)w << s; flip = 0;
        } else {        // mirror at the wall x = L: X -> 2 w 2^s - X, cell w-1 -> w
            src = t; cls = 2; a = -1; c = 2 * w - 1; b = 2 * ((long long)w << s); flip = 1;
        }
    }
}

__device__ __forceinline__ TileGeo tile_geo(const Sys &S, int tile)
{
    TileGeo G;
    G.tx = tile % S.ntx;
    G.ty = tile / S.ntx;
    const int x0 = S.x0tab[G.tx], y0 = S.y0tab[G.ty];
    G.tw = S.x0tab[G.tx + 1] - x0;
    G.th = S.y0tab[G.ty + 1] - y0;
    const int txl = G.tx > 0 ? G.tx - 1 : S.ntx - 1, txr = G.tx < S.ntx - 1 ? G.tx + 1 : 0;
    const int tyd = G.ty > 0 ? G.ty - 1 : S.nty - 1, tyu = G.ty < S.nty - 1 ? G.ty + 1 : 0;
    G.twL = S.x0tab[txl + 1] - S.x0tab[txl];
    G.twR = S.x0tab[txr + 1] - S.x0tab[txr];
    G.thD = S.y0tab[tyd + 1] - S.y0tab[tyd];
    G.thU = S.y0tab[tyu + 1] - S.y0tab[tyu];
    return G;
}

// Source segment s of a tile: s < 9 its own region s, then the 16 halo
// regions of the neighbour tiles (left, right, down, up edges, the corners)
// with their periodic shift or mirror map into the extended frame.
__device__ __forceinline__ Seg make_seg(const Sys &S, const TileGeo &G, int s, int cur)
{
    int bxo, byo, rx = -1, ry = -1;
    if (s < 9) {
        bxo = 0; byo = 0; rx = s % 3; ry = s / 3;
    } else {
        const int h = s - 9;
        if (h < 3)       { bxo = -1; byo = 0;  ry = h; }
        else if (h < 6)  { bxo = 1;  byo = 0;  ry = h - 3; }
        else if (h < 9)  { bxo = 0;  byo = -1; rx = h - 6; }
        else if (h < 12) { bxo = 0;  byo = 1;  rx = h - 9; }
        else { bxo = (h & 1) ? 1 : -1; byo = (h >= 14) ? 1 : -1; }
    }
    int srcx, clsx, ax, cx, fx, srcy, clsy, ay, cy, fy;
    long long bxx, byy;
    resolve_axis(bxo, G.tx, S.ntx, G.tw, G.twL, S.bx, S.sx, srcx, clsx, ax, cx, bxx, fx);
    resolve_axis(byo, G.ty, S.nty, G.th, G.thD, S.by, S.sy, srcy, clsy, ay, cy, byy, fy);
    if (clsx < 0) clsx = rx;
    if (clsy < 0) clsy = ry;
    Seg g;
    g.tile = srcy * S.ntx + srcx;
    g.region = clsy * 3 + clsx;
    g.base = S.rec[cur] + (long long)g.tile * S.tile_slots + S.off[g.region];
    const int c = S.cnt[cur][g.tile * kCntStride + g.region];
    g.count = min(c, S.cap[g.region]);
    g.ax = ax; g.ay = ay; g.cx = cx; g.cy = cy; g.bx = bxx; g.by = byy;
    g.flip = fx | (fy << 1);
    return g;
}

// Phase 1 of a tile: geometry, the 25 source segments (9 own regions, 16
// halo regions with their periodic or mirror maps), spill matches, and the
// number m of particles to stage.  The geometry and segments come from the
// read-ahead of the previous tile when it took this one.  Ends with the
// block synchronised.
template <int NT>
__device__ __forceinline__ void tile_setup(TileCtx &T, const Tables &tb, int cur, int nce_max,
                                           int *spill_e, unsigned char *spill_s, int spill_list_cap)
{
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const Sys &S = T.S;
    const bool pf = T.pf_tile == T.tile && T.pf_sys == T.sysi;
    const TileGeo G = pf ? T.pf_geo : tile_geo(S, T.tile);
    if (tid == 0) {
        T.tx = G.tx; T.ty = G.ty; T.tw = G.tw; T.th = G.th;
        T.W2 = G.tw + 2; T.H2 = G.th + 2; T.nce = (G.tw + 2) * (G.th + 2);
        T.twL = G.twL; T.twR = G.twR; T.thD = G.thD; T.thU = G.thU;
        T.n_spill = 0;
    }
    for (int i = tid; i < nce_max; i += NT) tb.hist[i] = 0;
    if (T.S.meas_until > 0)
        for (int i = tid; i < S.bins_theta + S.bins_nbr; i += NT) tb.mhist[i] = 0;
    if (tid < kSegs) T.seg[tid] = pf ? T.pf_seg[tid] : make_seg(S, G, tid, cur);
    const int nsp = pf ? T.pf_nsp : min(*((volatile int *)&S.spill_cnt[cur]), S.spill_cap);
    __syncthreads();
    if (tid == 0) T.pf_tile = -1;       // consumed (the read-ahead for the next tile comes later)
    if (warp == 0) {
        const int v = lane < kSegs ? T.seg[lane].count : 0;
        const int incl = warp_incl_scan(v);
        if (lane < kSegs) T.segpre[lane] = incl - v;
        if (lane == kSegs - 1) {
            T.segpre[kSegs] = incl;
            T.m_seg = incl;
        }
    }
    if (nsp > 0) {
        // particles parked in the spill list for one of our segments
        for (int e = tid; e < nsp; e += NT) {
            const int key = S.spill_key[cur][e];
            const int et = key / kCntStride, er = key % kCntStride;
            for (int s = 0; s < kSegs; ++s) {
                if (T.seg[s].tile == et && T.seg[s].region == er) {
                    const int j = atomicAdd(&T.n_spill, 1);
                    if (j < spill_list_cap) {
                        spill_e[j] = e;
                        spill_s[j] = (unsigned char)s;
                    }
                }
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (T.n_spill > spill_list_cap) {
            atomicOr(S.err, ERR_STAGE);
            T.n_spill = spill_list_cap;
        }
        T.m = T.m_seg + T.n_spill;
    }
    __syncthreads();
}

// The 3x3-cell neighbour sum of one particle (Eq. collision_VM / NVM, or the
// Langevin coupling sum): rows of three consecutive cells are contiguous in
// the cell order.  The particle itself is included: it adds e^{i theta_i} to
// the VM/NVM sum and sin 0 to the Langevin sum; cnt counts it.  The staged
// (cos, sin) are integers in units of 2^-22 (kFixNb), so the sums are exact and
// do not depend on the order of the particles inside a cell.  ACC is int for
// at most 511 candidates (|sum| < 2^31) and long long beyond.
template <int MODEL, typename ACC>
__device__ __forceinline__ void neighbour_sum(const float4 *__restrict__ P, const int *cstart, int ec,
                                              int W2, float4 pi, float r2, ACC &sc, ACC &ss, int &cnt)
{
    sc = 0;
    ss = 0;
    cnt = 0;
    const float pcf = (float)__float_as_int(pi.z), psf = (float)__float_as_int(pi.w);
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
        const int c0 = ec + dy * W2 - 1;
        const int a = cstart[c0], b = cstart[c0 + 3];
#pragma unroll 4
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

// Langevin sums with per-species couplings (Sec. 2.5): each neighbour's
// (cos o theta_j, sin o theta_j) weighted by grow[species of j] = Gamma_{s_i s_j} dt,
// rounded to integers in units of 2^-22 and summed exactly (order-free).
__device__ __forceinline__ void neighbour_sum_sp(const float4 *__restrict__ P, const unsigned short *spc,
                                                 const int *cstart, int ec, int W2, float4 pi, float r2,
                                                 const float *grow, long long &sc, long long &ss, int &cnt)
{
    sc = 0;
    ss = 0;
    cnt = 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
        const int c0 = ec + dy * W2 - 1;
        const int a = cstart[c0], b = cstart[c0 + 3];
        for (int j = a; j < b; ++j) {
            const float4 pj = P[j];
            const float dx = pj.x - pi.x, dyy = pj.y - pi.y;
            if (fmaf(dx, dx, dyy * dyy) <= r2) {
                const float g = grow[spc[j]];
                sc += __float2ll_rn(g * (float)__float_as_int(pj.z));
                ss += __float2ll_rn(g * (float)__float_as_int(pj.w));
                ++cnt;
            }
        }
    }
}

// Phase 2 of a tile, staged in A (shared memory or the block's scratch).
template <int NT, int MODEL>
__device__ __forceinline__ void tile_body(TileCtx &T, const Stage &A, const Tables &tb, long long step,
                                          const int *spill_e, const unsigned char *spill_s, int next_g)
{
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const Sys &S = T.S;
    const int cur = (int)(step & 1), nxt = cur ^ 1;
    const int m = T.m, m_seg = T.m_seg, W2 = T.W2, H2 = T.H2, nce = T.nce;
    const int tw = T.tw, th = T.th;
    PHASE_START();

    // --- segment of every 32nd staged index (chunk table) ---------------
    for (int i = tid; i * 32 < m_seg; i += NT) {
        const int k = i * 32;
        int lo = 0, hi = kSegs;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (T.segpre[mid] <= k) lo = mid; else hi = mid;
        }
        A.segc[i] = (unsigned char)lo;
    }
    __syncthreads();

    // --- stage: decode, map into the extended frame, histogram by cell ----
    for (int k = tid; k < m; k += NT) {
        int s;
        int4 r;
        if (k < m_seg) {
            s = A.segc[k >> 5];
            while (T.segpre[s + 1] <= k) ++s;
            r = T.seg[s].base[k - T.segpre[s]];
        } else {
            const int j = k - m_seg;
            s = spill_s[j];
            r = S.spill_rec[cur][spill_e[j]];
        }
        const Seg &g = T.seg[s];
        const int lx = r.x >> S.sx, ly = r.y >> S.sy;
        int ex = g.ax * lx + g.cx + 1, ey = g.ay * ly + g.cy + 1;
        if ((unsigned)ex >= (unsigned)W2 || (unsigned)ey >= (unsigned)H2) {
            atomicOr(S.err, ERR_BOUNDS);
            ex = min(max(ex, 0), W2 - 1);
            ey = min(max(ey, 0), H2 - 1);
        }
        const int ec = ey * W2 + ex;
        A.R[k] = make_int4((int)(g.ax * (long long)r.x + g.bx), (int)(g.ay * (long long)r.y + g.by), r.z, r.w);
        A.cell[k] = (unsigned short)(ec | (g.flip << 14));
        A.slot[k] = (unsigned short)atomicAdd(&tb.hist[ec], 1);
    }
    // the next tile's index, fetched by thread 0 at the start of this tile:
    // published only now, so that no warp waited for the atomic's round trip
    if (tid == 0) T.next = next_g;
    __syncthreads();
    PHASE_MARK(0);

    // --- block-level exclusive prefix scan of the cell histogram ----------
    {
        const int per = (nce + NT - 1) / NT;
        const int b0 = min(tid * per, nce), e0 = min(b0 + per, nce);
        int sum = 0;
        for (int i = b0; i < e0; ++i) sum += tb.hist[i];
        const int incl = warp_incl_scan(sum);
        if (lane == 31) T.warp_tot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int v = lane < NT / 32 ? T.warp_tot[lane] : 0;
            const int wi = warp_incl_scan(v);
            if (lane < NT / 32) T.warp_tot[lane] = wi - v;
            if (lane == NT / 32 - 1) tb.cstart[nce] = wi;
        }
        __syncthreads();
        int run = incl - sum + T.warp_tot[warp];
        for (int i = b0; i < e0; ++i) {
            tb.cstart[i] = run;
            run += tb.hist[i];
        }
    }
    __syncthreads();
    PHASE_MARK(1);

    // --- records into cell order (arrival order inside a cell: the sums are
    //     exact integers, so this order does not matter); own rows prefix ---
    const int xc = tw << (S.sx - 1), yc = th << (S.sy - 1);
    for (int k = tid; k < m; k += NT) {
        const unsigned short cf = A.cell[k];
        const int c = cf & 0x3fff;
        const int q = tb.cstart[c] + A.slot[k];
        const int4 rk = A.R[k];
        float thv = __int_as_float(rk.z);
        float sn, cs;
        if (MODEL == 1 && S.order != 1) {
            thv *= (float)S.order;
            sincosf(thv, &sn, &cs);
        } else {
            // |theta| <= pi: the hardware sine/cosine is within 2^-21.4 absolute
            __sincosf(thv, &sn, &cs);
        }
        const int flip = cf >> 14;
        if (flip & 1) {
            if (MODEL != 1 || (S.order & 1)) cs = -cs; else sn = -sn;
        }
        if (flip & 2) sn = -sn;
        A.P[q] = make_float4((float)(rk.x - xc) * S.ux, (float)(rk.y - yc) * S.uy,
                             __int_as_float(__float2int_rn(cs * kFixNbF)), __int_as_float(__float2int_rn(sn * kFixNbF)));
        A.sk[q] = (unsigned short)k;
        if (S.nsp > 1) A.gidx[q] = (unsigned short)species_of(S, (unsigned)rk.w);   // species by sorted position
    }
    if (warp == NT / 32 - 1) {
        int carry = 0;
        for (int r0 = 0; r0 < th; r0 += 32) {
            const int r = r0 + lane;
            int len = 0;
            if (r < th) len = tb.cstart[(r + 1) * W2 + tw + 1] - tb.cstart[(r + 1) * W2 + 1];
            const int incl = warp_incl_scan(len);
            if (r < th) tb.rowpre[r] = carry + incl - len;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) {
            tb.rowpre[th] = carry;
            T.n_own = carry;
        }
    }
    __syncthreads();
    PHASE_MARK(2);
    PHASE_MARK(3);

    // --- interact, update, scatter ---------------------------------------
    const int n_own = T.n_own;
    const float r2 = S.r2;
    const int TWs = tw << S.sx, THs = th << S.sy;
    const bool measure = step < S.meas_until;   // on-the-fly histograms (Sec. 3.4)
    long long acc_c = 0, acc_s = 0, acc_n = 0, acc_c2 = 0, acc_s2 = 0;
    for (int base = 0; base < n_own; base += NT) {
        const int o = base + tid;
        const bool act = o < n_own;
        int4 rec = make_int4(0, 0, 0, 0);
        int dtile = 0, region = 0;
        if (act) {
            // own particle o -> sorted position: the own row holding it
            int rlo = 0, rhi = th;
            while (rhi - rlo > 1) {
                const int mid = (rlo + rhi) >> 1;
                if (tb.rowpre[mid] <= o) rlo = mid; else rhi = mid;
            }
            const int q = tb.cstart[(rlo + 1) * W2 + 1] + (o - tb.rowpre[rlo]);
            const int k = A.sk[q];
            const int4 rk = A.R[k];
            const int X = rk.x, Y = rk.y;
            const float thi = __int_as_float(rk.z);
            const unsigned id = (unsigned)rk.w;
            const int ec = A.cell[k] & 0x3fff;
            const float4 pi = A.P[q];
            float sc, ss;                    // neighbour sums in units of 2^-22
            int cnt;
            const int sp = S.nsp > 1 ? species_of(S, id) : 0;
            if (MODEL == 1 && S.nsp > 1) {
                long long a, b;
                neighbour_sum_sp(A.P, A.gidx, tb.cstart, ec, W2, pi, r2, S.sp_gamma_dt + sp * kMaxSpecies, a, b,
                                 cnt);
                sc = (float)a;
                ss = (float)b;
            } else {
                const int ncand = tb.cstart[ec - W2 + 2] - tb.cstart[ec - W2 - 1] + tb.cstart[ec + 2] -
                                  tb.cstart[ec - 1] + tb.cstart[ec + W2 + 2] - tb.cstart[ec + W2 - 1];
                if (ncand < 512) {
                    int a, b;
                    neighbour_sum<MODEL, int>(A.P, tb.cstart, ec, W2, pi, r2, a, b, cnt);
                    sc = (float)a;
                    ss = (float)b;
                } else {
                    long long a, b;
                    neighbour_sum<MODEL, long long>(A.P, tb.cstart, ec, W2, pi, r2, a, b, cnt);
                    sc = (float)a;
                    ss = (float)b;
                }
            }
            const int nb = cnt - 1;          // the particle itself was counted
            if (measure) {
                int bt = (int)floorf((thi + AAP_PI_F) * ((float)S.bins_theta * (1.0f / AAP_2PI_F)));
                bt = min(max(bt, 0), S.bins_theta - 1);
                atomicAdd(&tb.mhist[bt], 1);
                atomicAdd(&tb.mhist[S.bins_theta + min(nb, S.bins_nbr - 1)], 1);
            }
            uint32_t c4[4] = {id, (uint32_t)step, (uint32_t)((unsigned long long)step >> 32), 0u};
            philox4x32_10(c4, S.seed_lo, S.seed_hi);
            const float u0 = u01f(c4[0]);
            float thn, cn, sn;
            int dX, dY;
            if (MODEL != 1) {
                // Eq. (collision_VM) / (collision_NVM) + noise; Eq. (streaming)
                thn = arg2(ss, sc) + S.sp_omega_step[sp] + S.sp_eta_pi[sp] * (2.0f * u0 - 1.0f);
                __sincosf(thn, &sn, &cn);
                dX = __float2int_rn(S.sp_kx[sp] * cn);
                dY = __float2int_rn(S.sp_ky[sp] * sn);
            } else {
                // Eq. (Langevin_dynamics), one Euler-Maruyama step
                const float u1 = u01f(c4[1]);
                const float h = S.wlen > 0 ? S.wtab[min(nb, S.wlen - 1)]
                                           : (S.weight ? 1.0f : 1.0f / (1.0f + (float)nb));
                // sum_j sin(o (theta_j - theta_i)) from the exact sums (units 2^-22 x 2^-22);
                // Gamma dt inside with several species
                const float tsum = ((float)__float_as_int(pi.z) * ss - (float)__float_as_int(pi.w) * sc) *
                                   (1.0f / (kFixNbF * kFixNbF));
                const float gz = sqrtf(-2.0f * logf(u0)) * cospif(2.0f * u1);
                const float drift = S.nsp > 1 ? h * tsum : S.gamma_dt * h * tsum;
                thn = thi + drift + S.sp_omega_step[sp] + S.sp_noise_amp[sp] * gz;
                float co, so;
                __sincosf(thi, &so, &co);    // streaming direction theta(t), |theta| <= pi
                dX = __float2int_rn(S.sp_kx[sp] * co);
                dY = __float2int_rn(S.sp_ky[sp] * so);
                cn = 0.f;
                sn = 0.f;
            }
            // boundary rule (Sec. 2.4) in exact fixed point
            int Xn = X + dX, Yn = Y + dY;
            int dtx = T.tx, dty = T.ty, twd = tw, thd = th;
            bool fx = false, fy = false;
            if (Xn < 0) {
                if (S.bx && T.tx == 0) { Xn = -Xn; fx = true; }
                else { dtx = T.tx > 0 ? T.tx - 1 : S.ntx - 1; twd = T.twL; Xn += T.twL << S.sx; }
            } else if (Xn >= TWs) {
                if (S.bx && T.tx == S.ntx - 1) {
                    if (Xn == TWs) Xn = TWs - 1; else { Xn = TWs - (Xn - TWs); fx = true; }
                } else { dtx = T.tx < S.ntx - 1 ? T.tx + 1 : 0; twd = T.twR; Xn -= TWs; }
            }
            if (Yn < 0) {
                if (S.by && T.ty == 0) { Yn = -Yn; fy = true; }
                else { dty = T.ty > 0 ? T.ty - 1 : S.nty - 1; thd = T.thD; Yn += T.thD << S.sy; }
            } else if (Yn >= THs) {
                if (S.by && T.ty == S.nty - 1) {
                    if (Yn == THs) Yn = THs - 1; else { Yn = THs - (Yn - THs); fy = true; }
                } else { dty = T.ty < S.nty - 1 ? T.ty + 1 : 0; thd = T.thU; Yn -= THs; }
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
            acc_c += __float2int_rn(cn * kFixStepF);
            acc_s += __float2int_rn(sn * kFixStepF);
            acc_c2 += __float2int_rn(fmaf(cn, cn, -sn * sn) * kFixStepF);
            acc_s2 += __float2int_rn(2.0f * cn * sn * kFixStepF);
            acc_n += nb;
            if (S.nbr_out && id < (unsigned long long)S.n) S.nbr_out[id] = nb;
        }
        warp_insert(S, nxt, act, dtile, region, rec);
    }
    // --- read ahead: the last warp (often idle in the last round of the
    //     update) prepares the next tile's geometry and segments, so that the
    //     next tile_setup starts without its chain of global loads ----------
    if (warp == NT / 32 - 1 && T.next < T.total) {
        const int g = T.next;
        const int si = T.nsys > 1 ? sys_of_tile(T.tile_base, T.nsys, g) : 0;
        if (si == T.sysi) {
            const TileGeo G = tile_geo(S, g - (T.nsys > 1 ? T.tile_base[si] : 0));
            if (lane < kSegs) T.pf_seg[lane] = make_seg(S, G, lane, cur);
            if (lane == 0) {
                T.pf_geo = G;
                T.pf_nsp = min(*((volatile int *)&S.spill_cnt[cur]), S.spill_cap);
                T.pf_tile = g - (T.nsys > 1 ? T.tile_base[si] : 0);
                T.pf_sys = si;
            }
        }
    }
    PHASE_MARK(4);
    // --- per-tile integer sums -> the step's accumulators ----------------
    acc_c = warp_sum_ll(acc_c);
    acc_s = warp_sum_ll(acc_s);
    acc_n = warp_sum_ll(acc_n);
    acc_c2 = warp_sum_ll(acc_c2);
    acc_s2 = warp_sum_ll(acc_s2);
    if (lane == 0) {
        T.red[0][warp] = acc_c;
        T.red[1][warp] = acc_s;
        T.red[2][warp] = acc_n;
        T.red[3][warp] = acc_c2;
        T.red[4][warp] = acc_s2;
    }
    __syncthreads();
    if (tid < 5) {
        long long v = 0;
        for (int w = 0; w < NT / 32; ++w) v += T.red[tid][w];
        unsigned long long *slot = S.acc + ((size_t)cur * kAccSlots + (T.tile & (kAccSlots - 1))) * kAccWords;
        atomicAdd(slot + tid, (unsigned long long)v);
    }
    if (measure) {
        for (int i = tid; i < S.bins_theta + S.bins_nbr; i += NT)
            if (tb.mhist[i]) atomicAdd(S.hist + i, (unsigned long long)tb.mhist[i]);
    }
    PHASE_MARK(5);
}

}  // namespace aapk
