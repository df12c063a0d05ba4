// aap_kernels.cu -- sm_103a kernels of the aligning-active-particles step.
//
// One time step (Sec. 2 of Kuersten, "Aligning Active Particles Py Package"):
//   k_step     per tile: stage the tile and its one-cell halo (cell lists,
//              Sec. 3.2, with periodic or mirror images, Sec. 2.4), counting
//              sort by cell in shared memory (block histogram + block prefix
//              scan), sum over the 3x3 cells (Eq. collision_VM / collision_NVM
//              or the Langevin sum of Eq. Langevin_dynamics), draw Philox
//              noise, stream (Eq. streaming or Euler-Maruyama), apply the
//              boundary rule, and scatter the new record into the region of
//              its new cell through a warp-aggregated atomic counter.  Also
//              accumulates p = |sum e^{i theta}| / N (Sec. 3.4) in exact
//              64-bit integers.
//   k_deferred the same for tiles whose staged set overflowed shared memory,
//              staging in global scratch instead.
//   k_finish   turns the step's integer sums into p(t), clears the counters
//              of the buffer just consumed and advances the step counter.
#include <cuda_runtime.h>

#include "aap_internal.cuh"
#include "aap_kernels.cuh"

namespace aapk {

#define AAP_PI_F 3.14159265358979f
#define AAP_2PI_F 6.28318530717959f

// ---------------------------------------------------------------- Philox --
// Philox4x32-10 (Salmon et al., SC'11): counter c, key (k0, k1).
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// (w >> 9 + 1/2) 2^-23: exact in FP32.
__device__ __forceinline__ float u01f(uint32_t w) { return ((float)(w >> 9) + 0.5f) * (1.0f / 8388608.0f); }
__device__ __forceinline__ double u01d(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }

// ------------------------------------------------------------ geometry ----
__device__ __forceinline__ int tile_x0(const Sys &S, int tx) { return (int)(((long long)tx * S.ncx) / S.ntx); }
__device__ __forceinline__ int tile_y0(const Sys &S, int ty) { return (int)(((long long)ty * S.ncy) / S.nty); }
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
    const unsigned peers = __match_any_sync(0xffffffffu, key);
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
                atomicOr(S.err, ERR_SPILL);
            } else {
                atomicOr(S.err, ERR_LOST);
            }
        }
    }
}

__device__ __forceinline__ long long warp_sum_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_incl_scan(int v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// ---------------------------------------------------------- tile context --
struct TileCtx {
    Sys S;
    int sysi, tile, tx, ty, tw, th, W2, H2, nce;
    int twL, twR, thD, thU;     // widths / heights of the neighbour tiles
    int m_seg, n_spill, m, n_own, defer;
    int segpre[kSegs + 1];
    int warp_tot[32];
    Seg seg[kSegs];
    long long red[3][32];
};

// Resolve the halo column (side -1: left, +1: right) of tile tx into a source
// tile column, the region column class there, and the position / cell maps.
__device__ __forceinline__ void resolve_axis(int side, int t, int nt, int w, int wlo, int whi,
                                             int refl, int s, int &src, int &cls, int &a,
                                             int &c, long long &b, int &flip)
{
    if (side == 0) {
        src = t; a = 1; c = 0; b = 0; flip = 0; cls = -1;
        return;
    }
    if (side < 0) {
        if (t > 0 || !refl) {
            src = (t > 0) ? t - 1 : nt - 1;
            cls = 2; a = 1; c = -wlo; b = -((long long)wlo << s); flip = 0;
        } else {
            src = t; cls = 0; a = -1; c = -1; b = 0; flip = 1;
        }
    } else {
        if (t < nt - 1 || !refl) {
            src = (t < nt - 1) ? t + 1 : 0;
            cls = 0; a = 1; c = w; b = (long long)w << s; flip = 0;
        } else {
            src = t; cls = 2; a = -1; c = 2 * w - 1; b = 2 * ((long long)w << s); flip = 1;
        }
    }
    (void)whi;
}

template <int NT>
__device__ void process_tile(TileCtx &T, const Stage &A, const Tables &tb, long long step,
                             Ctl *ctl, int *defer_list, int gtile, bool scratch)
{
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const Sys &S = T.S;
    const int cur = (int)(step & 1), nxt = cur ^ 1;

    // --- A. tile geometry ----------------------------------------------
    if (tid == 0) {
        const int tx = T.tile % S.ntx, ty = T.tile / S.ntx;
        T.tx = tx;
        T.ty = ty;
        const int x0 = tile_x0(S, tx), x1 = tile_x0(S, tx + 1);
        const int y0 = tile_y0(S, ty), y1 = tile_y0(S, ty + 1);
        T.tw = x1 - x0;
        T.th = y1 - y0;
        T.W2 = T.tw + 2;
        T.H2 = T.th + 2;
        T.nce = T.W2 * T.H2;
        const int txl = tx > 0 ? tx - 1 : S.ntx - 1, txr = tx < S.ntx - 1 ? tx + 1 : 0;
        const int tyd = ty > 0 ? ty - 1 : S.nty - 1, tyu = ty < S.nty - 1 ? ty + 1 : 0;
        T.twL = tile_x0(S, txl + 1) - tile_x0(S, txl);
        T.twR = tile_x0(S, txr + 1) - tile_x0(S, txr);
        T.thD = tile_y0(S, tyd + 1) - tile_y0(S, tyd);
        T.thU = tile_y0(S, tyu + 1) - tile_y0(S, tyu);
        T.n_spill = 0;
        T.defer = 0;
    }
    __syncthreads();

    // --- B. the 25 segments: 9 own regions, then the 16 halo regions ---
    if (tid < kSegs) {
        int bxo, byo, rx = -1, ry = -1;
        if (tid < 9) {
            bxo = 0; byo = 0; rx = tid % 3; ry = tid / 3;
        } else {
            const int h = tid - 9;
            if (h < 3)       { bxo = -1; byo = 0;  ry = h; }
            else if (h < 6)  { bxo = 1;  byo = 0;  ry = h - 3; }
            else if (h < 9)  { bxo = 0;  byo = -1; rx = h - 6; }
            else if (h < 12) { bxo = 0;  byo = 1;  rx = h - 9; }
            else { bxo = (h & 1) ? 1 : -1; byo = (h >= 14) ? 1 : -1; }
        }
        int srcx, clsx, ax, cx, fx, srcy, clsy, ay, cy, fy;
        long long bxx, byy;
        resolve_axis(bxo, T.tx, S.ntx, T.tw, T.twL, T.twR, S.bx, S.sx, srcx, clsx, ax, cx, bxx, fx);
        resolve_axis(byo, T.ty, S.nty, T.th, T.thD, T.thU, S.by, S.sy, srcy, clsy, ay, cy, byy, fy);
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
        T.seg[tid] = g;
    }
    __syncthreads();
    if (warp == 0) {
        const int v = lane < kSegs ? T.seg[lane].count : 0;
        const int incl = warp_incl_scan(v);
        if (lane < kSegs) T.segpre[lane] = incl - v;
        if (lane == kSegs - 1) {
            T.segpre[kSegs] = incl;
            T.m_seg = incl;
        }
    }
    // --- C. particles parked in the spill list for one of our segments ---
    const int nsp = min(*((volatile int *)&S.spill_cnt[cur]), S.spill_cap);
    __syncthreads();
    if (nsp > 0) {
        for (int e = tid; e < nsp; e += NT) {
            const int key = S.spill_key[cur][e];
            const int et = key / kCntStride, er = key % kCntStride;
            for (int s = 0; s < kSegs; ++s) {
                if (T.seg[s].tile == et && T.seg[s].region == er) {
                    const int j = atomicAdd(&T.n_spill, 1);
                    if (j < A.spill_list_cap) {
                        A.spill_e[j] = e;
                        A.spill_s[j] = (unsigned char)s;
                    }
                }
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        T.m = T.m_seg + T.n_spill;
        if (T.m > A.cap || T.n_spill > A.spill_list_cap) {
            if (!scratch) {
                const int d = atomicAdd(&ctl->defer_count, 1);
                defer_list[d] = gtile;
            } else {
                atomicOr(S.err, ERR_STAGE | ERR_LOST);
            }
            T.defer = 1;
        }
    }
    __syncthreads();
    if (T.defer) return;

    const int m = T.m, m_seg = T.m_seg, W2 = T.W2, H2 = T.H2, nce = T.nce;
    for (int i = tid; i < nce; i += NT) tb.hist[i] = 0;
    __syncthreads();

    // --- D. stage: decode, map into the extended frame, histogram by cell --
    for (int k = tid; k < m; k += NT) {
        int s;
        int4 r;
        if (k < m_seg) {
            int lo = 0, hi = kSegs;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (T.segpre[mid] <= k) lo = mid; else hi = mid;
            }
            s = lo;
            r = T.seg[s].base[k - T.segpre[s]];
        } else {
            const int j = k - m_seg;
            s = A.spill_s[j];
            r = S.spill_rec[cur][A.spill_e[j]];
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
        A.rX[k] = (int)(g.ax * (long long)r.x + g.bx);
        A.rY[k] = (int)(g.ay * (long long)r.y + g.by);
        A.rth[k] = __int_as_float(r.z);
        A.id[k] = (unsigned)r.w;
        A.cell[k] = (unsigned short)(ec | (g.flip << 14));
        A.slot[k] = (unsigned short)atomicAdd(&tb.hist[ec], 1);
    }
    __syncthreads();

    // --- E. block-level exclusive prefix scan of the cell histogram ------
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

    // --- F. group by cell -------------------------------------------------
    for (int k = tid; k < m; k += NT) {
        const int c = A.cell[k] & 0x3fff;
        A.gidx[tb.cstart[c] + A.slot[k]] = (unsigned short)k;
    }
    __syncthreads();

    // --- G. order each cell by particle id and lay out the sorted arrays --
    const int xc = T.tw << (S.sx - 1), yc = T.th << (S.sy - 1);
    for (int p = tid; p < m; p += NT) {
        const int k = A.gidx[p];
        const unsigned short cf = A.cell[k];
        const int c = cf & 0x3fff;
        const int a = tb.cstart[c], b = tb.cstart[c + 1];
        const unsigned myid = A.id[k];
        int rank = 0;
        for (int p2 = a; p2 < b; ++p2) {
            const int k2 = A.gidx[p2];
            const unsigned id2 = A.id[k2];
            rank += (id2 < myid) || (id2 == myid && k2 < k);
        }
        const int q = a + rank;
        float th = A.rth[k];
        if (S.model == 1 && S.order != 1) th *= (float)S.order;
        float sn, cs;
        sincosf(th, &sn, &cs);
        const int flip = cf >> 14;
        if (flip & 1) {
            if (S.model != 1 || (S.order & 1)) cs = -cs; else sn = -sn;
        }
        if (flip & 2) sn = -sn;
        A.px[q] = (float)(A.rX[k] - xc) * S.ux;
        A.py[q] = (float)(A.rY[k] - yc) * S.uy;
        A.pc[q] = cs;
        A.ps[q] = sn;
        A.sk[q] = (unsigned short)k;
    }
    __syncthreads();

    // --- H. own particles, in (cell, id) order, row by row ---------------
    if (warp == 0) {
        int carry = 0;
        for (int r0 = 0; r0 < T.th; r0 += 32) {
            const int r = r0 + lane;
            int len = 0;
            if (r < T.th) len = tb.cstart[(r + 1) * W2 + T.tw + 1] - tb.cstart[(r + 1) * W2 + 1];
            const int incl = warp_incl_scan(len);
            if (r < T.th) tb.rowpre[r] = carry + incl - len;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) {
            tb.rowpre[T.th] = carry;
            T.n_own = carry;
        }
    }
    __syncthreads();

    // --- I. interact, update, scatter ------------------------------------
    const int n_own = T.n_own, th_t = T.th, tw = T.tw, th = T.th;
    const float r2 = S.r2;
    const int model = S.model;
    const int TWs = tw << S.sx, THs = th << S.sy;
    long long acc_c = 0, acc_s = 0, acc_n = 0;
    for (int base = 0; base < n_own; base += NT) {
        const int o = base + tid;
        const bool act = o < n_own;
        int4 rec = make_int4(0, 0, 0, 0);
        int dtile = 0, region = 0;
        if (act) {
            int lo = 0, hi = th_t;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (tb.rowpre[mid] <= o) lo = mid; else hi = mid;
            }
            const int q = tb.cstart[(lo + 1) * W2 + 1] + (o - tb.rowpre[lo]);
            const int k = A.sk[q];
            const int X = A.rX[k], Y = A.rY[k];
            const float thi = A.rth[k];
            const unsigned id = A.id[k];
            const int ec = A.cell[k] & 0x3fff;   // clamped into the tile when staged
            const float xi = A.px[q], yi = A.py[q], ci = A.pc[q], si = A.ps[q];
            float sc = 0.f, ss = 0.f;
            int cnt = 0;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const int c0 = ec + dy * W2 - 1;
                const int a = tb.cstart[c0], b = tb.cstart[c0 + 3];
                for (int j = a; j < b; ++j) {
                    const float dx = A.px[j] - xi, dyy = A.py[j] - yi;
                    const float d2 = fmaf(dx, dx, dyy * dyy);
                    if (d2 <= r2) {
                        float cj = A.pc[j], sj = A.ps[j];
                        if (model == 2 && fmaf(ci, cj, si * sj) < 0.f) {
                            cj = -cj;
                            sj = -sj;
                        }
                        sc += cj;
                        ss += sj;
                        ++cnt;
                    }
                }
            }
            const int nb = cnt - 1;          // the particle itself was counted
            uint32_t c4[4] = {id, (uint32_t)step, (uint32_t)((unsigned long long)step >> 32), 0u};
            philox4x32_10(c4, S.seed_lo, S.seed_hi);
            const float u0 = u01f(c4[0]);
            float thn, cn, sn;
            int dX, dY;
            if (model != 1) {
                // Eq. (collision_VM) / (collision_NVM): the sum includes e^{i theta_i}.
                thn = atan2f(ss, sc) + S.omega_step + S.eta_pi * (2.0f * u0 - 1.0f);
                sincosf(thn, &sn, &cn);
                dX = __float2int_rn(S.kx * cn);
                dY = __float2int_rn(S.ky * sn);
            } else {
                // Eq. (Langevin_dynamics), Euler-Maruyama; the self term adds sin 0.
                const float u1 = u01f(c4[1]);
                const float h = S.weight ? 1.0f : 1.0f / (1.0f + (float)nb);
                const float tsum = ci * ss - si * sc;
                const float gz = sqrtf(-2.0f * logf(u0)) * cospif(2.0f * u1);
                thn = thi + S.gamma_dt * h * tsum + S.omega_step + S.noise_amp * gz;
                float co = ci, so = si;
                if (S.order != 1) sincosf(thi, &so, &co);
                dX = __float2int_rn(S.kx * co);
                dY = __float2int_rn(S.ky * so);
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
            if (thn >= AAP_PI_F || thn < -AAP_PI_F) thn -= AAP_2PI_F * floorf((thn + AAP_PI_F) * (1.0f / AAP_2PI_F));
            if (model == 1) sincosf(thn, &sn, &cn);
            if (!isfinite(thn)) atomicOr(S.err, ERR_NAN);
            dtile = dty * S.ntx + dtx;
            region = region_of(Xn >> S.sx, Yn >> S.sy, twd, thd);
            rec = make_int4(Xn, Yn, __float_as_int(thn), (int)id);
            acc_c += __float2ll_rn(cn * 4294967296.0f);
            acc_s += __float2ll_rn(sn * 4294967296.0f);
            acc_n += nb;
            if (S.nbr_out && id < (unsigned long long)S.n) S.nbr_out[id] = nb;
        }
        warp_insert(S, nxt, act, dtile, region, rec);
    }
    // --- J. per-tile integer sums -> the step's accumulators -------------
    acc_c = warp_sum_ll(acc_c);
    acc_s = warp_sum_ll(acc_s);
    acc_n = warp_sum_ll(acc_n);
    if (lane == 0) {
        T.red[0][warp] = acc_c;
        T.red[1][warp] = acc_s;
        T.red[2][warp] = acc_n;
    }
    __syncthreads();
    if (tid < 3) {
        long long v = 0;
        for (int w = 0; w < NT / 32; ++w) v += T.red[tid][w];
        unsigned long long *slot = S.acc + ((size_t)cur * kAccSlots + (T.tile & (kAccSlots - 1))) * kAccWords;
        atomicAdd(slot + tid, (unsigned long long)v);
    }
}

__device__ __forceinline__ int sys_of_tile(const int *tile_base, int nsys, int g)
{
    int lo = 0, hi = nsys;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tile_base[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void load_sys(TileCtx &T, const Sys *sys, int si)
{
    if (T.sysi == si) return;
    __syncthreads();
    const int words = (int)(sizeof(Sys) / 4);
    const int *src = reinterpret_cast<const int *>(sys + si);
    int *dst = reinterpret_cast<int *>(&T.S);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    if (threadIdx.x == 0) T.sysi = si;
    __syncthreads();
}

// Persistent blocks pull tiles (in raster order, so halos are L2-hot) from a
// device counter.
template <int NT>
__global__ void __launch_bounds__(NT) k_step(const Sys *__restrict__ sys, int nsys,
                                             const int *__restrict__ tile_base, Ctl *ctl,
                                             int *defer_list, int stage_cap, int nce_max)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ TileCtx T;
    __shared__ int s_next;
    const long long step = ctl->step;
    const int total = tile_base[nsys];
    Stage A;
    carve_particles(A, smem, stage_cap);
    unsigned char *p = smem + stage_particle_bytes(stage_cap);
    Tables tb;
    carve_tables(tb, p, nce_max);
    p += table_bytes(nce_max);
    A.spill_e = (int *)p;
    A.spill_s = (unsigned char *)(p + kSpillListFast * 4);
    A.spill_list_cap = kSpillListFast;
    if (threadIdx.x == 0) T.sysi = -1;
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(&ctl->tile_next, 1);
        __syncthreads();
        const int g = s_next;
        __syncthreads();
        if (g >= total) break;
        const int si = sys_of_tile(tile_base, nsys, g);
        load_sys(T, sys, si);
        if (threadIdx.x == 0) T.tile = g - tile_base[si];
        __syncthreads();
        process_tile<NT>(T, A, tb, step, ctl, defer_list, g, false);
        __syncthreads();
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_deferred(const Sys *__restrict__ sys, int nsys,
                                                 const int *__restrict__ tile_base, Ctl *ctl,
                                                 const int *defer_list, unsigned char *scratch,
                                                 size_t scratch_per_block, int scratch_cap,
                                                 int nce_max)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ TileCtx T;
    __shared__ int s_next;
    const int count = *((volatile int *)&ctl->defer_count);
    if (count == 0) return;
    const long long step = ctl->step;
    Stage A;
    unsigned char *mine = scratch + scratch_per_block * blockIdx.x;
    carve_particles(A, mine, scratch_cap);
    A.spill_e = (int *)(mine + stage_particle_bytes(scratch_cap));
    A.spill_s = (unsigned char *)(A.spill_e + scratch_cap);
    A.spill_list_cap = scratch_cap;
    Tables tb;
    carve_tables(tb, smem, nce_max);
    if (threadIdx.x == 0) T.sysi = -1;
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(&ctl->defer_next, 1);
        __syncthreads();
        const int i = s_next;
        __syncthreads();
        if (i >= count) break;
        const int g = defer_list[i];
        const int si = sys_of_tile(tile_base, nsys, g);
        load_sys(T, sys, si);
        if (threadIdx.x == 0) T.tile = g - tile_base[si];
        __syncthreads();
        process_tile<NT>(T, A, tb, step, ctl, nullptr, g, true);
        __syncthreads();
    }
}

// Close the step: p(t+1) from the integer sums, clear the consumed buffer's
// counters, advance the step.  The last block to arrive does the per-system
// work; every block clears a share of the counters.
__global__ void k_finish(Sys *sys, int nsys, Ctl *ctl)
{
    __shared__ int s_last;
    const long long step = ctl->step;
    const int cur = (int)(step & 1);
    for (int si = 0; si < nsys; ++si) {
        int *c = sys[si].cnt[cur];
        const long long nw = (long long)sys[si].ntiles * kCntStride;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nw;
             i += (long long)gridDim.x * blockDim.x)
            c[i] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = (atomicAdd(&ctl->finish_ticket, 1) == (int)gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    for (int si = threadIdx.x; si < nsys; si += blockDim.x) {
        Sys &S = sys[si];
        unsigned long long *a = S.acc + (size_t)cur * kAccSlots * kAccWords;
        long long sc = 0, ss = 0, sn = 0;
        for (int k = 0; k < kAccSlots; ++k) {
            sc += (long long)a[k * kAccWords + 0];
            ss += (long long)a[k * kAccWords + 1];
            sn += (long long)a[k * kAccWords + 2];
            a[k * kAccWords + 0] = 0;
            a[k * kAccWords + 1] = 0;
            a[k * kAccWords + 2] = 0;
        }
        const double n = (double)S.n;
        const double dc = (double)sc / kFix, ds = (double)ss / kFix;
        const double phi = n > 0 ? sqrt(dc * dc + ds * ds) / n : 0.0;
        const double nbar = n > 0 ? (double)sn / n : 0.0;
        if (S.trace) {
            const long long i1 = step + 1 - S.trace_base, i0 = step - S.trace_base;
            if (i1 >= 0 && i1 < S.trace_cap) S.trace[i1] = phi;
            if (i0 >= 0 && i0 < S.trace_cap) S.trace_nbar[i0] = nbar;
        }
        S.last[0] = phi;
        S.last[1] = nbar;
        S.last[2] = (double)(step + 1);
        S.spill_cnt[cur] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl->tile_next = 0;
        ctl->defer_next = 0;
        ctl->defer_count = 0;
        ctl->finish_ticket = 0;
        ctl->step = step + 1;
    }
}

// ------------------------------------------------- state in and out --------
// Place one particle given in box coordinates into buffer b (exact rounding
// of the position to the fixed-point grid).  mode 0: from arrays; mode 1: draw
// the uniform isotropic initial state from Philox, tag 1.
__global__ void k_insert(Sys S, int b, const double *x, const double *y, const float *th, int mode)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool act = i < S.n;
    int dtile = 0, region = 0;
    int4 rec = make_int4(0, 0, 0, 0);
    if (act) {
        double px, py;
        float pt;
        if (mode == 1) {
            uint32_t c4[4] = {(uint32_t)i, 0u, 0u, 1u};
            philox4x32_10(c4, S.seed_lo, S.seed_hi);
            px = S.lx * u01d(c4[0]);
            py = S.ly * u01d(c4[1]);
            pt = (float)(3.14159265358979323846 * (2.0 * u01d(c4[2]) - 1.0));
        } else {
            px = x[i];
            py = y[i];
            pt = th[i];
        }
        long long gx = llrint(px / S.csx_d * (double)(1ll << S.sx));
        long long gy = llrint(py / S.csy_d * (double)(1ll << S.sy));
        const long long wx = (long long)S.ncx << S.sx, wy = (long long)S.ncy << S.sy;
        if (gx >= wx) gx = S.bx ? wx - 1 : gx - wx;
        if (gx < 0) gx = S.bx ? 0 : gx + wx;
        if (gy >= wy) gy = S.by ? wy - 1 : gy - wy;
        if (gy < 0) gy = S.by ? 0 : gy + wy;
        const int cx = (int)(gx >> S.sx), cy = (int)(gy >> S.sy);
        const int tx = tile_of_x(S, cx), ty = tile_of_y(S, cy);
        const int x0 = tile_x0(S, tx), y0 = tile_y0(S, ty);
        const int X = (int)(gx - ((long long)x0 << S.sx)), Y = (int)(gy - ((long long)y0 << S.sy));
        const int tw = tile_x0(S, tx + 1) - x0, th_ = tile_y0(S, ty + 1) - y0;
        if (pt >= AAP_PI_F || pt < -AAP_PI_F) pt -= AAP_2PI_F * floorf((pt + AAP_PI_F) * (1.0f / AAP_2PI_F));
        dtile = ty * S.ntx + tx;
        region = region_of(X >> S.sx, Y >> S.sy, tw, th_);
        rec = make_int4(X, Y, __float_as_int(pt), (int)i);
    }
    warp_insert(S, b, act, dtile, region, rec);
}

// Visit every stored record of buffer b: slots [0, tiles * tile_slots) then
// the spill list.  Returns false for empty slots.
__device__ __forceinline__ bool fetch_record(const Sys &S, int b, long long g, int4 &r, int &tile)
{
    const long long nslot = (long long)S.ntiles * S.tile_slots;
    if (g < nslot) {
        tile = (int)(g / S.tile_slots);
        const int o = (int)(g - (long long)tile * S.tile_slots);
        int reg = 0;
#pragma unroll
        for (int k = 1; k < kRegions; ++k)
            if (o >= S.off[k]) reg = k;
        const int slot = o - S.off[reg];
        if (slot >= S.cap[reg]) return false;
        if (slot >= S.cnt[b][tile * kCntStride + reg]) return false;
        r = S.rec[b][g];
        return true;
    }
    const long long e = g - nslot;
    if (e >= min(S.spill_cnt[b], S.spill_cap)) return false;
    r = S.spill_rec[b][e];
    tile = S.spill_key[b][e] / kCntStride;
    return true;
}

__global__ void k_gather(Sys S, int b, double *x, double *y, float *th, int *seen)
{
    const long long total = (long long)S.ntiles * S.tile_slots + S.spill_cap;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        int4 r;
        int tile;
        if (!fetch_record(S, b, g, r, tile)) continue;
        const int tx = tile % S.ntx, ty = tile / S.ntx;
        const unsigned id = (unsigned)r.w;
        if (id >= (unsigned long long)S.n) {
            atomicOr(S.err, ERR_BOUNDS);
            continue;
        }
        const double gx = (double)((long long)tile_x0(S, tx) << S.sx) + (double)r.x;
        const double gy = (double)((long long)tile_y0(S, ty) << S.sy) + (double)r.y;
        x[id] = gx * (S.csx_d / (double)(1ll << S.sx));
        y[id] = gy * (S.csy_d / (double)(1ll << S.sy));
        th[id] = __int_as_float(r.z);
        atomicAdd(seen, 1);
    }
}

// p and q of buffer b (Sec. 3.4), in exact 64-bit integer sums (order-free,
// so the result is reproducible bit for bit), plus the number of records.
__global__ void k_observe(Sys S, int b, unsigned long long *out)
{
    __shared__ long long red[5][32];
    const long long total = (long long)S.ntiles * S.tile_slots + S.spill_cap;
    long long a[5] = {0, 0, 0, 0, 0};
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        int4 r;
        int tile;
        if (!fetch_record(S, b, g, r, tile)) continue;
        const float t = __int_as_float(r.z);
        if (!isfinite(t)) atomicOr(S.err, ERR_NAN);
        float s1, c1, s2, c2;
        sincosf(t, &s1, &c1);
        sincosf(2.0f * t, &s2, &c2);
        a[0] += __float2ll_rn(c1 * 4294967296.0f);
        a[1] += __float2ll_rn(s1 * 4294967296.0f);
        a[2] += __float2ll_rn(c2 * 4294967296.0f);
        a[3] += __float2ll_rn(s2 * 4294967296.0f);
        a[4] += 1;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const long long v = warp_sum_ll(a[k]);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        long long v = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
        atomicAdd(out + threadIdx.x, (unsigned long long)v);
    }
}

// --------------------------------------------------------------- launchers --
template <int NT>
static cudaError_t launch_step_t(const LaunchCfg &L, cudaStream_t st, cudaEvent_t *ev)
{
    const size_t smem = step_smem_bytes(L.stage_cap, L.nce_max);
    cudaError_t e;
    if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
    k_step<NT><<<L.grid_step, NT, smem, st>>>(L.sys, L.nsys, L.tile_base, L.ctl, L.defer_list,
                                               L.stage_cap, L.nce_max);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return e;
    k_deferred<NT><<<L.grid_defer, NT, table_bytes(L.nce_max), st>>>(
        L.sys, L.nsys, L.tile_base, L.ctl, L.defer_list, L.scratch, L.scratch_per_block,
        L.scratch_cap, L.nce_max);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[2], st)) != cudaSuccess) return e;
    k_finish<<<L.grid_finish, 256, 0, st>>>(L.sys, L.nsys, L.ctl);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[3], st)) != cudaSuccess) return e;
    return cudaSuccess;
}

size_t step_smem_bytes(int stage_cap, int nce_max)
{
    return stage_particle_bytes(stage_cap) + table_bytes(nce_max) + spill_list_bytes(kSpillListFast);
}

cudaError_t launch_step(const LaunchCfg &L, cudaStream_t st, cudaEvent_t *ev)
{
    switch (L.threads) {
    case 128: return launch_step_t<128>(L, st, ev);
    case 256: return launch_step_t<256>(L, st, ev);
    case 512: return launch_step_t<512>(L, st, ev);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t configure_step_kernels(int threads, size_t smem_bytes)
{
    cudaError_t e = cudaSuccess;
    switch (threads) {
    case 128: e = cudaFuncSetAttribute(k_step<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes); break;
    case 256: e = cudaFuncSetAttribute(k_step<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes); break;
    case 512: e = cudaFuncSetAttribute(k_step<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes); break;
    default: return cudaErrorInvalidValue;
    }
    return e;
}

cudaError_t step_blocks_per_sm(int threads, size_t smem_bytes, int *out)
{
    switch (threads) {
    case 128: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_step<128>, 128, smem_bytes);
    case 256: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_step<256>, 256, smem_bytes);
    case 512: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_step<512>, 512, smem_bytes);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_insert(const Sys &S, int b, const double *x, const double *y, const float *th,
                          int mode, cudaStream_t st)
{
    const long long n = S.n;
    if (n == 0) return cudaSuccess;
    const int bs = 256;
    const long long grid = (n + bs - 1) / bs;
    k_insert<<<(unsigned)grid, bs, 0, st>>>(S, b, x, y, th, mode);
    return cudaGetLastError();
}

cudaError_t launch_gather(const Sys &S, int b, double *x, double *y, float *th, int *seen,
                          cudaStream_t st)
{
    k_gather<<<1024, 256, 0, st>>>(S, b, x, y, th, seen);
    return cudaGetLastError();
}

cudaError_t launch_observe(const Sys &S, int b, unsigned long long *out, cudaStream_t st)
{
    k_observe<<<1024, 256, 0, st>>>(S, b, out);
    return cudaGetLastError();
}

}  // namespace aapk
