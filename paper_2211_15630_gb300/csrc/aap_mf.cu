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
//                  its rings: ring search with a sorted top-k list in
//                  registers, the VM / NVM / Langevin update with h = 1
//                  (Sec. 2.3), streaming, boundary rule, the new record, and
//                  exact integer sums for p, q and the histograms
// followed by the k_finish of the metric path.
//
// Determinism: the selected set is ordered by (distance, id, image) and the
// sums run in that order, so nothing depends on the arrival order in a cell.
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

__global__ void k_mf_count(const Sys *__restrict__ sys, const Ctl *__restrict__ ctl)
{
    const Sys &S = *sys;
    const int cur = (int)(ctl->step & 1);
    const int ncx = S.ncx, ncy = S.ncy, sx = S.sx, sy = S.sy;
    const int4 *__restrict__ rec = S.rec[cur];
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

// Offer every particle of virtual cell (vx, vy) to the list of particle q.
template <int KMAX>
__device__ __forceinline__ void visit_cell(const MfGeo &G, const int4 *__restrict__ srt, const int *__restrict__ st,
                                           const int *__restrict__ blk, int vx, int vy, int X, int Y, long long q,
                                           float (&d)[KMAX], unsigned (&key)[KMAX], unsigned (&ref)[KMAX])
{
    AxisMap mx, my;
    if (!map_axis(vx, G.ncx, G.W, G.bx, X, mx) || !map_axis(vy, G.ncy, G.H, G.by, Y, my)) return;
    const int c = my.real * G.ncx + mx.real;
    const int b = cell_begin(st, blk, c), e = cell_begin(st, blk, c + 1);
    const bool untransformed = mx.code == 0 && my.code == 0;
    const unsigned code = (unsigned)((mx.code + 1) + 3 * (my.code + 1));
    const unsigned flips = (G.bx && mx.code ? 1u : 0u) | (G.by && my.code ? 2u : 0u);
    for (int j = b; j < e; ++j) {
        if (untransformed && j == q) continue;             // j != i
        const int4 rj = srt[j];
        const float dx = (float)(mx.a * rj.x + mx.off) * G.ux;
        const float dy = (float)(my.a * rj.y + my.off) * G.uy;
        const float d2 = fmaf(dx, dx, dy * dy);
        topk_offer<KMAX>(d, key, ref, d2, (unsigned)rj.w * 9u + code, (unsigned)j | (flips << 30));
    }
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
            const float tj = __int_as_float(rj.z);
            float sn, cs;
            if (MODEL == 1 && order != 1) sincosf(tj * (float)order, &sn, &cs);
            else __sincosf(tj, &sn, &cs);
            if (rf & (1u << 30)) {                   // mirrored in x: theta -> pi - theta
                if (MODEL != 1 || (order & 1)) cs = -cs; else sn = -sn;
            }
            if (rf & (2u << 30)) sn = -sn;           // mirrored in y: theta -> -theta
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

// The k nearest by exhaustive scan of all n records (out of line: it only
// runs when a periodic window cannot certify the list, i.e. for systems with
// about k particles or fewer across half the box).  out: sum cos, sum sin,
// Langevin sum; returns |Omega_i|.
template <int MODEL, int KMAX>
__device__ __noinline__ int brute_sums(const MfGeo &G, const int4 *__restrict__ srt, const Sys &S, const float *grow,
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

template <int NT, int MODEL, int KMAX>
__global__ void __launch_bounds__(NT) k_mf_update(const Sys *__restrict__ sys, const Ctl *__restrict__ ctl)
{
    extern __shared__ int s_hist[];                 // [bins_theta + bins_nbr] while measuring
    __shared__ long long s_red[5][NT / 32];
    const Sys &S = *sys;
    const long long step = ctl->step;
    const int cur = (int)(step & 1), nxt = cur ^ 1;
    const long long n = S.n;
    const int sx = S.sx, sy = S.sy, k = S.knn;
    MfGeo G;
    G.ncx = S.ncx;
    G.ncy = S.ncy;
    G.W = S.ncx << sx;
    G.H = S.ncy << sy;
    G.ux = S.ux;
    G.uy = S.uy;
    G.bx = S.bx != 0;
    G.by = S.by != 0;
    const int4 *__restrict__ srt = S.mf_sorted;
    const int *__restrict__ st = S.mf_start;
    const int *__restrict__ blk = S.mf_blk;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool measure = step < S.meas_until;       // on-the-fly histograms (Sec. 3.4)
    const int nbins = S.bins_theta + S.bins_nbr;
    if (measure)
        for (int i = tid; i < nbins; i += NT) s_hist[i] = 0;
    __syncthreads();
    long long acc_c = 0, acc_s = 0, acc_n = 0, acc_c2 = 0, acc_s2 = 0;
    const long long q = blockIdx.x * (long long)NT + tid;
    if (q < n) {
        const int4 r = srt[q];
        const int X = r.x, Y = r.y;
        const float thi = __int_as_float(r.z);
        const unsigned id = (unsigned)r.w;
        const int cx = min(X >> sx, G.ncx - 1), cy = min(Y >> sy, G.ncy - 1);
        float d[KMAX];
        unsigned key[KMAX], ref[KMAX];
#pragma unroll
        for (int s = 0; s < KMAX; ++s) {
            const bool dummy = s < KMAX - k;
            d[s] = dummy ? -1.0f : __int_as_float(0x7f800000);
            key[s] = dummy ? 0u : 0xffffffffu;
            ref[s] = 0u;
        }
        // ring search (Sec. 3.3); a periodic window stops short of wrapping
        // onto itself, a reflecting one at the outermost mirror image
        const int rmx = G.bx ? max(cx + G.ncx, 2 * G.ncx - 1 - cx) : (G.ncx - 1) / 2;
        const int rmy = G.by ? max(cy + G.ncy, 2 * G.ncy - 1 - cy) : (G.ncy - 1) / 2;
        bool certified = false;
        for (int ring = 0;; ++ring) {
            const int rx = min(ring, rmx), ry = min(ring, rmy);
            for (int dy = -ry; dy <= ry; ++dy) {
                if (dy == -ring || dy == ring) {
                    for (int dx = -rx; dx <= rx; ++dx)
                        visit_cell<KMAX>(G, srt, st, blk, cx + dx, cy + dy, X, Y, q, d, key, ref);
                } else if (ring <= rmx) {
                    visit_cell<KMAX>(G, srt, st, blk, cx - ring, cy + dy, X, Y, q, d, key, ref);
                    visit_cell<KMAX>(G, srt, st, blk, cx + ring, cy + dy, X, Y, q, d, key, ref);
                }
            }
            // every unvisited candidate lies at least this far away
            float gx = __int_as_float(0x7f800000), gy = gx;
            const int lo = cx - rx, hi = cx + rx, lo2 = cy - ry, hi2 = cy + ry;
            if (!(G.bx && lo <= -G.ncx)) gx = (float)(X - lo * (1 << sx)) * G.ux;
            if (!(G.bx && hi >= 2 * G.ncx - 1)) gx = fminf(gx, (float)((hi + 1) * (1 << sx) - X) * G.ux);
            if (!(G.by && lo2 <= -G.ncy)) gy = (float)(Y - lo2 * (1 << sy)) * G.uy;
            if (!(G.by && hi2 >= 2 * G.ncy - 1)) gy = fminf(gy, (float)((hi2 + 1) * (1 << sy) - Y) * G.uy);
            const float g = fminf(gx, gy);
            if (d[KMAX - 1] <= g * g * 0.99999f) {
                certified = true;
                break;
            }
            if (ring >= rmx && ring >= rmy) break;
        }
        // sums over Omega_i in (distance, id, image) order
        float si, ci;
        __sincosf(thi, &si, &ci);                    // |theta| <= pi
        float oci = ci, osi = si;                    // cos, sin of o theta_i
        if (MODEL == 1 && S.order != 1) sincosf(thi * (float)S.order, &osi, &oci);
        float sc = MODEL == 1 ? 0.f : ci, ss = MODEL == 1 ? 0.f : si, tsum = 0.f;
        int nb = 0;
        const int sp = S.nsp > 1 ? species_of(S, id) : 0;
        const float *grow = (MODEL == 1 && S.nsp > 1) ? S.sp_gamma_dt + sp * kMaxSpecies : nullptr;
        if (certified) {
            list_sums<MODEL, KMAX>(d, ref, srt, S, grow, S.order, ci, si, oci, osi, sc, ss, tsum, nb);
        } else {
            // the periodic window is exhausted: the definition itself, over
            // every particle at its nearest periodic copy (and mirror images)
            float out[3];
            nb = brute_sums<MODEL, KMAX>(G, srt, S, grow, n, q, X, Y, k, S.order, ci, si, oci, osi, out);
            sc += out[0];
            ss += out[1];
            tsum = out[2];
        }
        if (measure) {
            int bt = (int)floorf((thi + AAP_PI_F) * ((float)S.bins_theta * (1.0f / AAP_2PI_F)));
            bt = min(max(bt, 0), S.bins_theta - 1);
            atomicAdd(&s_hist[bt], 1);
            atomicAdd(&s_hist[S.bins_theta + min(nb, S.bins_nbr - 1)], 1);
        }
        uint32_t c4[4] = {id, (uint32_t)step, (uint32_t)((unsigned long long)step >> 32), 0u};
        philox4x32_10(c4, S.seed_lo, S.seed_hi);
        const float u0 = u01f(c4[0]);
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
            thn = thi + (grow ? tsum : S.gamma_dt * tsum) + S.sp_omega_step[sp] + S.sp_noise_amp[sp] * gz;
            dX = __float2int_rn(S.sp_kx[sp] * ci);
            dY = __float2int_rn(S.sp_ky[sp] * si);
        }
        // boundary rule (Sec. 2.4) in exact fixed point
        int Xn = X + dX, Yn = Y + dY;
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
        S.rec[nxt][q] = make_int4(Xn, Yn, __float_as_int(thn), (int)id);
        acc_c = __float2int_rn(cn * kFixStepF);
        acc_s = __float2int_rn(sn * kFixStepF);
        acc_c2 = __float2int_rn(fmaf(cn, cn, -sn * sn) * kFixStepF);
        acc_s2 = __float2int_rn(2.0f * cn * sn * kFixStepF);
        acc_n = nb;
        if (S.nbr_out && id < (unsigned long long)n) S.nbr_out[id] = nb;
    }
    acc_c = warp_sum_ll(acc_c);
    acc_s = warp_sum_ll(acc_s);
    acc_n = warp_sum_ll(acc_n);
    acc_c2 = warp_sum_ll(acc_c2);
    acc_s2 = warp_sum_ll(acc_s2);
    if (lane == 0) {
        s_red[0][warp] = acc_c;
        s_red[1][warp] = acc_s;
        s_red[2][warp] = acc_n;
        s_red[3][warp] = acc_c2;
        s_red[4][warp] = acc_s2;
    }
    __syncthreads();
    if (tid < 5) {
        long long v = 0;
        for (int w = 0; w < NT / 32; ++w) v += s_red[tid][w];
        unsigned long long *slot = S.acc + ((size_t)cur * kAccSlots + (blockIdx.x & (kAccSlots - 1))) * kAccWords;
        atomicAdd(slot + tid, (unsigned long long)v);
    }
    if (measure)
        for (int i = tid; i < nbins; i += NT)
            if (s_hist[i]) atomicAdd(S.hist + i, (unsigned long long)s_hist[i]);
    if (blockIdx.x == 0 && tid == 0) S.cnt[nxt][0] = (int)n;   // all records in region 0 of tile 0
}

template <int MODEL, int KMAX>
cudaError_t launch_update(const LaunchCfg &L, cudaStream_t st)
{
    const long long blocks = (L.mf_n + kMfThreads - 1) / kMfThreads;
    k_mf_update<kMfThreads, MODEL, KMAX><<<(unsigned)blocks, kMfThreads, (size_t)L.hist_words * sizeof(int), st>>>(
        L.sys, L.ctl);
    return cudaGetLastError();
}

template <int MODEL>
cudaError_t launch_update_m(const LaunchCfg &L, cudaStream_t st)
{
    if (L.knn <= 8) return launch_update<MODEL, 8>(L, st);
    if (L.knn <= 16) return launch_update<MODEL, 16>(L, st);
    return launch_update<MODEL, kMaxKnn>(L, st);
}

}  // namespace

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
