// aap_kernels.cu -- sm_103a kernels of the aligning-active-particles step.
//
// One time step (Sec. 2 of Kuersten, "Aligning Active Particles Py Package"):
//   k_step     per tile: stage the tile and its one-cell halo (cell lists,
//              Sec. 3.2, with periodic or mirror images, Sec. 2.4), counting
//              sort by cell in shared memory (block histogram + block prefix
//              scan; arrival order inside a cell), sum over the 3x3 cells
//              (Eq. collision_VM / collision_NVM or the Langevin sum of
//              Eq. Langevin_dynamics) in exact integers, so that the result
//              does not depend on that arrival order, draw Philox
//              noise, stream (Eq. streaming or Euler-Maruyama), apply the
//              boundary rule, and scatter the new record into the region of
//              its new cell through a warp-aggregated atomic counter.  Also
//              accumulates p = |sum e^{i theta}| / N (Sec. 3.4) in exact
//              64-bit integers.
//              Tiles whose staged set does not fit shared memory are staged
//              in the block's slice of global scratch by the same code.
//   k_finish   turns the step's integer sums into p(t), clears the counters
//              of the buffer just consumed and advances the step counter.
#include <algorithm>

#include <atomic>
#include <cuda_runtime.h>

#include "aap_device.cuh"
#include "aap_internal.cuh"
#include "aap_kernels.cuh"
#include "aap_tile.cuh"

namespace aapk {

// Persistent blocks pull tiles in raster order (so halos are L2-hot) from a
// device counter; the next tile index is fetched while the current one runs.
// A tile whose staged set exceeds the shared-memory capacity is staged in the
// block's slice of global scratch instead.  All systems of one launch share
// the model.
template <int NT, int MODEL>
__global__ void __launch_bounds__(NT, NT >= 512 ? 2 : 3)
k_step(const Sys *__restrict__ sys, int nsys, const int *__restrict__ tile_base, Ctl *ctl,
       int stage_cap, int nce_max, unsigned char *scratch, size_t scratch_per_block, int scratch_cap,
       int spill_list_cap)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ TileCtx T;
    const long long step = ctl->step;
    const int cur = (int)(step & 1);
    const int total = tile_base[nsys];
    Stage As;
    carve_stage(As, smem, stage_cap);
    Tables tb;
    carve_tables(tb, smem + stage_bytes(stage_cap), nce_max);
    unsigned char *mine = scratch + scratch_per_block * blockIdx.x;
    Stage Ag;
    carve_stage(Ag, mine, scratch_cap);
    int *spill_e = (int *)(mine + stage_bytes(scratch_cap));
    unsigned char *spill_s = (unsigned char *)(spill_e + spill_list_cap);
    if (threadIdx.x == 0) {
        T.sysi = -1;
        T.pf_tile = -1;
        T.total = total;
        T.nsys = nsys;
        T.tile_base = tile_base;
        T.next = atomicAdd(&ctl->tile_next, 1);
    }
    __syncthreads();
    for (;;) {
        const int g = T.next;
        if (g >= total) break;
        const int si = nsys > 1 ? sys_of_tile(tile_base, nsys, g) : 0;
        if (si != T.sysi) {
            const int words = (int)(sizeof(Sys) / 4);
            const int *src = reinterpret_cast<const int *>(sys + si);
            int *dst = reinterpret_cast<int *>(&T.S);
            for (int i = threadIdx.x; i < words; i += NT) dst[i] = src[i];
        }
        __syncthreads();
        int next_g = 0;         // thread 0: the tile after this one (published in tile_body)
        if (threadIdx.x == 0) {
            T.sysi = si;
            T.tile = g - tile_base[si];
            next_g = atomicAdd(&ctl->tile_next, 1);
        }
        __syncthreads();
#ifdef AAP_PHASE_TIMING
        const long long ts0 = clock64();
#endif
        tile_setup<NT>(T, tb, cur, nce_max, spill_e, spill_s, spill_list_cap);
#ifdef AAP_PHASE_TIMING
        if (threadIdx.x == 0) {
            atomicAdd(&g_phase[6], (unsigned long long)(clock64() - ts0));
            atomicAdd(&g_phase[7], 1ull);
            atomicAdd(&g_phase[8], (unsigned long long)T.m);
            atomicAdd(&g_phase[9], (unsigned long long)(T.m > stage_cap));
        }
#endif
#ifdef AAP_PHASE_TIMING
        const long long tb0 = clock64();
#endif
        if (T.m <= stage_cap) {
            tile_body<NT, MODEL>(T, As, tb, step, spill_e, spill_s, next_g);
        } else if (T.m <= scratch_cap) {
            // a dense tile: staged in global scratch, except the records the
            // candidate loops read, which still fit the shared staging area
            Stage Ah = Ag;
            if ((size_t)T.m * sizeof(float4) <= stage_bytes(stage_cap)) Ah.P = reinterpret_cast<float4 *>(smem);
            tile_body<NT, MODEL>(T, Ah, tb, step, spill_e, spill_s, next_g);
        } else if (threadIdx.x == 0) {
            atomicOr(T.S.err, ERR_STAGE | ERR_LOST);
            T.next = next_g;
        }
#ifdef AAP_PHASE_TIMING
        if (threadIdx.x == 0)
            atomicAdd(&g_phase[T.m <= stage_cap ? 10 : 11], (unsigned long long)(clock64() - tb0));
#endif
        __syncthreads();
    }
}

// Close the step: p(t+1) from the integer sums, clear the consumed buffer's
// counters, advance the step.  Every thread clears counter words of the flat
// range over all systems' tiles; the warps of all blocks take one system each
// for the sums (its 64 accumulator slots loaded at once, then cleared); the
// last block to arrive advances the step.
__global__ void k_finish(Sys *sys, int nsys, const int *__restrict__ tile_base, Ctl *ctl)
{
    static_assert(kAccSlots == 64, "two accumulator slots per lane");
    __shared__ int s_last;
    const long long step = ctl->step;
    const int cur = (int)(step & 1);
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x, gs = (long long)gridDim.x * blockDim.x;
    if (nsys == 1) {
        // one system: its counter lines are one array (16-byte aligned, 64
        // bytes a tile), cleared by 16-byte stores through pointers read once
        int4 *c4 = reinterpret_cast<int4 *>(sys[0].cnt[cur]);
        unsigned *sb = sys[0].spill_bits[cur];
        const int nt = tile_base[1];
        const long long n4 = (long long)nt * (kCntStride / 4);
        for (long long i = gt; i < n4; i += gs) c4[i] = make_int4(0, 0, 0, 0);
        for (long long i = gt; i < (nt + 31) / 32; i += gs) sb[i] = 0u;    // the tiles' spill marks
    } else {
        const long long nw = (long long)tile_base[nsys] * kCntStride;
        for (long long i = gt; i < nw; i += gs) {
            const int g = (int)(i / kCntStride);
            const int si = sys_of_tile(tile_base, nsys, g);
            const int t = g - tile_base[si], w = (int)(i % kCntStride);
            sys[si].cnt[cur][(long long)t * kCntStride + w] = 0;
            if (w == 0 && (t & 31) == 0) sys[si].spill_bits[cur][t >> 5] = 0u;    // the tiles' spill marks
        }
    }
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    for (int si = gw; si < nsys; si += nwarps) {
        Sys &S = sys[si];
        unsigned long long *a = S.acc + (size_t)cur * kAccSlots * kAccWords;
        unsigned long long x0[5], x1[5];
#pragma unroll
        for (int w = 0; w < 5; ++w) {
            x0[w] = a[lane * kAccWords + w];
            x1[w] = a[(lane + 32) * kAccWords + w];
        }
#pragma unroll
        for (int w = 0; w < 5; ++w) {
            a[lane * kAccWords + w] = 0;
            a[(lane + 32) * kAccWords + w] = 0;
        }
        long long v[5];
#pragma unroll
        for (int w = 0; w < 5; ++w) v[w] = warp_sum_ll((long long)(x0[w] + x1[w]));   // exact, lane 0 holds it
        if (lane != 0) continue;
        const double n = (double)S.n;
        const double dc = (double)v[0] / kFixStep, ds = (double)v[1] / kFixStep;
        const double dc2 = (double)v[3] / kFixStep, ds2 = (double)v[4] / kFixStep;
        const double phi = n > 0 ? sqrt(dc * dc + ds * ds) / n : 0.0;
        const double q = n > 0 ? sqrt(dc2 * dc2 + ds2 * ds2) / n : 0.0;
        const double nbar = n > 0 ? (double)v[2] / n : 0.0;
        if (S.trace) {
            const long long i1 = step + 1 - S.trace_base, i0 = step - S.trace_base;
            if (i1 >= 0 && i1 < S.trace_cap) S.trace[i1] = phi;
            if (i0 >= 0 && i0 < S.trace_cap) S.trace_nbar[i0] = nbar;
        }
        if (step < S.meas_until) {
            // on-the-fly measurement (Sec. 3.4): state t contributes p(t),
            // q(t) and the mean neighbour number measured on it
            const double p0 = S.last[0], q0 = S.last[1];
            double pk = 1.0, qk = 1.0, nk = 1.0;
            for (int k = 0; k < 4; ++k) {
                pk *= p0;
                qk *= q0;
                nk *= nbar;
                S.stats[k] += pk;
                S.stats[4 + k] += qk;
                S.stats[8 + k] += nk;
            }
            S.stats[12] += 1.0;
        }
        S.last[0] = phi;
        S.last[1] = q;
        S.last[2] = nbar;
        S.last[3] = (double)(step + 1);
        S.spill_cnt[cur] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = (atomicAdd(&ctl->finish_ticket, 1) == (int)gridDim.x - 1);
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        ctl->tile_next = 0;
        ctl->finish_ticket = 0;
        ctl->dense_count = 0;
        ctl->dense_next = 0;
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
        region = S.flat ? 0 : region_of(X >> S.sx, Y >> S.sy, tw, th_);
        rec = make_int4(X, Y, __float_as_int(pt), (int)i);
    }
    warp_insert(S, b, act, dtile, region, rec);
}

// Visit every stored record of buffer b: slots [0, tiles * tile_slots) then
// the spill list.  Returns false for empty slots.
// The lowest index whose position lies outside [0, lx] x [0, ly] (bad[0])
// and whose orientation is not finite (bad[1]); both start at all ones.
__global__ void k_validate_state(const double *x, const double *y, const float *th, long long n, double lx,
                                 double ly, unsigned long long *bad)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (!(x[i] >= 0.0 && x[i] <= lx) || !(y[i] >= 0.0 && y[i] <= ly)) atomicMin(bad, (unsigned long long)i);
        if (!isfinite(th[i])) atomicMin(bad + 1, (unsigned long long)i);
    }
}

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
size_t step_smem_bytes(int stage_cap, int nce_max, int hist_words)
{
    return stage_bytes(stage_cap) + table_bytes(nce_max, hist_words);
}

template <int NT, int MODEL>
static cudaError_t launch_step_t(const LaunchCfg &L, cudaStream_t st, cudaEvent_t *ev)
{
    const size_t smem = step_smem_bytes(L.stage_cap, L.nce_max, L.hist_words);
    cudaError_t e;
    if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
    if (L.pipe) {
        e = launch_step_pipe(L, st);
    } else {
        k_step<NT, MODEL><<<L.grid_step, NT, smem, st>>>(L.sys, L.nsys, L.tile_base, L.ctl, L.stage_cap,
                                                          L.nce_max, L.scratch, L.scratch_per_block,
                                                          L.scratch_cap, L.spill_list_cap);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return e;
    k_finish<<<L.grid_finish, 256, 0, st>>>(L.sys, L.nsys, L.tile_base, L.ctl);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[2], st)) != cudaSuccess) return e;
    return cudaSuccess;
}

template <int MODEL>
static cudaError_t launch_step_m(const LaunchCfg &L, cudaStream_t st, cudaEvent_t *ev)
{
    if (L.pipe) return launch_step_t<512, MODEL>(L, st, ev);     // the pipelined kernel has its own shape
    switch (L.threads) {
    case 256: return launch_step_t<256, MODEL>(L, st, ev);
    case 512: return launch_step_t<512, MODEL>(L, st, ev);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step(const LaunchCfg &L, cudaStream_t st, cudaEvent_t *ev)
{
    if (L.knn > 0) {
        cudaError_t e = launch_mf_step(L, st, ev);
        if (e != cudaSuccess) return e;
        k_finish<<<L.grid_finish, 256, 0, st>>>(L.sys, L.nsys, L.tile_base, L.ctl);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (ev && (e = cudaEventRecord(ev[2], st)) != cudaSuccess) return e;
        return cudaSuccess;
    }
    switch (L.model) {
    case 0: return launch_step_m<0>(L, st, ev);
    case 1: return launch_step_m<1>(L, st, ev);
    case 2: return launch_step_m<2>(L, st, ev);
    default: return cudaErrorInvalidValue;
    }
}

template <int NT, int MODEL>
static cudaError_t config_t(size_t smem, int *bps)
{
    // The limit belongs to the kernel, not to a handle: raise it to the
    // largest size any handle of this process asked for, so that creating a
    // smaller system never breaks the launches of a larger one.
    static std::atomic<int> limit{0};
    int want = (int)smem, prev = limit.load();
    while (want > prev && !limit.compare_exchange_weak(prev, want)) {
    }
    cudaError_t e = cudaFuncSetAttribute(k_step<NT, MODEL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         std::max(want, limit.load()));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_step<NT, MODEL>, NT, smem);
}

cudaError_t configure_step_kernel(int model, int threads, size_t smem_bytes, int *blocks_per_sm)
{
    if (threads == 256) {
        if (model == 0) return config_t<256, 0>(smem_bytes, blocks_per_sm);
        if (model == 1) return config_t<256, 1>(smem_bytes, blocks_per_sm);
        if (model == 2) return config_t<256, 2>(smem_bytes, blocks_per_sm);
    } else if (threads == 512) {
        if (model == 0) return config_t<512, 0>(smem_bytes, blocks_per_sm);
        if (model == 1) return config_t<512, 1>(smem_bytes, blocks_per_sm);
        if (model == 2) return config_t<512, 2>(smem_bytes, blocks_per_sm);
    }
    return cudaErrorInvalidValue;
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

cudaError_t launch_validate(const double *x, const double *y, const float *th, long long n, double lx, double ly,
                            unsigned long long *bad, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(bad, 0xff, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess || n == 0) return e;
    k_validate_state<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, st>>>(x, y, th, n, lx, ly, bad);
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


#ifdef AAP_PHASE_TIMING
cudaError_t read_phase_times(unsigned long long *out16)
{
    return cudaMemcpyFromSymbol(out16, g_phase, sizeof(unsigned long long) * 16);
}
#endif

}  // namespace aapk
