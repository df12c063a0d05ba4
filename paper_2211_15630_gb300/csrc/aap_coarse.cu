// aap_coarse.cu -- coarse-grained fields of a state: density and
// polarisation per bin (the fields the learned surrogate advances), in exact
// 64-bit integer sums so that they are reproducible bit for bit.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "aap_internal.cuh"
#include "aap_kernels.cuh"

namespace aapk {

namespace {

// Bin of the fixed-point coordinate u = cell0 2^s + off (units of the box
// axis; cell0 the first cell of the record's tile, off >= 0 its offset in the
// tile): the definition is the FP64 product (int)(u * (cs / 2^s) * (nb / L))
// clamped to [0, nb).  It is evaluated in FP32 as cell0 * (bins per cell) +
// off * (bins per unit), with no 64-bit integer conversion (those run on
// the FP64 pipe, which is narrow on this GPU), and taken from there unless
// the FP32 value t lies within its error bound of a bin edge, where the FP64
// product decides.  Both terms are >= 0, so the five roundings of at most
// 2^-24 relative each (the two factors, off, the product, the fused sum)
// stay below 4 2^-24 t = 2.4e-7 t; the margin is 3e-7 t + 1e-6.  So the
// result is the FP64 one for every particle, with FP64 work for a few in ten
// thousand.
struct BinAxis {
    double cs_unit, f;          // cs / 2^s, nb / L
    float f_unit, f_cell;       // bins per unit, bins per cell
    int nb, s;
};

// The FP64 definition, out of line: inlined, the compiler predicates these
// FP64 instructions into every particle's path, where they occupy the FP64
// pipe even when the predicate is off.
__device__ __noinline__ int coarse_bin_fp64(long long u, double cs_unit, double f)
{
    return (int)((double)u * cs_unit * f);
}

__device__ __forceinline__ int coarse_bin(int cell0, int off, const BinAxis &a)
{
    const float t = fmaf((float)cell0, a.f_cell, (float)off * a.f_unit);
    const float fl = floorf(t), fr = t - fl, m = fmaf(t, 3e-7f, 1e-6f);
    int i = (int)fl;
    if (off < 0 || fr < m || fr > 1.0f - m) i = coarse_bin_fp64(((long long)cell0 << a.s) + off, a.cs_unit, a.f);
    return min(max(i, 0), a.nb - 1);
}

// cos or sin times 2^32 rounded to a 64-bit integer, equal to __float2ll_rn
// of it, from 32-bit conversions: below 2^31 in magnitude one conversion;
// above, |x| >= 1/2 carries at most 24 significant bits, so x 2^32 is a
// multiple of 2^8 and x 2^24 converts exactly.
__device__ __forceinline__ long long fix32_ll(float x)
{
    const float v = x * 4294967296.0f;
    if (fabsf(v) < 2147483648.0f) return (long long)__float2int_rn(v);
    return (long long)__float2int_rn(x * 16777216.0f) * 256;
}

__device__ __forceinline__ void coarse_add(unsigned long long *acc, long long nb, long long bin, float th)
{
    float sn, cs;
    sincosf(th, &sn, &cs);
    atomicAdd(acc + bin, 1ull);
    atomicAdd(acc + nb + bin, (unsigned long long)fix32_ll(cs));
    atomicAdd(acc + 2 * nb + bin, (unsigned long long)fix32_ll(sn));
}

// Counts and sums of cos theta, sin theta per bin of the state in buffer b,
// in exact 64-bit integers (cos scaled by 2^32), so that the fields are
// reproducible bit for bit.  acc: [3][nbx*nby], zeroed by the caller.  Blocks
// take whole tiles and read only the stored records (the valid slots of the
// nine regions, taken as one index range so that a tile costs one read of
// its counts and the block's threads stay busy across the small edge
// regions), then the spilled records, shared out over the blocks.  The sums
// go straight to acc, one atomic per record and field: merging a warp's
// lanes of one bin first (by match and reductions, or by runs of records per
// thread) was slower, as was a shared-memory window of the tile's bins
// (same-address shared atomics serialise).
template <int NT>
__global__ void __launch_bounds__(NT) k_coarse_tiles(Sys S, int b, BinAxis ax, BinAxis ay, unsigned long long *acc)
{
    const long long nb = (long long)ax.nb * ay.nb;
    __shared__ int s_pre[kRegions + 1];
    for (int tile = blockIdx.x; tile < S.ntiles; tile += gridDim.x) {
        const int tx = tile % S.ntx, ty = tile / S.ntx;
        const int cx0 = S.x0tab[tx], cy0 = S.y0tab[ty];
        const int4 *base = S.rec[b] + (long long)tile * S.tile_slots;
        if (threadIdx.x < 32) {
            // the regions' record counts and their prefix
            const int l = threadIdx.x;
            const int c = l < kRegions ? min(S.cnt[b][tile * kCntStride + l], S.cap[l]) : 0;
            int v = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, v, o);
                if (l >= o) v += t;
            }
            if (l < kRegions) s_pre[l + 1] = v;
            if (l == 0) s_pre[0] = 0;
        }
        __syncthreads();
        const int total = s_pre[kRegions];      // records of the tile; record k is in region r
                                                // for s_pre[r] <= k < s_pre[r + 1]
        for (int k = threadIdx.x; k < total; k += NT) {
            int r = 0;
            while (k >= s_pre[r + 1]) ++r;
            const int4 rec = base[S.off[r] + k - s_pre[r]];
            const int ix = coarse_bin(cx0, rec.x, ax), iy = coarse_bin(cy0, rec.y, ay);
            coarse_add(acc, nb, (long long)iy * ax.nb + ix, __int_as_float(rec.z));
        }
        __syncthreads();
    }
    const int nsp = min(S.spill_cnt[b], S.spill_cap);
    for (int e = blockIdx.x * NT + threadIdx.x; e < nsp; e += gridDim.x * NT) {
        const int4 rec = S.spill_rec[b][e];
        const int tile = S.spill_key[b][e] / kCntStride;
        const int tx = tile % S.ntx, ty = tile / S.ntx;
        const int ix = coarse_bin(S.x0tab[tx], rec.x, ax), iy = coarse_bin(S.y0tab[ty], rec.y, ay);
        coarse_add(acc, nb, (long long)iy * ax.nb + ix, __int_as_float(rec.z));
    }
}

// Fields per unit area: density, polarisation x, polarisation y (planes of
// nbx*nby floats, row-major with x fastest).
__global__ void k_coarse_finish(const unsigned long long *acc, int nbx, int nby, double inv_area, float *out)
{
    const long long nb = (long long)nbx * nby;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb;
         i += (long long)gridDim.x * blockDim.x) {
        out[i] = (float)((double)acc[i] * inv_area);
        out[nb + i] = (float)((double)(long long)acc[nb + i] / kFix * inv_area);
        out[2 * nb + i] = (float)((double)(long long)acc[2 * nb + i] / kFix * inv_area);
    }
}

}  // namespace

cudaError_t launch_coarse(const Sys &S, int b, int nbx, int nby, unsigned long long *acc, float *out,
                          cudaStream_t st)
{
    const long long nb = (long long)nbx * nby;
    cudaError_t e = cudaMemsetAsync(acc, 0, (size_t)nb * 3 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    BinAxis ax, ay;
    ax.cs_unit = S.csx_d / (double)(1ll << S.sx);
    ax.f = (double)nbx / S.lx;
    ax.f_unit = (float)(ax.cs_unit * ax.f);
    ax.f_cell = (float)(S.csx_d * ax.f);
    ax.nb = nbx;
    ax.s = S.sx;
    ay.cs_unit = S.csy_d / (double)(1ll << S.sy);
    ay.f = (double)nby / S.ly;
    ay.f_unit = (float)(ay.cs_unit * ay.f);
    ay.f_cell = (float)(S.csy_d * ay.f);
    ay.nb = nby;
    ay.s = S.sy;
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, std::min(S.ntiles, 8 * nsm));
    k_coarse_tiles<256><<<grid, 256, 0, st>>>(S, b, ax, ay, acc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const double inv_area = (double)nbx * nby / (S.lx * S.ly);
    k_coarse_finish<<<(unsigned)std::min<long long>((nb + 255) / 256, 4096), 256, 0, st>>>(acc, nbx, nby, inv_area, out);
    return cudaGetLastError();
}

}  // namespace aapk
