// aap_surrogate.cu -- coarse-grained convolutional surrogate of the particle
// fields (density and polarisation, from aap_coarse_grain).
//
// Network: F(t + 10) = F(t) + Net(F(t), eta), four 3x3 convolutions with
// circular padding, 4 (3 fields + the noise strength) -> 32 -> 32 -> 32 -> 3
// channels, ReLU between layers.  Activations are BF16 NHWC, weights BF16,
// every contraction accumulates in FP32; master weights and Adam moments are
// FP32.  Channel counts are padded for the tensor-core tiles: the first
// layer's 4 inputs to 16, the last layer's 3 outputs to 8 (the padded weights
// start at zero and receive zero gradient, so they stay zero).
//
// Kernels:
//   k_conv_ws<CIN, COUT, MODE> implicit-GEMM convolution on the tcgen05
//                             tensor cores (BF16 x BF16 -> FP32 accumulator in
//                             TMEM, M = 128 pixels, N = COUT), warp-specialised
//                             (halo copies, MMA issue and epilogue overlap over
//                             a block's tiles): forward with bias + ReLU,
//                             forward with the residual update, or the data
//                             gradient (flipped, transposed weights) masked by
//                             the ReLU of the layer input
//   k_conv_dw_tc<CIN, COUT>   weight and bias gradients on the tcgen05
//                             tensor cores (shifted input rows and the
//                             transposed dy as K-major operands, pixels along
//                             K, the three row shifts stacked along M, one TMEM
//                             accumulator per column shift for all of a block's
//                             tiles), one partial per block, reduced in a fixed
//                             order (deterministic)
//   k_adam                    Adam step on the FP32 master weights
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/aap.h"
#include "../../include/aap_surrogate.h"

namespace aaps {

typedef __nv_bfloat16 bf16;

// tcgen05 convolution tile: 16 rows x 8 columns = 128 output pixels, the M of
// one tensor-core MMA (cta_group::1, M = 128), one pixel per TMEM lane.
constexpr int kTH = 16, kTW = 8;
constexpr int kHaloPix = (kTH + 2) * (kTW + 2);     // 180 input pixels with the 1-pixel ring
constexpr int kPlane = kHaloPix * 16;               // bytes of one 8-channel plane of the halo tile

__device__ int g_sur_err;                           // sticky: 1 = a tensor-core wait gave up

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor, no swizzle, K-major core matrices of
// 8 rows x 16 bytes: start address, LBO = byte step between core matrices
// along K, SBO = byte step between core matrices along M (or N); bit 46 is
// the descriptor version of this tensor-core generation.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= 1ull << 46;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, BF16 A
// and B, both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                 ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// 8, 16 or 32 FP32 columns of this warp's 32 TMEM lanes (one row each).
template <int NC>
__device__ __forceinline__ void tmem_load(uint32_t taddr, uint32_t (&r)[NC])
{
    if constexpr (NC == 8) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                       "=r"(r[7])
                     : "r"(taddr));
    } else if constexpr (NC == 16) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                     "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                       "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                       "=r"(r[14]), "=r"(r[15])
                     : "r"(taddr));
    } else {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                     "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                     "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                       "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                       "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                       "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                       "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                     : "r"(taddr));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;");
}

enum { MODE_RELU = 0, MODE_RESID = 1, MODE_MASK = 2, MODE_LINEAR = 3 };

constexpr int kConvThreads = 256;

// out[b, y, x, co] = sum_{tap, ci} w[tap][co][ci] * in[b, (y+dy-1) mod H, (x+dx-1) mod W, ci]
// (tap = 3 dy + dx), then per MODE:
//   MODE_RELU   + bias, ReLU, BF16 NHWC out
//   MODE_LINEAR + bias, BF16 NHWC out
//   MODE_RESID  + bias, FP32: resid_out = resid_in + value (NHWC, 8 channels)
//   MODE_MASK   value where mask > 0 else 0, BF16 NHWC out (data gradient)
// An implicit GEMM on the 5th-generation tensor cores.  Each 16 x 8 pixel
// tile is one MMA row block (M = 128) for all COUT channels (N = COUT, at
// least 16) with K = 9 taps x CIN in steps of 16.  The input tile and its
// ring are staged as 8-channel planes of 16-byte pixels, so the A operand of
// every tap is a descriptor view of the same planes (start moved by the tap
// offset; core matrices 8 pixels of a row, LBO one plane, SBO one halo row).
// The weights are staged once per block, per (tap, K step) as N x 16 core
// matrices.  k_conv_ws below runs the tiles of a block as a pipeline.
// The halo of tile t staged by nthr threads (thread index i0) of the calling
// role, asynchronously (cp.async, 16 bytes each, circular padding).
template <int CIN>
__device__ __forceinline__ void stage_halo_part(unsigned char *s_in, const bf16 *__restrict__ in, int H, int W, int t,
                                                int i0, int nthr)
{
    constexpr int G = CIN / 8;
    const int tx = W / kTW, ty = H / kTH;
    const int b = t / (tx * ty), r = t - b * (tx * ty);
    const int y0 = (r / tx) * kTH, x0 = (r % tx) * kTW;
    for (int i = i0; i < kHaloPix * G; i += nthr) {
        const int hp = i / G, g = i - hp * G;
        const int hy = hp / (kTW + 2), hx = hp - hy * (kTW + 2);
        int gy = y0 + hy - 1, gx = x0 + hx - 1;
        gy += (gy < 0) ? H : 0;
        gy -= (gy >= H) ? H : 0;
        gx += (gx < 0) ? W : 0;
        gx -= (gx >= W) ? W : 0;
        const uint4 *src = reinterpret_cast<const uint4 *>(in + (((size_t)b * H + gy) * W + gx) * CIN) + g;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(s_in + g * kPlane + hp * 16)),
                     "l"(src)
                     : "memory");
    }
}

__device__ __forceinline__ void bar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ void bar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Wait for the completion of the phase of the given parity, bounded by about
// two seconds of SM clock (the hint lets the hardware suspend the warp while
// it waits); false when the bound ran out (the sticky error flag is set).
constexpr long long kConvWaitCycles = 4000000000ll;
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done) : "r"(smem_addr(bar)), "r"(parity), "r"(20000u) : "memory");
        if (done) return true;
        if (clock64() - t0 > kConvWaitCycles) {
            atomicOr(&g_sur_err, 1);
            return false;
        }
    }
}

constexpr int kConvStages = 4;      // halo buffers
constexpr int kConvAccs = 4;        // TMEM accumulators of 32 columns
constexpr int kConvProducers = 96;  // threads of warps 1-3

template <int CIN, int COUT>
__host__ __device__ constexpr size_t conv_ws_smem()
{
    constexpr int NP = COUT < 16 ? 16 : COUT;
    return ((size_t)kConvStages * (CIN / 8) * kPlane + 1023) / 1024 * 1024 + (size_t)9 * (CIN / 16) * ((NP / 8) * 2 * 128) +
           1024;
}

// The same convolution as a warp-specialised pipeline over the block's tiles
// (t = blockIdx.x + i gridDim.x).  Warp 0, one thread: issues the 9 x CIN/16
// MMAs of tile i from halo buffer i % 4 into accumulator i % 4 and commits
// them to that buffer's "empty" and that accumulator's "full" mbarrier.
// Warps 1-3: stage the halo of tile i into buffer i % 4 with cp.async as soon
// as the buffer's previous MMAs are done (up to four tiles ahead); once a
// thread's copies of a tile have landed it fences them for the tensor core and
// arrives on the buffer's "full" mbarrier.  Warps 4-7 (TMEM lane quarters 0-3,
// one output pixel per thread): read the accumulator, free it, and write the
// tile's outputs (bias, ReLU, mask or residual per MODE).  Every wait is
// bounded; a role whose wait runs out stops, and the block drains its copies
// and MMAs before it frees TMEM.
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(kConvThreads) k_conv_ws(const bf16 *__restrict__ in, int H, int W, int ntiles,
                                                          const bf16 *__restrict__ wt, const float *__restrict__ bias,
                                                          bf16 *__restrict__ out, const bf16 *__restrict__ mask,
                                                          const float *__restrict__ resid_in,
                                                          float *__restrict__ resid_out)
{
    constexpr int NP = COUT < 16 ? 16 : COUT;       // MMA N
    constexpr int G = CIN / 8;                      // 8-channel groups of the input
    constexpr int KC = CIN / 16;                    // K steps per tap
    constexpr int WBLK = (NP / 8) * 2 * 128;        // bytes of one (tap, K step) weight block
    constexpr int NS = kConvStages, NA = kConvAccs;
    extern __shared__ unsigned char s_dyn[];
    unsigned char *base = (unsigned char *)(((uintptr_t)s_dyn + 1023) & ~(uintptr_t)1023);
    unsigned char *s_in = base;                     // [NS][G * kPlane]
    unsigned char *s_w = base + ((size_t)NS * G * kPlane + 1023) / 1024 * 1024;
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t full[NS], empty[NS], afull[NA], aempty[NA];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < 9 * NP * G; i += kConvThreads) {
        const int tap = i / (NP * G), rem = i - tap * (NP * G), co = rem / G, g = rem - co * G;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (co < COUT) v = *(reinterpret_cast<const uint4 *>(wt + ((size_t)tap * COUT + co) * CIN) + g);
        *reinterpret_cast<uint4 *>(s_w + (tap * KC + (g >> 1)) * WBLK + ((co >> 3) * 2 + (g & 1)) * 128 +
                                   (co & 7) * 16) = v;
    }
    if (tid == 0) {
        for (int k = 0; k < NS; ++k) {
            bar_init(&full[k], kConvProducers);
            bar_init(&empty[k], 1);
        }
        for (int k = 0; k < NA; ++k) {
            bar_init(&afull[k], 1);
            bar_init(&aempty[k], 128);
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(32 * NA));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;");   // the staged weights, for the tensor core
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;
    const int tx = W / kTW, ty = H / kTH;
    if (warp == 0) {
        // ------------------------------------------------------------ MMA --
        if (lane == 0) {
            constexpr uint32_t idesc = umma_idesc_bf16(128, NP);
            const uint32_t w0 = smem_addr(s_w);
            int i = 0;
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
                const int st = i % NS, ac = i % NA;
                if (!bar_wait(&full[st], (uint32_t)(i / NS) & 1u)) break;
                if (i >= NA && !bar_wait(&aempty[ac], (uint32_t)((i / NA) & 1) ^ 1u)) break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t a0 = smem_addr(s_in + (size_t)st * G * kPlane);
                uint32_t acc = 0;
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int dy = tap / 3, dx = tap - dy * 3;
#pragma unroll
                    for (int kc = 0; kc < KC; ++kc) {
                        const uint64_t ad =
                            umma_desc(a0 + 2 * kc * kPlane + (dy * (kTW + 2) + dx) * 16, kPlane, (kTW + 2) * 16);
                        const uint64_t bd = umma_desc(w0 + (tap * KC + kc) * WBLK, 128, 256);
                        umma_bf16(tmem + ac * 32, ad, bd, idesc, acc);
                        acc = 1;
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(smem_addr(&empty[st])));
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(smem_addr(&afull[ac])));
            }
            // MMAs still running (only when a wait ran out): the last commit
            // covers every earlier MMA of this thread
            if (i > 0 && blockIdx.x + (long long)i * gridDim.x < ntiles) {
                const int last = i - 1;
                if (!bar_wait(&afull[last % NA], (uint32_t)(last / NA) & 1u))
                    bar_wait(&afull[last % NA], (uint32_t)(last / NA) & 1u);
            }
        }
        __syncwarp();
    } else if (warp < 4) {
        // -------------------------------------------------------- producers --
        const int pt = tid - 32;
        int i = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
            const int st = i % NS;
            if (i >= NS && !bar_wait(&empty[st], (uint32_t)((i / NS) & 1) ^ 1u)) {
                ok = false;
                break;
            }
            stage_halo_part<CIN>(s_in + (size_t)st * G * kPlane, in, H, W, t, pt, kConvProducers);
            asm volatile("cp.async.commit_group;" ::: "memory");
            if (i >= 1) {
                // the previous tile's copies of this thread have landed
                asm volatile("cp.async.wait_group 1;" ::: "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                bar_arrive(&full[(i - 1) % NS]);
            }
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        if (ok && i >= 1) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            bar_arrive(&full[(i - 1) % NS]);
        }
    } else {
        // --------------------------------------------------------- epilogue --
        const int q = warp & 3;                     // TMEM lane quarter of this warp
        const int m = q * 32 + lane;                // output pixel of the tile
        int i = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
            const int ac = i % NA;
            // warp-uniform: the TMEM load below is a whole-warp instruction
            if (!__all_sync(0xffffffffu, bar_wait(&afull[ac], (uint32_t)(i / NA) & 1u))) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            uint32_t r[NP];
            tmem_load<NP>(tmem + ac * 32 + ((uint32_t)(q * 32) << 16), r);
            asm volatile("tcgen05.fence::before_thread_sync;");
            bar_arrive(&aempty[ac]);
            const int b = t / (tx * ty), rr = t - b * (tx * ty);
            const int y = (rr / tx) * kTH + m / kTW, x = (rr % tx) * kTW + m % kTW;
            const size_t pix = ((size_t)b * H + y) * W + x;
            if (MODE == MODE_RESID) {
#pragma unroll
                for (int co = 0; co < COUT; ++co)
                    resid_out[pix * 8 + co] = resid_in[pix * 8 + co] + (__uint_as_float(r[co]) + bias[co]);
            } else {
                // COUT bf16 outputs of this pixel, written 16 bytes at a time
#pragma unroll
                for (int c0 = 0; c0 < COUT; c0 += 8) {
                    uint32_t pk[4];
#pragma unroll
                    for (int j = 0; j < 8; j += 2) {
                        const int co = c0 + j;
                        float v0 = __uint_as_float(r[co]), v1 = __uint_as_float(r[co + 1]);
                        if (MODE != MODE_MASK) {
                            v0 += bias[co];
                            v1 += bias[co + 1];
                        }
                        if (MODE == MODE_RELU) {
                            v0 = fmaxf(v0, 0.f);
                            v1 = fmaxf(v1, 0.f);
                        }
                        if (MODE == MODE_MASK) {
                            const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162 *>(mask + pix * COUT + co);
                            if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
                            if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
                        }
                        const __nv_bfloat162 h2 = __floats2bfloat162_rn(v0, v1);
                        pk[j / 2] = *reinterpret_cast<const uint32_t *>(&h2);
                    }
                    *reinterpret_cast<uint4 *>(out + pix * COUT + c0) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32 * NA));
}

// Weight / bias gradient on the tensor cores.  For every column shift dx the
// block accumulates D_dx[(dy, ci)][co] = sum_p x[p + (dy, dx) - 1][ci] dy[p][co]
// over all its tiles in TMEM (accumulator dx at columns 32 dx): one MMA per dx
// and K step of 16 pixels (two tile rows), M = 128 rows (dy, ci) -- the three
// row shifts stacked, since the rows of shift dy + 1 are one halo row further
// on (rows past the third shift are padding the tensor core requires and are
// never read back) -- N = COUT (at least 16), both operands K-major (pixels
// along K):
//   A = xT[dx][hy][ci][8 px]    halo row hy seen from column dx
//                               (LBO: one halo row, SBO: 8 channels = 128 B)
//   B = dyT[py][co][8 px]       (LBO: one tile row, SBO: 128 B)
// Warps 1-7 fetch a tile's halo and dy into one of two raw staging areas
// (cp.async, one tile ahead), then write the transposed operands into one of
// two stages with ldmatrix.trans / stmatrix (8 x 8 blocks of 16-bit values)
// and add up db in FP32 (each thread always for the same output channel, in
// a fixed order); warp 0, one thread, issues the 24 MMAs of a stage and
// commits them to its "empty" mbarrier; after the last tile warps 4-7 (TMEM
// lane quarters 0-3 = rows (dy, ci)) write the block's partial dw and the
// threads' db partials are summed in a fixed order.
// part[block][COUT * 9 * CIN + COUT].
constexpr int kDwThreads = 256;
constexpr int kDwT = kDwThreads - 32;          // transposing threads (warps 1-7)

template <int CIN, int COUT>
__host__ __device__ constexpr int dw_coutp() { return COUT < 8 ? 8 : COUT; }

template <int CIN, int COUT>
__host__ __device__ constexpr size_t dw_xt_bytes() { return (size_t)3 * (kTH + 2) * CIN * 16; }

template <int CIN, int COUT>
__host__ __device__ constexpr size_t dw_dyt_bytes()
{
    // 16 tile rows of COUTP channel rows, plus what the 128 MMA rows of the
    // last K step read beyond them
    return ((size_t)(kTH - 1) * dw_coutp<CIN, COUT>() * 16 + 2048 + 1023) / 1024 * 1024;
}

template <int CIN, int COUT>
__host__ __device__ constexpr size_t dw_tc_smem()
{
    return 2 * ((size_t)kHaloPix * CIN * 2 + (size_t)kTH * kTW * COUT * 2) + 1024 +
           2 * (dw_xt_bytes<CIN, COUT>() + dw_dyt_bytes<CIN, COUT>()) + 1024;
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(kDwThreads, 1) k_conv_dw_tc(const bf16 *__restrict__ x, const bf16 *__restrict__ dy,
                                                             int dy_stride, int H, int W, int ntiles,
                                                             float *__restrict__ part)
{
    constexpr int COUTP = dw_coutp<CIN, COUT>();
    constexpr size_t XT = dw_xt_bytes<CIN, COUT>(), DYT = dw_dyt_bytes<CIN, COUT>();
    extern __shared__ unsigned char s_dyn[];
    unsigned char *base = (unsigned char *)(((uintptr_t)s_dyn + 1023) & ~(uintptr_t)1023);
    unsigned char *stage0 = base;                                    // [2][XT + DYT]
    bf16 *raw_x = reinterpret_cast<bf16 *>(base + 2 * (XT + DYT));   // [2][18 * 10][CIN]
    bf16 *raw_dy = raw_x + 2 * kHaloPix * CIN;                       // [2][128][COUT]
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t tfull[2], tempty[2], done;
    __shared__ float s_db[kDwT];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int k = 0; k < 2; ++k) {
            bar_init(&tfull[k], kDwT);
            bar_init(&tempty[k], 1);
        }
        bar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(128));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;
    const int tx = W / kTW, ty = H / kTH;
    bool ok = true;
    if (warp == 0) {
        // ------------------------------------------------------------ MMA --
        if (lane == 0) {
            constexpr int NB = COUT < 16 ? 16 : COUT;     // MMA N (output channels, padded)
            constexpr uint32_t idesc = umma_idesc_bf16(128, NB);
            int i = 0;
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
                const int st = i & 1;
                if (!bar_wait(&tfull[st], (uint32_t)(i >> 1) & 1u)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t xt = smem_addr(stage0 + st * (XT + DYT)), dyt = xt + (uint32_t)XT;
#pragma unroll
                for (int ks = 0; ks < kTH / 2; ++ks) {
                    const uint64_t bd = umma_desc(dyt + 2 * ks * COUTP * 16, COUTP * 16, 128);
#pragma unroll
                    for (int ddx = 0; ddx < 3; ++ddx) {
                        // rows (dy, ci): the halo rows 2 ks + dy of column
                        // shift ddx, one halo row (CIN x 16 bytes) per dy
                        const uint64_t ad = umma_desc(xt + (ddx * (kTH + 2) + 2 * ks) * CIN * 16, CIN * 16, 128);
                        umma_bf16(tmem + ddx * 32, ad, bd, idesc, (i > 0 || ks > 0) ? 1u : 0u);
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(smem_addr(&tempty[st])));
            }
            // every MMA of this block (or, after a wait ran out, those issued)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_addr(&done)));
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------- transposers --
        const int pt = tid - 32;
        float db = 0.f;                              // for output channel pt % COUT
        // the raw halo and dy of tile t into raw buffer rb, asynchronously
        const auto fetch = [&](int t, int rb) {
            const int b = t / (tx * ty), rr = t - b * (tx * ty);
            const int y0 = (rr / tx) * kTH, x0 = (rr % tx) * kTW;
            bf16 *rx = raw_x + rb * (kHaloPix * CIN), *rd = raw_dy + rb * (kTH * kTW * COUT);
            for (int k = pt; k < kHaloPix * (CIN / 8); k += kDwT) {
                const int hp = k / (CIN / 8), g = k - hp * (CIN / 8);
                const int hy = hp / (kTW + 2), hx = hp - hy * (kTW + 2);
                int gy = y0 + hy - 1, gx = x0 + hx - 1;
                gy += (gy < 0) ? H : 0;
                gy -= (gy >= H) ? H : 0;
                gx += (gx < 0) ? W : 0;
                gx -= (gx >= W) ? W : 0;
                const uint4 *src = reinterpret_cast<const uint4 *>(x + (((size_t)b * H + gy) * W + gx) * CIN) + g;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(rx + hp * CIN + g * 8)),
                             "l"(src)
                             : "memory");
            }
            for (int k = pt; k < kTH * kTW * (COUT / 8); k += kDwT) {
                const int px = k / (COUT / 8), g = k - px * (COUT / 8);
                const int yy = y0 + px / kTW, xx = x0 + px % kTW;
                const uint4 *src = reinterpret_cast<const uint4 *>(dy + (((size_t)b * H + yy) * W + xx) * dy_stride) + g;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(rd + px * COUT + g * 8)),
                             "l"(src)
                             : "memory");
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        if ((int)blockIdx.x < ntiles) fetch(blockIdx.x, 0);
        int i = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
            const int st = i & 1, rb = i & 1;
            // the next tile's raw data in flight while this one is transposed
            const bool more = t + (int)gridDim.x < ntiles;
            if (more) {
                fetch(t + gridDim.x, rb ^ 1);
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
            // the stage must be free (its previous tile's MMAs are done); the
            // outcome is made the same for every transposing thread, and the
            // barrier also completes every thread's copies of this tile
            const bool free_ok = i < 2 || bar_wait(&tempty[st], (uint32_t)((i >> 1) - 1) & 1u);
            int all_ok;
            asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
                         "bar.red.and.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
                         : "=r"(all_ok) : "r"((int)free_ok), "r"(kDwT) : "memory");
            if (!all_ok) {
                ok = false;
                break;
            }
            const bf16 *rx = raw_x + rb * (kHaloPix * CIN), *rd = raw_dy + rb * (kTH * kTW * COUT);
            unsigned char *xt = stage0 + st * (XT + DYT), *dyt = xt + XT;
            // The transposes are 8 x 8 blocks of 16-bit values: ldmatrix.trans
            // reads 8 rows of 16 bytes (8 pixels x 8 channels) and stmatrix
            // writes them back as 8 rows of 8 pixels (one per channel); one
            // warp instruction each moves four blocks.  Lane l addresses row
            // l % 8 of block l / 8.
            const int tw8 = pt >> 5, rr8 = lane & 7, mm = lane >> 3;
            // xT[dx][hy][ci][j] = halo[hy][dx + j][ci]: blocks (dx, hy, g)
            constexpr int G = CIN / 8;
            for (int item = tw8; item < 3 * (kTH + 2) * G / 4; item += kDwT / 32) {
                const int mi = 4 * item + mm, g = mi % G, pr = mi / G, hy = pr % (kTH + 2), dxx = pr / (kTH + 2);
                uint32_t v[4];
                asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                             : "r"(smem_addr(rx + (hy * (kTW + 2) + dxx + rr8) * CIN + 8 * g)));
                asm volatile("stmatrix.sync.aligned.m8n8.x4.shared.b16 [%0], {%1,%2,%3,%4};"
                             ::"r"(smem_addr(xt + ((size_t)(dxx * (kTH + 2) + hy) * CIN + 8 * g + rr8) * 16)),
                               "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
                             : "memory");
            }
            // dyT[py][co][j] = dy[py][j][co]: blocks (py, q)
            constexpr int Q = COUT / 8;
            for (int item = tw8; item < kTH * Q / 4; item += kDwT / 32) {
                const int mi = 4 * item + mm, q = mi % Q, py = mi / Q;
                uint32_t v[4];
                asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                             : "r"(smem_addr(rd + (py * kTW + rr8) * COUT + 8 * q)));
                asm volatile("stmatrix.sync.aligned.m8n8.x4.shared.b16 [%0], {%1,%2,%3,%4};"
                             ::"r"(smem_addr(dyt + ((size_t)py * COUTP + 8 * q + rr8) * 16)),
                               "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
                             : "memory");
            }
            // db of this thread's output channel (pt % COUT), pixels in order
            {
                const unsigned short *src = reinterpret_cast<const unsigned short *>(rd);
                for (int k = pt; k < kTH * kTW * COUT; k += kDwT) db += __uint_as_float((uint32_t)src[k] << 16);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // for the tensor core
            bar_arrive(&tfull[st]);
            asm volatile("bar.sync 1, %0;" ::"r"(kDwT) : "memory");       // raw buffer rb read by all
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        s_db[pt] = db;
    }
    __syncthreads();
    // all MMAs issued by this block are complete before TMEM is read or freed
    const bool fin = __syncthreads_and(bar_wait(&done, 0u)) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    float *pb = part + (size_t)blockIdx.x * (COUT * 9 * CIN + COUT);
    if (fin && warp >= 4) {
        // TMEM lane quarter q = warp % 4 holds rows 32 q .. 32 q + 31 = (dy, ci)
        const int m = (warp & 3) * 32 + lane, ddy = m / CIN, ci = m % CIN;
#pragma unroll 1
        for (int ddx = 0; ddx < 3; ++ddx) {
            uint32_t r[32];
            tmem_load<32>(tmem + ddx * 32 + ((uint32_t)((warp & 3) * 32) << 16), r);
            if (ddy < 3)
                for (int co = 0; co < COUT; ++co)
                    pb[((size_t)co * 9 + 3 * ddy + ddx) * CIN + ci] = __uint_as_float(r[co]);
        }
    }
    if (tid < COUT) {
        float sdb = 0.f;
        for (int k = tid; k < kDwT; k += COUT) sdb += s_db[k];
        pb[COUT * 9 * CIN + tid] = sdb;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
    (void)ok;
}

// out[i] = sum_k part[k][i] in a fixed order (deterministic): a block takes
// 32 consecutive i; its eight warps sum eight consecutive ranges of k, and
// the eight partial sums are added in warp order.
__global__ void __launch_bounds__(256) k_reduce_parts(const float *__restrict__ part, int nparts, int len,
                                                      float *__restrict__ w_out, int wlen, float *__restrict__ b_out)
{
    __shared__ float s_sum[8][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    const int per = (nparts + 7) / 8, k0 = min(w * per, nparts), k1 = min(k0 + per, nparts);
    float acc = 0.f;
    if (i < len)
        for (int k = k0; k < k1; ++k) acc += part[(size_t)k * len + i];
    s_sum[w][lane] = acc;
    __syncthreads();
    if (w == 0 && i < len) {
        float t = 0.f;
#pragma unroll
        for (int v = 0; v < 8; ++v) t += s_sum[v][lane];
        if (i < wlen) w_out[i] = t; else b_out[i - wlen] = t;
    }
}

// Fields in (FP32 planes [B][3][H][W]) -> normalised residual state (FP32 NHWC 8)
// and the BF16 network input (NHWC 16: 3 fields, the noise strength, zeros).
// One pixel of a BF16 NHWC 16 tensor: channels 0-3 = (a, b, c, d), the rest
// zero, written as two 16-byte stores.
__device__ __forceinline__ void store_input_pixel(bf16 *px, float a, float b, float c, float d)
{
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(a, b), h1 = __floats2bfloat162_rn(c, d);
    uint4 *o = reinterpret_cast<uint4 *>(px);
    o[0] = make_uint4(*reinterpret_cast<const uint32_t *>(&h0), *reinterpret_cast<const uint32_t *>(&h1), 0u, 0u);
    o[1] = make_uint4(0u, 0u, 0u, 0u);
}

__global__ void k_fields_in(const float *__restrict__ f, const float *__restrict__ eta, int B, int H, int W,
                            float rho0, float eta_c, float eta_s, float *__restrict__ state, bf16 *__restrict__ x0)
{
    const long long n = (long long)B * H * W;
    const long long plane = (long long)H * W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / plane, p = i - b * plane;
        const float u0 = f[(b * 3 + 0) * plane + p] / rho0 - 1.f;
        const float u1 = f[(b * 3 + 1) * plane + p] / rho0;
        const float u2 = f[(b * 3 + 2) * plane + p] / rho0;
        float4 *s = reinterpret_cast<float4 *>(state + i * 8);
        s[0] = make_float4(u0, u1, u2, 0.f);
        s[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        const float e = (eta[b] - eta_c) / eta_s;
        store_input_pixel(x0 + i * 16, u0, u1, u2, e);
    }
}

// Residual state -> the next network input (after one application).
__global__ void k_state_to_input(const float *__restrict__ state, const float *__restrict__ eta, int B, int H,
                                 int W, float eta_c, float eta_s, bf16 *__restrict__ x0)
{
    const long long n = (long long)B * H * W;
    const long long plane = (long long)H * W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / plane;
        const float4 u = *reinterpret_cast<const float4 *>(state + i * 8);
        const float e = (eta[b] - eta_c) / eta_s;
        store_input_pixel(x0 + i * 16, u.x, u.y, u.z, e);
    }
}

// Normalised state -> fields (FP32 planes).
__global__ void k_fields_out(const float *__restrict__ state, int B, int H, int W, float rho0, float *__restrict__ f)
{
    const long long n = (long long)B * H * W;
    const long long plane = (long long)H * W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / plane, p = i - b * plane;
        const float *s = state + i * 8;
        f[(b * 3 + 0) * plane + p] = rho0 * (s[0] + 1.f);
        f[(b * 3 + 1) * plane + p] = rho0 * s[1];
        f[(b * 3 + 2) * plane + p] = rho0 * s[2];
    }
}

// Mean squared error over the 3 field channels of pred vs target (both
// normalised FP32 NHWC 8), per-block partial sums; dout = d loss / d pred in
// BF16 NHWC 16 (channels >= 3 zero), minus the per-sample means dmean of the
// conserved channels when a projection is on (plane = pixels per sample).
__global__ void k_mse(const float *__restrict__ pred, const float *__restrict__ target, long long npix,
                      float scale, float *__restrict__ part, bf16 *__restrict__ dout, const float *__restrict__ dmean,
                      int plane)
{
    __shared__ float red[256];
    float s = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npix; i += (long long)gridDim.x * blockDim.x) {
        const float4 u = *reinterpret_cast<const float4 *>(pred + i * 8);
        const float4 v = *reinterpret_cast<const float4 *>(target + i * 8);
        float d[3] = {u.x - v.x, u.y - v.y, u.z - v.z};
        for (int c = 0; c < 3; ++c) s += d[c] * d[c];
        if (dmean) {
            const long long b = i / plane;
            for (int c = 0; c < 3; ++c) d[c] -= dmean[b * 3 + c];     // through the projection P
        }
        store_input_pixel(dout + i * 16, 2.f * scale * d[0], 2.f * scale * d[1], 2.f * scale * d[2], 0.f);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Channels whose per-sample grid mean one application keeps (conserve bits:
// 1 the density, 2 both polarisation channels).
__host__ __device__ inline bool conserved(int conserve, int c) { return c == 0 ? (conserve & 1) : (conserve & 2); }

// Conservation projection in two passes over chunks of kCenterChunk pixels
// of a sample (NHWC 8 FP32, channels 0..2 read as one float4 per pixel):
// k_center_part writes each chunk's sums of a - b per channel (fixed order,
// so the result is deterministic); the means follow from a sample's chunk
// sums in chunk order.
constexpr int kCenterChunk = 2048;

__global__ void __launch_bounds__(256) k_center_part(const float *__restrict__ a, const float *__restrict__ b,
                                                     int npix, int nchunk, float *__restrict__ part)
{
    __shared__ float red[3][256];
    const int smp = blockIdx.x / nchunk, ch = blockIdx.x % nchunk;
    const long long base = (long long)smp * npix;
    const int p0 = ch * kCenterChunk, p1 = min(npix, p0 + kCenterChunk);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int p = p0 + threadIdx.x; p < p1; p += 256) {
        const float4 u = *reinterpret_cast<const float4 *>(a + (base + p) * 8);
        const float4 v = *reinterpret_cast<const float4 *>(b + (base + p) * 8);
        s0 += u.x - v.x;
        s1 += u.y - v.y;
        s2 += u.z - v.z;
    }
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    red[2][threadIdx.x] = s2;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 3) part[(long long)blockIdx.x * 4 + threadIdx.x] = red[threadIdx.x][0];
}

// Grid mean of channel c of sample smp from its chunk sums.
__device__ __forceinline__ float chunk_mean(const float *__restrict__ part, int smp, int nchunk, int c, int npix)
{
    float t = 0.f;
    for (int k = 0; k < nchunk; ++k) t += part[((long long)smp * nchunk + k) * 4 + c];
    return t / (float)npix;
}

// Remove the mean of out - in from the conserved channels of out (one block
// per chunk of a sample).
__global__ void __launch_bounds__(256) k_center_apply(float *__restrict__ out, const float *__restrict__ part,
                                                      int npix, int nchunk, int conserve)
{
    __shared__ float mean[3];
    const int smp = blockIdx.x / nchunk, ch = blockIdx.x % nchunk;
    if (threadIdx.x < 3)
        mean[threadIdx.x] = conserved(conserve, threadIdx.x) ? chunk_mean(part, smp, nchunk, threadIdx.x, npix) : 0.f;
    __syncthreads();
    const long long base = (long long)smp * npix;
    const int p0 = ch * kCenterChunk, p1 = min(npix, p0 + kCenterChunk);
    for (int p = p0 + threadIdx.x; p < p1; p += 256) {
        float4 *o = reinterpret_cast<float4 *>(out + (base + p) * 8);
        float4 u = *o;
        u.x -= mean[0];
        u.y -= mean[1];
        u.z -= mean[2];
        *o = u;
    }
}

// dmean[smp * 3 + c] = grid mean of pred - target for the conserved channels
// (0 otherwise), from the chunk sums: the loss gradient minus it is the
// gradient through the projection.
__global__ void k_dmean(const float *__restrict__ part, int B, int npix, int nchunk, int conserve,
                        float *__restrict__ dmean)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * 3) return;
    const int smp = i / 3, c = i % 3;
    dmean[i] = conserved(conserve, c) ? chunk_mean(part, smp, nchunk, c, npix) : 0.f;
}

// Adam (Kingma & Ba) on the FP32 master parameters.
__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Master weights [co][tap][ci] -> BF16 forward layout [tap][co][ci] and the
// data-gradient layout [tap'][ci][cob] with tap' = 8 - tap the flipped tap and
// cob >= cout output channels (zero beyond cout; the buffer is cleared first).
__global__ void k_pack(const float *__restrict__ w, int cout, int cin, bf16 *__restrict__ wf, bf16 *__restrict__ wb,
                       int cob)
{
    const int n = cout * 9 * cin;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int co = i / (9 * cin), r = i - co * 9 * cin, tap = r / cin, ci = r - tap * cin;
        const bf16 v = __float2bfloat16_rn(w[i]);
        wf[((size_t)tap * cout + co) * cin + ci] = v;
        if (wb) wb[((size_t)(8 - tap) * cin + ci) * cob + co] = v;
    }
}

}  // namespace aaps

using namespace aaps;

// ------------------------------------------------------------------ host --
namespace {

// NVTX range around an entry point (tracing; free unless a tool is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

thread_local std::string s_err;

int sfail(int code, const std::string &m)
{
    s_err = m;
    return code;
}

// The sticky flag of the tensor-core waits (AAP_ETIMEOUT once set).
int check_tc(cudaStream_t st)
{
    int v = 0;
    if (cudaMemcpyFromSymbolAsync(&v, g_sur_err, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return sfail(AAP_ECUDA, "reading the tensor-core wait flag");
    return v ? sfail(AAP_ETIMEOUT, "a tensor-core completion wait gave up") : AAP_OK;
}

#define SCK(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return sfail(AAP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    } while (0)

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 148;
    return n;
}

// The dynamic shared memory of each convolution (above the 48 KB default),
// set once per instantiation.
template <int CIN, int COUT, int MODE>
cudaError_t conv_configure()
{
    static std::atomic<int> configured{0};
    if (configured.load()) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(k_conv_ws<CIN, COUT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)conv_ws_smem<CIN, COUT>());
    if (e == cudaSuccess) configured.store(1);
    return e;
}

// Every instantiation the library launches (called before a predict call
// can be captured into a graph).
cudaError_t conv_configure_all()
{
    const cudaError_t es[] = {conv_configure<16, 32, MODE_RELU>(),   conv_configure<32, 32, MODE_RELU>(),
                              conv_configure<32, 8, MODE_RESID>(),   conv_configure<16, 32, MODE_MASK>(),
                              conv_configure<32, 32, MODE_MASK>(),   conv_configure<16, 32, MODE_LINEAR>(),
                              conv_configure<32, 32, MODE_LINEAR>(), conv_configure<32, 8, MODE_RELU>(),
                              conv_configure<32, 8, MODE_LINEAR>(),  conv_configure<16, 8, MODE_RELU>(),
                              conv_configure<16, 8, MODE_LINEAR>()};
    for (cudaError_t e : es)
        if (e != cudaSuccess) return e;
    return cudaSuccess;
}

template <int CIN, int COUT, int MODE>
cudaError_t conv(const bf16 *in, int B, int H, int W, const bf16 *w, const float *bias, bf16 *out, const bf16 *mask,
                 const float *rin, float *rout, cudaStream_t st)
{
    const int ntiles = (W / kTW) * (H / kTH) * B;
    constexpr size_t smem = conv_ws_smem<CIN, COUT>();
    const cudaError_t ce = conv_configure<CIN, COUT, MODE>();
    if (ce != cudaSuccess) return ce;
    k_conv_ws<CIN, COUT, MODE><<<std::min(ntiles, 2 * sm_count()), kConvThreads, smem, st>>>(in, H, W, ntiles, w, bias,
                                                                                            out, mask, rin, rout);
    return cudaGetLastError();
}

int dw_rows(int H) { return H % 4 == 0 ? 4 : (H % 2 == 0 ? 2 : 1); }

template <int CIN, int COUT>
cudaError_t conv_dw(const bf16 *x, const bf16 *dy, int dy_stride, int B, int H, int W, float *part, float *dw,
                    float *db, cudaStream_t st)
{
    constexpr size_t smem = dw_tc_smem<CIN, COUT>();
    static std::atomic<int> configured{0};
    if (!configured.load()) {
        const cudaError_t e0 = cudaFuncSetAttribute(k_conv_dw_tc<CIN, COUT>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e0 != cudaSuccess) return e0;
        configured.store(1);
    }
    const int ntiles = (W / kTW) * (H / kTH) * B;
    // one persistent block per SM (about 117 KB of shared memory each), no
    // more partials than the documented scratch holds
    const int nblk = std::max(1, std::min(std::min(ntiles, sm_count()), (H / dw_rows(H)) * B));
    k_conv_dw_tc<CIN, COUT><<<nblk, kDwThreads, smem, st>>>(x, dy, dy_stride, H, W, ntiles, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int len = COUT * 9 * CIN + COUT;
    k_reduce_parts<<<std::max(1, (len + 31) / 32), 256, 0, st>>>(part, nblk, len, dw, COUT * 9 * CIN, db);
    return cudaGetLastError();
}

bool valid_shape(int H, int W) { return H >= 16 && W >= 16 && H % 16 == 0 && W % 16 == 0 && H <= 4096 && W <= 4096; }

}  // namespace

// Layer table: (cin, cout) padded.
static const int kLayerCin[4] = {16, 32, 32, 32};
static const int kLayerCout[4] = {32, 32, 32, 8};

struct aap_sur {
    aap_sur_params p{};
    cudaStream_t stream = nullptr;
    int H = 0, W = 0, maxb = 0;
    long long nparam = 0;
    long long woff[4], boff[4];
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;       // FP32 master, grad, Adam moments
    bf16 *wf[4] = {}, *wb[4] = {};                                     // packed BF16 weights
    bf16 *x0 = nullptr, *a[3] = {}, *d[3] = {}, *dout = nullptr;       // activations and gradients
    float *state = nullptr, *state2 = nullptr, *target = nullptr, *eta = nullptr;
    float *part = nullptr, *loss_part = nullptr;
    float *dmean = nullptr;                                            // [max_batch * 3] projected gradient means
    float *cpart = nullptr;                                            // chunk sums of the projection
    // the last predict call, captured as a CUDA graph (replayed while the
    // buffers, batch and number of applications stay the same)
    cudaGraphExec_t pexec = nullptr;
    cudaStream_t pstream = nullptr;
    const void *pkey[3] = {nullptr, nullptr, nullptr};
    int pbatch = -1, papps = -1;
    size_t part_floats = 0;
    int loss_blocks = 0;
    long long t = 0;                                                   // Adam step
    std::vector<void *> allocs;
};

namespace {

template <typename T>
int salloc(aap_sur *s, T **p, size_t bytes)
{
    void *q = nullptr;
    if (cudaMalloc(&q, bytes ? bytes : 16) != cudaSuccess) {
        cudaGetLastError();
        return sfail(AAP_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    s->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return AAP_OK;
}

void sfree(aap_sur *s)
{
    if (s->pexec) cudaGraphExecDestroy(s->pexec);
    s->pexec = nullptr;
    if (s->pstream) cudaStreamDestroy(s->pstream);
    s->pstream = nullptr;
    for (void *q : s->allocs) cudaFree(q);
    s->allocs.clear();
}

// Output channels of the data-gradient weight layout of layer l (the last
// layer's 8 are padded to 16, the smallest input width of k_conv_ws).
int cob_of(int l) { return std::max(kLayerCout[l], 16); }

int pack_all(aap_sur *s)
{
    for (int l = 0; l < 4; ++l) {
        const int n = kLayerCout[l] * 9 * kLayerCin[l];
        if (l > 0) SCK(cudaMemsetAsync(s->wb[l], 0, (size_t)cob_of(l) * 9 * kLayerCin[l] * 2, s->stream));
        k_pack<<<(n + 255) / 256, 256, 0, s->stream>>>(s->w + s->woff[l], kLayerCout[l], kLayerCin[l], s->wf[l],
                                                       l > 0 ? s->wb[l] : nullptr, cob_of(l));
        SCK(cudaGetLastError());
    }
    return AAP_OK;
}

// Forward of `batch` samples from s->x0; the result (normalised state after
// one application) goes to s->state2 from s->state.
int forward(aap_sur *s, int batch)
{
    const int H = s->H, W = s->W;
    cudaStream_t st = s->stream;
    SCK((conv<16, 32, MODE_RELU>(s->x0, batch, H, W, s->wf[0], s->w + s->boff[0], s->a[0], nullptr, nullptr, nullptr, st)));
    SCK((conv<32, 32, MODE_RELU>(s->a[0], batch, H, W, s->wf[1], s->w + s->boff[1], s->a[1], nullptr, nullptr, nullptr, st)));
    SCK((conv<32, 32, MODE_RELU>(s->a[1], batch, H, W, s->wf[2], s->w + s->boff[2], s->a[2], nullptr, nullptr, nullptr, st)));
    SCK((conv<32, 8, MODE_RESID>(s->a[2], batch, H, W, s->wf[3], s->w + s->boff[3], nullptr, nullptr, s->state, s->state2, st)));
    if (s->p.conserve) {
        const int nchunk = (H * W + kCenterChunk - 1) / kCenterChunk;
        k_center_part<<<batch * nchunk, 256, 0, st>>>(s->state2, s->state, H * W, nchunk, s->cpart);
        k_center_apply<<<batch * nchunk, 256, 0, st>>>(s->state2, s->cpart, H * W, nchunk, s->p.conserve);
        SCK(cudaGetLastError());
    }
    return AAP_OK;
}

// The kernels of one predict call on s->stream: normalise, `applications`
// forward passes, denormalise into dev_out.
int enqueue_predict(aap_sur *s, const float *dev_in, const float *dev_eta, int batch, int applications, float *dev_out)
{
    const int H = s->H, W = s->W;
    const int grid = 1024;
    SCK(cudaMemcpyAsync(s->eta, dev_eta, (size_t)batch * 4, cudaMemcpyDeviceToDevice, s->stream));
    k_fields_in<<<grid, 256, 0, s->stream>>>(dev_in, s->eta, batch, H, W, (float)s->p.rho0, (float)s->p.eta_center,
                                             (float)s->p.eta_scale, s->state, s->x0);
    SCK(cudaGetLastError());
    for (int k = 0; k < applications; ++k) {
        if (k > 0) {
            k_state_to_input<<<grid, 256, 0, s->stream>>>(s->state, s->eta, batch, H, W, (float)s->p.eta_center,
                                                          (float)s->p.eta_scale, s->x0);
            SCK(cudaGetLastError());
        }
        int rc = forward(s, batch);
        if (rc) return rc;
        std::swap(s->state, s->state2);
    }
    k_fields_out<<<grid, 256, 0, s->stream>>>(s->state, batch, H, W, (float)s->p.rho0, dev_out);
    SCK(cudaGetLastError());
    return AAP_OK;
}

unsigned long long splitmix(unsigned long long &x)
{
    unsigned long long z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" {

const char *aap_sur_last_error(void) { return s_err.c_str(); }

void aap_sur_params_default(aap_sur_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->nbx = p->nby = 128;
    p->max_batch = 32;
    p->rho0 = 2.0;
    p->eta_center = 0.4;
    p->eta_scale = 0.1;
    p->lr = 1e-3;
    p->beta1 = 0.9;
    p->beta2 = 0.999;
    p->eps = 1e-8;
    p->seed = 1;
}

int aap_sur_create(const aap_sur_params *p, void *stream, aap_sur **out)
{
    Range range_("aap_sur_create");
    s_err.clear();
    if (!p || !out) return sfail(AAP_EINVAL, "NULL argument");
    *out = nullptr;
    if (!valid_shape(p->nby, p->nbx)) return sfail(AAP_EINVAL, "nby and nbx must be multiples of 16 (<= 4096)");
    if (p->max_batch < 1 || p->max_batch > 4096) return sfail(AAP_EINVAL, "max_batch must be in [1, 4096]");
    if (!(p->rho0 > 0) || !(p->eta_scale > 0) || !(p->lr > 0) || !(p->eps > 0))
        return sfail(AAP_EINVAL, "rho0, eta_scale, lr and eps must be positive");
    if (p->conserve < 0 || p->conserve > 3) return sfail(AAP_EINVAL, "conserve must be in [0, 3]");
    if (conv_configure_all() != cudaSuccess) return sfail(AAP_ECUDA, "configuring the convolution kernels");
    aap_sur *s = new aap_sur();
    s->p = *p;
    s->stream = static_cast<cudaStream_t>(stream);
    s->H = p->nby;
    s->W = p->nbx;
    s->maxb = p->max_batch;
    long long off = 0;
    for (int l = 0; l < 4; ++l) {
        s->woff[l] = off;
        off += (long long)kLayerCout[l] * 9 * kLayerCin[l];
        s->boff[l] = off;
        off += kLayerCout[l];
    }
    s->nparam = off;
    const size_t pix = (size_t)s->maxb * s->H * s->W;
    int rc = AAP_OK;
    auto A = [&](auto **ptr, size_t bytes) {
        if (rc == AAP_OK) rc = salloc(s, ptr, bytes);
    };
    A(&s->w, off * 4);
    A(&s->g, off * 4);
    A(&s->m, off * 4);
    A(&s->v, off * 4);
    for (int l = 0; l < 4; ++l) {
        A(&s->wf[l], (size_t)kLayerCout[l] * 9 * kLayerCin[l] * 2);
        A(&s->wb[l], (size_t)std::max(kLayerCout[l], 16) * 9 * kLayerCin[l] * 2);
    }
    A(&s->x0, pix * 16 * 2);
    for (int l = 0; l < 3; ++l) {
        A(&s->a[l], pix * 32 * 2);
        A(&s->d[l], pix * 32 * 2);
    }
    A(&s->dout, pix * 16 * 2);
    A(&s->state, pix * 8 * 4);
    A(&s->state2, pix * 8 * 4);
    A(&s->target, pix * 8 * 4);
    A(&s->eta, (size_t)s->maxb * 4);
    // weight-gradient partials: one per block of the gradient kernel (at most
    // one per row band and sample)
    const size_t nblk = (size_t)(s->H / dw_rows(s->H)) * s->maxb;
    s->part_floats = nblk * (32 * 9 * 32 + 32);
    A(&s->part, s->part_floats * 4);
    s->loss_blocks = 256;
    A(&s->loss_part, (size_t)s->loss_blocks * 4);
    A(&s->dmean, (size_t)s->maxb * 3 * 4);
    A(&s->cpart, (size_t)s->maxb * ((s->H * s->W + kCenterChunk - 1) / kCenterChunk) * 4 * 4);
    if (rc) {
        sfree(s);
        delete s;
        return rc;
    }
    // He-uniform initial weights (splitmix64 stream from the seed); the last
    // layer starts small so that the residual map starts near the identity;
    // padded inputs / outputs are zero.
    std::vector<float> hw((size_t)off, 0.f);
    unsigned long long st = p->seed;
    for (int l = 0; l < 4; ++l) {
        const int cin_real = l == 0 ? 4 : 32, cout_real = l == 3 ? 3 : 32;
        const double bound = std::sqrt(6.0 / (9.0 * cin_real)) * (l == 3 ? 0.1 : 1.0);
        for (int co = 0; co < kLayerCout[l]; ++co)
            for (int tap = 0; tap < 9; ++tap)
                for (int ci = 0; ci < kLayerCin[l]; ++ci) {
                    const double u = (double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
                    if (co < cout_real && ci < cin_real)
                        hw[(size_t)s->woff[l] + ((size_t)co * 9 + tap) * kLayerCin[l] + ci] = (float)((2.0 * u - 1.0) * bound);
                }
    }
    if (cudaMemcpy(s->w, hw.data(), (size_t)off * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(s->m, 0, (size_t)off * 4) != cudaSuccess || cudaMemset(s->v, 0, (size_t)off * 4) != cudaSuccess ||
        cudaMemset(s->g, 0, (size_t)off * 4) != cudaSuccess) {
        sfree(s);
        delete s;
        return sfail(AAP_ECUDA, "surrogate initialisation");
    }
    if ((rc = pack_all(s)) || cudaStreamSynchronize(s->stream) != cudaSuccess) {
        sfree(s);
        delete s;
        return rc ? rc : sfail(AAP_ECUDA, "surrogate initialisation");
    }
    *out = s;
    return AAP_OK;
}

int aap_sur_destroy(aap_sur *s)
{
    if (!s) return AAP_OK;
    cudaStreamSynchronize(s->stream);
    sfree(s);
    delete s;
    return AAP_OK;
}

int aap_sur_param_count(aap_sur *s, int64_t *count)
{
    if (!s || !count) return sfail(AAP_EINVAL, "NULL argument");
    *count = s->nparam;
    return AAP_OK;
}

int aap_sur_get_params(aap_sur *s, float *host, int64_t count)
{
    if (!s || !host || count != s->nparam) return sfail(AAP_EINVAL, "bad arguments");
    SCK(cudaMemcpyAsync(host, s->w, (size_t)count * 4, cudaMemcpyDeviceToHost, s->stream));
    SCK(cudaStreamSynchronize(s->stream));
    return AAP_OK;
}

int aap_sur_set_params(aap_sur *s, const float *host, int64_t count)
{
    if (!s || !host || count != s->nparam) return sfail(AAP_EINVAL, "bad arguments");
    SCK(cudaMemcpyAsync(s->w, host, (size_t)count * 4, cudaMemcpyHostToDevice, s->stream));
    SCK(cudaMemsetAsync(s->m, 0, (size_t)count * 4, s->stream));
    SCK(cudaMemsetAsync(s->v, 0, (size_t)count * 4, s->stream));
    s->t = 0;
    int rc = pack_all(s);
    if (rc) return rc;
    SCK(cudaStreamSynchronize(s->stream));
    return AAP_OK;
}

int aap_sur_predict(aap_sur *s, const float *dev_in, const float *dev_eta, int32_t batch, int32_t applications,
                    float *dev_out)
{
    Range range_("aap_sur_predict");
    if (!s || !dev_in || !dev_eta || !dev_out) return sfail(AAP_EINVAL, "NULL argument");
    if (batch < 1 || batch > s->maxb || applications < 0) return sfail(AAP_EINVAL, "bad batch or applications");
    // a call is tens of short launches (4 convolutions per application): it
    // is captured once as a graph on a private stream and replayed on the
    // caller's stream while the buffers, batch and applications stay the same
    const bool same = s->pexec && s->pkey[0] == dev_in && s->pkey[1] == dev_eta && s->pkey[2] == dev_out &&
                      s->pbatch == batch && s->papps == applications;
    if (!same) {
        if (s->pexec) cudaGraphExecDestroy(s->pexec);
        s->pexec = nullptr;
        if (!s->pstream) SCK(cudaStreamCreateWithFlags(&s->pstream, cudaStreamNonBlocking));
        cudaStream_t user = s->stream;
        s->stream = s->pstream;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s->pstream, cudaStreamCaptureModeThreadLocal);
        int rc = e == cudaSuccess ? enqueue_predict(s, dev_in, dev_eta, batch, applications, dev_out) : AAP_OK;
        cudaError_t e2 = cudaStreamEndCapture(s->pstream, &g);
        s->stream = user;
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return sfail(AAP_ECUDA, std::string("capturing the predict call: ") +
                                        cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        e = cudaGraphInstantiate(&s->pexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            s->pexec = nullptr;
            return sfail(AAP_ECUDA, std::string("instantiating the predict graph: ") + cudaGetErrorString(e));
        }
        s->pkey[0] = dev_in;
        s->pkey[1] = dev_eta;
        s->pkey[2] = dev_out;
        s->pbatch = batch;
        s->papps = applications;
    }
    SCK(cudaGraphLaunch(s->pexec, s->stream));
    return AAP_OK;
}

int aap_sur_train_step(aap_sur *s, const float *dev_in, const float *dev_target, const float *dev_eta, int32_t batch,
                       double *loss_out)
{
    Range range_("aap_sur_train_step");
    if (!s || !dev_in || !dev_target || !dev_eta) return sfail(AAP_EINVAL, "NULL argument");
    if (batch < 1 || batch > s->maxb) return sfail(AAP_EINVAL, "bad batch");
    const int H = s->H, W = s->W;
    cudaStream_t st = s->stream;
    const int grid = 1024;
    SCK(cudaMemcpyAsync(s->eta, dev_eta, (size_t)batch * 4, cudaMemcpyDeviceToDevice, st));
    // targets: normalised through the same path (x0 is overwritten below)
    k_fields_in<<<grid, 256, 0, st>>>(dev_target, s->eta, batch, H, W, (float)s->p.rho0, (float)s->p.eta_center,
                                      (float)s->p.eta_scale, s->target, s->x0);
    k_fields_in<<<grid, 256, 0, st>>>(dev_in, s->eta, batch, H, W, (float)s->p.rho0, (float)s->p.eta_center,
                                      (float)s->p.eta_scale, s->state, s->x0);
    SCK(cudaGetLastError());
    int rc = forward(s, batch);
    if (rc) return rc;
    const long long npix = (long long)batch * H * W;
    if (s->p.conserve) {
        const int nchunk = (H * W + kCenterChunk - 1) / kCenterChunk;
        k_center_part<<<batch * nchunk, 256, 0, st>>>(s->state2, s->target, H * W, nchunk, s->cpart);
        k_dmean<<<(batch * 3 + 127) / 128, 128, 0, st>>>(s->cpart, batch, H * W, nchunk, s->p.conserve, s->dmean);
        SCK(cudaGetLastError());
    }
    k_mse<<<s->loss_blocks, 256, 0, st>>>(s->state2, s->target, npix, (float)(1.0 / (3.0 * (double)npix)),
                                          s->loss_part, s->dout, s->p.conserve ? s->dmean : nullptr, H * W);
    SCK(cudaGetLastError());
    float *g = s->g;
    // layer 4: weight gradient from a[2] and dout (16-channel pixels, 8 used);
    // data gradient through the flipped weights, masked by ReLU(a[2]) > 0
    SCK((conv_dw<32, 8>(s->a[2], s->dout, 16, batch, H, W, s->part, g + s->woff[3], g + s->boff[3], st)));
    SCK((conv<16, 32, MODE_MASK>(s->dout, batch, H, W, s->wb[3], nullptr, s->d[2], s->a[2], nullptr, nullptr, st)));
    // layer 3
    SCK((conv_dw<32, 32>(s->a[1], s->d[2], 32, batch, H, W, s->part, g + s->woff[2], g + s->boff[2], st)));
    SCK((conv<32, 32, MODE_MASK>(s->d[2], batch, H, W, s->wb[2], nullptr, s->d[1], s->a[1], nullptr, nullptr, st)));
    // layer 2
    SCK((conv_dw<32, 32>(s->a[0], s->d[1], 32, batch, H, W, s->part, g + s->woff[1], g + s->boff[1], st)));
    SCK((conv<32, 32, MODE_MASK>(s->d[1], batch, H, W, s->wb[1], nullptr, s->d[0], s->a[0], nullptr, nullptr, st)));
    // layer 1 (its input needs no gradient)
    SCK((conv_dw<16, 32>(s->x0, s->d[0], 32, batch, H, W, s->part, g + s->woff[0], g + s->boff[0], st)));
    // Adam step and the BF16 copies
    s->t += 1;
    const double c1 = 1.0 - std::pow(s->p.beta1, (double)s->t), c2 = 1.0 - std::pow(s->p.beta2, (double)s->t);
    k_adam<<<(int)std::min<long long>(1024, (s->nparam + 255) / 256), 256, 0, st>>>(
        s->w, s->g, s->m, s->v, (int)s->nparam, (float)s->p.lr, (float)s->p.beta1, (float)s->p.beta2,
        (float)s->p.eps, (float)c1, (float)c2);
    SCK(cudaGetLastError());
    if ((rc = pack_all(s))) return rc;
    if (loss_out) {
        std::vector<float> lp(s->loss_blocks);
        SCK(cudaMemcpyAsync(lp.data(), s->loss_part, lp.size() * 4, cudaMemcpyDeviceToHost, st));
        SCK(cudaStreamSynchronize(st));
        double tot = 0.0;
        for (float v : lp) tot += v;
        *loss_out = tot / (3.0 * (double)npix);
        return check_tc(st);
    }
    return AAP_OK;
}

// Gradient of the last train step (FP32, the layout of aap_sur_get_params).
int aap_sur_get_grads(aap_sur *s, float *host, int64_t count)
{
    if (!s || !host || count != s->nparam) return sfail(AAP_EINVAL, "bad arguments");
    SCK(cudaMemcpyAsync(host, s->g, (size_t)count * 4, cudaMemcpyDeviceToHost, s->stream));
    SCK(cudaStreamSynchronize(s->stream));
    return check_tc(s->stream);
}

// ---- the convolution kernels alone (device buffers, BF16 as raw 16-bit) ----
int aap_conv3x3_forward(const uint16_t *x, int32_t batch, int32_t h, int32_t w, int32_t cin, int32_t cout,
                        const uint16_t *wt, const float *bias, int32_t relu, uint16_t *y, void *stream)
{
    if (!x || !wt || !bias || !y || batch < 1 || !valid_shape(h, w)) return sfail(AAP_EINVAL, "bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bf16 *X = reinterpret_cast<const bf16 *>(x), *Wt = reinterpret_cast<const bf16 *>(wt);
    bf16 *Y = reinterpret_cast<bf16 *>(y);
    cudaError_t e;
    if (cin == 16 && cout == 32) e = relu ? conv<16, 32, MODE_RELU>(X, batch, h, w, Wt, bias, Y, nullptr, nullptr, nullptr, st)
                                          : conv<16, 32, MODE_LINEAR>(X, batch, h, w, Wt, bias, Y, nullptr, nullptr, nullptr, st);
    else if (cin == 32 && cout == 32) e = relu ? conv<32, 32, MODE_RELU>(X, batch, h, w, Wt, bias, Y, nullptr, nullptr, nullptr, st)
                                               : conv<32, 32, MODE_LINEAR>(X, batch, h, w, Wt, bias, Y, nullptr, nullptr, nullptr, st);
    else if (cin == 32 && cout == 8) e = relu ? conv<32, 8, MODE_RELU>(X, batch, h, w, Wt, bias, Y, nullptr, nullptr, nullptr, st)
                                              : conv<32, 8, MODE_LINEAR>(X, batch, h, w, Wt, bias, Y, nullptr, nullptr, nullptr, st);
    else if (cin == 16 && cout == 8) e = relu ? conv<16, 8, MODE_RELU>(X, batch, h, w, Wt, bias, Y, nullptr, nullptr, nullptr, st)
                                              : conv<16, 8, MODE_LINEAR>(X, batch, h, w, Wt, bias, Y, nullptr, nullptr, nullptr, st);
    else return sfail(AAP_EINVAL, "supported (cin, cout): (16, 32), (32, 32), (32, 8), (16, 8)");
    if (e != cudaSuccess) return sfail(AAP_ECUDA, cudaGetErrorString(e));
    return AAP_OK;
}

int aap_conv3x3_backward_data(const uint16_t *dy, int32_t batch, int32_t h, int32_t w, int32_t cin, int32_t cout,
                              const uint16_t *wt_t, const uint16_t *mask, uint16_t *dx, void *stream)
{
    // dx[., ci] = sum_{tap', co} wt_t[tap'][ci][co] dy[p + tap' - 1][co], zeroed where mask <= 0
    if (!dy || !wt_t || !mask || !dx || batch < 1 || !valid_shape(h, w)) return sfail(AAP_EINVAL, "bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bf16 *D = reinterpret_cast<const bf16 *>(dy), *Wt = reinterpret_cast<const bf16 *>(wt_t);
    const bf16 *M = reinterpret_cast<const bf16 *>(mask);
    bf16 *X = reinterpret_cast<bf16 *>(dx);
    cudaError_t e;
    if (cout == 32 && cin == 32) e = conv<32, 32, MODE_MASK>(D, batch, h, w, Wt, nullptr, X, M, nullptr, nullptr, st);
    else if (cout == 16 && cin == 32) e = conv<16, 32, MODE_MASK>(D, batch, h, w, Wt, nullptr, X, M, nullptr, nullptr, st);
    else return sfail(AAP_EINVAL, "supported (cout, cin): (32, 32), (16, 32)");
    if (e != cudaSuccess) return sfail(AAP_ECUDA, cudaGetErrorString(e));
    return AAP_OK;
}

int aap_conv3x3_backward_weight(const uint16_t *x, const uint16_t *dy, int32_t dy_stride, int32_t batch, int32_t h,
                                int32_t w, int32_t cin, int32_t cout, float *part, int64_t part_floats, float *dw,
                                float *db, void *stream)
{
    if (!x || !dy || !part || !dw || !db || batch < 1 || !valid_shape(h, w)) return sfail(AAP_EINVAL, "bad arguments");
    const long long need = (long long)(h / dw_rows(h)) * batch * (cout * 9 * cin + cout);
    if (part_floats < need) return sfail(AAP_EINVAL, "part buffer too small: need " + std::to_string(need) + " floats");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bf16 *X = reinterpret_cast<const bf16 *>(x), *D = reinterpret_cast<const bf16 *>(dy);
    cudaError_t e;
    if (cin == 32 && cout == 32) e = conv_dw<32, 32>(X, D, dy_stride, batch, h, w, part, dw, db, st);
    else if (cin == 16 && cout == 32) e = conv_dw<16, 32>(X, D, dy_stride, batch, h, w, part, dw, db, st);
    else if (cin == 32 && cout == 8) e = conv_dw<32, 8>(X, D, dy_stride, batch, h, w, part, dw, db, st);
    else return sfail(AAP_EINVAL, "supported (cin, cout): (32, 32), (16, 32), (32, 8)");
    if (e != cudaSuccess) return sfail(AAP_ECUDA, cudaGetErrorString(e));
    return AAP_OK;
}

}  // extern "C"
