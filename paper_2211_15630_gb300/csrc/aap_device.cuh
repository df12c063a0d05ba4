// aap_device.cuh -- device helpers shared by the step kernels: Philox
// noise, uniform conversion and warp reductions.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

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
        // each 32 x 32 -> 64-bit product as one wide multiply (high and low words)
        const unsigned long long p0 = 0xD2511F53ull * c[0], p1 = 0xCD9E8D57ull * c[2];
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
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

// arg(x + i y) in [-pi, pi] (the angle of the VM sum, Eq. collision_VM), with
// arg(0) = 0.  The octant symmetries of the arctangent reduce the argument to
// t = min(|x|, |y|) / max(|x|, |y|) in [0, 1]; atan(t) there is an odd
// polynomial t P(t^2) of degree 15 whose coefficients were fitted in the
// minimax sense on [0, 1] (Lawson's iteratively reweighted least squares):
// 3.7e-8 rad in exact arithmetic, 1.4e-7 rad evaluated in FP32 with FMAs, plus
// the error of the fast quotient (2 ulp of t, times atan' <= 1).  No branches.
constexpr float kAtan0 = 9.999993443e-01f, kAtan1 = -3.332985938e-01f, kAtan2 = 1.994656622e-01f,
                kAtan3 = -1.390862912e-01f, kAtan4 = 9.642197192e-02f, kAtan5 = -5.591231957e-02f,
                kAtan6 = 2.186295204e-02f, kAtan7 = -4.054565448e-03f;

__device__ __forceinline__ float arg2(float y, float x)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float hi = fmaxf(ax, ay), lo = fminf(ax, ay);
    const float t = hi > 0.f ? __fdividef(lo, hi) : 0.f;      // |sums| < 2^126: the fast quotient is valid
    const float t2 = t * t;
    float r = fmaf(kAtan7, t2, kAtan6);
    r = fmaf(r, t2, kAtan5);
    r = fmaf(r, t2, kAtan4);
    r = fmaf(r, t2, kAtan3);
    r = fmaf(r, t2, kAtan2);
    r = fmaf(r, t2, kAtan1);
    r = fmaf(r, t2, kAtan0);
    r *= t;
    if (ay > ax) r = 1.57079632679490f - r;
    if (x < 0.f) r = AAP_PI_F - r;
    return copysignf(r, y);
}

}  // namespace aapk
