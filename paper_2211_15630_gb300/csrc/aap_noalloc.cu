// aap_noalloc.cu -- coarse-graining of caller-owned particle arrays without
// any device allocation.
//
// Some callers cannot allocate device memory at all: code running inside a
// memory pool or arena that owns every byte, callers that must not call
// cudaMalloc (it can synchronise the device and is not allowed while a
// stream is being captured), and embedded users with a fixed memory budget.
// For them aap_coarse_grain_noalloc does what aap_coarse_grain does, but
// keeps its integer accumulators in a file-scope __device__ array of fixed
// size instead of memory the library allocates.
//
// The array lives in every device that loads this library, until the process
// exits.  Host code must not pass the array's name to a kernel (on the host
// it is only a stand-in symbol); its device address is looked up once per
// device with cudaGetSymbolAddress, on the first call made on that device.
// Every call shares the one array, so calls whose work overlaps on the GPU
// (different streams, or different host threads) race; calls ordered on one
// stream are safe.  The array is cleared at the start of each call.  The
// looked-up address is kept for the life of the process: it does not survive
// cudaDeviceReset (or any other teardown of the device's primary context),
// after which this entry point must not be called again on that device.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "../../include/aap.h"

namespace {

constexpr long long kNoAllocMaxBins = 256 * 256;      // 3 x 65,536 x 8 bytes = 1.5 MiB

__device__ __align__(256) unsigned long long g_cg_scratch[3 * kNoAllocMaxBins];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long *g_scratch_ptr[kMaxDevices] = {};

thread_local std::string g_na_err;

int na_fail(int code, const std::string &m)
{
    g_na_err = m;
    return code;
}

__global__ void k_na_clear(unsigned long long *acc, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc[i] = 0ull;
}

// Bin floor(u f) of one coordinate, clamped to [0, nb): a position below 0
// or a NaN goes to bin 0, one at or beyond the far edge to bin nb - 1 (the
// comparisons decide before any conversion, so no value is converted out of
// the int range).
__device__ __forceinline__ int na_bin(double u, double f, int nb)
{
    const double t = u * f;
    if (!(t >= 0.0)) return 0;
    if (t >= (double)nb) return nb - 1;
    return min((int)t, nb - 1);
}

// Same binning and the same exact integer sums as aap_coarse_grain.  A
// non-finite orientation adds to the count of its bin but nothing to the
// polarisation sums.
__global__ void k_na_accumulate(const double *__restrict__ x, const double *__restrict__ y,
                                const float *__restrict__ th, long long n, double fx, double fy, int nbx, int nby,
                                unsigned long long *acc)
{
    const long long nb = (long long)nbx * nby;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long bin = (long long)na_bin(y[i], fy, nby) * nbx + na_bin(x[i], fx, nbx);
        const float t = th[i];
        float sn = 0.f, cs = 0.f;
        if (isfinite(t)) sincosf(t, &sn, &cs);
        atomicAdd(acc + bin, 1ull);
        atomicAdd(acc + nb + bin, (unsigned long long)__float2ll_rn(cs * 4294967296.0f));
        atomicAdd(acc + 2 * nb + bin, (unsigned long long)__float2ll_rn(sn * 4294967296.0f));
    }
}

__global__ void k_na_finish(const unsigned long long *acc, int nbx, int nby, double inv_area, float *out)
{
    const long long nb = (long long)nbx * nby;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x) {
        out[i] = (float)((double)acc[i] * inv_area);
        out[nb + i] = (float)((double)(long long)acc[nb + i] / 4294967296.0 * inv_area);
        out[2 * nb + i] = (float)((double)(long long)acc[2 * nb + i] / 4294967296.0 * inv_area);
    }
}

// Device address of the scratch array on the current device (looked up once).
int scratch_for_current_device(unsigned long long **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(AAP_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return na_fail(AAP_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_cg_scratch);
        if (e != cudaSuccess || !p)
            return na_fail(AAP_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<unsigned long long *>(p);
    }
    *out = g_scratch_ptr[dev];
    return AAP_OK;
}

}  // namespace

extern "C" {

const char *aap_noalloc_last_error(void) { return g_na_err.c_str(); }

int aap_coarse_grain_noalloc(const double *x, const double *y, const float *theta, int64_t n, double lx, double ly,
                             int32_t nbx, int32_t nby, float *dev_out, void *stream)
{
    g_na_err.clear();
    if (!dev_out || (n > 0 && (!x || !y || !theta))) return na_fail(AAP_EINVAL, "NULL argument");
    if (n < 0) return na_fail(AAP_EINVAL, "n < 0");
    if (!std::isfinite(lx) || !std::isfinite(ly) || !(lx > 0) || !(ly > 0))
        return na_fail(AAP_EINVAL, "lx and ly must be finite and positive");
    if (nbx < 1 || nby < 1) return na_fail(AAP_EINVAL, "nbx and nby must be >= 1");
    const long long nb = (long long)nbx * nby;
    if (nb > kNoAllocMaxBins)
        return na_fail(AAP_EINVAL, "nbx * nby = " + std::to_string(nb) + " exceeds the fixed scratch of " +
                                       std::to_string(kNoAllocMaxBins) + " bins");
    unsigned long long *acc = nullptr;
    int rc = scratch_for_current_device(&acc);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_na_clear<<<(unsigned)std::min<long long>((3 * nb + 255) / 256, 1024), 256, 0, st>>>(acc, 3 * nb);
    if (n > 0)
        k_na_accumulate<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, st>>>(
            x, y, theta, n, (double)nbx / lx, (double)nby / ly, nbx, nby, acc);
    k_na_finish<<<(unsigned)std::min<long long>((nb + 255) / 256, 4096), 256, 0, st>>>(acc, nbx, nby,
                                                                                        (double)nb / (lx * ly), dev_out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(AAP_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return AAP_OK;
}

}  // extern "C"
