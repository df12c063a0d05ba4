// aap_kernels.cuh -- host-callable launchers of the step kernels.
#pragma once

#include <cuda_runtime.h>

#include "aap_internal.cuh"

namespace aapk {

// Everything one step launch needs; the step index and buffer parity are read
// on the device from Ctl, so a captured CUDA graph of steps can be replayed.
struct LaunchCfg {
    Sys *sys;                    // device array [nsys]
    int nsys;
    int model;                   // shared by all systems of the launch
    const int *tile_base;        // device [nsys + 1]: prefix of tiles per system
    Ctl *ctl;
    unsigned char *scratch;      // device [grid_step * scratch_per_block]
    size_t scratch_per_block;
    int scratch_cap;             // particles a block can stage in global scratch
    int spill_list_cap;          // spill matches a block can hold
    int threads;                 // 256 or 512
    int stage_cap;               // particles staged in shared memory
    int nce_max;                 // cells of the largest tile plus its ring
    int hist_words;              // histogram bins (theta + |Omega|) of the widest system
    int grid_step, grid_finish;
    // pipelined step (one system, one species): shared buffers of pipe_cap
    // staged / pipe_cap_own own particles per tile, one block per SM; tiles
    // that do not fit go to dense_list (device [ntiles], zero between steps)
    int pipe;
    int pipe_cap, pipe_cap_own, pipe_grid;
    int pipe_nceh;               // half cells (split along x) of the largest extended tile, (2 tw + 4)(th + 2)
    int *dense_list;
    // metric-free step (knn > 0): cell count, scan, scatter, k-nearest update
    int knn;
    long long mf_n, mf_ncell;
    int mf_grid;                 // persistent blocks of the k-nearest update
};

size_t step_smem_bytes(int stage_cap, int nce_max, int hist_words);
// Set the dynamic shared-memory limit of the step kernel and report how many
// of its blocks fit on one SM.
cudaError_t configure_step_kernel(int model, int threads, size_t smem_bytes, int *blocks_per_sm);

// Dynamic shared memory of the pipelined step kernel.
__host__ __device__ size_t pipe_smem_bytes(int cap, int cap_own, int nceh, int hist_words);
// Static shared memory of the pipelined step kernel of a model.
cudaError_t pipe_static_smem(int model, size_t *bytes);
// Set the dynamic shared-memory limit of the pipelined step kernel.
cudaError_t configure_pipe_kernel(int model, size_t smem);
// test hook: the wait bound of the pipelined kernel (<= 0: default) and the stall injection
cudaError_t set_pipe_test(long long wait_cycles, int stall);
// The pipelined step kernel alone (launch_step adds k_finish).
cudaError_t launch_step_pipe(const LaunchCfg &L, cudaStream_t st);

// One full step: k_step (or the pipelined step kernel) then k_finish.  With ev != nullptr, ev[0..2] are
// recorded before k_step, after k_step and after k_finish.
cudaError_t launch_step(const LaunchCfg &L, cudaStream_t st, cudaEvent_t *ev = nullptr);

// Blocks of the metric-free update that are resident at once on sm_count SMs.
cudaError_t configure_mf_kernels(int model, int knn, int hist_words, int sm_count, int *grid);

// The metric-free step (knn > 0): the kernels of launch_step for a flat system.
cudaError_t launch_mf_step(const LaunchCfg &L, cudaStream_t st, cudaEvent_t *ev);

cudaError_t launch_insert(const Sys &S, int b, const double *x, const double *y, const float *th,
                          int mode, cudaStream_t st);
// bad[0]: the lowest index with a position outside [0, lx] x [0, ly]; bad[1]:
// the lowest with a non-finite orientation; ~0 where there is none.
cudaError_t launch_validate(const double *x, const double *y, const float *th, long long n, double lx, double ly,
                            unsigned long long *bad, cudaStream_t st);
cudaError_t launch_gather(const Sys &S, int b, double *x, double *y, float *th, int *seen,
                          cudaStream_t st);
cudaError_t launch_observe(const Sys &S, int b, unsigned long long *out, cudaStream_t st);
// Coarse-grained fields of buffer b into out[3][nby][nbx] (device), using
// acc[3 * nbx * nby] (device scratch) for the integer sums.
cudaError_t launch_coarse(const Sys &S, int b, int nbx, int nby, unsigned long long *acc, float *out,
                          cudaStream_t st);

}  // namespace aapk
