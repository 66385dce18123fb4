// dugks_internal.h -- host-side declarations shared by the translation units of libdugks.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dugks_device.cuh"

namespace dugks {

// Launch one fused step (fused_step<Q, S, TX, TY>) on `stream`. store: DUGKS_STORE_*.
// Returns cudaSuccess or the launch error; cudaErrorNotSupported for a tile that was not
// instantiated.
cudaError_t launch_step_q9(const StepParams &p, int store, int tx, int ty, cudaStream_t stream);
cudaError_t launch_step_q19(const StepParams &p, int store, int tx, int ty, cudaStream_t stream);
cudaError_t launch_step_q27(const StepParams &p, int store, int tx, int ty, cudaStream_t stream);
// Throughput kernel for D3Q19 with F32/BF16/F16 storage (dugks_step3d.cuh); ry = CTA rows.
cudaError_t launch_step3d_q19(const StepParams &p, int store, int ry, cudaStream_t stream);
// The same throughput kernel for D3Q27 (32 x 8 columns per CTA).
cudaError_t launch_step3d_q27(const StepParams &p, int store, cudaStream_t stream);
// Throughput kernel for D2Q9 with F32/BF16/F16 storage (dugks_step2d.cuh); ry = CTA rows
// (4, 8 or 16; the inner tile is 30 x (ry - 2) cells). The batch form walks a work list of
// (instance, x0, y0) inner-tile origins over params[2 i + parity] on a persistent grid.
cudaError_t launch_step2d_q9(const StepParams &p, int store, int ry, cudaStream_t stream);
cudaError_t launch_step2d_batch(const StepParams *params, const int4 *items, int nitems, int parity, int store,
                                int ry, bool force, cudaStream_t stream);

// Whether a TMA wait of the 3D throughput kernel gave up since the last call (the kernel then
// skipped its step); clears the flag. 1: yes, 0: no, -1: the flag could not be read.
int tma_wait_failures();

// Auxiliary kernels (aux.cu).
cudaError_t launch_init(int q, int store, const StepParams &p, const double *pres, const double *vel, double rt,
                        cudaStream_t stream);
cudaError_t launch_moments(int q, int store, const StepParams &p, double t, double rt, float *out,
                           cudaStream_t stream);
// FP64 residual and totals: per-block partial sums into `partials` ([nblocks][8] doubles),
// then a fixed-order final sum into `out` (8 doubles on the device).
cudaError_t launch_residual(int q, int store, const StepParams &p, double t, double rt, double *uprev,
                            int have_prev, double *partials, int nblocks, double *out, cudaStream_t stream);
int residual_blocks(int64_t ncell);
cudaError_t launch_advance(long long *ctr, long long n, cudaStream_t stream);

// Sets the message that dugks_last_error(NULL) returns in this thread (api.cu).
void set_null_handle_error(const char *msg);

}  // namespace dugks
