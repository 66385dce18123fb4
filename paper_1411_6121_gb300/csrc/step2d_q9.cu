// step2d_q9.cu -- instantiations and launchers of the D2Q9 throughput kernel
// (dugks_step2d.cuh): one instance on a grid of tiles, or a batch on a persistent grid.
#include "dugks_internal.h"
#include "dugks_step2d.cuh"

namespace dugks {

namespace {

template <class S, int RY, bool FORCE, bool BATCH>
cudaError_t configure(int *blocks_per_sm, int *sms) {
    using K = Shape2<RY, S>;
    static int configured_dev = -1;
    static int cached_bps = 0, cached_sms = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_dev != dev) {
        cudaError_t e;
        if (BATCH)
            e = cudaFuncSetAttribute(fused_step2d_batch<S, RY, FORCE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)K::smem_bytes);
        else
            e = cudaFuncSetAttribute(fused_step2d<S, RY, FORCE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)K::smem_bytes);
        if (e != cudaSuccess) return e;
        if (BATCH)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cached_bps, fused_step2d_batch<S, RY, FORCE>, 32 * RY,
                                                          K::smem_bytes);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cached_bps, fused_step2d<S, RY, FORCE>, 32 * RY,
                                                          K::smem_bytes);
        cudaDeviceGetAttribute(&cached_sms, cudaDevAttrMultiProcessorCount, dev);
        configured_dev = dev;
    }
    if (blocks_per_sm) *blocks_per_sm = cached_bps < 1 ? 1 : cached_bps;
    if (sms) *sms = cached_sms;
    return cudaSuccess;
}

template <class S, int RY, bool FORCE>
cudaError_t launch_one(const StepParams &p, cudaStream_t stream) {
    using K = Shape2<RY, S>;
    cudaError_t e = configure<S, RY, FORCE, false>(nullptr, nullptr);
    if (e != cudaSuccess) return e;
    dim3 grid((p.nx + K::TXI - 1) / K::TXI, (p.ny + K::TYI - 1) / K::TYI);
    fused_step2d<S, RY, FORCE><<<grid, dim3(32, RY), K::smem_bytes, stream>>>(p);
    return cudaGetLastError();
}

template <class S, int RY, bool FORCE>
cudaError_t launch_many(const StepParams *params, const int4 *items, int nitems, int parity, cudaStream_t stream) {
    using K = Shape2<RY, S>;
    int bps = 1, sms = 1;
    cudaError_t e = configure<S, RY, FORCE, true>(&bps, &sms);
    if (e != cudaSuccess) return e;
    const int grid = nitems < sms * bps ? nitems : sms * bps;  // persistent: resident CTAs, at most the items
    if (grid < 1) return cudaSuccess;
    fused_step2d_batch<S, RY, FORCE><<<grid, dim3(32, RY), K::smem_bytes, stream>>>(params, items, nitems, parity);
    return cudaGetLastError();
}

template <class S, bool FORCE>
cudaError_t one_ry(const StepParams &p, int ry, cudaStream_t st) {
    if (ry == 4) return launch_one<S, 4, FORCE>(p, st);
    if (ry == 8) return launch_one<S, 8, FORCE>(p, st);
    if (ry == 16) return launch_one<S, 16, FORCE>(p, st);
    return cudaErrorNotSupported;
}

template <class S, bool FORCE>
cudaError_t many_ry(const StepParams *params, const int4 *items, int nitems, int parity, int ry, cudaStream_t st) {
    if (ry == 4) return launch_many<S, 4, FORCE>(params, items, nitems, parity, st);
    if (ry == 8) return launch_many<S, 8, FORCE>(params, items, nitems, parity, st);
    if (ry == 16) return launch_many<S, 16, FORCE>(params, items, nitems, parity, st);
    return cudaErrorNotSupported;
}

}  // namespace

cudaError_t launch_step2d_q9(const StepParams &p, int store, int ry, cudaStream_t stream) {
    const bool force = p.field != nullptr || p.g[0] != 0.0 || p.g[1] != 0.0;
    switch (store) {
        case 0: return force ? one_ry<float, true>(p, ry, stream) : one_ry<float, false>(p, ry, stream);
        case 1: return force ? one_ry<__nv_bfloat16, true>(p, ry, stream) : one_ry<__nv_bfloat16, false>(p, ry, stream);
        case 2: return force ? one_ry<__half, true>(p, ry, stream) : one_ry<__half, false>(p, ry, stream);
    }
    return cudaErrorNotSupported;
}

cudaError_t launch_step2d_batch(const StepParams *params, const int4 *items, int nitems, int parity, int store,
                                int ry, bool force, cudaStream_t stream) {
    switch (store) {
        case 0:
            return force ? many_ry<float, true>(params, items, nitems, parity, ry, stream)
                         : many_ry<float, false>(params, items, nitems, parity, ry, stream);
        case 1:
            return force ? many_ry<__nv_bfloat16, true>(params, items, nitems, parity, ry, stream)
                         : many_ry<__nv_bfloat16, false>(params, items, nitems, parity, ry, stream);
        case 2:
            return force ? many_ry<__half, true>(params, items, nitems, parity, ry, stream)
                         : many_ry<__half, false>(params, items, nitems, parity, ry, stream);
    }
    return cudaErrorNotSupported;
}

}  // namespace dugks
