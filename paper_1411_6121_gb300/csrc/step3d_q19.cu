// step3d_q19.cu -- instantiations of the D3Q19 throughput kernel (dugks_step3d.cuh).
#include "dugks_internal.h"
#include "dugks_step3d.cuh"

namespace dugks {

template <int RY, class S, bool FORCE>
static cudaError_t launch_ry(const StepParams &p, cudaStream_t stream) {
    using K = Shape3<19, RY, S>;
    static int configured_dev = -1;
    static int sms = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(fused_step3d<19, S, RY, FORCE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem_bytes);
        if (e != cudaSuccess) return e;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        configured_dev = dev;
    }
    int blocks_per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, fused_step3d<19, S, RY, FORCE>, 32 * RY,
                                                  K::smem_bytes);
    if (blocks_per_sm < 1) blocks_per_sm = 1;
    const int tiles_x = (p.nx + K::TXI - 1) / K::TXI;
    const int tiles_y = (p.ny + K::TYI - 1) / K::TYI;
    const int64_t tiles = (int64_t)tiles_x * tiles_y;
    // number of z chunks: maximise (useful waves / launched waves) / (1 + 2 / chunk length)
    // (each chunk recomputes two extra planes of fbar+ in its prologue)
    const int64_t slots = (int64_t)sms * blocks_per_sm;
    int best = 1;
    double best_eff = -1.0;
    for (int nc = 1; nc <= 16; nc++) {
        const int zc = (p.nz + nc - 1) / nc;
        if (nc > 1 && zc < 8) break;
        const int ncr = (p.nz + zc - 1) / zc;
        const double waves = (double)(tiles * ncr) / (double)slots;
        const double eff = waves / ceil(waves) / (1.0 + 2.0 / zc);
        if (eff > best_eff + 1e-9) { best_eff = eff; best = nc; }
    }
    const int zchunk = (p.nz + best - 1) / best;
    const int nchunks = (p.nz + zchunk - 1) / zchunk;
    dim3 grid(tiles_x, tiles_y, nchunks);
    dim3 block(32, RY);
    fused_step3d<19, S, RY, FORCE><<<grid, block, K::smem_bytes, stream>>>(p, zchunk);
    return cudaGetLastError();
}

template <class S>
static cudaError_t launch_s(const StepParams &p, int ry, bool force, cudaStream_t stream) {
    if (ry == 10) return force ? launch_ry<10, S, true>(p, stream) : launch_ry<10, S, false>(p, stream);
    if (ry == 8) return force ? launch_ry<8, S, true>(p, stream) : launch_ry<8, S, false>(p, stream);
    return cudaErrorNotSupported;
}

cudaError_t launch_step3d_q19(const StepParams &p, int store, int ry, cudaStream_t stream) {
    const bool force = p.field != nullptr || p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0;
    switch (store) {
        case 0: return launch_s<float>(p, ry, force, stream);
        case 1: return launch_s<__nv_bfloat16>(p, ry, force, stream);
        case 2: return launch_s<__half>(p, ry, force, stream);
    }
    return cudaErrorNotSupported;
}

}  // namespace dugks
