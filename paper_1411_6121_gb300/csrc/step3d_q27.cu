// step3d_q27.cu -- the throughput kernel of dugks_step3d.cuh instantiated for D3Q27 (the
// paper's 3D velocity set, Sec. 2.3): 32 x 8 columns per CTA, F32/BF16/F16 storage. At
// 27 velocities the TMA stages do not fit beside the ring, so every plane is loaded
// directly (the kernel's tensor-map argument is unused).
#include <string.h>

#include "dugks_internal.h"
#include "dugks_step3d.cuh"

namespace dugks {

template <class S, bool FORCE>
static cudaError_t launch27(const StepParams &p, cudaStream_t stream) {
    using K = Shape3<27, 8, S>;
    static int configured_dev = -1;
    static int sms = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(fused_step3d<27, S, 8, FORCE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)K::smem_bytes);
        if (e != cudaSuccess) return e;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        configured_dev = dev;
    }
    const int tiles_x = (p.nx + K::TXI - 1) / K::TXI;
    const int tiles_y = (p.ny + K::TYI - 1) / K::TYI;
    const int64_t tiles = (int64_t)tiles_x * tiles_y;
    // z chunks: maximise (useful waves / launched waves) / (1 + 2 / chunk length), one CTA
    // per SM (each chunk recomputes two extra planes of fbar+ in its prologue)
    int best = 1;
    double best_eff = -1.0;
    for (int nc = 1; nc <= 16; nc++) {
        const int zc = (p.nz + nc - 1) / nc;
        if (nc > 1 && zc < 8) break;
        const int ncr = (p.nz + zc - 1) / zc;
        const double waves = (double)(tiles * ncr) / (double)sms;
        const double eff = waves / ceil(waves) / (1.0 + 2.0 / zc);
        if (eff > best_eff + 1e-9) { best_eff = eff; best = nc; }
    }
    const int zchunk = (p.nz + best - 1) / best;
    const int nchunks = (p.nz + zchunk - 1) / zchunk;
    static_assert(!K::TMA, "D3Q27 loads its planes directly");
    CUtensorMap unused;
    memset(&unused, 0, sizeof unused);
    fused_step3d<27, S, 8, FORCE><<<dim3(tiles_x, tiles_y, nchunks), dim3(32, 8), K::smem_bytes, stream>>>(p, unused,
                                                                                                          zchunk);
    return cudaGetLastError();
}

cudaError_t launch_step3d_q27(const StepParams &p, int store, cudaStream_t stream) {
    const bool force = p.field != nullptr || p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0;
    switch (store) {
        case 0: return force ? launch27<float, true>(p, stream) : launch27<float, false>(p, stream);
        case 1: return force ? launch27<__nv_bfloat16, true>(p, stream) : launch27<__nv_bfloat16, false>(p, stream);
        case 2: return force ? launch27<__half, true>(p, stream) : launch27<__half, false>(p, stream);
    }
    return cudaErrorNotSupported;
}

}  // namespace dugks
