// step3d_q19.cu -- instantiations of the D3Q19 throughput kernel (dugks_step3d.cuh), the
// tensor maps its TMA stages read through, and the flag of a copy that never landed.
#include <string.h>

#include <cudaTypedefs.h>

#include "dugks_internal.h"
#include "dugks_step3d.cuh"
#include "dugks_step3d_ws.cuh"

namespace dugks {

int tma_wait_failures() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tma_wait_failed, sizeof v) != cudaSuccess) return -1;
    if (v) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_tma_wait_failed, &zero, sizeof zero);
    }
    return v;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (the library
// links the runtime only).
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool looked = false;
    if (!looked) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
        looked = true;
    }
    return fn;
}

cudaError_t encode_state_map(CUtensorMap *map, const void *base, int esize, bool bf16, int64_t px, int64_t ny,
                             int64_t nz, int q, int bx, int ry) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const CUtensorMapDataType dt = esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                              : (bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
    const cuuint64_t dims[4] = {(cuuint64_t)px, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)q};
    const cuuint64_t strides[3] = {(cuuint64_t)(px * esize), (cuuint64_t)(px * ny * esize),
                                   (cuuint64_t)(px * ny * nz * esize)};
    const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)ry, 1u, (cuuint32_t)q};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    const CUresult r = fn(map, dt, 4, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

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
    CUtensorMap map;
    memset(&map, 0, sizeof map);
    if (K::TMA) {
        const cudaError_t e = encode_state_map(&map, p.src, (int)sizeof(S), std::is_same<S, __nv_bfloat16>::value, p.px,
                                               p.ny, p.nz, 19, K::BX, RY);
        if (e != cudaSuccess) return e;
    }
    fused_step3d<19, S, RY, FORCE><<<grid, block, K::smem_bytes, stream>>>(p, map, zchunk);
    return cudaGetLastError();
}

// z chunks per tile column for one CTA per SM: maximise (useful waves / launched waves) /
// (1 + 2 / chunk length) (each chunk makes two extra planes of fbar+ in its prologue).
static int zchunk_for(int64_t tiles, int nz, int64_t slots) {
    int best = 1;
    double best_eff = -1.0;
    for (int nc = 1; nc <= 16; nc++) {
        const int zc = (nz + nc - 1) / nc;
        if (nc > 1 && zc < 8) break;
        const int ncr = (nz + zc - 1) / zc;
        const double waves = (double)(tiles * ncr) / (double)slots;
        const double eff = waves / ceil(waves) / (1.0 + 2.0 / zc);
        if (eff > best_eff + 1e-9) { best_eff = eff; best = nc; }
    }
    return (nz + best - 1) / best;
}

// The warp-specialised kernel (dugks_step3d_ws.cuh): 8 producer + 8 consumer warps, one CTA
// per SM, 32 x 8 columns per tile.
template <class S, bool FORCE>
static cudaError_t launch_ws(const StepParams &p, cudaStream_t stream) {
    using K = ShapeWS<19, S>;
    static int configured_dev = -1;
    static int sms = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(fused_step3d_ws<19, S, FORCE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)K::smem_bytes);
        if (e != cudaSuccess) return e;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        configured_dev = dev;
    }
    const int tiles_x = (p.nx + K::TXI - 1) / K::TXI;
    const int tiles_y = (p.ny + K::TYI - 1) / K::TYI;
    const int zchunk = zchunk_for((int64_t)tiles_x * tiles_y, p.nz, sms);
    const int nchunks = (p.nz + zchunk - 1) / zchunk;
    CUtensorMap map;
    memset(&map, 0, sizeof map);
    const cudaError_t e = encode_state_map(&map, p.src, (int)sizeof(S), std::is_same<S, __nv_bfloat16>::value, p.px,
                                           p.ny, p.nz, 19, K::BX, K::RY);
    if (e != cudaSuccess) return e;
    fused_step3d_ws<19, S, FORCE><<<dim3(tiles_x, tiles_y, nchunks), K::NTHREADS, K::smem_bytes, stream>>>(p, map,
                                                                                                          zchunk);
    return cudaGetLastError();
}

template <class S>
static cudaError_t launch_s(const StepParams &p, int ry, bool force, cudaStream_t stream) {
    if (ry == 0) return force ? launch_ws<S, true>(p, stream) : launch_ws<S, false>(p, stream);
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
