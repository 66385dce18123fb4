// step_q19.cu -- instantiations of the fused DUGKS step for the Q = 19 velocity set.
#include "dugks_internal.h"
#include "dugks_step.cuh"

#include <type_traits>

namespace dugks {

template <int TX, int TY, class S, bool NU = false>
static cudaError_t launch_tile(const StepParams &p, cudaStream_t stream) {
    using K = StepShape<19, TX, TY, typename Arith<S>::T>;
    if (K::smem_bytes > 227 * 1024) return cudaErrorNotSupported;
    static int configured_dev = -1;  // per template instance: device it was configured for
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(fused_step<19, S, TX, TY, NU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)K::smem_bytes);
        if (e != cudaSuccess) return e;
        configured_dev = dev;
    }
    int nchunks = 1;
    if (K::D == 3) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t tiles = (int64_t)((p.nx + TX - 1) / TX) * ((p.ny + TY - 1) / TY);
        // about four CTAs per SM in flight over the whole grid, at least 8 planes a chunk
        int64_t want = (4LL * sms + tiles - 1) / tiles;
        if (want < 1) want = 1;
        int64_t maxc = (p.nz + 7) / 8;
        if (want > maxc) want = maxc < 1 ? 1 : maxc;
        nchunks = (int)want;
    }
    const int zchunk = (p.nz + nchunks - 1) / nchunks;
    nchunks = (p.nz + zchunk - 1) / zchunk;
    dim3 grid((p.nx + TX - 1) / TX, (p.ny + TY - 1) / TY, nchunks);
    fused_step<19, S, TX, TY, NU><<<grid, TX * TY, K::smem_bytes, stream>>>(p, zchunk);
    return cudaGetLastError();
}

template <class S>
static cudaError_t launch_store(const StepParams &p, int tx, int ty, cudaStream_t stream) {
    if constexpr (std::is_same<S, float>::value || std::is_same<S, double>::value) {
        if (p.metric[0]) {  // non-uniform mesh (FP32 and FP64 storage)
            if (tx == 32 && ty == 8) return launch_tile<32, 8, S, true>(p, stream);
            if (tx == 16 && ty == 8) return launch_tile<16, 8, S, true>(p, stream);
            return cudaErrorNotSupported;
        }
    } else {
        if (p.metric[0]) return cudaErrorNotSupported;
    }
    if (tx == 32 && ty == 8) return launch_tile<32, 8, S>(p, stream);
    if (tx == 16 && ty == 8) return launch_tile<16, 8, S>(p, stream);
    return cudaErrorNotSupported;
}

cudaError_t launch_step_q19(const StepParams &p, int store, int tx, int ty, cudaStream_t stream) {
    switch (store) {
        case 0: return launch_store<float>(p, tx, ty, stream);
        case 1: return launch_store<__nv_bfloat16>(p, tx, ty, stream);
        case 2: return launch_store<__half>(p, tx, ty, stream);
        case 3: return launch_store<double>(p, tx, ty, stream);
    }
    return cudaErrorNotSupported;
}

}  // namespace dugks
