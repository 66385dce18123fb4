// noalloc.cu -- the FP64 residual / conservation reduction for callers that cannot allocate.
//
// dugks_residual (api.cu) reduces through a per-block partial-sum buffer that the handle
// allocates with cudaMalloc at creation. Some callers cannot make that call: code embedded in
// a host framework whose allocator already owns the device memory (cudaMalloc there fails or
// fragments it), and loops that must not take cudaMalloc's implicit device synchronisation.
// They need the same reduction with nothing allocated on their behalf. This file gives them
// one entry point, dugks_residual_static, which runs the very same kernels, on the same
// number of blocks, with the partial sums placed in a fixed array in device memory that the
// library reserves when it is loaded. The call copies its sums to host memory and
// synchronises its stream before it returns, so it cannot be called while that stream is
// being captured into a CUDA graph.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/dugks.h"
#include "dugks_internal.h"

namespace dugks {

// The reduction runs residual_blocks(ncell) blocks, as dugks_residual does: one per 2048
// cells, at most 4096, each block striding over its cells in a fixed order and writing 8
// doubles; the final sum takes 8 more. The array holds the 4096 blocks' partials. The entry
// point accepts meshes up to STATIC_RES_MAX_CELLS = 4096 * 4096 = 16,777,216 cells (a 256^3
// mesh, at most 4096 cells per block). Size: (4096 + 1) * 8 doubles = 256 KB, held by every
// GPU that loads the library until the process exits.
constexpr int STATIC_RES_MAX_BLOCKS = 4096;
constexpr int64_t STATIC_RES_MAX_CELLS = (int64_t)4096 * 4096;

static __device__ __align__(256) double g_res_scratch[(STATIC_RES_MAX_BLOCKS + 1) * 8];

// Device address of g_res_scratch per device. In host code the name g_res_scratch is only a
// host-side stand-in for the symbol, so the address is looked up with cudaGetSymbolAddress,
// once per device, with that device current.
static double *g_scratch_addr[256];
static std::mutex g_scratch_mutex;

static cudaError_t scratch_for_current_device(double **ptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_res_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *ptr = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace dugks

using namespace dugks;

// Failures are reported through dugks_last_error(NULL), as for dugks_create.
static thread_local char g_static_err[256];
static int fail_static(int code) {
    set_null_handle_error(g_static_err);
    return code;
}

extern "C" int dugks_residual_static(int32_t lattice, int32_t store, const void *state, int64_t nx, int64_t ny,
                                     int64_t nz, double rt, double rho0, const double *shift,
                                     const float *shift_field, double *uprev, int32_t have_prev, double *out,
                                     void *stream) {
    const int dim = lattice == DUGKS_D2Q9 ? 2 : 3;
    if (!(lattice == DUGKS_D2Q9 || lattice == DUGKS_D3Q19 || lattice == DUGKS_D3Q27) || store < 0 || store > 3 ||
        !state || !uprev || !out || nx < 1 || ny < 1 || nz < 1 || (dim == 2 && nz != 1) || !(rt > 0) ||
        !(rho0 > 0)) {
        snprintf(g_static_err, sizeof g_static_err, "dugks_residual_static: invalid argument");
        return fail_static(DUGKS_E_INVAL);
    }
    const int64_t ncell = nx * ny * nz;
    if (ncell > STATIC_RES_MAX_CELLS) {
        snprintf(g_static_err, sizeof g_static_err,
                 "dugks_residual_static: %lld cells exceed the static scratch limit of %lld cells (4096 partial-sum blocks of at most 4096 cells)",
                 (long long)ncell, (long long)STATIC_RES_MAX_CELLS);
        return fail_static(DUGKS_E_INVAL);
    }
    double *scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) {
        snprintf(g_static_err, sizeof g_static_err, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return fail_static(DUGKS_E_CUDA);
    }
    const int nblocks = residual_blocks(ncell);  // <= STATIC_RES_MAX_BLOCKS
    double *partials = scratch;                               // [nblocks][8], fully rewritten
    double *final_sum = scratch + (int64_t)STATIC_RES_MAX_BLOCKS * 8;  // [8], fully rewritten

    // Unpadded layout [Q][nz][ny][nx]; the velocity shift u = c/rho0 sum e g + shift (+
    // shift_field per cell) is passed through the reduction's force slots with dt = 2 and
    // omega = 0 (so the kernel's G dt/2 cos(omega t) factor is exactly the shift). The model
    // field stays 0: the incompressible model's u = c j / rho0 + shift.
    StepParams p;
    memset(&p, 0, sizeof p);
    p.nx = (int)nx;
    p.ny = (int)ny;
    p.nz = (int)nz;
    p.px = nx;
    p.plane = nx * ny;
    p.dstride = nx * ny * nz;
    p.rho0 = rho0;
    p.inv_c = 1.0 / sqrt(3.0 * rt);
    for (int a = 0; a < 3; a++) p.g[a] = shift ? shift[a] : 0.0;
    p.field = shift_field;
    p.omega = 0.0;
    p.dt = 2.0;
    p.src = state;
    cudaStream_t st = (cudaStream_t)stream;
    e = launch_residual(lattice, store, p, 0.0, rt, uprev, have_prev ? 1 : 0, partials, nblocks, final_sum, st);
    double s[8];
    if (e == cudaSuccess) e = cudaMemcpyAsync(s, final_sum, sizeof s, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        snprintf(g_static_err, sizeof g_static_err, "reduction: %s", cudaGetErrorString(e));
        return fail_static(DUGKS_E_CUDA);
    }
    out[0] = have_prev ? (s[1] > 0 ? sqrt(s[0]) / sqrt(s[1]) : (s[0] > 0 ? INFINITY : 0.0)) : INFINITY;
    out[1] = s[2];
    for (int a = 0; a < dim; a++) out[2 + a] = s[3 + a];
    for (int i = 0; i < 3 + dim; i++)
        if (!isfinite(s[i])) {
            snprintf(g_static_err, sizeof g_static_err, "non-finite moments (slot %d)", i);
            return fail_static(DUGKS_E_UNSTABLE);
        }
    return DUGKS_OK;
}
