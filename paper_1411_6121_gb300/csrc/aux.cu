// aux.cu -- initialisation, moments and FP64 reductions of the DUGKS state (sm_103a).
// The per-cell sums of 32- and 16-bit states run in compensated FP32; the reductions (residual,
// conservation totals) accumulate in FP64.
#include "dugks_internal.h"

namespace dugks {

// Initial state (Sec. 3: the equilibrium is initialised from the given fields):
// g~ = f_eq(rho0 + p/RT, u) - W rho0 of eq. (6) (eq. (5) for the original model: rho in
// place of rho0 in the velocity part), evaluated in double and rounded once.
template <int Q, class S>
__global__ void init_kernel(const StepParams p, const double *pres, const double *vel, double rt, double c) {
    constexpr int D = Lat<Q>::D;
    const int64_t ncell = (int64_t)p.nx * p.ny * p.nz;
    S *dst = reinterpret_cast<S *>(p.dst);
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < ncell; n += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(n % p.nx);
        const int y = (int)((n / p.nx) % p.ny);
        const int z = (int)(n / ((int64_t)p.nx * p.ny));
        const double drho = pres ? pres[n] / rt : 0.0;
        double uh[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < D; a++) uh[a] = vel ? vel[a * ncell + n] / c : 0.0;
        const double uu = uh[0] * uh[0] + uh[1] * uh[1] + uh[2] * uh[2];
        const int64_t off = (int64_t)z * p.plane + (int64_t)y * p.px + x;
#pragma unroll
        for (int k = 0; k < Q; k++) {
            double eu = 0.0;
            for (int a = 0; a < D; a++) eu += Lat<Q>::e(k, a) * uh[a];
            const double rv = p.model == 1 ? (double)p.rho0 + drho : (double)p.rho0;
            const double g = Lat<Q>::template wt<double>(k) * (drho + rv * (3.0 * eu + 4.5 * eu * eu - 1.5 * uu));
            Store<S>::st(dst + k * p.dstride + off, (typename Arith<S>::T)g);
        }
    }
}

// Cell moments in double from the stored state: drho = sum g, u = c/rho0 sum e g + G dt/2.
template <int Q, class S>
__device__ __forceinline__ void cell_moments_d(const StepParams &p, const S *src, int64_t n, int64_t ncell, double ct,
                                               double dtc, double c, double &drho, double u[3]) {
    constexpr int D = Lat<Q>::D;
    const int x = (int)(n % p.nx);
    const int y = (int)((n / p.nx) % p.ny);
    const int z = (int)(n / ((int64_t)p.nx * p.ny));
    const int64_t off = (int64_t)z * p.plane + (int64_t)y * p.px + x;
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < Q; k++) {
        const double g = (double)Store<S>::ld(src + k * p.dstride + off);
        r += g;
#pragma unroll
        for (int a = 0; a < D; a++) j[a] += Lat<Q>::e(k, a) * g;
    }
    drho = r;
    // u = c j / rho0 + G dt/2 (eq. (27)); c j / rho + G dt/2 in the original model
    const double rd = p.model == 1 ? (double)p.rho0 + r : (double)p.rho0;
    for (int a = 0; a < 3; a++) {
        double G = a < D ? (double)p.g[a] : 0.0;
        if (p.field && a < D) G += (double)p.field[a * ncell + n];
        u[a] = a < D ? c / rd * j[a] + G * ct * dtc : 0.0;
    }
}

// Knuth's TwoSum: s + e == a + b exactly (round to nearest; the intrinsics keep the
// compiler from reassociating or contracting).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Cell sums of a 32- or 16-bit state in FP32, each carried as an unevaluated pair
// (compensated summation with TwoSum): drho = r[0] + r[1], sum_k e_ka g_k = j[a][0] + j[a][1].
// The pair holds the sum to about 2^-48 of sum |g|, as an FP64 sum of the same values would,
// while the FP64 unit (a small fraction of the FP32 rate on this part) stays free.
template <int Q, class S>
__device__ __forceinline__ void cell_sums_f(const StepParams &p, const S *src, int64_t off, float r[2],
                                            float j[3][2]) {
    constexpr int D = Lat<Q>::D;
    r[0] = r[1] = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; a++) j[a][0] = j[a][1] = 0.0f;
#pragma unroll
    for (int k = 0; k < Q; k++) {
        const float g = (float)Store<S>::ld(src + k * p.dstride + off);
        float t, e;
        two_sum(r[0], g, t, e);
        r[0] = t;
        r[1] += e;
#pragma unroll
        for (int a = 0; a < D; a++) {
            if (Lat<Q>::e(k, a) == 0) continue;
            two_sum(j[a][0], Lat<Q>::e(k, a) > 0 ? g : -g, t, e);
            j[a][0] = t;
            j[a][1] += e;
        }
    }
}

// Element offset of cell n (x fastest) in the padded state layout: n itself when the rows carry
// no padding, which spares the 64-bit divisions.
__device__ __forceinline__ int64_t cell_offset(const StepParams &p, int64_t n) {
    if (p.px == p.nx) return n;
    const int x = (int)(n % p.nx);
    const int y = (int)((n / p.nx) % p.ny);
    const int z = (int)(n / ((int64_t)p.nx * p.ny));
    return (int64_t)z * p.plane + (int64_t)y * p.px + x;
}

// Cell moments in double from the stored state: drho = sum g, u = c/rho0 sum e g + G dt/2
// (the sums of 32- and 16-bit states in compensated FP32, converted once). cr0 = c / rho0,
// divided once by the caller (the incompressible model's factor).
template <int Q, class S>
__device__ __forceinline__ void cell_moments_dd(const StepParams &p, const S *src, int64_t n, int64_t ncell, double ct,
                                                double dtc, double c, double cr0, double &drho, double u[3]) {
    if constexpr (sizeof(S) == 8) {
        cell_moments_d<Q, S>(p, src, n, ncell, ct, dtc, c, drho, u);
    } else {
        constexpr int D = Lat<Q>::D;
        float r[2], j[3][2];
        cell_sums_f<Q, S>(p, src, cell_offset(p, n), r, j);
        drho = (double)r[0] + (double)r[1];
        const double cr = p.model == 1 ? c / ((double)p.rho0 + drho) : cr0;
        for (int a = 0; a < 3; a++) {
            double G = a < D ? (double)p.g[a] : 0.0;
            if (p.field && a < D) G += (double)p.field[a * ncell + n];
            u[a] = a < D ? cr * ((double)j[a][0] + (double)j[a][1]) + G * ct * dtc : 0.0;
        }
    }
}

// Moments as FP32 output from a 32- or 16-bit state, without FP64 arithmetic.
template <int Q, class S>
__device__ __forceinline__ void cell_moments_out_f(const StepParams &p, const S *src, int64_t n, int64_t ncell,
                                                   float ctdt, float c_over_rho0, float rt, float *out) {
    constexpr int D = Lat<Q>::D;
    float r[2], j[3][2];
    cell_sums_f<Q, S>(p, src, cell_offset(p, n), r, j);
    out[n] = (r[0] + r[1]) * rt;
    // c / rho0, or c / rho in the original model
    const float cr = p.model == 1 ? c_over_rho0 * (float)p.rho0 / ((float)p.rho0 + (r[0] + r[1])) : c_over_rho0;
#pragma unroll
    for (int a = 0; a < D; a++) {
        float G = (float)p.g[a];
        if (p.field) G += p.field[a * ncell + n];
        out[(a + 1) * ncell + n] = fmaf(cr, j[a][0] + j[a][1], G * ctdt);
    }
}

// Moments (eq. (27)): out[0] = p = (rho - rho0) RT, out[1+a] = u_a; [dim+1][ncell].
template <int Q, class S>
__global__ void moments_kernel(const StepParams p, double ct, double rt, double c, float *out) {
    constexpr int D = Lat<Q>::D;
    const int64_t ncell = (int64_t)p.nx * p.ny * p.nz;
    const S *src = reinterpret_cast<const S *>(p.src);
    if constexpr (sizeof(S) != 8) {
        const float ctdt = (float)(ct * 0.5 * p.dt), cr = (float)(c / p.rho0), rtf = (float)rt;
        for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < ncell; n += (int64_t)gridDim.x * blockDim.x)
            cell_moments_out_f<Q, S>(p, src, n, ncell, ctdt, cr, rtf, out);
    } else {
        for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < ncell;
             n += (int64_t)gridDim.x * blockDim.x) {
            double drho, u[3];
            cell_moments_d<Q, S>(p, src, n, ncell, ct, 0.5 * p.dt, c, drho, u);
            out[n] = (float)(drho * rt);
            for (int a = 0; a < D; a++) out[(a + 1) * ncell + n] = (float)u[a];
        }
    }
}

// Steady-state residual of Sec. 3.1 and conservation totals, in FP64. Per block:
// s[0] = sum |u - u_prev|^2, s[1] = sum |u|^2, s[2] = sum rho, s[3+a] = sum rho0 u_a.
// u_prev is overwritten with u. Deterministic: fixed per-block order, fixed final order.
constexpr int RES_THREADS = 256;
constexpr int RES_SLOTS = 8;

template <int Q, class S>
__global__ void __launch_bounds__(RES_THREADS) residual_kernel(const StepParams p, double ct, double c, double cr0,
                                                                double *uprev, int have_prev, double *partials) {
    constexpr int D = Lat<Q>::D;
    const int64_t ncell = (int64_t)p.nx * p.ny * p.nz;
    const S *src = reinterpret_cast<const S *>(p.src);
    double s[RES_SLOTS] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < ncell; n += (int64_t)gridDim.x * blockDim.x) {
        double drho, u[3];
        cell_moments_dd<Q, S>(p, src, n, ncell, ct, 0.5 * p.dt, c, cr0, drho, u);
        for (int a = 0; a < D; a++) {
            const double du = u[a] - (have_prev ? uprev[a * ncell + n] : 0.0);
            s[0] += du * du;
            s[1] += u[a] * u[a];
            s[3 + a] += (p.model == 1 ? (double)p.rho0 + drho : (double)p.rho0) * u[a];  // rho0 u, or rho u
            uprev[a * ncell + n] = u[a];
        }
        s[2] += (double)p.rho0 + drho;
    }
    __shared__ double red[RES_THREADS / 32][RES_SLOTS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < RES_SLOTS; i++) {
        double v = s[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < RES_SLOTS) {
        double v = 0.0;
        for (int w = 0; w < RES_THREADS / 32; w++) v += red[w][threadIdx.x];
        partials[blockIdx.x * RES_SLOTS + threadIdx.x] = v;
    }
}

__global__ void residual_final(const double *partials, int nblocks, double *out) {
    // one thread per slot, blocks summed in index order
    if (threadIdx.x < RES_SLOTS) {
        double v = 0.0;
        for (int b = 0; b < nblocks; b++) v += partials[b * RES_SLOTS + threadIdx.x];
        out[threadIdx.x] = v;
    }
}

__global__ void advance_kernel(long long *ctr, long long n) { *ctr += n; }

static int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > 65535 * 8 ? 65535 * 8 : b));
}

int residual_blocks(int64_t ncell) {
    int64_t b = (ncell + RES_THREADS * 8 - 1) / (RES_THREADS * 8);
    if (b < 1) b = 1;
    if (b > 4096) b = 4096;
    return (int)b;
}

template <int Q>
static cudaError_t init_q(int store, const StepParams &p, const double *pres, const double *vel, double rt,
                          cudaStream_t st) {
    const int64_t ncell = (int64_t)p.nx * p.ny * p.nz;
    const double c = sqrt(3.0 * rt);
    const int g = grid_for(ncell, 256);
    if (store == 0) init_kernel<Q, float><<<g, 256, 0, st>>>(p, pres, vel, rt, c);
    else if (store == 1) init_kernel<Q, __nv_bfloat16><<<g, 256, 0, st>>>(p, pres, vel, rt, c);
    else if (store == 2) init_kernel<Q, __half><<<g, 256, 0, st>>>(p, pres, vel, rt, c);
    else init_kernel<Q, double><<<g, 256, 0, st>>>(p, pres, vel, rt, c);
    return cudaGetLastError();
}

template <int Q>
static cudaError_t moments_q(int store, const StepParams &p, double t, double rt, float *out, cudaStream_t st) {
    const int64_t ncell = (int64_t)p.nx * p.ny * p.nz;
    const double c = sqrt(3.0 * rt);
    const double ct = cos(p.omega * t);
    const int g = grid_for(ncell, 256);
    if (store == 0) moments_kernel<Q, float><<<g, 256, 0, st>>>(p, ct, rt, c, out);
    else if (store == 1) moments_kernel<Q, __nv_bfloat16><<<g, 256, 0, st>>>(p, ct, rt, c, out);
    else if (store == 2) moments_kernel<Q, __half><<<g, 256, 0, st>>>(p, ct, rt, c, out);
    else moments_kernel<Q, double><<<g, 256, 0, st>>>(p, ct, rt, c, out);
    return cudaGetLastError();
}

template <int Q>
static cudaError_t residual_q(int store, const StepParams &p, double t, double rt, double *uprev, int have_prev,
                              double *partials, int nblocks, double *out, cudaStream_t st) {
    const double c = sqrt(3.0 * rt);
    const double ct = cos(p.omega * t);
    const double cr0 = c / p.rho0;
    if (store == 0) residual_kernel<Q, float><<<nblocks, RES_THREADS, 0, st>>>(p, ct, c, cr0, uprev, have_prev, partials);
    else if (store == 1)
        residual_kernel<Q, __nv_bfloat16><<<nblocks, RES_THREADS, 0, st>>>(p, ct, c, cr0, uprev, have_prev, partials);
    else if (store == 2)
        residual_kernel<Q, __half><<<nblocks, RES_THREADS, 0, st>>>(p, ct, c, cr0, uprev, have_prev, partials);
    else residual_kernel<Q, double><<<nblocks, RES_THREADS, 0, st>>>(p, ct, c, cr0, uprev, have_prev, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    residual_final<<<1, 32, 0, st>>>(partials, nblocks, out);
    return cudaGetLastError();
}

cudaError_t launch_init(int q, int store, const StepParams &p, const double *pres, const double *vel, double rt,
                        cudaStream_t st) {
    switch (q) {
        case 9: return init_q<9>(store, p, pres, vel, rt, st);
        case 19: return init_q<19>(store, p, pres, vel, rt, st);
        case 27: return init_q<27>(store, p, pres, vel, rt, st);
    }
    return cudaErrorNotSupported;
}

cudaError_t launch_moments(int q, int store, const StepParams &p, double t, double rt, float *out, cudaStream_t st) {
    switch (q) {
        case 9: return moments_q<9>(store, p, t, rt, out, st);
        case 19: return moments_q<19>(store, p, t, rt, out, st);
        case 27: return moments_q<27>(store, p, t, rt, out, st);
    }
    return cudaErrorNotSupported;
}

cudaError_t launch_residual(int q, int store, const StepParams &p, double t, double rt, double *uprev,
                            int have_prev, double *partials, int nblocks, double *out, cudaStream_t st) {
    switch (q) {
        case 9: return residual_q<9>(store, p, t, rt, uprev, have_prev, partials, nblocks, out, st);
        case 19: return residual_q<19>(store, p, t, rt, uprev, have_prev, partials, nblocks, out, st);
        case 27: return residual_q<27>(store, p, t, rt, uprev, have_prev, partials, nblocks, out, st);
    }
    return cudaErrorNotSupported;
}

cudaError_t launch_advance(long long *ctr, long long n, cudaStream_t st) {
    advance_kernel<<<1, 1, 0, st>>>(ctr, n);
    return cudaGetLastError();
}

}  // namespace dugks
