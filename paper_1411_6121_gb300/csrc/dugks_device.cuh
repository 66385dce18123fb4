// dugks_device.cuh -- device-side building blocks of the fused DUGKS time step (sm_103a).
//
// Notation follows Wu, Shi, Chai and Wang (arXiv 1411.6121): f~ cell averages, fbar+ the
// auxiliary distribution of eq. (24), fbar the interface distribution at t + h
// (eq. (21)), f the original distribution at the interface (eq. (20)).
// Storage and arithmetic use the deviation from the rest equilibrium, g = f - W rho0: every
// linear map of the scheme has coefficients summing to one (steps 1, 3, 7, 9) or zero
// (gradients, the closed-surface flux), so the deviation form is the same algebra with
// W rho0 removed; f_eq becomes geq = W [drho + rho0 (3 e.u^ + 4.5 (e.u^)^2 - 1.5 u^2)]
// with u^ = u / c and c = sqrt(3 RT), and the force term S keeps the full f_eq = W rho0 + geq.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace dugks {

// Compile-time loop: f(std::integral_constant<int, i>) for i = 0 .. N-1, so that indices
// derived from i (direction components, compact flux indices) are constant expressions and
// register arrays are never indexed at run time.
template <class F, int... I>
__host__ __device__ __forceinline__ void sfor_impl(F &&f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__host__ __device__ __forceinline__ void sfor(F &&f) {
    sfor_impl(f, std::make_integer_sequence<int, N>{});
}

// ---------------------------------------------------------------------------------
// Velocity sets (Sec. 2.3). Paper index order: x component slowest.
// ---------------------------------------------------------------------------------
template <int Q>
struct Lat;

template <>
struct Lat<9> {
    static constexpr int D = 2;
    __host__ __device__ static constexpr int e(int k, int a) {
        return a == 0 ? k / 3 - 1 : (a == 1 ? k % 3 - 1 : 0);
    }
    template <class T>
    __host__ __device__ static constexpr T wt(int k) {
        return (e(k, 0) == 0 && e(k, 1) == 0) ? T(4) / T(9) : (e(k, 0) == 0 || e(k, 1) == 0) ? T(1) / T(9) : T(1) / T(36);
    }
    __host__ __device__ static constexpr float w(int k) { return wt<float>(k); }
};

template <>
struct Lat<27> {
    static constexpr int D = 3;
    __host__ __device__ static constexpr int e(int k, int a) {
        return a == 0 ? k / 9 - 1 : (a == 1 ? (k / 3) % 3 - 1 : k % 3 - 1);
    }
    __host__ __device__ static constexpr int nnz(int k) {
        return (e(k, 0) != 0) + (e(k, 1) != 0) + (e(k, 2) != 0);
    }
    template <class T>
    __host__ __device__ static constexpr T wt(int k) {
        return nnz(k) == 0 ? T(8) / T(27) : nnz(k) == 1 ? T(2) / T(27) : nnz(k) == 2 ? T(1) / T(54) : T(1) / T(216);
    }
    __host__ __device__ static constexpr float w(int k) { return wt<float>(k); }
};

template <>
struct Lat<19> {
    static constexpr int D = 3;
    // D3Q27 index of the k-th D3Q19 velocity (the 8 corners removed, order kept).
    __host__ __device__ static constexpr int k27(int k) {
        // 1, 3, 4, 5, 7, 9, 10, ..., 17, 19, 21, 22, 23, 25
        return k < 1 ? 1 : k < 4 ? k + 2 : k < 5 ? 7 : k < 14 ? k + 4 : k < 15 ? 19 : k < 18 ? k + 6 : 25;
    }
    __host__ __device__ static constexpr int e(int k, int a) { return Lat<27>::e(k27(k), a); }
    template <class T>
    __host__ __device__ static constexpr T wt(int k) {
        return Lat<27>::nnz(k27(k)) == 0 ? T(1) / T(3) : Lat<27>::nnz(k27(k)) == 1 ? T(1) / T(18) : T(1) / T(36);
    }
    __host__ __device__ static constexpr float w(int k) { return wt<float>(k); }
};

// Index of the velocity opposite to k.
template <int Q>
__host__ __device__ constexpr int opposite(int k) {
    int r = -1;
    for (int j = 0; j < Q; j++)
        if (Lat<Q>::e(j, 0) == -Lat<Q>::e(k, 0) && Lat<Q>::e(j, 1) == -Lat<Q>::e(k, 1) &&
            Lat<Q>::e(j, 2) == -Lat<Q>::e(k, 2))
            r = j;
    return r;
}

// Number of velocities with a non-zero component along axis d (the directions that carry
// flux through a face normal to d) and the compact index of velocity k among them.
template <int Q>
__host__ __device__ constexpr int n_flux(int d) {
    int n = 0;
    for (int k = 0; k < Q; k++) n += Lat<Q>::e(k, d) != 0;
    return n;
}
template <int Q>
__host__ __device__ constexpr int flux_index(int d, int k) {
    int n = 0;
    for (int j = 0; j < k; j++) n += Lat<Q>::e(j, d) != 0;
    return n;
}

// ---------------------------------------------------------------------------------
// Storage types
// ---------------------------------------------------------------------------------
template <class S>
struct Store;
template <>
struct Store<float> {
    __device__ static __forceinline__ float ld(const float *p) { return __ldg(p); }
    __device__ static __forceinline__ void st(float *p, float v) { *p = v; }
};
template <>
struct Store<__nv_bfloat16> {
    __device__ static __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    __device__ static __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};
template <>
struct Store<double> {
    __device__ static __forceinline__ double ld(const double *p) { return __ldg(p); }
    __device__ static __forceinline__ void st(double *p, double v) { *p = v; }
};
// FP16 holds g~ * 2^12: the exact power-of-two scale moves FP16's normal range
// [6.1e-5, 65504] to [1.5e-8, 16], so slowly developing flows (deviations of 1e-6 and less)
// stay out of the subnormals while any physical deviation still fits.
constexpr float F16_SCALE = 4096.0f, F16_UNSCALE = 1.0f / 4096.0f;
template <>
struct Store<__half> {
    __device__ static __forceinline__ float ld(const __half *p) { return __half2float(__ldg(p)) * F16_UNSCALE; }
    __device__ static __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v * F16_SCALE); }
};

// BF16 keeps 8 significant bits and FP16 11. Rounded to nearest, a slowly varying stored
// value makes nearly the same rounding error at every step, and those errors add up like a
// bias; an increment below half a unit in the last place is lost at every step (a slowly
// accelerating flow stagnates). The state stores therefore round both stochastically
// (unbiased: up with probability equal to the discarded fraction), drawing the random bits
// from a counter-based hash of the destination address and the step. The hash is the 32-bit
// finalizer of MurmurHash3 (A. Appleby).
__device__ __forceinline__ uint32_t mix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}
// Seed of one step's stores (t: the step index).
__device__ __forceinline__ uint32_t store_seed(long long t) { return mix32((uint32_t)t * 0x9e3779b9u + 0x7f4a7c15u); }

// Random bits for the stores of one cell: a 32-bit word per pair of velocities, hashed from
// the step seed and the cell's element offset; velocity k takes the low (k even) or the
// high (k odd) half.
struct CellRandom {
    uint32_t base;
    __device__ __forceinline__ CellRandom(uint32_t seed, int64_t cell) : base(mix32(seed ^ (uint32_t)cell)) {}
    template <int k>
    __device__ __forceinline__ uint32_t bits() const {
        const uint32_t h = mix32(base + (uint32_t)(k >> 1));
        return (k & 1) ? (h >> 16) : h;
    }
    // the whole word of velocities 2 i and 2 i + 1
    template <int i>
    __device__ __forceinline__ uint32_t word() const { return mix32(base + (uint32_t)i); }
};

// Stores a state value: round to nearest for FP32/FP64; stochastic rounding for BF16 and
// FP16 with the random bits r: they are added below the kept significand of the FP32
// pattern, then the pattern is truncated (BF16: 16 bits dropped; FP16: 13, within its
// normal range, which the 2^12 scale covers).
template <class S>
__device__ __forceinline__ void store_state(S *p, typename std::conditional<sizeof(S) == 8, double, float>::type v,
                                            uint32_t r) {
    if constexpr (std::is_same<S, __nv_bfloat16>::value) {
        *p = __ushort_as_bfloat16((unsigned short)((__float_as_uint(v) + (r & 0xffffu)) >> 16));
    } else if constexpr (std::is_same<S, __half>::value) {
        *p = __float2half_rz(__uint_as_float(__float_as_uint(v * F16_SCALE) + (r & 0x1fffu)));
    } else {
        Store<S>::st(p, v);
    }
}

// Stores two state values, v0 at p0 and v1 at p1 (usually two velocities of one cell). For BF16
// and FP16 one hardware conversion rounds both stochastically (cvt.rs.satfinite.{bf16,f16}x2:
// the random bits r[31:16] round v0 and r[15:0] round v1, up with probability equal to the
// discarded fraction); FP16 holds the value times 2^12 (its normal range then spans
// [1.5e-8, 16], which the state never leaves). FP32 stores round to nearest.
template <class S>
__device__ __forceinline__ void store_state_pair(S *p0, float v0, S *p1, float v1, uint32_t r) {
    if constexpr (std::is_same<S, __nv_bfloat16>::value) {
        uint32_t d;
        asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v0), "f"(v1), "r"(r));
        *p0 = __ushort_as_bfloat16((unsigned short)(d >> 16));
        *p1 = __ushort_as_bfloat16((unsigned short)(d & 0xffffu));
    } else if constexpr (std::is_same<S, __half>::value) {
        uint32_t d;
        asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v0 * F16_SCALE), "f"(v1 * F16_SCALE), "r"(r));
        *p0 = __ushort_as_half((unsigned short)(d >> 16));
        *p1 = __ushort_as_half((unsigned short)(d & 0xffffu));
    } else {
        *p0 = v0;
        *p1 = v1;
    }
}
// The same for one value (the rounding takes r[31:16]).
template <class S>
__device__ __forceinline__ void store_state_one(S *p0, float v0, uint32_t r) {
    if constexpr (std::is_same<S, __nv_bfloat16>::value) {
        uint32_t d;
        asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v0), "f"(0.0f), "r"(r));
        *p0 = __ushort_as_bfloat16((unsigned short)(d >> 16));
    } else if constexpr (std::is_same<S, __half>::value) {
        uint32_t d;
        asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v0 * F16_SCALE), "f"(0.0f), "r"(r));
        *p0 = __ushort_as_half((unsigned short)(d >> 16));
    } else {
        *p0 = v0;
    }
}

// Arithmetic type for a storage type: FP32 for FP32/BF16/F16 storage, FP64 for FP64.
template <class S>
struct Arith { using T = float; };
template <>
struct Arith<double> { using T = double; };

__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }

// Sums of products written as explicit fused multiply-adds: left to the compiler, an
// expression like a*a + b*b may be contracted differently in two instantiations of the same
// code (e.g. with and without the force term), and the bits of a step would then depend on
// the instantiation. v.v over the first D components and the ghost value 2 a - b (step 2).
template <int D, class T>
__device__ __forceinline__ T dotD(const T u[3], const T v[3]) {
    return D == 3 ? fmaT(u[0], v[0], fmaT(u[1], v[1], u[2] * v[2])) : fmaT(u[0], v[0], u[1] * v[1]);
}
template <class T>
__device__ __forceinline__ T ghost_value(T a, T b) { return fmaT(T(2), a, -b); }
// A product rounded on its own (never fused into a later addition).
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
// The correctly rounded reciprocal (the value of 1 / x, without the divide's slow path).
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }

// ---------------------------------------------------------------------------------
// Parameters of one fused step launch (coefficients precomputed on the host in double;
// the kernel rounds them once to its arithmetic type).
// ---------------------------------------------------------------------------------
struct StepParams {
    int nx, ny, nz;
    int64_t px;         // row pitch (elements)
    int64_t plane;      // px * ny
    int64_t dstride;    // plane * nz: distance between directions
    double rho0;
    double inv_c;       // 1 / c
    double a1, b1, c1;  // step 1 (eq. (24)): fbar+ = a1 g~ + b1 geq + c1 S
    double a7, b7, c7;  // step 7 (eq. (20)): f = a7 fbar + b7 geq + c7 S
    double kappa;       // h c / dx: reconstruction (eq. (23))
    double two_kappa;   // dt c / dx: flux (eq. (16))
    double c_over_rho0; // c / rho0: velocity moment
    double wcell;       // dt / 2: force weight in the cell moments (eq. (27))
    double wface;       // h / 2: force weight in the interface moments (Appendix step 6)
    double g[3];        // uniform acceleration
    const float *field;        // [dim][ncell] acceleration field or null
    double omega, dt;          // G(t) = (g + field) cos(omega t)
    const long long *step_ctr; // device step counter: t_n = (*step_ctr + step_off) dt
    int step_off;
    int model;                 // 0: incompressible model (eq. (6)); 1: original DUGKS (eq. (5))
    // non-uniform mesh (Sec. 3.4): per axis a, metric[a] = [wf (n+1) | idc (n+1) | idx (n)]:
    // the weight of the high cell at interface i, 1 / (centre distance across i), 1 / (width
    // of cell i); eg[a][side]: the ghost extrapolation coefficient, ghost = f0 + eg (f1 - f0)
    const double *metric[3];
    double eg[3][2];
    int bc[6];                 // DUGKS_BC_* per face
    double bc_u[6][3];         // wall velocity
    double bc_drho[6];         // pressure condition: rho_a - rho0 = p_w / RT
    double bc_drho1[6];        // its oscillating part: + bc_drho1 cos(omega t)
    // The same wall data and acceleration rounded once to FP32 on the host
    // (finish_step_params), for the FP32 kernels: GB300's FP64 rate is a small fraction of its
    // FP32 rate, so no FP64 operation is left on their per-interface paths. Each is the FP32
    // rounding of the FP64 value the FP64 kernels use.
    float fwm[6][3];           // rho0 u_w / c
    float fwu[6][3];           // u_w / c
    float fdrho[6], fdrho1[6]; // bc_drho, bc_drho1
    float fg[3];               // g
    float fcoef[11];           // rho0, 1/rho0, 1/c, b1, c1, b7, c7, kappa, two_kappa, wcell, wface
    const void *src;
    void *dst;
};

// Fills the FP32 copies above from the FP64 fields (host).
inline void finish_step_params(StepParams &p) {
    for (int w = 0; w < 6; w++) {
        for (int a = 0; a < 3; a++) {
            p.fwm[w][a] = (float)(p.bc_u[w][a] * p.rho0 * p.inv_c);
            p.fwu[w][a] = (float)(p.bc_u[w][a] * p.inv_c);
        }
        p.fdrho[w] = (float)p.bc_drho[w];
        p.fdrho1[w] = (float)p.bc_drho1[w];
    }
    for (int a = 0; a < 3; a++) p.fg[a] = (float)p.g[a];
    const double c[11] = {p.rho0, 1.0 / p.rho0, p.inv_c, p.b1, p.c1, p.b7, p.c7, p.kappa, p.two_kappa, p.wcell, p.wface};
    for (int i = 0; i < 11; i++) p.fcoef[i] = (float)c[i];
}

// Coefficients in the arithmetic type T.
template <class T>
struct Coef {
    T rho0, inv_rho0, inv_c, b1, c1, b7, c7, kappa, two_kappa, wcell, wface;
    T cwh;  // cos(omega (t_n + h)): the time factor of an oscillating wall pressure
    __device__ __forceinline__ explicit Coef(const StepParams &p) : cwh(T(1)) {
        if constexpr (sizeof(T) == 4) {  // rounded on the host (finish_step_params)
            rho0 = p.fcoef[0]; inv_rho0 = p.fcoef[1]; inv_c = p.fcoef[2]; b1 = p.fcoef[3]; c1 = p.fcoef[4];
            b7 = p.fcoef[5]; c7 = p.fcoef[6]; kappa = p.fcoef[7]; two_kappa = p.fcoef[8]; wcell = p.fcoef[9];
            wface = p.fcoef[10];
        } else {
            rho0 = (T)p.rho0; inv_rho0 = (T)(1.0 / p.rho0); inv_c = (T)p.inv_c; b1 = (T)p.b1; c1 = (T)p.c1;
            b7 = (T)p.b7; c7 = (T)p.c7; kappa = (T)p.kappa; two_kappa = (T)p.two_kappa; wcell = (T)p.wcell;
            wface = (T)p.wface;
        }
        if (p.omega != 0.0)
            cwh = (T)cos(p.omega * (((double)(*p.step_ctr) + (double)p.step_off) * p.dt + 0.5 * p.dt));
    }
};

// ---------------------------------------------------------------------------------
// Weights in the arithmetic type. In FP32 a weight like 1/9 carries a relative
// representation error of ~1e-8 that is the same at every step, so the momentum of the
// equilibrium, 3 sum_k W_k e_k e_k . m, would differ from m by a fixed factor and the
// relaxation would drift by that much per step. Splitting each weight into a head and a
// tail (W = hi + lo to ~1e-16) leaves only unbiased rounding.
// ---------------------------------------------------------------------------------
template <int Q, class T>
__device__ __forceinline__ T wmul(int k, T x) {
    // k is a compile-time constant after loop unrolling, so these fold to literals
    const double W = Lat<Q>::template wt<double>(k);
    if constexpr (sizeof(T) == 4) {
        const float hi = (float)W;
        const float lo = (float)(W - (double)hi);
        return fmaf(lo, x, hi * x);
    } else {
        return (T)W * x;
    }
}

// ---------------------------------------------------------------------------------
// Moments of a deviation distribution g = f - W rho0 (eq. (27) / Appendix step 6),
// in units of the particle speed c: drho = sum_k g_k, m = sum_k e_k g_k + rho0 Gh w, where
// Gh = G / c and w the force weight (dt/2 at cells, h/2 at interfaces). The velocity is
// u = c m / rho0. Working with m keeps every constant that feeds back into the momentum
// exactly 1 (no c or 1/rho0 factor inside the relaxation loop).
// ---------------------------------------------------------------------------------
//
// EXACT_J (FP32 only; used for the cell moments of step 1): the momentum sums are formed
// without the rounding of a plain FP32 sum. The cell stage rounds the same way at every step
// of a slowly varying flow, so a momentum rounded at the scale of the largest |g_k| biases
// the momentum that the relaxation aims at, and the bias accumulates over the steps. Each
// g_k is split exactly into a head on the grid of 2^(e-19) and a tail, where 2^e bounds the
// cell's largest |g_k| (Dekker's splitting by adding and subtracting 1.5 * 2^(e+4)); the
// head sums are exact in FP32 (at most 10 terms below 2^(e+4) on that grid) and the tails
// are below 2^(e-20), so m = heads + tails is rounded once, at the scale of m.
template <int Q, class T, bool EXACT_J = false>
__device__ __forceinline__ void moments(const T g[Q], const T rGh[3], T w, T &drho, T m[3]) {
    constexpr int D = Lat<Q>::D;
    T r = T(0), j[3] = {T(0), T(0), T(0)};
    if constexpr (EXACT_J && sizeof(T) == 4) {
        float amax = 0.0f;
#pragma unroll
        for (int k = 0; k < Q; k++) {
            r += g[k];
            if (Lat<Q>::e(k, 0) != 0 || Lat<Q>::e(k, 1) != 0 || Lat<Q>::e(k, 2) != 0) amax = fmaxf(amax, fabsf(g[k]));
        }
        // 1.5 * 2^(E + 5) for amax in [2^E, 2^(E+1)): exponent field + 5, significand 1.5
        const float split = __uint_as_float((__float_as_uint(amax) & 0x7f800000u) + 0x02c00000u);
        float hi[3] = {0.0f, 0.0f, 0.0f}, lo[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int k = 0; k < Q; k++) {
            if (Lat<Q>::e(k, 0) == 0 && Lat<Q>::e(k, 1) == 0 && Lat<Q>::e(k, 2) == 0) continue;
            const float h = __fsub_rn(__fadd_rn(g[k], split), split);
            const float l = __fsub_rn(g[k], h);
#pragma unroll
            for (int a = 0; a < D; a++) {
                if (Lat<Q>::e(k, a) > 0) { hi[a] = __fadd_rn(hi[a], h); lo[a] = __fadd_rn(lo[a], l); }
                if (Lat<Q>::e(k, a) < 0) { hi[a] = __fsub_rn(hi[a], h); lo[a] = __fsub_rn(lo[a], l); }
            }
        }
        drho = r;
#pragma unroll
        for (int a = 0; a < 3; a++) m[a] = (a < D) ? __fadd_rn(hi[a], fmaf(rGh[a], w, lo[a])) : 0.0f;
    } else {
#pragma unroll
        for (int k = 0; k < Q; k++) {
            r += g[k];
#pragma unroll
            for (int a = 0; a < D; a++) {
                if (Lat<Q>::e(k, a) > 0) j[a] += g[k];
                if (Lat<Q>::e(k, a) < 0) j[a] -= g[k];
            }
        }
        drho = r;
#pragma unroll
        for (int a = 0; a < 3; a++) m[a] = (a < D) ? fmaT(rGh[a], w, j[a]) : T(0);
    }
}

// Equilibrium deviation of eq. (6) in the variables above:
//   geq_k = W_k [ drho + 3 e_k.m + (4.5 (e_k.m)^2 - 1.5 m.m) / rho0 ].
template <int Q, class T>
__device__ __forceinline__ T geq_k(int k, T drho, const T m[3], T mm, T inv_rho0) {
    constexpr int D = Lat<Q>::D;
    T em = T(0);
#pragma unroll
    for (int a = 0; a < D; a++) {
        if (Lat<Q>::e(k, a) > 0) em += m[a];
        if (Lat<Q>::e(k, a) < 0) em -= m[a];
    }
    const T x = fmaT(em, T(3), fmaT(inv_rho0 * em, T(4.5) * em, fmaT(T(-1.5) * inv_rho0, mm, drho)));
    return wmul<Q, T>(k, x);
}

// Relaxation with the force term, in increment form (coefficients that sum to one in the
// paper's equations are applied as y = g + b (geq - g) + c S, which keeps exact levels
// exact in finite precision):
//   out_k = g_k + b (geq_k - g_k) + c S_k,  S_k = 3 (Gh.e_k - Gh.m / rho0) (W_k rho0 + geq_k)
// (eq. (9) with G.(xi - u)/RT = 3 (Gh.e - Gh.u/c) for xi = c e, c^2 = 3 RT).
// Step 1 (eq. (24)) uses b = 3h/(2tau+dt), c = 3 tau h/(2tau+dt); step 7
// (eq. (20)) uses b = h/(2tau+h), c = tau h/(2tau+h). FORCE = false drops S
// (G = 0 everywhere). Opposite velocities share e.m and the quadratic part of geq.
// In FP32 the equilibrium is rounded once at the scale of its odd term 3 W e.m: with
// 3W = W3h + W3l and W = Wh + Wl split into heads and tails, geq = W3h e.m + (W3l e.m + W q)
// with the small terms formed first and the odd term added by one fused multiply-add
// (forming W (q + 3 e.m) instead rounds several times at that scale, and at a steady flow
// those roundings repeat from step to step and bias the relaxation).
template <int Q, class T>
__device__ __forceinline__ void geq_pair(int k, T em, T q, T &geq, T &geqb) {
    const double W = Lat<Q>::template wt<double>(k);
    if constexpr (sizeof(T) == 4) {
        const float wh = (float)W, wl = (float)(W - (double)wh);
        const float w3h = (float)(3.0 * W), w3l = (float)(3.0 * W - (double)w3h);
        const float wq = fmaf(wl, q, wh * q);
        geq = fmaf(w3h, em, fmaf(w3l, em, wq));
        geqb = fmaf(-w3h, em, fmaf(-w3l, em, wq));
    } else {
        geq = (T)W * fmaT(em, T(3), q);
        geqb = (T)W * fmaT(em, T(-3), q);
    }
}

template <int Q, class T, bool FORCE = true>
__device__ __forceinline__ void relax(const T g[Q], T drho, const T m[3], const T rGh[3], T rho0, T inv_rho0, T b,
                                      T c, T out[Q]) {
    constexpr int D = Lat<Q>::D;
    const T mm = dotD<D, T>(m, m);
    T gm = T(0);
    if constexpr (FORCE) gm = dotD<D, T>(rGh, m) * inv_rho0;
    const T base = fmaT(T(-1.5) * inv_rho0, mm, drho);
    const T c45 = T(4.5) * inv_rho0;
    sfor<Q>([&](auto kc) {
        constexpr int k = kc;
        constexpr int kb = opposite<Q>(k);
        if constexpr (k <= kb) {  // handle the pair (k, -k) once (k == kb for the rest velocity)
            T em = T(0), ge = T(0);
#pragma unroll
            for (int a = 0; a < D; a++) {
                if (Lat<Q>::e(k, a) > 0) { em += m[a]; if (FORCE) ge += rGh[a]; }
                if (Lat<Q>::e(k, a) < 0) { em -= m[a]; if (FORCE) ge -= rGh[a]; }
            }
            const T q = fmaT(c45 * em, em, base);   // even part of the bracket
            T geq, geqb;
            if constexpr (kb != k) geq_pair<Q, T>(k, em, q, geq, geqb);
            else geq = wmul<Q, T>(k, q);             // the rest velocity (e = 0)
            T v = fmaT(b, geq - g[k], g[k]);
            if constexpr (FORCE) {
                const T feq = fmaT((T)Lat<Q>::template wt<double>(k), rho0, geq);
                v = fmaT(c, T(3) * (ge - gm) * feq, v);
            }
            out[k] = v;
            if constexpr (kb != k) {
                T vb = fmaT(b, geqb - g[kb], g[kb]);
                if constexpr (FORCE) {
                    const T feqb = fmaT((T)Lat<Q>::template wt<double>(kb), rho0, geqb);
                    vb = fmaT(c, T(3) * (-ge - gm) * feqb, vb);
                }
                out[kb] = vb;
            }
        }
    });
}

}  // namespace dugks
