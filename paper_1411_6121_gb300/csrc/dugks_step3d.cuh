// dugks_step3d.cuh -- throughput kernel of the fused DUGKS time step for 3D velocity sets
// (D3Q19) on sm_103a, FP32 arithmetic, F32/BF16/F16 storage.
//
// Same scheme and the same readings as the reference kernel in dugks_step.cuh (Appendix
// steps 1-10 of arXiv 1411.6121); what differs is how the work is organised:
//
//  * A CTA is 32 x RY threads, one per cell column; the 30 x (RY-2) inner columns are
//    updated, the outer ring is halo. The CTA marches through its z range keeping fbar+
//    (step 1) of three planes in a shared-memory ring.
//  * Step 3-4 reconstruction is split per cell. For the interface normal to d between
//    cells L and R (eq. gradient with the cross-point tangential gradients):
//        F_k = alpha_k(L) + beta_k(R),
//        alpha_k = (1/2 + kappa e_dk) fbar+_k - kappa/4 sum_t e_tk C^t_k,
//        beta_k  = (1/2 - kappa e_dk) fbar+_k - kappa/4 sum_t e_tk C^t_k,
//    with C^t_k the central difference of fbar+_k along the tangential axis t. Only the
//    velocities that cross the interface (e_dk != 0) are formed per direction.
//  * Step 6 interface moments are sums of the same per-cell parts, taken in moment space:
//        sum_k F_k = A0(L) + B0(R),  sum_k e_k F_k = A1(L) + B1(R),
//    A0 = M0/2 + kappa M_d - kappa/4 (E_t1 + E_t2) etc., where M are moments of fbar+ and
//    E moments of the central differences. This avoids reconstructing the velocities that
//    do not cross the interface just to sum them.
//  * Each cell forms the relaxed interface values (step 7) for its +x, +y, +z interfaces;
//    neighbours exchange the beta parts and the finished interface values through shared
//    memory, so every interface is computed once and both cells use the same bits.
//  * Wall interfaces (and the chunk's first z interface) take the direct path of
//    dugks_step.cuh: all velocities reconstructed from the ring, NEQ (step 5), relax.
#pragma once

#include "dugks_step.cuh"

namespace dugks {

template <int Q, int RY>
struct Shape3 {
    static constexpr int D = 3;
    static constexpr int RX = 32;
    static constexpr int NT = RX * RY;
    static constexpr int TXI = RX - 2, TYI = RY - 2;  // inner columns
    static constexpr int NF = n_flux<Q>(0);           // same for every axis
    static constexpr int XS = (2 * (NF + 4)) | 1;     // exchange slots per cell (odd stride)
    static constexpr int PLANE = RY * RX * Q;
    static constexpr size_t smem_floats = 3 * (size_t)PLANE + (size_t)NT * XS;
    static constexpr size_t smem_bytes = smem_floats * sizeof(float);
};

// Moments of fbar+ of one cell.
struct Mom {
    float M0, M1[3], M2[3][3];
};

// Moments of fbar+ of one cell: M0, M1[a] = sum e_a f, M2[a][b] = sum e_a e_b f.
template <int Q>
__device__ __forceinline__ void phi_moments(const float f[Q], float &M0, float M1[3], float M2[3][3]) {
    M0 = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        M1[a] = 0.0f;
#pragma unroll
        for (int b = 0; b < 3; b++) M2[a][b] = 0.0f;
    }
#pragma unroll
    for (int k = 0; k < Q; k++) {
        M0 += f[k];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (Lat<Q>::e(k, a) > 0) M1[a] += f[k];
            if (Lat<Q>::e(k, a) < 0) M1[a] -= f[k];
#pragma unroll
            for (int b = a; b < 3; b++) {
                const int s = Lat<Q>::e(k, a) * Lat<Q>::e(k, b);
                if (s > 0) M2[a][b] += f[k];
                if (s < 0) M2[a][b] -= f[k];
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < a; b++) M2[a][b] = M2[b][a];
}

// Moments of the central differences along t: E0 = sum_k e_tk C_k, E1[a] = sum_k e_ak e_tk C_k
// (C_k defined for e_tk != 0).
template <int Q, int t>
__device__ __forceinline__ void diff_moments(const float C[Q], float &E0, float E1[3]) {
    E0 = 0.0f;
    E1[0] = E1[1] = E1[2] = 0.0f;
#pragma unroll
    for (int k = 0; k < Q; k++) {
        if (Lat<Q>::e(k, t) == 0) continue;
        const float c = Lat<Q>::e(k, t) > 0 ? C[k] : -C[k];  // e_t C
        E0 += c;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (Lat<Q>::e(k, a) > 0) E1[a] += c;
            if (Lat<Q>::e(k, a) < 0) E1[a] -= c;
        }
    }
}

// Per-cell parts of the interface normal to d (see the file comment). ph: fbar+ of the
// cell; C1, C2: central differences along the tangential axes t1 < t2; E: their moments.
// Writes alpha, beta (compact flux index) and A = (A0, A1[3]), B = (B0, B1[3]).
template <int Q, int d>
__device__ __forceinline__ void face_parts(const float ph[Q], const float C1[Q], const float C2[Q], float E01,
                                           const float E11[3], float E02, const float E12[3], float M0,
                                           const float M1[3], const float M2[3][3], float kappa, float *alpha,
                                           float *beta, float A[4], float B[4]) {
    constexpr int t1 = d == 0 ? 1 : 0;
    constexpr int t2 = d == 2 ? 1 : 2;
    const float qk = -0.25f * kappa;
    const float g0 = qk * (E01 + E02);
    A[0] = fmaf(0.5f, M0, fmaf(kappa, M1[d], g0));
    B[0] = fmaf(0.5f, M0, fmaf(-kappa, M1[d], g0));
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float g1 = qk * (E11[a] + E12[a]);
        A[1 + a] = fmaf(0.5f, M1[a], fmaf(kappa, M2[a][d], g1));
        B[1 + a] = fmaf(0.5f, M1[a], fmaf(-kappa, M2[a][d], g1));
    }
    sfor<Q>([&](auto kc) {
        constexpr int k = kc;
        if constexpr (Lat<Q>::e(k, d) != 0) {
            constexpr int i = flux_index<Q>(d, k);
            float tg = 0.0f;
            if constexpr (Lat<Q>::e(k, t1) != 0) tg = Lat<Q>::e(k, t1) > 0 ? C1[k] : -C1[k];
            if constexpr (Lat<Q>::e(k, t2) != 0) tg += Lat<Q>::e(k, t2) > 0 ? C2[k] : -C2[k];
            const float gam = qk * tg;
            constexpr float ed = (float)Lat<Q>::e(k, d);
            alpha[i] = fmaf(fmaf(kappa, ed, 0.5f), ph[k], gam);
            beta[i] = fmaf(fmaf(-kappa, ed, 0.5f), ph[k], gam);
        }
    });
}

// Step 6-7 for the crossing velocities of the interface normal to d from its step-4 values
// F (compact) and moments (drho, j): f = F + b7 (geq - F) + c7 S.
template <int Q, int d, bool FORCE>
__device__ __forceinline__ void face_relax(const Coef<float> &cf, const float *F, float drho, const float j[3],
                                           const float Gh[3], float *out) {
    float m[3];
#pragma unroll
    for (int a = 0; a < 3; a++) m[a] = FORCE ? fmaf(Gh[a], cf.wface * cf.rho0, j[a]) : j[a];
    const float mm = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
    const float base = fmaf(-1.5f * cf.inv_rho0, mm, drho);
    float gm = 0.0f;
    if (FORCE) gm = (Gh[0] * m[0] + Gh[1] * m[1] + Gh[2] * m[2]) * cf.inv_rho0;
    sfor<Q>([&](auto kc) {
        constexpr int k = kc;
        if constexpr (Lat<Q>::e(k, d) != 0) {
            float em = 0.0f, ge = 0.0f;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                if (Lat<Q>::e(k, a) > 0) { em += m[a]; if (FORCE) ge += Gh[a]; }
                if (Lat<Q>::e(k, a) < 0) { em -= m[a]; if (FORCE) ge -= Gh[a]; }
            }
            constexpr int i = flux_index<Q>(d, k);
            constexpr float w = Lat<Q>::w(k);
            // interface values need no conservation-exact form (the same value is used by
            // both cells, so the flux telescopes exactly whatever its rounding)
            const float geq = w * fmaf(em, 3.0f, fmaf(cf.inv_rho0 * em, 4.5f * em, base));
            float v = fmaf(cf.b7, geq - F[i], F[i]);
            if (FORCE) v = fmaf(cf.c7 * 3.0f * (ge - gm), fmaf(w, cf.rho0, geq), v);
            out[i] = v;
        }
    });
}

template <int Q, class S, int RY, bool FORCE>
__global__ void __launch_bounds__(32 * RY, 1) fused_step3d(const __grid_constant__ StepParams p, int zchunk) {
    using K = Shape3<Q, RY>;
    constexpr int NF = K::NF;
    constexpr int XS = K::XS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *phi = reinterpret_cast<float *>(smem_raw);  // [3][RY][32][Q]
    float *xch = phi + 3 * K::PLANE;                   // [RY][32][XS]
    const Coef<float> cf(p);

    const int lane = threadIdx.x, row = threadIdx.y;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int x0 = blockIdx.x * K::TXI, y0 = blockIdx.y * K::TYI;
    const int gx = x0 - 1 + lane, gy = y0 - 1 + row;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(nz, z0 + zchunk);
    const int64_t ncell = (int64_t)nx * ny * nz;
    const bool perx = p.bc[0] == 0, pery = p.bc[2] == 0, perz = p.bc[4] == 0;
    const S *src = reinterpret_cast<const S *>(p.src);
    S *dst = reinterpret_cast<S *>(p.dst);

    // column classification
    const bool inner = lane >= 1 && lane <= K::TXI && row >= 1 && row <= K::TYI;
    const bool own_real = gx >= 0 && gx < nx && gy >= 0 && gy < ny;       // a cell of the domain
    const bool upd = inner && own_real;                                  // this thread updates cells
    int cx = gx, cy = gy;                                                // column whose data is loaded
    bool load = true;                                                    // real or periodic image
    if (gx < 0 || gx >= nx) { if (perx && gx >= -1 && gx <= nx) cx = wrap_idx(gx, nx); else load = false; }
    if (gy < 0 || gy >= ny) { if (pery && gy >= -1 && gy <= ny) cy = wrap_idx(gy, ny); else load = false; }
    const bool xghost = !perx && (gx == -1 || gx == nx) && ((gy >= 0 && gy < ny) || (pery && gy >= -1 && gy <= ny));
    const bool yghost = !pery && (gy == -1 || gy == ny) && gx >= -1 && gx <= nx;
    const bool xwall_tile = !perx && (x0 == 0 || x0 + K::TXI >= nx);
    const bool ywall_tile = !pery && (y0 == 0 || y0 + K::TYI >= ny);

    float ct = (float)p.inv_c, cth = (float)p.inv_c;
    if (FORCE && p.omega != 0.0) {
        const double tn = ((double)(*p.step_ctr) + (double)p.step_off) * p.dt;
        ct = (float)(cos(p.omega * tn) * p.inv_c);
        cth = (float)(cos(p.omega * (tn + 0.5 * p.dt)) * p.inv_c);
    }

    auto P = [&](int slot, int r, int l) __attribute__((always_inline)) -> float * { return phi + ((slot * RY + r) * 32 + l) * Q; };
    auto slot_of = [](int pz) __attribute__((always_inline)) { return (pz + 3) % 3; };
    auto X = [&](int r, int l) __attribute__((always_inline)) -> float * { return xch + (r * 32 + l) * XS; };

    // cell G / c (with time factor) at (x, y, z) of the domain
    auto cellG = [&](int x, int y, int z, float Gh[3]) __attribute__((always_inline)) {
        const int64_t c = (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
        cell_G<3, float>(p, c, ncell, ct, Gh);
    };
    // interface G / c at time t+h: mean of the two cells (one cell at a wall)
    auto faceG = [&](int d, int x, int y, int z, float Gh[3]) __attribute__((always_inline)) {
        // interface between (x,y,z) - e_d and (x,y,z)
        int lo[3] = {x, y, z}, hi[3] = {x, y, z};
        const int nd = d == 0 ? nx : (d == 1 ? ny : nz);
        const bool per = d == 0 ? perx : (d == 1 ? pery : perz);
        lo[d] -= 1;
        if (per) { lo[d] = wrap_idx(lo[d], nd); hi[d] = wrap_idx(hi[d], nd); }
        else { lo[d] = max(lo[d], 0); hi[d] = min(hi[d], nd - 1); }
        const int64_t il = (int64_t)lo[0] + (int64_t)nx * ((int64_t)lo[1] + (int64_t)ny * lo[2]);
        const int64_t ih = (int64_t)hi[0] + (int64_t)nx * ((int64_t)hi[1] + (int64_t)ny * hi[2]);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            float v = (float)p.g[a];
            if (p.field) v += 0.5f * (__ldg(p.field + a * ncell + il) + __ldg(p.field + a * ncell + ih));
            Gh[a] = v * cth;
        }
    };

    // ---- step 1 for the own column at plane pz into the ring (returns the moments) ----
    auto make_phi = [&](int pz) __attribute__((always_inline)) -> Mom {
        Mom r;
        float *o = P(slot_of(pz), row, lane);
        if (!load) {
#pragma unroll
            for (int k = 0; k < Q; k++) o[k] = 0.0f;
            r.M0 = 0.0f;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                r.M1[a] = 0.0f;
#pragma unroll
                for (int b = 0; b < 3; b++) r.M2[a][b] = 0.0f;
            }
            return r;
        }
        const int gz = wrap_idx(pz, nz);
        const int64_t off = (int64_t)gz * p.plane + (int64_t)cy * p.px + cx;
        float g[Q];
#pragma unroll
        for (int k = 0; k < Q; k++) g[k] = (float)Store<S>::ld(src + k * p.dstride + off);
        float Gh[3] = {0.0f, 0.0f, 0.0f}, drho, m[3];
        if (FORCE) cellG(cx, cy, gz, Gh);
        moments<Q, float>(g, Gh, cf.wcell * cf.rho0, drho, m);
        float f[Q];
        relax<Q, float>(g, drho, m, Gh, cf.rho0, cf.inv_rho0, cf.b1, cf.c1, f);
#pragma unroll
        for (int k = 0; k < Q; k++) o[k] = f[k];
        phi_moments<Q>(f, r.M0, r.M1, r.M2);
        return r;
    };
    auto ring_moments = [&](int pz) __attribute__((always_inline)) -> Mom {
        Mom r;
        const float *q = P(slot_of(pz), row, lane);
        float fv[Q];
#pragma unroll
        for (int k = 0; k < Q; k++) fv[k] = q[k];
        phi_moments<Q>(fv, r.M0, r.M1, r.M2);
        return r;
    };
    // step 2 in x and y for the ghost columns of a plane (reading R3: linear, x then y)
    auto ghosts_xy = [&](int pz) __attribute__((always_inline)) {
        const int s = slot_of(pz);
        if (xwall_tile) {
            __syncthreads();
            if (xghost) {
                const int d1 = gx < 0 ? 1 : -1;
                float *o = P(s, row, lane);
                const float *a = P(s, row, lane + d1), *b = P(s, row, lane + 2 * d1);
#pragma unroll
                for (int k = 0; k < Q; k++) o[k] = 2.0f * a[k] - b[k];
            }
        }
        if (ywall_tile) {
            __syncthreads();
            if (yghost) {
                const int d1 = gy < 0 ? 1 : -1;
                float *o = P(s, row, lane);
                const float *a = P(s, row + d1, lane), *b = P(s, row + 2 * d1, lane);
#pragma unroll
                for (int k = 0; k < Q; k++) o[k] = 2.0f * a[k] - b[k];
            }
        }
    };
    // step 2 along z: whole plane by extrapolation from the two inner planes (own column)
    auto ghost_z = [&](int pz) __attribute__((always_inline)) {
        float *o = P(slot_of(pz), row, lane);
        const float *a = P(slot_of(pz < 0 ? 0 : nz - 1), row, lane), *b = P(slot_of(pz < 0 ? 1 : nz - 2), row, lane);
#pragma unroll
        for (int k = 0; k < Q; k++) o[k] = 2.0f * a[k] - b[k];
    };

    // central differences of the own column at plane pz along x or y (from the ring)
    auto cdiff_x = [&](int pz, float C[Q]) __attribute__((always_inline)) {
        const int s = slot_of(pz);
        const float *lo = P(s, row, max(lane - 1, 0)), *hi = P(s, row, min(lane + 1, 31));
#pragma unroll
        for (int k = 0; k < Q; k++)
            if (Lat<Q>::e(k, 0) != 0) C[k] = hi[k] - lo[k];
    };
    auto cdiff_y = [&](int pz, float C[Q]) __attribute__((always_inline)) {
        const int s = slot_of(pz);
        const float *lo = P(s, max(row - 1, 0), lane), *hi = P(s, min(row + 1, RY - 1), lane);
#pragma unroll
        for (int k = 0; k < Q; k++)
            if (Lat<Q>::e(k, 1) != 0) C[k] = hi[k] - lo[k];
    };
    auto cdiff_z = [&](int pz, float C[Q]) __attribute__((always_inline)) {
        const float *lo = P(slot_of(pz - 1), row, lane), *hi = P(slot_of(pz + 1), row, lane);
#pragma unroll
        for (int k = 0; k < Q; k++)
            if (Lat<Q>::e(k, 2) != 0) C[k] = hi[k] - lo[k];
    };

    // direct path for one interface (walls, chunk start): all velocities from the ring,
    // NEQ at walls, relax. Interface normal to d, L at (rl, ll, plane pl) and R the next cell.
    auto direct_face = [&](int d, int pl, int gfd, float *out) __attribute__((always_inline)) {
        const int sL = slot_of(pl), sR = d == 2 ? slot_of(pl + 1) : sL;
        const int rl = row, ll = lane;
        auto ptr = [&](int s, int r, int l) __attribute__((always_inline)) -> const float * { return P(s, r, l); };
        auto rec = [&](int sl, int sr, int r, int l, float F[Q]) __attribute__((always_inline)) {
            if (d == 0)
                reconstruct<Q, 0, float>(ptr(sl, r, l), ptr(sl, r, l + 1), ptr(sl, r - 1, l), ptr(sl, r - 1, l + 1),
                                         ptr(sl, r + 1, l), ptr(sl, r + 1, l + 1), ptr(slot_of(pl - 1), r, l),
                                         ptr(slot_of(pl - 1), r, l + 1), ptr(slot_of(pl + 1), r, l),
                                         ptr(slot_of(pl + 1), r, l + 1), cf.kappa, F);
            else if (d == 1)
                reconstruct<Q, 1, float>(ptr(sl, r, l), ptr(sl, r + 1, l), ptr(sl, r, l - 1), ptr(sl, r + 1, l - 1),
                                         ptr(sl, r, l + 1), ptr(sl, r + 1, l + 1), ptr(slot_of(pl - 1), r, l),
                                         ptr(slot_of(pl - 1), r + 1, l), ptr(slot_of(pl + 1), r, l),
                                         ptr(slot_of(pl + 1), r + 1, l), cf.kappa, F);
            else
                reconstruct<Q, 2, float>(ptr(sl, r, l), ptr(sr, r, l), ptr(sl, r, l - 1), ptr(sr, r, l - 1),
                                         ptr(sl, r, l + 1), ptr(sr, r, l + 1), ptr(sl, r - 1, l), ptr(sr, r - 1, l),
                                         ptr(sl, r + 1, l), ptr(sr, r + 1, l), cf.kappa, F);
        };
        float F[Q];
        rec(sL, sR, rl, ll, F);
        const int nd = d == 0 ? nx : (d == 1 ? ny : nz);
        const bool per = d == 0 ? perx : (d == 1 ? pery : perz);
        const int wall = !per && (gfd == 0 || gfd == nd);
        float Gb[3] = {0.0f, 0.0f, 0.0f}, Gc[3] = {0.0f, 0.0f, 0.0f};
        const int fx = d == 0 ? gfd : min(max(gx, 0), nx - 1);
        const int fy = d == 1 ? gfd : min(max(gy, 0), ny - 1);
        const int fz = d == 2 ? gfd : pl;
        if (FORCE) faceG(d, fx, fy, fz, Gb);
        float Fc[Q];
        if (wall) {
            // x_c: the boundary cell's opposite interface, one cell inward
            const int sh = gfd == 0 ? 1 : -1;
            if (d == 0) rec(sL, sR, rl, ll + sh, Fc);
            else if (d == 1) rec(sL, sR, rl + sh, ll, Fc);
            else {
                const int pc = gfd == 0 ? 0 : nz - 2;
                const int cL = slot_of(pc), cR = slot_of(pc + 1);
                reconstruct<Q, 2, float>(ptr(cL, rl, ll), ptr(cR, rl, ll), ptr(cL, rl, ll - 1), ptr(cR, rl, ll - 1),
                                         ptr(cL, rl, ll + 1), ptr(cR, rl, ll + 1), ptr(cL, rl - 1, ll),
                                         ptr(cR, rl - 1, ll), ptr(cL, rl + 1, ll), ptr(cR, rl + 1, ll), cf.kappa, Fc);
            }
            if (FORCE) faceG(d, d == 0 ? gfd + sh : fx, d == 1 ? gfd + sh : fy, d == 2 ? gfd + sh : fz, Gc);
        }
        if (d == 0) interface_f<Q, 0, float>(p, cf, F, Gb, wall, gfd == 0 ? 0 : 1, Fc, Gc, out);
        else if (d == 1) interface_f<Q, 1, float>(p, cf, F, Gb, wall, gfd == 0 ? 0 : 1, Fc, Gc, out);
        else interface_f<Q, 2, float>(p, cf, F, Gb, wall, gfd == 0 ? 0 : 1, Fc, Gc, out);
    };

    // ---------------- prologue: planes z0-1, z0, z0+1 ----------------
    Mom mc, mn;  // moments of fbar+ at the current and the next plane
    {
        for (int pz = z0 - 1; pz <= z0 + 1; pz++) {
            if (!perz && (pz < 0 || pz >= nz)) continue;
            const Mom t = make_phi(pz);
            if (pz == z0) mc = t;
            if (pz == z0 + 1) mn = t;
        }
        for (int pz = z0 - 1; pz <= z0 + 1; pz++) {
            if (!perz && (pz < 0 || pz >= nz)) continue;
            ghosts_xy(pz);
        }
        __syncthreads();
        for (int pz = z0 - 1; pz <= z0 + 1; pz++)
            if (!perz && (pz < 0 || pz >= nz)) ghost_z(pz);
        __syncthreads();
        // ghost columns and ghost planes: moments from the ring
        if (!load) mc = ring_moments(z0);
        if (!load || (!perz && z0 + 1 >= nz)) mn = ring_moments(z0 + 1);
    }
    // carried: alpha_z, A_z of the current plane and f at its -z interface
    float alz[NF], Az[4], fzm[NF];
    if (upd) {
        float C1[Q], C2[Q], E01, E11[3], E02, E12[3], bz[NF], Bz[4];
        cdiff_x(z0, C1);
        cdiff_y(z0, C2);
        diff_moments<Q, 0>(C1, E01, E11);
        diff_moments<Q, 1>(C2, E02, E12);
        face_parts<Q, 2>(P(slot_of(z0), row, lane), C1, C2, E01, E11, E02, E12, mc.M0, mc.M1, mc.M2, cf.kappa, alz,
                         bz, Az, Bz);
        float t[NF];
        direct_face(2, z0 - 1, z0, t);
#pragma unroll
        for (int i = 0; i < NF; i++) fzm[i] = t[i];
    }

    const bool xrow = row >= 1 && row <= K::TYI && gy >= 0 && gy < ny;       // needs x parts
    const bool ycol = lane >= 1 && lane <= K::TXI && gx >= 0 && gx < nx;     // needs y parts
    const bool need_x = xrow && lane <= K::TXI && gx >= -1 && gx < nx;       // owns its +x interface
    const bool need_y = ycol && row <= K::TYI && gy >= -1 && gy < ny;        // owns its +y interface

    for (int kz = z0; kz < z1; kz++) {
        // ---- P2a: z parts of plane kz+1 and the z interface kz+1/2 ----
        float alzn[NF], Azn[4], fzp[NF];
        if (upd) {
            float Cxn[Q], Cyn[Q], Exn0, Exn1[3], Eyn0, Eyn1[3], bezn[NF], Bzn[4];
            cdiff_x(kz + 1, Cxn);
            cdiff_y(kz + 1, Cyn);
            diff_moments<Q, 0>(Cxn, Exn0, Exn1);
            diff_moments<Q, 1>(Cyn, Eyn0, Eyn1);
            face_parts<Q, 2>(P(slot_of(kz + 1), row, lane), Cxn, Cyn, Exn0, Exn1, Eyn0, Eyn1, mn.M0, mn.M1, mn.M2,
                             cf.kappa, alzn, bezn, Azn, Bzn);
            if (!perz && kz + 1 == nz) {
                float t[NF];
                direct_face(2, kz, kz + 1, t);
#pragma unroll
                for (int i = 0; i < NF; i++) fzp[i] = t[i];
            } else {
                float F[NF], jb[3];
#pragma unroll
                for (int i = 0; i < NF; i++) F[i] = alz[i] + bezn[i];
#pragma unroll
                for (int a = 0; a < 3; a++) jb[a] = Az[1 + a] + Bzn[1 + a];
                float Gb[3] = {0.0f, 0.0f, 0.0f};
                if (FORCE) faceG(2, gx, gy, kz + 1, Gb);
                face_relax<Q, 2, FORCE>(cf, F, Az[0] + Bzn[0], jb, Gb, fzp);
            }
        }
        // ---- P2b: x and y parts of plane kz; publish the beta parts ----
        float alx[NF], Ax[4], aly[NF], Ay[4];
        {
            float Cz[Q], Ez0, Ez1[3];
            cdiff_z(kz, Cz);
            diff_moments<Q, 2>(Cz, Ez0, Ez1);
            const float *phk = P(slot_of(kz), row, lane);
            float *x = X(row, lane);
            if (xrow) {
                float Cy[Q], Ey0, Ey1[3], bex[NF], Bx[4];
                cdiff_y(kz, Cy);
                diff_moments<Q, 1>(Cy, Ey0, Ey1);
                face_parts<Q, 0>(phk, Cy, Cz, Ey0, Ey1, Ez0, Ez1, mc.M0, mc.M1, mc.M2, cf.kappa, alx, bex, Ax, Bx);
#pragma unroll
                for (int i = 0; i < NF; i++) x[i] = bex[i];
#pragma unroll
                for (int i = 0; i < 4; i++) x[NF + i] = Bx[i];
            }
            if (ycol) {
                float Cx[Q], Ex0, Ex1[3], bey[NF], By[4];
                cdiff_x(kz, Cx);
                diff_moments<Q, 0>(Cx, Ex0, Ex1);
                face_parts<Q, 1>(phk, Cx, Cz, Ex0, Ex1, Ez0, Ez1, mc.M0, mc.M1, mc.M2, cf.kappa, aly, bey, Ay, By);
#pragma unroll
                for (int i = 0; i < NF; i++) x[NF + 4 + i] = bey[i];
#pragma unroll
                for (int i = 0; i < 4; i++) x[2 * NF + 4 + i] = By[i];
            }
        }
        __syncthreads();

        // ---- P3: +x and +y interfaces of the own cell ----
        float fxp[NF], fyp[NF];
        if (need_x) {
            if (!perx && (gx == -1 || gx == nx - 1)) {
                float t[NF];
                direct_face(0, kz, gx + 1, t);
#pragma unroll
                for (int i = 0; i < NF; i++) fxp[i] = t[i];
            } else {
                const float *nb = X(row, lane + 1);
                float F[NF], jb[3];
#pragma unroll
                for (int i = 0; i < NF; i++) F[i] = alx[i] + nb[i];
#pragma unroll
                for (int a = 0; a < 3; a++) jb[a] = Ax[1 + a] + nb[NF + 1 + a];
                float Gb[3] = {0.0f, 0.0f, 0.0f};
                if (FORCE) faceG(0, gx + 1, gy, kz, Gb);
                face_relax<Q, 0, FORCE>(cf, F, Ax[0] + nb[NF], jb, Gb, fxp);
            }
        }
        if (need_y) {
            if (!pery && (gy == -1 || gy == ny - 1)) {
                float t[NF];
                direct_face(1, kz, gy + 1, t);
#pragma unroll
                for (int i = 0; i < NF; i++) fyp[i] = t[i];
            } else {
                const float *nb = X(row + 1, lane) + NF + 4;
                float F[NF], jb[3];
#pragma unroll
                for (int i = 0; i < NF; i++) F[i] = aly[i] + nb[i];
#pragma unroll
                for (int a = 0; a < 3; a++) jb[a] = Ay[1 + a] + nb[NF + 1 + a];
                float Gb[3] = {0.0f, 0.0f, 0.0f};
                if (FORCE) faceG(1, gx, gy + 1, kz, Gb);
                face_relax<Q, 1, FORCE>(cf, F, Ay[0] + nb[NF], jb, Gb, fyp);
            }
        }
        __syncthreads();
        {
            float *x = X(row, lane);
            if (need_x)
#pragma unroll
                for (int i = 0; i < NF; i++) x[i] = fxp[i];
            if (need_y)
#pragma unroll
                for (int i = 0; i < NF; i++) x[NF + 4 + i] = fyp[i];
        }
        __syncthreads();

        // ---- P4: steps 8-9, update of cell (gx, gy, kz) ----
        if (upd) {
            const float *xm = X(row, lane - 1), *ym = X(row - 1, lane) + NF + 4;
            const float *ph = P(slot_of(kz), row, lane);
            const int64_t off = (int64_t)kz * p.plane + (int64_t)gy * p.px + gx;
            sfor<Q>([&](auto kc) {
                constexpr int k = kc;
                float acc = 0.0f;
                if constexpr (Lat<Q>::e(k, 0) != 0) {
                    constexpr int i = flux_index<Q>(0, k);
                    acc = fmaf((float)Lat<Q>::e(k, 0), fxp[i] - xm[i], acc);
                }
                if constexpr (Lat<Q>::e(k, 1) != 0) {
                    constexpr int i = flux_index<Q>(1, k);
                    acc = fmaf((float)Lat<Q>::e(k, 1), fyp[i] - ym[i], acc);
                }
                if constexpr (Lat<Q>::e(k, 2) != 0) {
                    constexpr int i = flux_index<Q>(2, k);
                    acc = fmaf((float)Lat<Q>::e(k, 2), fzp[i] - fzm[i], acc);
                }
                // eq. f_tilde_+ in increment form, then eq. evolution_equation
                const float gold = (float)Store<S>::ld(src + k * p.dstride + off);
                const float u0 = fmaf(1.0f / 3.0f, ph[k] - gold, ph[k]);
                Store<S>::st(dst + k * p.dstride + off, fmaf(-cf.two_kappa, acc, u0));
            });
#pragma unroll
            for (int i = 0; i < NF; i++) { fzm[i] = fzp[i]; alz[i] = alzn[i]; }
#pragma unroll
            for (int i = 0; i < 4; i++) Az[i] = Azn[i];
        }
        // ---- P1: fbar+ of plane kz+2 into the ring slot of plane kz-1 ----
        mc = mn;
        if (kz + 1 < z1) {
            const int pn = kz + 2;
            __syncthreads();  // every thread is done with the ring slot of kz-1
            if (perz || pn < nz) {
                mn = make_phi(pn);
                ghosts_xy(pn);
                __syncthreads();
                if (!load) mn = ring_moments(pn);
            } else if (pn == nz) {
                ghost_z(pn);
                __syncthreads();
                mn = ring_moments(pn);
            }
        }
    }
}

}  // namespace dugks
