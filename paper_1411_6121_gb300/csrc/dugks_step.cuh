// dugks_step.cuh -- the fused DUGKS time step (Appendix steps 1-10 of arXiv 1411.6121) as
// one kernel per step on sm_103a.
//
// A CTA owns a TX x TY tile of cell columns and marches through its z range (2.5D
// blocking). For every z plane it
//   1. loads g~ for the tile plus a one-cell halo and forms fbar+ (step 1, eq. (24))
//      into a three-plane shared-memory ring, filling wall ghost cells by linear
//      extrapolation (step 2) in the order x, y, z;
//   2. reconstructs fbar at every x, y and z interface of the tile's cells (steps 3-4,
//      eq. (23): two-cell mean, normal difference, cross-point tangential
//      differences), applies the NEQ condition at wall interfaces (step 5, eq. (32)),
//      takes the interface moments (step 6) and forms the original f (step 7,
//      eq. (20)) for the directions that cross the interface;
//   3. updates the cell: f~(t+dt) = 4/3 fbar+ - 1/3 f~ - dt/|V| flux (steps 8-9,
//      eqs. (25) and (16)).
// Each interface value is computed once and used by both adjacent cells, so the discrete
// flux telescopes exactly (mass conservation to rounding).
#pragma once

#include "dugks_device.cuh"

namespace dugks {

template <int Q, int TX, int TY, class T = float>
struct StepShape {
    static constexpr int D = Lat<Q>::D;
    static constexpr int RX = TX + 2, RY = TY + 2;      // tile + halo
    static constexpr int NP = D == 3 ? 3 : 1;           // fbar+ planes held
    static constexpr int NT = TX * TY;
    static constexpr int NFX = n_flux<Q>(0), NFY = n_flux<Q>(1), NFZ = D == 3 ? n_flux<Q>(2) : 1;
    static constexpr int SX = NFX | 1, SY = NFY | 1;    // odd strides: no bank conflicts
    static constexpr int PLANE = RY * RX * Q;
    static constexpr size_t smem_floats = (size_t)NP * PLANE + (size_t)TY * (TX + 1) * SX + (size_t)(TY + 1) * TX * SY;
    static constexpr size_t smem_bytes = smem_floats * sizeof(T);
};

// Step 4 (eq. (23)): fbar(x_b, t+h) = fbar+(x_b) - h xi . sigma_b for every velocity,
// at the interface normal to axis d between cells L and R. fbar+(x_b) is the mean of L and
// R (step 3); the normal gradient is (R - L)/dx; the gradient along a tangential axis t is
// the difference of the two cross points on the interface, each the mean of the 4 cells
// around it (step 3), which reduces to [(L+R)_{t+1} - (L+R)_{t-1}] / (4 dx).
// T1m/T1p (T2m/T2p) point at the (L, R) pairs one cell below/above along the first (second)
// tangential axis; in 2D the second pair is unused.
template <int Q, int d, class T>
__device__ __forceinline__ void reconstruct(const T *L, const T *R, const T *L1m, const T *R1m, const T *L1p,
                                            const T *R1p, const T *L2m, const T *R2m, const T *L2p, const T *R2p,
                                            T kappa, T F[Q]) {
    constexpr int D = Lat<Q>::D;
    constexpr int t1 = d == 0 ? 1 : 0;
    constexpr int t2 = d == 2 ? 1 : 2;
    const T qk = T(0.25) * kappa;
#pragma unroll
    for (int k = 0; k < Q; k++) {
        const T l = L[k], r = R[k];
        T v = mul_rn(T(0.5), l + r);
        if (Lat<Q>::e(k, d) != 0) v = fmaT(-kappa * (T)Lat<Q>::e(k, d), r - l, v);
        if (Lat<Q>::e(k, t1) != 0) v = fmaT(-qk * (T)Lat<Q>::e(k, t1), (L1p[k] + R1p[k]) - (L1m[k] + R1m[k]), v);
        if (D == 3 && Lat<Q>::e(k, t2) != 0)
            v = fmaT(-qk * (T)Lat<Q>::e(k, t2), (L2p[k] + R2p[k]) - (L2m[k] + R2m[k]), v);
        F[k] = v;
    }
}

// Density deviation rho_a - rho0 of a pressure wall at the interface time t_n + h (Sec. 2.4:
// rho_a from the wall pressure p_w(t) = p + p_amp cos(omega t), divided by RT on the host;
// cf.cwh holds the cosine).
template <class T>
__device__ __forceinline__ T wall_drho(const StepParams &p, const Coef<T> &cf, int wid) {
    if constexpr (sizeof(T) == 4) return p.fdrho[wid] + p.fdrho1[wid] * cf.cwh;
    else return (T)p.bc_drho[wid] + (T)p.bc_drho1[wid] * cf.cwh;
}

// Steps 3-4 on a non-uniform mesh (Sec. 3.4, the same reading as the oracle): the interface
// value interpolates linearly between the two centres (weight w of the high cell), the normal
// gradient divides their difference by the centre distance, and each tangential gradient
// divides the difference of the interface's two cross points, each bilinear in the four cells
// around it (weights wm, wp of the high row along that axis), by the interface's extent along it:
//   F = M - hc e_d (R - L) idc - sum_t hc e_t (Vp - Vm) idt,  M = (1 - w) L + w R,
//   Vp = (1 - wp) M + wp Mp,  Vm = (1 - wm) Mm + wm M.
// hcn = h c idc and hct1/hct2 = h c idt. Pointers as in reconstruct (first and, in 3D, second
// tangential pair; the second pair is not read in 2D).
template <int Q, int d, class T>
__device__ __forceinline__ void reconstruct_nu(const T *L, const T *R, const T *L1m, const T *R1m, const T *L1p,
                                               const T *R1p, const T *L2m, const T *R2m, const T *L2p,
                                               const T *R2p, T w, T w1m, T w1p, T w2m, T w2p, T hcn, T hct1,
                                               T hct2, T F[Q]) {
    constexpr int D = Lat<Q>::D;
    constexpr int t1 = d == 0 ? 1 : 0;
    constexpr int t2 = d == 2 ? 1 : 2;
    for (int k = 0; k < Q; k++) {
        const T l = L[k], r = R[k];
        const T mid = fmaT(w, r - l, l);
        T v = mid;
        if (Lat<Q>::e(k, d) != 0) v = fmaT(-hcn * (T)Lat<Q>::e(k, d), r - l, v);
        if (Lat<Q>::e(k, t1) != 0) {
            const T midp = fmaT(w, R1p[k] - L1p[k], L1p[k]), midm = fmaT(w, R1m[k] - L1m[k], L1m[k]);
            const T vp = fmaT(w1p, midp - mid, mid), vm = fmaT(w1m, mid - midm, midm);
            v = fmaT(-hct1 * (T)Lat<Q>::e(k, t1), vp - vm, v);
        }
        if (D == 3 && Lat<Q>::e(k, t2) != 0) {
            const T midp = fmaT(w, R2p[k] - L2p[k], L2p[k]), midm = fmaT(w, R2m[k] - L2m[k], L2m[k]);
            const T vp = fmaT(w2p, midp - mid, mid), vm = fmaT(w2m, mid - midm, midm);
            v = fmaT(-hct2 * (T)Lat<Q>::e(k, t2), vp - vm, v);
        }
        F[k] = v;
    }
}

// The model switch of the reference path. For the incompressible model (eq. (6),
// eq. (27)) the momentum variable is m = rho0 u / c and f_eq, S divide by rho0;
// returns 1/rho0. For the original DUGKS (p.model == 1: eq. (5), rho u = sum xi f~ + rho G w)
// m = rho u / c: the force shift that moments() applied with rho0 is completed to
// rho = rho0 + drho, and 1/rho is returned for f_eq and S. ORIG = false compiles the switch
// out (kernels that only run the incompressible model).
template <class T, bool ORIG = true>
__device__ __forceinline__ T original_model(const StepParams &p, const Coef<T> &cf, const T Gh[3], T w, T drho,
                                            T m[3]) {
    if (!ORIG || p.model != 1) return cf.inv_rho0;
#pragma unroll
    for (int a = 0; a < 3; a++) m[a] = fmaT(Gh[a], w * drho, m[a]);
    return rcp_rn(cf.rho0 + drho);
}

// Steps 5-7 at one interface normal to axis d. F: step-4 values (modified in place by the
// wall condition, NEQ or bounce-back, when wall != 0). Fc: step-4 values at x_c, the boundary
// cell's opposite interface (read only by NEQ). side: 0 for the low wall (outward normal -e_d),
// 1 for the high wall. Writes the original f of eq. (20) for the velocities with
// e_d != 0 into out[flux_index(d, k)] (stride 1). ORIG as in original_model.
template <int Q, int d, class T, bool ORIG = true>
__device__ __forceinline__ void interface_f(const StepParams &p, const Coef<T> &cf, T F[Q], const T Gh[3], int wall,
                                            int side, const T *Fc, const T Ghc[3], T *out) {
    constexpr int D = Lat<Q>::D;
    if (wall && p.bc[2 * d + side] == 3) {
        // Step 5, eq. (31): F_k = F_-k + 2 rho0 W_k xi_k.u_w / RT for xi . n < 0, i.e.
        // g_k = g_-k + 6 W_k e_k.m_w with m_w = rho0 u_w / c (deviations: W_k = W_-k)
        const int wid = 2 * d + side;
        T mw[3];
#pragma unroll
        for (int a = 0; a < 3; a++) mw[a] = sizeof(T) == 4 ? (T)p.fwm[wid][a] : (T)(p.bc_u[wid][a] * p.rho0 * p.inv_c);
        const int sgn = side == 0 ? -1 : 1;
        sfor<Q>([&](auto kc) {
            constexpr int k = kc;
            if constexpr (Lat<Q>::e(k, d) != 0) {
                if (sgn * Lat<Q>::e(k, d) < 0) {
                    T em = T(0);
#pragma unroll
                    for (int a = 0; a < D; a++) {
                        if (Lat<Q>::e(k, a) > 0) em += mw[a];
                        if (Lat<Q>::e(k, a) < 0) em -= mw[a];
                    }
                    F[k] = F[opposite<Q>(k)] + wmul<Q, T>(k, T(6) * em);
                }
            }
        });
    } else if (wall) {
        // Step 5, eq. (32): f(x_w) = f_eq(rho_a, u_a) + [f(x_c) - f_eq(rho_c, u_c)] for
        // xi . n < 0, applied to fbar (Appendix step 5) with the moments of step 6 at x_c.
        const int wid = 2 * d + side;
        T drc, mc[3];
        moments<Q, T>(Fc, Ghc, cf.wface * cf.rho0, drc, mc);
        const T irc = original_model<T, ORIG>(p, cf, Ghc, cf.wface, drc, mc);
        T dra, ma[3];
        if (p.bc[wid] == 1) {  // velocity condition: u_a = u_w, rho_a = rho_c
            dra = drc;
            // m = rho u / c: rho0 u_w / c, or rho_a u_w / c in the original model
            if (ORIG && p.model == 1) {
                const double ra = p.rho0 + (double)drc;
                ma[0] = (T)(p.bc_u[wid][0] * ra * p.inv_c);
                ma[1] = (T)(p.bc_u[wid][1] * ra * p.inv_c);
                ma[2] = (T)(p.bc_u[wid][2] * ra * p.inv_c);
            } else if constexpr (sizeof(T) == 4) {
                ma[0] = p.fwm[wid][0];
                ma[1] = p.fwm[wid][1];
                ma[2] = p.fwm[wid][2];
            } else {
                ma[0] = (T)(p.bc_u[wid][0] * p.rho0 * p.inv_c);
                ma[1] = (T)(p.bc_u[wid][1] * p.rho0 * p.inv_c);
                ma[2] = (T)(p.bc_u[wid][2] * p.rho0 * p.inv_c);
            }
        } else {               // pressure condition: rho_a = rho0 + p_w/RT, u_a = u_c
            dra = wall_drho<T>(p, cf, wid);
            // m_a = rho0 u_c / c = m_c, or rho_a u_c / c = m_c rho_a / rho_c (original model)
            const T sc = (ORIG && p.model == 1) ? (cf.rho0 + dra) * irc : T(1);
            ma[0] = mc[0] * sc; ma[1] = mc[1] * sc; ma[2] = mc[2] * sc;
        }
        const T ira = (ORIG && p.model == 1) ? rcp_rn(cf.rho0 + dra) : cf.inv_rho0;
        const T mma = dotD<D, T>(ma, ma);
        const T mmc = dotD<D, T>(mc, mc);
        const int sgn = side == 0 ? -1 : 1;
#pragma unroll
        for (int k = 0; k < Q; k++) {
            if (Lat<Q>::e(k, d) == 0) continue;
            if (sgn * Lat<Q>::e(k, d) < 0)
                F[k] = geq_k<Q, T>(k, dra, ma, mma, ira) + (Fc[k] - geq_k<Q, T>(k, drc, mc, mmc, irc));
        }
    }
    // Step 6: interface moments (weight h/2 on G). Step 7: original distribution.
    T drb, mb[3];
    moments<Q, T>(F, Gh, cf.wface * cf.rho0, drb, mb);
    const T irb = original_model<T, ORIG>(p, cf, Gh, cf.wface, drb, mb);
    T t[Q];
    relax<Q, T>(F, drb, mb, Gh, cf.rho0, irb, cf.b7, cf.c7, t);
    sfor<Q>([&](auto kc) {
        constexpr int k = kc;
        if constexpr (Lat<Q>::e(k, d) != 0) out[flux_index<Q>(d, k)] = t[k];
    });
}

__device__ __forceinline__ int wrap_idx(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Acceleration at a cell (unpadded index) in units of c, times the time factor:
// Gh = (g + field) cos(omega t) / c.
template <int D, class T>
__device__ __forceinline__ void cell_G(const StepParams &p, int64_t cell, int64_t ncell, T ct_over_c, T G[3]) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        T v = (a < D) ? (sizeof(T) == 4 ? (T)p.fg[a] : (T)p.g[a]) : T(0);
        if (p.field && a < D) v += (T)__ldg(p.field + a * ncell + cell);
        G[a] = v * ct_over_c;
    }
}

// One tile of the fused step: cells [x0, x0+TX) x [y0, y0+TY) x [z0, z1) of the instance
// described by p, with the CTA's TX*TY threads and its dynamic shared memory.
template <int Q, class S, int TX, int TY, bool NU = false, bool ORIG = true>
__device__ __forceinline__ void step_tile(const StepParams &p, int x0, int y0, int z0, int z1,
                                          unsigned char *smem_raw) {
    using T = typename Arith<S>::T;
    using K = StepShape<Q, TX, TY, T>;
    constexpr int D = K::D;
    constexpr int RX = K::RX, RY = K::RY, NT = K::NT;
    T *smem = reinterpret_cast<T *>(smem_raw);
    T *phi = smem;                                       // [NP][RY][RX][Q]
    T *xf = phi + K::NP * K::PLANE;                      // [TY][TX+1][SX]
    T *yf = xf + TY * (TX + 1) * K::SX;                  // [TY+1][TX][SY]
    const Coef<T> cf(p);

    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = tid / TX;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int64_t ncell = (int64_t)nx * ny * nz;
    const bool perx = p.bc[0] == 0, pery = p.bc[2] == 0, perz = D == 3 ? p.bc[4] == 0 : true;
    const S *src = reinterpret_cast<const S *>(p.src);
    S *dst = reinterpret_cast<S *>(p.dst);

    uint32_t seed = 0;  // stochastic rounding of 16-bit stores
    if constexpr (sizeof(S) == 2) seed = store_seed(*p.step_ctr + p.step_off);
    // time factors of G(t) (reading: cells at t_n, interfaces at t_n + h), over c
    T ct = (T)p.inv_c, cth = (T)p.inv_c;
    if (p.omega != 0.0) {
        const double tn = ((double)(*p.step_ctr) + (double)p.step_off) * p.dt;
        ct = (T)(cos(p.omega * tn) * p.inv_c);
        cth = (T)(cos(p.omega * (tn + 0.5 * p.dt)) * p.inv_c);
    }

    // Non-uniform mesh metrics (Sec. 3.4): interpolation weight of the high cell at interface i
    // of axis a, 1 / centre distance across it, 1 / width of cell i; hc = h c.
    auto mptr = [&](int a) __attribute__((always_inline)) { return a == 0 ? p.metric[0] : (a == 1 ? p.metric[1] : p.metric[2]); };
    auto nax = [&](int a) __attribute__((always_inline)) { return a == 0 ? nx : (a == 1 ? ny : nz); };
    auto mwf = [&](int a, int i) __attribute__((always_inline)) -> T { return (T)__ldg(mptr(a) + i); };
    auto midc = [&](int a, int i) __attribute__((always_inline)) -> T {
        return (T)__ldg(mptr(a) + nax(a) + 1 + i);
    };
    auto midx = [&](int a, int i) __attribute__((always_inline)) -> T {
        return (T)__ldg(mptr(a) + 2 * nax(a) + 2 + i);
    };
    const T hc = NU ? (T)(0.5 * p.dt / p.inv_c) : T(0);
    // z metrics of plane-level quantities (3D only; a 2D mesh has no z block)
    auto zw = [&](int i) __attribute__((always_inline)) -> T { return D == 3 ? mwf(2, i) : T(0); };
    auto zhc = [&](int i) __attribute__((always_inline)) -> T { return D == 3 ? hc * midx(2, i) : T(0); };

    auto slot_of = [](int pz) __attribute__((always_inline)) { return D == 3 ? (pz + 3) % 3 : 0; };
    auto cellp = [&](int slot, int ry, int rx) __attribute__((always_inline)) -> T * { return phi + slot * K::PLANE + (ry * RX + rx) * Q; };

    // ---- step 1 (+ step 2 in x and y) for global plane pz (real or periodic image) ----
    auto make_plane = [&](int pz) __attribute__((always_inline)) {
        const int slot = slot_of(pz);
        const int gz = D == 3 ? wrap_idx(pz, nz) : 0;
        for (int r = tid; r < RX * RY; r += NT) {
            const int rx = r % RX, ry = r / RX;
            int gx = x0 + rx - 1, gy = y0 + ry - 1;
            T *out = cellp(slot, ry, rx);
            bool ok = true;
            if (gx < 0 || gx >= nx) { if (perx && gx >= -1 && gx <= nx) gx = wrap_idx(gx, nx); else ok = false; }
            if (gy < 0 || gy >= ny) { if (pery && gy >= -1 && gy <= ny) gy = wrap_idx(gy, ny); else ok = false; }
            if (!ok) {
#pragma unroll
                for (int k = 0; k < Q; k++) out[k] = T(0);
                continue;
            }
            const int64_t cell = (int64_t)gx + (int64_t)nx * ((int64_t)gy + (int64_t)ny * gz);
            const int64_t off = (int64_t)gz * p.plane + (int64_t)gy * p.px + gx;
            T g[Q];
#pragma unroll
            for (int k = 0; k < Q; k++) g[k] = (T)Store<S>::ld(src + k * p.dstride + off);
            T Gh[3], drho, m[3];
            cell_G<D, T>(p, cell, ncell, ct, Gh);
            moments<Q, T, true>(g, Gh, cf.wcell * cf.rho0, drho, m);
            const T ir = original_model<T, ORIG>(p, cf, Gh, cf.wcell, drho, m);
            relax<Q, T>(g, drho, m, Gh, cf.rho0, ir, cf.b1, cf.c1, out);
        }
        // Step 2 (reading: linear extrapolation ghost = 2 f0 - f1, axis by axis).
        const bool xwall = !perx && (x0 == 0 || x0 + TX >= nx);
        const bool ywall = !pery && (y0 == 0 || y0 + TY >= ny);
        if (xwall) {
            __syncthreads();
            for (int r = tid; r < 2 * RY; r += NT) {
                const int ry = r >> 1, hi = r & 1;
                const int gy = y0 + ry - 1;
                if (!((gy >= 0 && gy < ny) || (pery && gy >= -1 && gy <= ny))) continue;
                const int rx = hi ? nx - x0 + 1 : -x0;  // region index of gx = nx or gx = -1
                if (rx < 0 || rx >= RX) continue;
                const int s1 = hi ? -1 : 1;
                T *o = cellp(slot, ry, rx);
                const T *a = cellp(slot, ry, rx + s1), *b = cellp(slot, ry, rx + 2 * s1);
                if constexpr (NU) {  // linear through the two boundary centres (ghost centre mirrored)
                    const T eg = (T)p.eg[0][hi];
#pragma unroll
                    for (int k = 0; k < Q; k++) o[k] = fmaT(eg, b[k] - a[k], a[k]);
                } else {
#pragma unroll
                    for (int k = 0; k < Q; k++) o[k] = ghost_value(a[k], b[k]);
                }
            }
        }
        if (ywall) {
            __syncthreads();
            for (int r = tid; r < 2 * RX; r += NT) {
                const int rx = r >> 1, hi = r & 1;
                const int gx = x0 + rx - 1;
                if (gx < -1 || gx > nx) continue;
                const int ry = hi ? ny - y0 + 1 : -y0;
                if (ry < 0 || ry >= RY) continue;
                const int s1 = hi ? -1 : 1;
                T *o = cellp(slot, ry, rx);
                const T *a = cellp(slot, ry + s1, rx), *b = cellp(slot, ry + 2 * s1, rx);
                if constexpr (NU) {
                    const T eg = (T)p.eg[1][hi];
#pragma unroll
                    for (int k = 0; k < Q; k++) o[k] = fmaT(eg, b[k] - a[k], a[k]);
                } else {
#pragma unroll
                    for (int k = 0; k < Q; k++) o[k] = ghost_value(a[k], b[k]);
                }
            }
        }
    };
    // z ghost plane (step 2 along z): 2 fbar+(inner) - fbar+(next inner), whole region.
    auto ghost_plane = [&](int pz) __attribute__((always_inline)) {
        const int s = slot_of(pz);
        const int sa = slot_of(pz < 0 ? 0 : nz - 1), sb = slot_of(pz < 0 ? 1 : nz - 2);
        if constexpr (NU) {  // linear through the two boundary centres (ghost centre mirrored)
            const T eg = (T)p.eg[2][pz < 0 ? 0 : 1];
            for (int i = tid; i < K::PLANE; i += NT)
                phi[s * K::PLANE + i] = fmaT(eg, phi[sb * K::PLANE + i] - phi[sa * K::PLANE + i], phi[sa * K::PLANE + i]);
        } else {
            for (int i = tid; i < K::PLANE; i += NT)
                phi[s * K::PLANE + i] = ghost_value(phi[sa * K::PLANE + i], phi[sb * K::PLANE + i]);
        }
    };
    auto plane = [&](int pz) __attribute__((always_inline)) {  // real or periodic planes only
        make_plane(pz);
    };

    // Field index for interface G (reading: mean of the two adjacent cells; at a wall the
    // one adjacent cell).
    auto face_G = [&](int d, int gx, int gy, int gz, int gfd, T G[3]) __attribute__((always_inline)) {
        // gfd: interface index along d (between cells gfd-1 and gfd)
        int nd = d == 0 ? nx : (d == 1 ? ny : nz);
        bool per = d == 0 ? perx : (d == 1 ? pery : perz);
        int lo = gfd - 1, hi = gfd;
        if (per) { lo = wrap_idx(lo, nd); hi = wrap_idx(hi, nd); }
        else { if (lo < 0) lo = 0; if (hi >= nd) hi = nd - 1; }
        int cl[3] = {gx, gy, gz}, ch[3] = {gx, gy, gz};
        cl[d] = lo; ch[d] = hi;
        const int64_t il = (int64_t)cl[0] + (int64_t)nx * ((int64_t)cl[1] + (int64_t)ny * cl[2]);
        const int64_t ih = (int64_t)ch[0] + (int64_t)nx * ((int64_t)ch[1] + (int64_t)ny * ch[2]);
        // non-uniform mesh: linear interpolation to the interface between distinct cells
        const T wh = (NU && lo != hi) ? mwf(d, gfd) : T(0.5);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            T v = (a < D) ? (sizeof(T) == 4 ? (T)p.fg[a] : (T)p.g[a]) : T(0);
            if (p.field && a < D) {
                const T fl = (T)__ldg(p.field + a * ncell + il), fh = (T)__ldg(p.field + a * ncell + ih);
                v += NU ? fmaT(wh, fh - fl, fl) : T(0.5) * (fl + fh);
            }
            G[a] = v * cth;
        }
    };

    // z interface between global planes pl and pl+1 for the thread's own column (3D only).
    auto zface = [&](int pl, int gfz, T *out) __attribute__((always_inline)) {
        if constexpr (D == 3) {
            const int sL = slot_of(pl), sR = slot_of(pl + 1);
            const int gx = min(x0 + lx, nx - 1), gy = min(y0 + ly, ny - 1);
            // the interface between planes a and a + 1 (its index along z is a + 1)
            auto recz = [&](int a, T *out) __attribute__((always_inline)) {
                const int cL = slot_of(a), cR = slot_of(a + 1);
                if constexpr (NU)
                    reconstruct_nu<Q, 2, T>(cellp(cL, ly + 1, lx + 1), cellp(cR, ly + 1, lx + 1), cellp(cL, ly + 1, lx),
                                            cellp(cR, ly + 1, lx), cellp(cL, ly + 1, lx + 2), cellp(cR, ly + 1, lx + 2),
                                            cellp(cL, ly, lx + 1), cellp(cR, ly, lx + 1), cellp(cL, ly + 2, lx + 1),
                                            cellp(cR, ly + 2, lx + 1), mwf(2, a + 1), mwf(0, gx), mwf(0, gx + 1),
                                            mwf(1, gy), mwf(1, gy + 1), hc * midc(2, a + 1), hc * midx(0, gx),
                                            hc * midx(1, gy), out);
                else
                    reconstruct<Q, 2, T>(cellp(cL, ly + 1, lx + 1), cellp(cR, ly + 1, lx + 1), cellp(cL, ly + 1, lx),
                                         cellp(cR, ly + 1, lx), cellp(cL, ly + 1, lx + 2), cellp(cR, ly + 1, lx + 2),
                                         cellp(cL, ly, lx + 1), cellp(cR, ly, lx + 1), cellp(cL, ly + 2, lx + 1),
                                         cellp(cR, ly + 2, lx + 1), cf.kappa, out);
            };
            T F[Q];
            (void)sL;
            (void)sR;
            recz(pl, F);
            T Gb[3];
            face_G(2, gx, gy, 0, gfz, Gb);
            const int wall = !perz && (gfz == 0 || gfz == nz);
            T Fc[Q], Gc[3] = {T(0), T(0), T(0)};
            if (wall) {
                const int pc = gfz == 0 ? 0 : nz - 2;  // x_c between planes pc and pc+1
                recz(pc, Fc);
                face_G(2, gx, gy, 0, gfz == 0 ? 1 : nz - 1, Gc);
            }
            interface_f<Q, 2, T, ORIG>(p, cf, F, Gb, wall, gfz == 0 ? 0 : 1, Fc, Gc, out);
        }
    };

    // ---- prologue: planes z0-1, z0, z0+1 ----
    if constexpr (D == 3) {
        const bool wz = !perz;
        for (int pz = z0 - 1; pz <= z0 + 1; pz++) {
            if (wz && (pz < 0 || pz >= nz)) continue;
            plane(pz);
        }
        __syncthreads();
        for (int pz = z0 - 1; pz <= z0 + 1; pz++) {
            if (wz && (pz < 0 || pz >= nz)) { ghost_plane(pz); }
        }
        __syncthreads();
    } else {
        plane(0);
        __syncthreads();
    }

    T zf_lo[K::NFZ], zf_hi[K::NFZ];
    if constexpr (D == 3) zface(z0 - 1, z0, zf_lo);

    for (int kz = z0; kz < z1; kz++) {
        const int s = slot_of(kz);
        const int sm = slot_of(kz - 1), sp = slot_of(kz + 1);
        // ---- x interfaces of plane kz ----
        for (int f = tid; f < (TX + 1) * TY; f += NT) {
            const int fx = f % (TX + 1), fy = f / (TX + 1);
            const int gfx = x0 + fx, gy = y0 + fy;
            if (gy >= ny || gfx > nx) continue;
            T F[Q];
            if constexpr (NU)
                reconstruct_nu<Q, 0, T>(cellp(s, fy + 1, fx), cellp(s, fy + 1, fx + 1), cellp(s, fy, fx),
                                        cellp(s, fy, fx + 1), cellp(s, fy + 2, fx), cellp(s, fy + 2, fx + 1),
                                        cellp(sm, fy + 1, fx), cellp(sm, fy + 1, fx + 1), cellp(sp, fy + 1, fx),
                                        cellp(sp, fy + 1, fx + 1), mwf(0, gfx), mwf(1, gy), mwf(1, gy + 1),
                                        zw(kz), zw(kz + 1), hc * midc(0, gfx), hc * midx(1, gy), zhc(kz), F);
            else
                reconstruct<Q, 0, T>(cellp(s, fy + 1, fx), cellp(s, fy + 1, fx + 1), cellp(s, fy, fx),
                                     cellp(s, fy, fx + 1), cellp(s, fy + 2, fx), cellp(s, fy + 2, fx + 1),
                                     cellp(sm, fy + 1, fx), cellp(sm, fy + 1, fx + 1), cellp(sp, fy + 1, fx),
                                     cellp(sp, fy + 1, fx + 1), cf.kappa, F);
            T Gb[3];
            face_G(0, gfx, gy, kz, gfx, Gb);
            const int wall = !perx && (gfx == 0 || gfx == nx);
            T Fc[Q], Gc[3] = {T(0), T(0), T(0)};
            if (wall) {
                const int cx = gfx == 0 ? fx + 1 : fx - 1;  // x_c: interface 1 or nx-1
                const int gcx = gfx == 0 ? 1 : nx - 1;
                if constexpr (NU)
                    reconstruct_nu<Q, 0, T>(cellp(s, fy + 1, cx), cellp(s, fy + 1, cx + 1), cellp(s, fy, cx),
                                            cellp(s, fy, cx + 1), cellp(s, fy + 2, cx), cellp(s, fy + 2, cx + 1),
                                            cellp(sm, fy + 1, cx), cellp(sm, fy + 1, cx + 1), cellp(sp, fy + 1, cx),
                                            cellp(sp, fy + 1, cx + 1), mwf(0, gcx), mwf(1, gy), mwf(1, gy + 1),
                                            zw(kz), zw(kz + 1), hc * midc(0, gcx), hc * midx(1, gy), zhc(kz), Fc);
                else
                    reconstruct<Q, 0, T>(cellp(s, fy + 1, cx), cellp(s, fy + 1, cx + 1), cellp(s, fy, cx),
                                         cellp(s, fy, cx + 1), cellp(s, fy + 2, cx), cellp(s, fy + 2, cx + 1),
                                         cellp(sm, fy + 1, cx), cellp(sm, fy + 1, cx + 1), cellp(sp, fy + 1, cx),
                                         cellp(sp, fy + 1, cx + 1), cf.kappa, Fc);
                face_G(0, gfx, gy, kz, gcx, Gc);
            }
            interface_f<Q, 0, T, ORIG>(p, cf, F, Gb, wall, gfx == 0 ? 0 : 1, Fc, Gc, xf + (fy * (TX + 1) + fx) * K::SX);
        }
        // ---- y interfaces of plane kz ----
        for (int f = tid; f < TX * (TY + 1); f += NT) {
            const int fx = f % TX, fy = f / TX;
            const int gx = x0 + fx, gfy = y0 + fy;
            if (gx >= nx || gfy > ny) continue;
            T F[Q];
            if constexpr (NU)
                reconstruct_nu<Q, 1, T>(cellp(s, fy, fx + 1), cellp(s, fy + 1, fx + 1), cellp(s, fy, fx),
                                        cellp(s, fy + 1, fx), cellp(s, fy, fx + 2), cellp(s, fy + 1, fx + 2),
                                        cellp(sm, fy, fx + 1), cellp(sm, fy + 1, fx + 1), cellp(sp, fy, fx + 1),
                                        cellp(sp, fy + 1, fx + 1), mwf(1, gfy), mwf(0, gx), mwf(0, gx + 1),
                                        zw(kz), zw(kz + 1), hc * midc(1, gfy), hc * midx(0, gx), zhc(kz), F);
            else
                reconstruct<Q, 1, T>(cellp(s, fy, fx + 1), cellp(s, fy + 1, fx + 1), cellp(s, fy, fx),
                                     cellp(s, fy + 1, fx), cellp(s, fy, fx + 2), cellp(s, fy + 1, fx + 2),
                                     cellp(sm, fy, fx + 1), cellp(sm, fy + 1, fx + 1), cellp(sp, fy, fx + 1),
                                     cellp(sp, fy + 1, fx + 1), cf.kappa, F);
            T Gb[3];
            face_G(1, gx, gfy, kz, gfy, Gb);
            const int wall = !pery && (gfy == 0 || gfy == ny);
            T Fc[Q], Gc[3] = {T(0), T(0), T(0)};
            if (wall) {
                const int cy = gfy == 0 ? fy + 1 : fy - 1;
                const int gcy = gfy == 0 ? 1 : ny - 1;
                if constexpr (NU)
                    reconstruct_nu<Q, 1, T>(cellp(s, cy, fx + 1), cellp(s, cy + 1, fx + 1), cellp(s, cy, fx),
                                            cellp(s, cy + 1, fx), cellp(s, cy, fx + 2), cellp(s, cy + 1, fx + 2),
                                            cellp(sm, cy, fx + 1), cellp(sm, cy + 1, fx + 1), cellp(sp, cy, fx + 1),
                                            cellp(sp, cy + 1, fx + 1), mwf(1, gcy), mwf(0, gx), mwf(0, gx + 1),
                                            zw(kz), zw(kz + 1), hc * midc(1, gcy), hc * midx(0, gx), zhc(kz), Fc);
                else
                    reconstruct<Q, 1, T>(cellp(s, cy, fx + 1), cellp(s, cy + 1, fx + 1), cellp(s, cy, fx),
                                         cellp(s, cy + 1, fx), cellp(s, cy, fx + 2), cellp(s, cy + 1, fx + 2),
                                         cellp(sm, cy, fx + 1), cellp(sm, cy + 1, fx + 1), cellp(sp, cy, fx + 1),
                                         cellp(sp, cy + 1, fx + 1), cf.kappa, Fc);
                face_G(1, gx, gcy, kz, gcy, Gc);
            }
            interface_f<Q, 1, T, ORIG>(p, cf, F, Gb, wall, gfy == 0 ? 0 : 1, Fc, Gc, yf + (fy * TX + fx) * K::SY);
        }
        // ---- z interface kz+1/2 of the own column ----
        if constexpr (D == 3) zface(kz, kz + 1, zf_hi);
        __syncthreads();

        // ---- steps 8-9: update of cell (lx, ly, kz) ----
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx < nx && gy < ny) {
            const int64_t off = (int64_t)kz * p.plane + (int64_t)gy * p.px + gx;
            const T *ph = cellp(s, ly + 1, lx + 1);
            const T *xm = xf + (ly * (TX + 1) + lx) * K::SX, *xp = xm + K::SX;
            const T *ym = yf + (ly * TX + lx) * K::SY, *yp = ym + TX * K::SY;
            const CellRandom rnd(seed, off);
            // non-uniform mesh: the flux of each axis is divided by the cell's width along it
            const T dcx = NU ? (T)(p.dt / p.inv_c) * midx(0, gx) : T(0);
            const T dcy = NU ? (T)(p.dt / p.inv_c) * midx(1, gy) : T(0);
            const T dcz = (NU && D == 3) ? (T)(p.dt / p.inv_c) * midx(2, kz) : T(0);
            sfor<Q>([&](auto kc) {
                constexpr int k = kc;
                T acc = T(0);
                if constexpr (NU) {
                    T ax = T(0), ay = T(0), az = T(0);
                    if constexpr (Lat<Q>::e(k, 0) != 0) ax = (T)Lat<Q>::e(k, 0) * (xp[flux_index<Q>(0, k)] - xm[flux_index<Q>(0, k)]);
                    if constexpr (Lat<Q>::e(k, 1) != 0) ay = (T)Lat<Q>::e(k, 1) * (yp[flux_index<Q>(1, k)] - ym[flux_index<Q>(1, k)]);
                    if constexpr (D == 3 && Lat<Q>::e(k, 2) != 0) az = (T)Lat<Q>::e(k, 2) * (zf_hi[flux_index<Q>(2, k)] - zf_lo[flux_index<Q>(2, k)]);
                    const T gold = (T)Store<S>::ld(src + k * p.dstride + off);
                    // the flux of each axis divided by the cell's width along it
                    const T v = fmaT(T(1) / T(3), ph[k] - gold, ph[k]) -
                                (D == 3 ? fmaT(dcx, ax, fmaT(dcy, ay, dcz * az)) : fmaT(dcx, ax, dcy * ay));
                    store_state<S>(dst + k * p.dstride + off, v, sizeof(S) == 2 ? rnd.bits<k>() : 0u);
                    return;
                }
                if constexpr (Lat<Q>::e(k, 0) != 0) {
                    constexpr int i = flux_index<Q>(0, k);
                    acc = fmaT((T)Lat<Q>::e(k, 0), xp[i] - xm[i], acc);
                }
                if constexpr (Lat<Q>::e(k, 1) != 0) {
                    constexpr int i = flux_index<Q>(1, k);
                    acc = fmaT((T)Lat<Q>::e(k, 1), yp[i] - ym[i], acc);
                }
                if constexpr (D == 3 && Lat<Q>::e(k, 2) != 0) {
                    constexpr int i = flux_index<Q>(2, k);
                    acc = fmaT((T)Lat<Q>::e(k, 2), zf_hi[i] - zf_lo[i], acc);
                }
                const T gold = (T)Store<S>::ld(src + k * p.dstride + off);
                // eq. (25) in increment form: 4/3 fbar+ - 1/3 f~ = fbar+ + (fbar+ - f~)/3
                const T v = fmaT(T(1) / T(3), ph[k] - gold, ph[k]) - cf.two_kappa * acc;
                store_state<S>(dst + k * p.dstride + off, v, sizeof(S) == 2 ? rnd.bits<k>() : 0u);
            });
        }
        if constexpr (D == 3) {
#pragma unroll
            for (int j = 0; j < K::NFZ; j++) zf_lo[j] = zf_hi[j];
            // next plane kz+2 into the slot of kz-1
            if (kz + 1 < z1) {
                const int pz = kz + 2;
                __syncthreads();  // every thread is done reading the slot of kz-1 and the faces
                if (perz || pz < nz) {
                    plane(pz);
                    __syncthreads();
                } else if (pz == nz) {
                    ghost_plane(pz);
                    __syncthreads();
                }
            }
        }
    }
}

// NU: a non-uniform mesh (p.metric: interface coordinates per axis, Sec. 3.4).
template <int Q, class S, int TX, int TY, bool NU = false>
__global__ void __launch_bounds__(TX *TY) fused_step(const __grid_constant__ StepParams p, int zchunk) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(p.nz, z0 + zchunk);
    step_tile<Q, S, TX, TY, NU>(p, blockIdx.x * TX, blockIdx.y * TY, z0, z1, smem_raw);
}

// Batched form: many independent 2D instances in one persistent launch. params holds two
// descriptors per instance (source/destination buffers swapped: index 2 i + parity); items
// is the work list of (instance, x0, y0) tiles, largest instances first; CTA b takes items
// b, b + gridDim.x, ...
template <int Q, class S, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) fused_step_batch(const StepParams *__restrict__ params,
                                                           const int4 *__restrict__ items, int nitems, int parity) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 w = items[it];
        const StepParams &p = params[2 * w.x + parity];
        step_tile<Q, S, TX, TY>(p, w.y, w.z, 0, 1, smem_raw);
        __syncthreads();  // the next item reuses the shared buffers
    }
}

}  // namespace dugks
