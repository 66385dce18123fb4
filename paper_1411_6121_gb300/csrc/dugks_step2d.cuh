// dugks_step2d.cuh -- throughput kernel of the fused DUGKS time step for the D2Q9 velocity
// set on sm_103a, FP32 arithmetic, F32/BF16/F16 storage.
//
// Same scheme and readings as the reference kernel in dugks_step.cuh (Appendix steps 1-10
// of arXiv 1411.6121); the work is organised like the 3D throughput kernel
// (dugks_step3d.cuh), without its z march:
//
//  * A CTA is 32 x RY threads, one per cell (lanes along x, warps along y); the inner
//    30 x (RY-2) cells are updated, the outer ring is halo. fbar+ (step 1) and its six
//    moments are made once per cell into shared memory.
//  * The reconstruction is split per cell, F_k = alpha_k(L) + beta_k(R) with
//        alpha_k = (1/2 + kappa e_dk) fbar+_k - kappa/4 e_tk C_k,
//        beta_k  = (1/2 - kappa e_dk) fbar+_k - kappa/4 e_tk C_k
//    (C_k the central difference of fbar+_k along the tangential axis t), for the six
//    velocities that cross the interface; the interface moments are the same split taken in
//    moment space, A(L) + B(R), from the cells' moments and their tangential differences.
//  * x neighbours exchange beta through warp shuffles, y neighbours through shared memory;
//    every interface is computed once and both cells use the same bits.
//  * Wall interfaces take the direct path of dugks_step.cuh (all nine velocities, NEQ,
//    relax).
// A launch takes either a grid of tiles (one instance) or a work list of (instance, tile)
// items walked by a persistent grid (the batched form).
#pragma once

#include "dugks_step.cuh"

namespace dugks {

template <int RY, class S = float>
struct Shape2 {
    static constexpr int Q = 9;
    static constexpr int RX = 32;
    static constexpr int NT = RX * RY;
    static constexpr int TXI = RX - 2, TYI = RY - 2;  // inner cells
    static constexpr int NF = n_flux<9>(0);           // crossing velocities per interface (6)
    static constexpr int NM = 6;                      // moments kept per cell
    static constexpr int CS = Q + NM;                 // floats per cell (odd: no conflicts)
    static constexpr int BS = (NF + 3) | 1;           // y exchange: beta_y + B_y
    static constexpr int FS = NF | 1;                 // y exchange: f at +y
    static constexpr size_t smem_floats = (size_t)NT * (CS + BS + FS);
    static constexpr size_t smem_bytes = smem_floats * sizeof(float);
};

// Moment slots: 0 M0, 1 M_x, 2 M_y, 3 M_xx, 4 M_yy, 5 M_xy.
__host__ __device__ constexpr int mslot2_2d(int a, int b) { return a == b ? 3 + a : 5; }

// Moments of fbar+ of one cell into m[6], from partial sums over e_a = +1, -1, 0.
__device__ __forceinline__ void phi_moments_2d(const float f[9], float m[6]) {
    float sp[2] = {0.0f, 0.0f}, sn[2] = {0.0f, 0.0f}, s0 = 0.0f, mxy = 0.0f;
    sfor<9>([&](auto kc) {
        constexpr int k = kc;
        constexpr int ex = Lat<9>::e(k, 0), ey = Lat<9>::e(k, 1);
        if constexpr (ex > 0) sp[0] += f[k];
        if constexpr (ex < 0) sn[0] += f[k];
        if constexpr (ex == 0) s0 += f[k];
        if constexpr (ey > 0) sp[1] += f[k];
        if constexpr (ey < 0) sn[1] += f[k];
        if constexpr (ex * ey != 0) mxy += ex * ey > 0 ? f[k] : -f[k];
    });
    m[0] = s0 + (sp[0] + sn[0]);
#pragma unroll
    for (int a = 0; a < 2; a++) {
        m[1 + a] = sp[a] - sn[a];
        m[3 + a] = sp[a] + sn[a];
    }
    m[5] = mxy;
}

// Per-cell parts of the interface normal to d (t = the other axis): alpha, beta for the
// crossing velocities (compact index), A = (A0, A1x, A1y), B likewise. ph: fbar+ of the cell;
// m: its moments; C: per-velocity central differences along t (read for the crossing
// velocities with a component along t); dM: tangential differences of (M_t, M_xt, M_yt).
template <int d>
__device__ __forceinline__ void face_parts_2d(const float *ph, const float *m, const float C[9], const float dM[3],
                                              float kappa, float *alpha, float *beta, float A[3], float B[3]) {
    constexpr int t = 1 - d;
    const float qk = -0.25f * kappa;
    const float g0 = qk * dM[0];
    A[0] = fmaf(0.5f, m[0], fmaf(kappa, m[1 + d], g0));
    B[0] = fmaf(0.5f, m[0], fmaf(-kappa, m[1 + d], g0));
#pragma unroll
    for (int a = 0; a < 2; a++) {
        const float g1 = qk * dM[1 + a];
        const float mad = m[mslot2_2d(a, d)];
        A[1 + a] = fmaf(0.5f, m[1 + a], fmaf(kappa, mad, g1));
        B[1 + a] = fmaf(0.5f, m[1 + a], fmaf(-kappa, mad, g1));
    }
    sfor<9>([&](auto kc) {
        constexpr int k = kc;
        if constexpr (Lat<9>::e(k, d) != 0) {
            constexpr int i = flux_index<9>(d, k);
            constexpr int et = Lat<9>::e(k, t);
            constexpr float ed = (float)Lat<9>::e(k, d);
            const float f = ph[k];
            if constexpr (et != 0) {
                const float gam = qk * (et > 0 ? C[k] : -C[k]);
                alpha[i] = fmaf(fmaf(kappa, ed, 0.5f), f, gam);
                beta[i] = fmaf(fmaf(-kappa, ed, 0.5f), f, gam);
            } else {
                alpha[i] = mul_rn(fmaf(kappa, ed, 0.5f), f);
                beta[i] = mul_rn(fmaf(-kappa, ed, 0.5f), f);
            }
        }
    });
}

// Steps 6-7 for the crossing velocities of the interface normal to d from its step-4 values
// F (compact) and moments (drho, j): f = F + b7 (geq - F) + c7 S; opposite velocities share
// e.m and the quadratic part of geq.
template <int d, bool FORCE>
__device__ __forceinline__ void face_relax_2d(const Coef<float> &cf, const float *F, float drho, const float j[2],
                                              const float Gh[2], float *out) {
    float m[2];
#pragma unroll
    for (int a = 0; a < 2; a++) m[a] = FORCE ? fmaf(Gh[a], cf.wface * cf.rho0, j[a]) : j[a];
    const float m3[3] = {m[0], m[1], 0.0f}, G3[3] = {Gh[0], Gh[1], 0.0f};
    const float mm = dotD<2, float>(m3, m3);
    const float base = fmaf(-1.5f * cf.inv_rho0, mm, drho);
    float gm = 0.0f;
    if (FORCE) gm = dotD<2, float>(G3, m3) * cf.inv_rho0;
    const float c45 = 4.5f * cf.inv_rho0;
    sfor<9>([&](auto kc) {
        constexpr int k = kc;
        constexpr int kb = opposite<9>(k);
        if constexpr (Lat<9>::e(k, d) > 0) {  // the pair (k, kb), e_d = +1 / -1
            float em = 0.0f, ge = 0.0f;
#pragma unroll
            for (int a = 0; a < 2; a++) {
                if (Lat<9>::e(k, a) > 0) { em += m[a]; if (FORCE) ge += Gh[a]; }
                if (Lat<9>::e(k, a) < 0) { em -= m[a]; if (FORCE) ge -= Gh[a]; }
            }
            constexpr int i = flux_index<9>(d, k), ib = flux_index<9>(d, kb);
            constexpr float w = Lat<9>::w(k);
            // interface values need no conservation-exact form (both cells use the same bits)
            const float q = fmaf(c45 * em, em, base);
            const float geq = mul_rn(w, fmaf(em, 3.0f, q)), geqb = mul_rn(w, fmaf(em, -3.0f, q));
            float v = fmaf(cf.b7, geq - F[i], F[i]), vb = fmaf(cf.b7, geqb - F[ib], F[ib]);
            if (FORCE) {
                v = fmaf(cf.c7 * 3.0f * (ge - gm), fmaf(w, cf.rho0, geq), v);
                vb = fmaf(cf.c7 * 3.0f * (-ge - gm), fmaf(w, cf.rho0, geqb), vb);
            }
            out[i] = v;
            out[ib] = vb;
        }
    });
}

// One tile: inner cells [x0, x0 + 30) x [y0, y0 + RY - 2) of the instance p.
template <class S, int RY, bool FORCE>
__device__ __forceinline__ void step2d_tile(const StepParams &p, unsigned char *smem_raw, int x0, int y0) {
    using K = Shape2<RY, S>;
    constexpr int Q = 9, NF = K::NF, CS = K::CS;
    float *cell = reinterpret_cast<float *>(smem_raw);  // [RY][32][CS]: fbar+ then moments
    float *xb = cell + K::NT * CS;                      // [RY][32][BS]: beta_y, B_y
    float *xf = xb + K::NT * K::BS;                     // [RY][32][FS]: f at +y
    const Coef<float> cf(p);

    const int lane = threadIdx.x, row = threadIdx.y;
    const int nx = p.nx, ny = p.ny;
    const int gx = x0 - 1 + lane, gy = y0 - 1 + row;
    const int64_t ncell = (int64_t)nx * ny;
    const bool perx = p.bc[0] == 0, pery = p.bc[2] == 0;
    const S *src = reinterpret_cast<const S *>(p.src);
    S *dst = reinterpret_cast<S *>(p.dst);

    // cell classification (as in the 3D kernel)
    const bool inner = lane >= 1 && lane <= K::TXI && row >= 1 && row <= K::TYI;
    const bool upd = inner && gx < nx && gy < ny;
    int cx = gx, cy = gy;
    bool load = true;
    if (gx < 0 || gx >= nx) { if (perx && gx >= -1 && gx <= nx) cx = wrap_idx(gx, nx); else load = false; }
    if (gy < 0 || gy >= ny) { if (pery && gy >= -1 && gy <= ny) cy = wrap_idx(gy, ny); else load = false; }
    const bool yreal = (gy >= 0 && gy < ny) || (pery && gy >= -1 && gy <= ny);
    const bool xghost = !perx && (gx == -1 || gx == nx) && yreal;
    const bool yghost = !pery && (gy == -1 || gy == ny) && gx >= -1 && gx <= nx;
    const bool xwall_tile = !perx && (x0 == 0 || x0 + K::TXI >= nx);
    const bool ywall_tile = !pery && (y0 == 0 || y0 + K::TYI >= ny);
    const bool need_x = row >= 1 && row <= K::TYI && gy >= 0 && gy < ny && lane <= K::TXI && gx >= -1 && gx < nx;
    const bool ycol = lane >= 1 && lane <= K::TXI && gx >= 0 && gx < nx && gy >= -1 && gy <= ny;
    const bool need_y = ycol && row <= K::TYI && gy < ny;

    uint32_t seed = 0;  // stochastic rounding of 16-bit stores
    if constexpr (sizeof(S) == 2) seed = store_seed(*p.step_ctr + p.step_off);
    float ct = p.fcoef[2], cth = p.fcoef[2];
    if (FORCE && p.omega != 0.0) {
        const double tn = ((double)(*p.step_ctr) + (double)p.step_off) * p.dt;
        ct = (float)(cos(p.omega * tn) * p.inv_c);
        cth = (float)(cos(p.omega * (tn + 0.5 * p.dt)) * p.inv_c);
    }
    auto Rp = [&](int r, int l) __attribute__((always_inline)) -> float * { return cell + (r * 32 + l) * CS; };

    // interface acceleration / c at t+h between (x, y) - e_d and (x, y) (reading R2)
    auto faceG = [&](int d, int x, int y, float Gh[2]) __attribute__((always_inline)) {
        int lo[2] = {x, y}, hi[2] = {x, y};
        const int nd = d == 0 ? nx : ny;
        const bool per = d == 0 ? perx : pery;
        lo[d] -= 1;
        if (per) { lo[d] = wrap_idx(lo[d], nd); hi[d] = wrap_idx(hi[d], nd); }
        else { lo[d] = max(lo[d], 0); hi[d] = min(hi[d], nd - 1); }
        const int64_t il = (int64_t)lo[0] + (int64_t)nx * lo[1], ih = (int64_t)hi[0] + (int64_t)nx * hi[1];
#pragma unroll
        for (int a = 0; a < 2; a++) {
            float v = p.fg[a];
            if (p.field) v += 0.5f * (__ldg(p.field + a * ncell + il) + __ldg(p.field + a * ncell + ih));
            Gh[a] = v * cth;
        }
    };

    // ---- step 1 for the own cell; g and fbar+ stay in registers for the update ----
    float g[Q], f[Q];
    {
        float *o = Rp(row, lane);
        if (load) {
            const int64_t off = (int64_t)cy * p.px + cx;
#pragma unroll
            for (int k = 0; k < Q; k++) g[k] = (float)Store<S>::ld(src + k * p.dstride + off);
            float Gh[3] = {0.0f, 0.0f, 0.0f}, drho, m[3];
            if (FORCE) cell_G<2, float>(p, (int64_t)cx + (int64_t)nx * cy, ncell, ct, Gh);
            moments<Q, float, true>(g, Gh, cf.wcell * cf.rho0, drho, m);
            relax<Q, float, FORCE>(g, drho, m, Gh, cf.rho0, cf.inv_rho0, cf.b1, cf.c1, f);
            float mo[6];
            phi_moments_2d(f, mo);
#pragma unroll
            for (int k = 0; k < Q; k++) o[k] = f[k];
#pragma unroll
            for (int i = 0; i < 6; i++) o[Q + i] = mo[i];
        } else {
#pragma unroll
            for (int k = 0; k < CS; k++) o[k] = 0.0f;
#pragma unroll
            for (int k = 0; k < Q; k++) g[k] = f[k] = 0.0f;
        }
    }
    // step 2 (reading R3: ghost = 2 f0 - f1, x then y): fbar+ and its moments
    if (xwall_tile) {
        __syncthreads();
        if (xghost) {
            const int d1 = gx < 0 ? 1 : -1;
            float *o = Rp(row, lane);
            const float *a = Rp(row, lane + d1), *b = Rp(row, lane + 2 * d1);
#pragma unroll
            for (int k = 0; k < CS; k++) o[k] = ghost_value(a[k], b[k]);
        }
    }
    if (ywall_tile) {
        __syncthreads();
        if (yghost) {
            const int d1 = gy < 0 ? 1 : -1;
            float *o = Rp(row, lane);
            const float *a = Rp(row + d1, lane), *b = Rp(row + 2 * d1, lane);
#pragma unroll
            for (int k = 0; k < CS; k++) o[k] = ghost_value(a[k], b[k]);
        }
    }
    __syncthreads();

    // direct path for one interface (walls): all velocities from shared memory, NEQ, relax.
    // Interface normal to d between the own cell and its +d neighbour; gfd its index along d.
    auto direct_face = [&](int d, int gfd, float *out) {
        auto rec = [&](int r, int l, float F[Q]) __attribute__((always_inline)) {
            // interface normal to d whose low cell is (r, l)
            if (d == 0)
                reconstruct<Q, 0, float>(Rp(r, l), Rp(r, l + 1), Rp(r - 1, l), Rp(r - 1, l + 1), Rp(r + 1, l),
                                         Rp(r + 1, l + 1), Rp(r, l), Rp(r, l + 1), Rp(r, l), Rp(r, l + 1), cf.kappa, F);
            else
                reconstruct<Q, 1, float>(Rp(r, l), Rp(r + 1, l), Rp(r, l - 1), Rp(r + 1, l - 1), Rp(r, l + 1),
                                         Rp(r + 1, l + 1), Rp(r, l), Rp(r + 1, l), Rp(r, l), Rp(r + 1, l), cf.kappa, F);
        };
        float F[Q];
        rec(row, lane, F);
        const int nd = d == 0 ? nx : ny;
        const bool per = d == 0 ? perx : pery;
        const int wall = !per && (gfd == 0 || gfd == nd);
        float Gb[3] = {0.0f, 0.0f, 0.0f}, Gc[3] = {0.0f, 0.0f, 0.0f};
        const int fx = d == 0 ? gfd : min(max(gx, 0), nx - 1);
        const int fy = d == 1 ? gfd : min(max(gy, 0), ny - 1);
        if (FORCE) faceG(d, fx, fy, Gb);
        float Fc[Q];
        if (wall) {
            // x_c: the boundary cell's opposite interface, one cell inward (reading R4)
            const int sh = gfd == 0 ? 1 : -1;
            if (d == 0) rec(row, lane + sh, Fc);
            else rec(row + sh, lane, Fc);
            if (FORCE) faceG(d, d == 0 ? gfd + sh : fx, d == 1 ? gfd + sh : fy, Gc);
        }
        if (d == 0) interface_f<Q, 0, float, false>(p, cf, F, Gb, wall, gfd == 0 ? 0 : 1, Fc, Gc, out);
        else interface_f<Q, 1, float, false>(p, cf, F, Gb, wall, gfd == 0 ? 0 : 1, Fc, Gc, out);
    };

    // central differences along t of the own cell: per velocity (diagonals only) and of
    // the moments (M_t, M_xt, M_yt)
    auto cdiff = [&](auto tc, float C[Q], float dM[3]) __attribute__((always_inline)) {
        constexpr int t = decltype(tc)::value;
        const float *lo, *hi;
        if constexpr (t == 0) { lo = Rp(row, max(lane - 1, 0)); hi = Rp(row, min(lane + 1, 31)); }
        else { lo = Rp(max(row - 1, 0), lane); hi = Rp(min(row + 1, RY - 1), lane); }
        sfor<Q>([&](auto kc) {
            constexpr int k = kc;
            if constexpr (Lat<9>::e(k, 0) != 0 && Lat<9>::e(k, 1) != 0) C[k] = hi[k] - lo[k];
            else C[k] = 0.0f;
        });
        dM[0] = hi[Q + 1 + t] - lo[Q + 1 + t];
#pragma unroll
        for (int a = 0; a < 2; a++) dM[1 + a] = hi[Q + mslot2_2d(a, t)] - lo[Q + mslot2_2d(a, t)];
    };
    constexpr std::integral_constant<int, 0> AX{};
    constexpr std::integral_constant<int, 1> AY{};
    const float *cur = Rp(row, lane);

    // ---- x interfaces (beta parts exchanged by shuffles) ----
    float fxp[NF];
#pragma unroll
    for (int i = 0; i < NF; i++) fxp[i] = 0.0f;
    if (row >= 1 && row <= K::TYI) {  // warp-uniform: halo rows own no x interface
        float alx[NF], bex[NF], Ax[3], Bx[3], Cy[Q], dy[3];
        cdiff(AY, Cy, dy);
        face_parts_2d<0>(cur, cur + Q, Cy, dy, cf.kappa, alx, bex, Ax, Bx);
        float F[NF], jb[2];
#pragma unroll
        for (int i = 0; i < NF; i++) F[i] = alx[i] + __shfl_down_sync(0xffffffffu, bex[i], 1);
        const float drb = Ax[0] + __shfl_down_sync(0xffffffffu, Bx[0], 1);
#pragma unroll
        for (int a = 0; a < 2; a++) jb[a] = Ax[1 + a] + __shfl_down_sync(0xffffffffu, Bx[1 + a], 1);
        if (need_x) {
            if (!perx && (gx == -1 || gx == nx - 1)) {
                float t[NF];
                direct_face(0, gx + 1, t);
#pragma unroll
                for (int i = 0; i < NF; i++) fxp[i] = t[i];
            } else {
                float Gb[2] = {0.0f, 0.0f};
                if (FORCE) {
                    float G3[3];
                    faceG(0, gx + 1, gy, G3);
                    Gb[0] = G3[0];
                    Gb[1] = G3[1];
                }
                face_relax_2d<0, FORCE>(cf, F, drb, jb, Gb, fxp);
            }
        }
    }
    // ---- y interfaces: publish beta_y, B_y; then the interface above the own cell ----
    float aly[NF], Ay[3];
    if (ycol) {
        float bey[NF], By[3], Cx[Q], dx[3];
        cdiff(AX, Cx, dx);
        face_parts_2d<1>(cur, cur + Q, Cx, dx, cf.kappa, aly, bey, Ay, By);
        float *b = xb + (row * 32 + lane) * K::BS;
#pragma unroll
        for (int i = 0; i < NF; i++) b[i] = bey[i];
#pragma unroll
        for (int i = 0; i < 3; i++) b[NF + i] = By[i];
    }
    __syncthreads();
    float fyp[NF];
#pragma unroll
    for (int i = 0; i < NF; i++) fyp[i] = 0.0f;
    if (need_y) {
        if (!pery && (gy == -1 || gy == ny - 1)) {
            direct_face(1, gy + 1, fyp);
        } else {
            const float *nb = xb + ((row + 1) * 32 + lane) * K::BS;
            float F[NF], jb[2];
#pragma unroll
            for (int i = 0; i < NF; i++) F[i] = aly[i] + nb[i];
#pragma unroll
            for (int a = 0; a < 2; a++) jb[a] = Ay[1 + a] + nb[NF + 1 + a];
            float Gb[2] = {0.0f, 0.0f};
            if (FORCE) {
                float G3[3];
                faceG(1, gx, gy + 1, G3);
                Gb[0] = G3[0];
                Gb[1] = G3[1];
            }
            face_relax_2d<1, FORCE>(cf, F, Ay[0] + nb[NF], jb, Gb, fyp);
        }
        float *o = xf + (row * 32 + lane) * K::FS;
#pragma unroll
        for (int i = 0; i < NF; i++) o[i] = fyp[i];
    }
    __syncthreads();

    // ---- steps 8-9: update of the own cell ----
    float fxm[NF];
    if (row >= 1 && row <= K::TYI) {
#pragma unroll
        for (int i = 0; i < NF; i++) fxm[i] = __shfl_up_sync(0xffffffffu, fxp[i], 1);
    }
    if (upd) {
        const float *ym = xf + ((row - 1) * 32 + lane) * K::FS;
        const int64_t off = (int64_t)gy * p.px + gx;
        const CellRandom rnd(seed, off);
        sfor<Q>([&](auto kc) {
            constexpr int k = kc;
            float acc = 0.0f;
            if constexpr (Lat<9>::e(k, 0) != 0) {
                constexpr int i = flux_index<9>(0, k);
                acc = fmaf((float)Lat<9>::e(k, 0), fxp[i] - fxm[i], acc);
            }
            if constexpr (Lat<9>::e(k, 1) != 0) {
                constexpr int i = flux_index<9>(1, k);
                acc = fmaf((float)Lat<9>::e(k, 1), fyp[i] - ym[i], acc);
            }
            // eq. (25) in increment form (4/3 fbar+ - 1/3 f~), then the flux of
            // eq. (16)
            const float u0 = fmaf(1.0f / 3.0f, f[k] - g[k], f[k]);
            store_state<S>(dst + k * p.dstride + off, fmaf(-cf.two_kappa, acc, u0), sizeof(S) == 2 ? rnd.bits<k>() : 0u);
        });
    }
}

template <class S, int RY, bool FORCE>
__global__ void __launch_bounds__(32 * RY) fused_step2d(const __grid_constant__ StepParams p) {
    using K = Shape2<RY, S>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    step2d_tile<S, RY, FORCE>(p, smem_raw, blockIdx.x * K::TXI, blockIdx.y * K::TYI);
}

// Batched form: params holds two descriptors per instance (source/destination swapped:
// index 2 i + parity); items is the work list of (instance, x0, y0, -) inner-tile origins,
// largest instances first; CTA b takes items b, b + gridDim.x, ...
template <class S, int RY, bool FORCE>
__global__ void __launch_bounds__(32 * RY) fused_step2d_batch(const StepParams *__restrict__ params,
                                                              const int4 *__restrict__ items, int nitems, int parity) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 w = items[it];
        step2d_tile<S, RY, FORCE>(params[2 * w.x + parity], smem_raw, w.y, w.z);
        __syncthreads();  // the next item reuses the shared buffers
    }
}

}  // namespace dugks
