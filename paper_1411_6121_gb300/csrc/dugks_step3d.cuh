// dugks_step3d.cuh -- throughput kernel of the fused DUGKS time step for 3D velocity sets
// (D3Q19) on sm_103a, FP32 arithmetic, F32/BF16/F16 storage.
//
// Same scheme and the same readings as the reference kernel in dugks_step.cuh (Appendix
// steps 1-10 of arXiv 1411.6121); what differs is how the work is organised:
//
//  * A CTA is 32 x RY threads, one per cell column (lanes along x, warps along y); the
//    30 x (RY-2) inner columns are updated, the outer ring is halo. The CTA marches through
//    its z range keeping fbar+ (step 1) and its moments for three planes in a
//    shared-memory ring.
//  * Step 3-4 reconstruction is split per cell. For the interface normal to d between
//    cells L and R (eq. (23) with the cross-point tangential gradients):
//        F_k = alpha_k(L) + beta_k(R),
//        alpha_k = (1/2 + kappa e_dk) fbar+_k - kappa/4 sum_t e_tk C^t_k,
//        beta_k  = (1/2 - kappa e_dk) fbar+_k - kappa/4 sum_t e_tk C^t_k,
//    with C^t_k the central difference of fbar+_k along the tangential axis t. Only the
//    velocities that cross the interface (e_dk != 0) are formed per direction.
//  * Step 6 interface moments are sums of the same per-cell parts taken in moment space:
//        sum_k F_k = A0(L) + B0(R),  sum_k e_k F_k = A1(L) + B1(R),
//        A0 = M0/2 + kappa M_d - kappa/4 (dM_t1 + dM_t2),
//        A1_a = M_a/2 + kappa M_ad - kappa/4 (dM_a,t1 + dM_a,t2),
//    (B with -kappa), where M are moments of fbar+ and dM_.,t their central differences
//    along t, read from the neighbours' moments in the ring.
//  * Each cell forms the relaxed interface values (step 7) of its +x, +y, +z interfaces;
//    x neighbours exchange through warp shuffles, y neighbours through shared memory, so
//    every interface is computed once and both cells use the same bits.
//  * x-wall interfaces take the regular path and then step 5 (NEQ) as a correction, with
//    the values at x_c (the boundary cell's opposite interface) shuffled from the next lane
//    inward. y- and z-wall interfaces (and the chunk's first z interface) take the direct
//    path of dugks_step.cuh: all velocities reconstructed from the ring, NEQ, relax.
#pragma once

#include "dugks_step.cuh"
#include "tma.cuh"

namespace dugks {

// Velocity whose compact flux index along d is i.
template <int Q>
__host__ __device__ constexpr int flux_vel(int d, int i) {
    int r = -1;
    for (int k = 0; k < Q; k++)
        if (Lat<Q>::e(k, d) != 0 && flux_index<Q>(d, k) == i) r = k;
    return r;
}

template <int Q, int RY, class S = float>
struct Shape3 {
    static constexpr int RX = 32;
    static constexpr int NT = RX * RY;
    static constexpr int TXI = RX - 2, TYI = RY - 2;  // inner columns
    static constexpr int NF = n_flux<Q>(0);           // crossing velocities per interface
    static constexpr int NM = 10;                     // moments kept per cell
    static constexpr int CS = Q + NM;                 // ring floats per cell (odd: no conflicts)
    static constexpr int BS = (NF + 4) | 1;           // y exchange: beta_y + B_y
    static constexpr int FS = NF | 1;                 // y exchange: f at +y
    static constexpr int PLANE = RY * RX * CS;
    static constexpr int US = Q | 1;                  // u0 of a plane (own column), two planes
    static constexpr size_t BASE_FLOATS = 3 * (size_t)PLANE + (size_t)NT * (BS + FS + 2 * US);
    // The state of the tile's planes arrives by TMA into NSTAGE shared-memory stages of
    // [Q][RY][BX] elements: BX covers the 32 columns from x0 - 1 after rounding the box's
    // start down to a 16-byte boundary (3 floats or 7 16-bit values at most). Three stages
    // keep two planes in flight while the third is read. Where the stages do not fit beside
    // the ring (27 velocities), every plane is loaded directly.
    static constexpr int BX = 32 + (sizeof(S) == 4 ? 4 : 8);
    static constexpr int NSTAGE = 3;
    static constexpr size_t STAGE_BYTES = (size_t)Q * RY * BX * sizeof(S);
    // stages start at the first 128-byte boundary after the other arrays (aligned at run
    // time; 128 bytes are reserved for it), the barriers follow them
    static constexpr size_t STAGE_OFF = BASE_FLOATS * 4;
    static constexpr size_t BAR_OFF = NSTAGE * STAGE_BYTES;  // from the aligned stage start
    static constexpr size_t TMA_BYTES = STAGE_OFF + 128 + BAR_OFF + NSTAGE * 8;
    static constexpr bool TMA = sizeof(S) <= 4 && TMA_BYTES <= 227 * 1024;
    static constexpr size_t smem_bytes = TMA ? TMA_BYTES : BASE_FLOATS * 4;
};

// Moment slots in the ring: 0 M0, 1..3 M_x,y,z, 4..6 M_xx,yy,zz, 7 M_xy, 8 M_xz, 9 M_yz.
__host__ __device__ constexpr int mslot2(int a, int b) {
    return a == b ? 4 + a : (a + b == 1 ? 7 : (a + b == 2 ? 8 : 9));
}

// Moments of fbar+ of one cell into m[10] (layout above), from partial sums over the
// velocities with e_a = +1, -1 and 0.
template <int Q>
__device__ __forceinline__ void phi_moments(const float f[Q], float m[10]) {
    float sp[3] = {0.0f, 0.0f, 0.0f}, sn[3] = {0.0f, 0.0f, 0.0f}, s0 = 0.0f, mxy = 0.0f, mxz = 0.0f, myz = 0.0f;
    sfor<Q>([&](auto kc) {
        constexpr int k = kc;
        constexpr int ex = Lat<Q>::e(k, 0), ey = Lat<Q>::e(k, 1), ez = Lat<Q>::e(k, 2);
        if constexpr (ex > 0) sp[0] += f[k];
        if constexpr (ex < 0) sn[0] += f[k];
        if constexpr (ex == 0) s0 += f[k];
        if constexpr (ey > 0) sp[1] += f[k];
        if constexpr (ey < 0) sn[1] += f[k];
        if constexpr (ez > 0) sp[2] += f[k];
        if constexpr (ez < 0) sn[2] += f[k];
        if constexpr (ex * ey != 0) mxy += ex * ey > 0 ? f[k] : -f[k];
        if constexpr (ex * ez != 0) mxz += ex * ez > 0 ? f[k] : -f[k];
        if constexpr (ey * ez != 0) myz += ey * ez > 0 ? f[k] : -f[k];
    });
    m[0] = s0 + (sp[0] + sn[0]);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        m[1 + a] = sp[a] - sn[a];
        m[4 + a] = sp[a] + sn[a];
    }
    m[7] = mxy;
    m[8] = mxz;
    m[9] = myz;
}

// Tangential moment differences of a cell along t from its two neighbours' moments:
// dM[0] = difference of M_t, dM[1+a] = difference of M_at.
template <int t>
__device__ __forceinline__ void moment_diff(const float *lo, const float *hi, float dM[4]) {
    dM[0] = hi[1 + t] - lo[1 + t];
#pragma unroll
    for (int a = 0; a < 3; a++) dM[1 + a] = hi[mslot2(a, t)] - lo[mslot2(a, t)];
}

// Per-cell parts of the interface normal to d (see the file comment): alpha, beta for the
// crossing velocities (compact index), A = (A0, A1[3]), B = (B0, B1[3]). ph: fbar+ of the
// cell; m: its moments; C1/C2: per-velocity central differences along t1 < t2 (only the
// velocities that cross d and have a component along t are read); dM1/dM2: moment
// differences along t1, t2.
template <int Q, int d>
__device__ __forceinline__ void face_parts(const float *ph, const float *m, const float C1[Q], const float C2[Q],
                                           const float dM1[4], const float dM2[4], float kappa, float *alpha,
                                           float *beta, float A[4], float B[4]) {
    constexpr int t1 = d == 0 ? 1 : 0;
    constexpr int t2 = d == 2 ? 1 : 2;
    const float qk = -0.25f * kappa;
    const float g0 = qk * (dM1[0] + dM2[0]);
    A[0] = fmaf(0.5f, m[0], fmaf(kappa, m[1 + d], g0));
    B[0] = fmaf(0.5f, m[0], fmaf(-kappa, m[1 + d], g0));
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float g1 = qk * (dM1[1 + a] + dM2[1 + a]);
        const float mad = m[mslot2(a, d)];
        A[1 + a] = fmaf(0.5f, m[1 + a], fmaf(kappa, mad, g1));
        B[1 + a] = fmaf(0.5f, m[1 + a], fmaf(-kappa, mad, g1));
    }
    sfor<Q>([&](auto kc) {
        constexpr int k = kc;
        if constexpr (Lat<Q>::e(k, d) != 0) {
            constexpr int i = flux_index<Q>(d, k);
            constexpr int e1 = Lat<Q>::e(k, t1), e2 = Lat<Q>::e(k, t2);
            constexpr float ed = (float)Lat<Q>::e(k, d);
            const float f = ph[k];
            if constexpr (e1 != 0 || e2 != 0) {
                float tg = 0.0f;
                if constexpr (e1 != 0) tg = e1 > 0 ? C1[k] : -C1[k];
                if constexpr (e2 != 0) tg += e2 > 0 ? C2[k] : -C2[k];
                const float gam = qk * tg;
                alpha[i] = fmaf(fmaf(kappa, ed, 0.5f), f, gam);
                beta[i] = fmaf(fmaf(-kappa, ed, 0.5f), f, gam);
            } else {
                alpha[i] = mul_rn(fmaf(kappa, ed, 0.5f), f);
                beta[i] = mul_rn(fmaf(-kappa, ed, 0.5f), f);
            }
        }
    });
}

// Step 6-7 for the crossing velocities of the interface normal to d from its step-4 values
// F (compact) and moments (drho, j): f = F + b7 (geq - F) + c7 S. Opposite velocities (both
// cross the interface) share e.m and the quadratic part of geq.
template <int Q, int d, bool FORCE>
__device__ __forceinline__ void face_relax(const Coef<float> &cf, const float *F, float drho, const float j[3],
                                           const float Gh[3], float *out) {
    float m[3];
#pragma unroll
    for (int a = 0; a < 3; a++) m[a] = FORCE ? fmaf(Gh[a], cf.wface * cf.rho0, j[a]) : j[a];
    const float mm = dotD<3, float>(m, m);
    const float base = fmaf(-1.5f * cf.inv_rho0, mm, drho);
    float gm = 0.0f;
    if (FORCE) gm = dotD<3, float>(Gh, m) * cf.inv_rho0;
    const float c45 = 4.5f * cf.inv_rho0;
    sfor<Q>([&](auto kc) {
        constexpr int k = kc;
        constexpr int kb = opposite<Q>(k);
        if constexpr (Lat<Q>::e(k, d) > 0) {  // the pair (k, kb), e_d = +1 / -1
            float em = 0.0f, ge = 0.0f;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                if (Lat<Q>::e(k, a) > 0) { em += m[a]; if (FORCE) ge += Gh[a]; }
                if (Lat<Q>::e(k, a) < 0) { em -= m[a]; if (FORCE) ge -= Gh[a]; }
            }
            constexpr int i = flux_index<Q>(d, k), ib = flux_index<Q>(d, kb);
            constexpr float w = Lat<Q>::w(k);  // = W of the opposite velocity
            // interface values need no conservation-exact form (the same value is used by
            // both cells, so the flux telescopes exactly whatever its rounding)
            const float q = fmaf(c45 * em, em, base);
            if constexpr (FORCE) {
                const float geq = mul_rn(w, fmaf(em, 3.0f, q)), geqb = mul_rn(w, fmaf(em, -3.0f, q));
                float v = fmaf(cf.b7, geq - F[i], F[i]), vb = fmaf(cf.b7, geqb - F[ib], F[ib]);
                v = fmaf(cf.c7 * 3.0f * (ge - gm), fmaf(w, cf.rho0, geq), v);
                vb = fmaf(cf.c7 * 3.0f * (-ge - gm), fmaf(w, cf.rho0, geqb), vb);
                out[i] = v;
                out[ib] = vb;
            } else {
                // (1 - b7) F + (b7 W) (q +- 3 e.m): one operation less than F + b7 (geq - F)
                const float bw = cf.b7 * w, ob = 1.0f - cf.b7;
                out[i] = fmaf(bw, fmaf(em, 3.0f, q), ob * F[i]);
                out[ib] = fmaf(bw, fmaf(em, -3.0f, q), ob * F[ib]);
            }
        }
    });
}

// Step 5 at a wall interface normal to d, formed from the values of the regular path: F
// (compact step-4 values of the crossing velocities) and its interface moments (drb, jb: sums
// over all velocities, without the force shift), and the same at x_c, the boundary cell's
// opposite interface (Fc, drc, jc, with its acceleration Ghc). The velocities that enter from
// the wall (e_d > 0 at the low wall, SIDE 0; e_d < 0 at the high wall, SIDE 1) become
// f_eq(rho_a, u_a) + [Fc - f_eq(rho_c, u_c)] (eq. (32)), or, at a bounce-back wall, the
// opposite velocity's value plus the wall term of eq. (31). The interface moments take the
// moments of that change, so step 6 sees the moments of the modified values.
template <int Q, int d, bool FORCE, int SIDE>
__device__ __forceinline__ void neq_wall(const StepParams &p, const Coef<float> &cf, float *F, float &drb,
                                         float jb[3], const float *Fc, float drc, const float jc[3],
                                         const float Ghc[3]) {
    constexpr int wid = 2 * d + SIDE;
    if (p.bc[wid] == 3) {
        // eq. (31) instead: F_k = F_-k + 6 W_k e_k.m_w (m_w = rho0 u_w / c), from this
        // interface's own values
        float mw[3];
#pragma unroll
        for (int a = 0; a < 3; a++) mw[a] = p.fwm[wid][a];
        sfor<Q>([&](auto kc) {
            constexpr int k = kc;
            constexpr int ed = Lat<Q>::e(k, d);
            if constexpr (SIDE == 0 ? ed > 0 : ed < 0) {
                constexpr int i = flux_index<Q>(d, k), ib = flux_index<Q>(d, opposite<Q>(k));
                float em = 0.0f;
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    if (Lat<Q>::e(k, a) > 0) em += mw[a];
                    if (Lat<Q>::e(k, a) < 0) em -= mw[a];
                }
                const float v = F[ib] + wmul<Q, float>(k, 6.0f * em);
                const float dv = v - F[i];
                drb += dv;
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    if (Lat<Q>::e(k, a) > 0) jb[a] += dv;
                    if (Lat<Q>::e(k, a) < 0) jb[a] -= dv;
                }
                F[i] = v;
            }
        });
        return;
    }
    float mc[3];
#pragma unroll
    for (int a = 0; a < 3; a++) mc[a] = FORCE ? fmaf(Ghc[a], cf.wface * cf.rho0, jc[a]) : jc[a];
    float dra, ma[3];
    if (p.bc[wid] == 1) {  // velocity condition: u_a = u_w, rho_a = rho_c
        dra = drc;
#pragma unroll
        for (int a = 0; a < 3; a++) ma[a] = p.fwm[wid][a];
    } else {  // pressure condition: rho_a = rho0 + p_w / RT, u_a = u_c
        dra = wall_drho<float>(p, cf, wid);
#pragma unroll
        for (int a = 0; a < 3; a++) ma[a] = mc[a];
    }
    const float mma = dotD<3, float>(ma, ma), mmc = dotD<3, float>(mc, mc);
    sfor<Q>([&](auto kc) {
        constexpr int k = kc;
        constexpr int ed = Lat<Q>::e(k, d);
        if constexpr (SIDE == 0 ? ed > 0 : ed < 0) {
            constexpr int i = flux_index<Q>(d, k);
            const float v = geq_k<Q, float>(k, dra, ma, mma, cf.inv_rho0) +
                            (Fc[i] - geq_k<Q, float>(k, drc, mc, mmc, cf.inv_rho0));
            const float dv = v - F[i];
            drb += dv;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                if (Lat<Q>::e(k, a) > 0) jb[a] += dv;
                if (Lat<Q>::e(k, a) < 0) jb[a] -= dv;
            }
            F[i] = v;
        }
    });
}

// One segment of work: the z planes [z0, z1) of the tile whose inner columns start at
// (x0, y0). The kernel below walks a contiguous run of (tile, plane) units.
// A stored state value in a TMA stage (shared memory), as FP32 (FP16 holds g~ * 2^12).
template <class S>
__device__ __forceinline__ float stage_value(const S *p) {
    if constexpr (std::is_same<S, __nv_bfloat16>::value) return __bfloat162float(*p);
    else if constexpr (std::is_same<S, __half>::value) return __half2float(*p) * F16_UNSCALE;
    else return (float)*p;
}

// Exit path after a copy that never landed: thread 0 gives the copies that may still be in
// flight (planes next - 3 .. next - 1 of the stage sequence) a bounded time to land before the
// CTA leaves, so no copy writes into the shared memory of a finished CTA.
__device__ __forceinline__ void drain_stages(int tid, uint64_t *bars, int first, int lastp, int next) {
    if (tid != 0) return;
    for (int pz = max(first, next - 3); pz <= min(lastp, next - 1); pz++) {
        const int n = pz - first;
        mbar_wait(bars + n % 3, (uint32_t)((n / 3) & 1));
    }
}

template <int Q, class S, int RY, bool FORCE>
__device__ __forceinline__ void step3d_segment(const StepParams &p, const CUtensorMap *tmap, unsigned char *smem_raw,
                                               int x0, int y0, int z0, int z1);

// Grid: (tiles along x, tiles along y, z chunks); neighbouring CTAs stream the same z
// planes of neighbouring tiles together, so the halo columns they share hit in L2. tmap: the
// tensor map of p.src with the box [Q][RY][BX] (read only where Shape3::TMA).
template <int Q, class S, int RY, bool FORCE>
__global__ void __launch_bounds__(32 * RY, 1)
    fused_step3d(const __grid_constant__ StepParams p, const __grid_constant__ CUtensorMap tmap, int zchunk) {
    using K = Shape3<Q, RY, S>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(p.nz, z0 + zchunk);
    step3d_segment<Q, S, RY, FORCE>(p, &tmap, smem_raw, blockIdx.x * K::TXI, blockIdx.y * K::TYI, z0, z1);
}

template <int Q, class S, int RY, bool FORCE>
__device__ __forceinline__ void step3d_segment(const StepParams &p, const CUtensorMap *tmap, unsigned char *smem_raw,
                                               int x0, int y0, int z0, int z1) {
    using K = Shape3<Q, RY, S>;
    constexpr int NF = K::NF;
    constexpr int CS = K::CS;
    float *ring = reinterpret_cast<float *>(smem_raw);  // [3][RY][32][CS]: fbar+ then moments
    float *xb = ring + 3 * K::PLANE;                     // [RY][32][BS]: beta_y, B_y
    float *xf = xb + K::NT * K::BS;                      // [RY][32][FS]: f at +y
    const Coef<float> cf(p);

    const int lane = threadIdx.x, row = threadIdx.y;
    // own u0 = fbar+ + (fbar+ - f~)/3 (the cell's part of eq. (25)) of planes with
    // even / odd index
    float *usb = xf + K::NT * K::FS + (row * 32 + lane) * (2 * K::US);
    auto US = [&](int pz) __attribute__((always_inline)) -> float * { return usb + (pz & 1) * K::US; };
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int gx = x0 - 1 + lane, gy = y0 - 1 + row;
    const int64_t ncell = (int64_t)nx * ny * nz;
    const bool perx = p.bc[0] == 0, pery = p.bc[2] == 0, perz = p.bc[4] == 0;
    const S *src = reinterpret_cast<const S *>(p.src);
    S *dst = reinterpret_cast<S *>(p.dst);

    // column classification
    const bool inner = lane >= 1 && lane <= K::TXI && row >= 1 && row <= K::TYI;
    const bool upd = inner && gx < nx && gy < ny;            // this thread updates cells
    int cx = gx, cy = gy;                                    // column whose data is loaded
    bool load = true;                                        // real cell or periodic image
    if (gx < 0 || gx >= nx) { if (perx && gx >= -1 && gx <= nx) cx = wrap_idx(gx, nx); else load = false; }
    if (gy < 0 || gy >= ny) { if (pery && gy >= -1 && gy <= ny) cy = wrap_idx(gy, ny); else load = false; }
    const bool yreal = (gy >= 0 && gy < ny) || (pery && gy >= -1 && gy <= ny);
    const bool xghost = !perx && (gx == -1 || gx == nx) && yreal;
    const bool yghost = !pery && (gy == -1 || gy == ny) && gx >= -1 && gx <= nx;
    const bool xwall_tile = !perx && (x0 == 0 || x0 + K::TXI >= nx);
    const bool ywall_tile = !pery && (y0 == 0 || y0 + K::TYI >= ny);
    // which interfaces this column owns
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

    auto R = [&](int slot, int r, int l) __attribute__((always_inline)) -> float * {
        return ring + ((slot * RY + r) * 32 + l) * CS;
    };
    auto slot_of = [](int pz) __attribute__((always_inline)) { return (pz + 3) % 3; };

    // interface G / c at time t+h between (x,y,z) - e_d and (x,y,z): mean of the two cells,
    // one cell at a wall (reading R2)
    auto faceG = [&](int d, int x, int y, int z, float Gh[3]) __attribute__((always_inline)) {
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
            float v = p.fg[a];
            if (p.field) v += 0.5f * (__ldg(p.field + a * ncell + il) + __ldg(p.field + a * ncell + ih));
            Gh[a] = v * cth;
        }
    };

    // ---- TMA stages: the real planes first .. lastp of this chunk (planes z0 - 1 .. z1, less
    //      the ghost planes beyond non-periodic z walls) go in order to stage n % 3 with
    //      phase (n / 3) & 1, n = pz - first; thread 0 issues each copy once its stage has
    //      been read by every thread (a barrier lies between) ----
    const int tid = row * 32 + lane;
    unsigned char *stages = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw + K::STAGE_OFF) + 127) & ~(uintptr_t)127);
    uint64_t *bars = reinterpret_cast<uint64_t *>(stages + K::BAR_OFF);
    const int first = (!perz && z0 - 1 < 0) ? z0 : z0 - 1;
    const int lastp = (!perz && z1 >= nz) ? nz - 1 : z1;
    constexpr int XA = 16 / (int)sizeof(S);                       // box start: multiple of 16 bytes
    const int xs = (x0 - 1 >= 0) ? (x0 - 1) / XA * XA : -XA;       // x0 - 1 >= -1
    const int xcol = (x0 - 1) - xs + lane;                         // this lane's column in the box
    const bool boxed = load && cx == gx && cy == gy;               // not a periodic image
    auto issue = [&](int pz) __attribute__((always_inline)) {
        if constexpr (K::TMA) {
            if (tid == 0 && pz >= first && pz <= lastp) {
                const int s = (pz - first) % 3;
                mbar_arrive_expect_tx(bars + s, (uint32_t)K::STAGE_BYTES);
                tma_load_4d(stages + s * K::STAGE_BYTES, tmap, bars + s, xs, y0 - 1, wrap_idx(pz, nz), 0);
            }
        }
    };
    if constexpr (K::TMA) {
        if (tid == 0) {
#pragma unroll
            for (int s = 0; s < 3; s++) mbar_init(bars + s, 1);
            mbar_fence_init();
        }
        __syncthreads();
        issue(first);
        issue(first + 1);
        issue(first + 2);
    }
    bool wait_ok = true;  // false once a copy did not land (the CTA then leaves, see below)

    // ---- step 1 for the own column at plane pz into the ring; u0 = fbar+ + (fbar+ - f~)/3
    //      (the cell's part of eq. (25), applied in increment form) is returned ----
    auto make_phi = [&](int pz, float *u0) __attribute__((always_inline)) {
        float *o = R(slot_of(pz), row, lane);
        const S *sb = nullptr;
        if constexpr (K::TMA) {
            const int n = pz - first;
            wait_ok = wait_ok && mbar_wait(bars + n % 3, (uint32_t)((n / 3) & 1));
            sb = reinterpret_cast<const S *>(stages + (n % 3) * K::STAGE_BYTES) + row * K::BX + xcol;
        }
        if (!load) {
#pragma unroll
            for (int k = 0; k < CS; k++) o[k] = 0.0f;
            return;
        }
        const int gz = wrap_idx(pz, nz);
        const int64_t off = (int64_t)gz * p.plane + (int64_t)cy * p.px + cx;
        float g[Q];
        if (K::TMA && boxed) {
#pragma unroll
            for (int k = 0; k < Q; k++) g[k] = stage_value(sb + k * (RY * K::BX));
        } else {
#pragma unroll
            for (int k = 0; k < Q; k++) g[k] = (float)Store<S>::ld(src + k * p.dstride + off);
        }
        float Gh[3] = {0.0f, 0.0f, 0.0f}, drho, m[3];
        if (FORCE) {
            const int64_t c = (int64_t)cx + (int64_t)nx * ((int64_t)cy + (int64_t)ny * gz);
            cell_G<3, float>(p, c, ncell, ct, Gh);
        }
        moments<Q, float, true>(g, Gh, cf.wcell * cf.rho0, drho, m);
        float f[Q];
        relax<Q, float, FORCE>(g, drho, m, Gh, cf.rho0, cf.inv_rho0, cf.b1, cf.c1, f);
        float mo[10];
        phi_moments<Q>(f, mo);
#pragma unroll
        for (int k = 0; k < Q; k++) {
            o[k] = f[k];
            u0[k] = fmaf(1.0f / 3.0f, f[k] - g[k], f[k]);
        }
#pragma unroll
        for (int i = 0; i < 10; i++) o[Q + i] = mo[i];
    };
    // step 2 (reading R3: ghost = 2 f0 - f1, x then y then z): fbar+ and, by linearity,
    // its moments extrapolate the same way
    auto ghosts_xy = [&](int pz) __attribute__((always_inline)) {
        const int s = slot_of(pz);
        if (xwall_tile) {
            __syncthreads();
            if (xghost) {
                const int d1 = gx < 0 ? 1 : -1;
                float *o = R(s, row, lane);
                const float *a = R(s, row, lane + d1), *b = R(s, row, lane + 2 * d1);
#pragma unroll
                for (int k = 0; k < CS; k++) o[k] = ghost_value(a[k], b[k]);
            }
        }
        if (ywall_tile) {
            __syncthreads();
            if (yghost) {
                const int d1 = gy < 0 ? 1 : -1;
                float *o = R(s, row, lane);
                const float *a = R(s, row + d1, lane), *b = R(s, row + 2 * d1, lane);
#pragma unroll
                for (int k = 0; k < CS; k++) o[k] = ghost_value(a[k], b[k]);
            }
        }
    };
    auto ghost_z = [&](int pz) __attribute__((always_inline)) {
        float *o = R(slot_of(pz), row, lane);
        const float *a = R(slot_of(pz < 0 ? 0 : nz - 1), row, lane);
        const float *b = R(slot_of(pz < 0 ? 1 : nz - 2), row, lane);
#pragma unroll
        for (int k = 0; k < CS; k++) o[k] = ghost_value(a[k], b[k]);
    };

    // direct path for one interface (walls, chunk start): all velocities from the ring,
    // NEQ at walls, relax. Interface normal to d between the own cell at plane pl and the
    // next cell along d; gfd is its index along d.
    auto direct_face = [&](int d, int pl, int gfd, float *out) {
        auto ptr = [&](int s, int r, int l) __attribute__((always_inline)) -> const float * { return R(s, r, l); };
        auto rec = [&](int r, int l, int pc, float F[Q]) __attribute__((always_inline)) {
            // interface normal to d whose low cell is (r, l) at plane pc
            const int a = slot_of(pc - 1), b = slot_of(pc), c = slot_of(pc + 1);
            if (d == 0)
                reconstruct<Q, 0, float>(ptr(b, r, l), ptr(b, r, l + 1), ptr(b, r - 1, l), ptr(b, r - 1, l + 1),
                                         ptr(b, r + 1, l), ptr(b, r + 1, l + 1), ptr(a, r, l), ptr(a, r, l + 1),
                                         ptr(c, r, l), ptr(c, r, l + 1), cf.kappa, F);
            else if (d == 1)
                reconstruct<Q, 1, float>(ptr(b, r, l), ptr(b, r + 1, l), ptr(b, r, l - 1), ptr(b, r + 1, l - 1),
                                         ptr(b, r, l + 1), ptr(b, r + 1, l + 1), ptr(a, r, l), ptr(a, r + 1, l),
                                         ptr(c, r, l), ptr(c, r + 1, l), cf.kappa, F);
            else
                reconstruct<Q, 2, float>(ptr(b, r, l), ptr(c, r, l), ptr(b, r, l - 1), ptr(c, r, l - 1),
                                         ptr(b, r, l + 1), ptr(c, r, l + 1), ptr(b, r - 1, l), ptr(c, r - 1, l),
                                         ptr(b, r + 1, l), ptr(c, r + 1, l), cf.kappa, F);
        };
        float F[Q];
        rec(row, lane, pl, F);
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
            // x_c: the boundary cell's opposite interface, one cell inward (reading R4)
            const int sh = gfd == 0 ? 1 : -1;
            if (d == 0) rec(row, lane + sh, pl, Fc);
            else if (d == 1) rec(row + sh, lane, pl, Fc);
            else rec(row, lane, gfd == 0 ? 0 : nz - 2, Fc);
            if (FORCE) faceG(d, d == 0 ? gfd + sh : fx, d == 1 ? gfd + sh : fy, d == 2 ? gfd + sh : fz, Gc);
        }
        if (d == 0) interface_f<Q, 0, float, false>(p, cf, F, Gb, wall, gfd == 0 ? 0 : 1, Fc, Gc, out);
        else if (d == 1) interface_f<Q, 1, float, false>(p, cf, F, Gb, wall, gfd == 0 ? 0 : 1, Fc, Gc, out);
        else interface_f<Q, 2, float, false>(p, cf, F, Gb, wall, gfd == 0 ? 0 : 1, Fc, Gc, out);
    };

    // per-velocity central differences of the own column at plane pz along t (edge
    // velocities only: a velocity along one axis has no tangential part)
    auto cdiff = [&](int pz, auto tc, float C[Q]) __attribute__((always_inline)) {
        constexpr int t = decltype(tc)::value;
        const float *lo, *hi;
        if constexpr (t == 0) { lo = R(slot_of(pz), row, max(lane - 1, 0)); hi = R(slot_of(pz), row, min(lane + 1, 31)); }
        else if constexpr (t == 1) { lo = R(slot_of(pz), max(row - 1, 0), lane); hi = R(slot_of(pz), min(row + 1, RY - 1), lane); }
        else { lo = R(slot_of(pz - 1), row, lane); hi = R(slot_of(pz + 1), row, lane); }
        sfor<Q>([&](auto kc) {
            constexpr int k = kc;
            constexpr int nzc = (Lat<Q>::e(k, 0) != 0) + (Lat<Q>::e(k, 1) != 0) + (Lat<Q>::e(k, 2) != 0);
            if constexpr (nzc >= 2 && Lat<Q>::e(k, t) != 0) C[k] = hi[k] - lo[k];
            else C[k] = 0.0f;
        });
    };
    auto mdiff = [&](int pz, auto tc, float dM[4]) __attribute__((always_inline)) {
        constexpr int t = decltype(tc)::value;
        const float *lo, *hi;
        if constexpr (t == 0) { lo = R(slot_of(pz), row, max(lane - 1, 0)); hi = R(slot_of(pz), row, min(lane + 1, 31)); }
        else if constexpr (t == 1) { lo = R(slot_of(pz), max(row - 1, 0), lane); hi = R(slot_of(pz), min(row + 1, RY - 1), lane); }
        else { lo = R(slot_of(pz - 1), row, lane); hi = R(slot_of(pz + 1), row, lane); }
        moment_diff<t>(lo + Q, hi + Q, dM);
    };
    constexpr std::integral_constant<int, 0> AX{};
    constexpr std::integral_constant<int, 1> AY{};
    constexpr std::integral_constant<int, 2> AZ{};

    // ---------------- prologue: planes z0-1, z0, z0+1 ----------------
    // plane z0+2 is made at the first iteration of the loop below, if there is one
    int consumed = 0;
    for (int pz = z0 - 1; pz <= z0 + 1; pz++) {
        if (!perz && (pz < 0 || pz >= nz)) continue;
        make_phi(pz, US(pz));  // (plane z0+1 overwrites the u0 of plane z0-1: same parity)
        consumed++;
    }
    for (int pz = z0 - 1; pz <= z0 + 1; pz++) {
        if (!perz && (pz < 0 || pz >= nz)) continue;
        ghosts_xy(pz);
    }
    // a copy that never landed: every thread leaves together (after thread 0 gave the copies
    // in flight a bounded time to land)
    if (__syncthreads_or(!wait_ok)) {
        if constexpr (K::TMA) drain_stages(tid, bars, first, lastp, first + 3);
        return;
    }
    // the stages read above are free again
    for (int i = 0; i < consumed; i++) issue(first + 3 + i);
    for (int pz = z0 - 1; pz <= z0 + 1; pz++)
        if (!perz && (pz < 0 || pz >= nz)) ghost_z(pz);
    __syncthreads();

    // carried: alpha_z, A_z of the current plane and f at its -z interface
    float alz[NF], Az[4], fzm[NF];
#pragma unroll
    for (int i = 0; i < NF; i++) alz[i] = fzm[i] = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; i++) Az[i] = 0.0f;
    // carried too (D3Q19), by the rows that own x interfaces: the x and y differences of the
    // current plane (per velocity and of the moments), formed with the z parts of the previous
    // iteration and used again by the x and y parts of this one. With 27 velocities carrying
    // them costs more registers than recomputing them (the kernel would spill), so there they
    // are formed again where they are used.
    constexpr bool CARRY = Q == 19;
    const bool xrow = row >= 1 && row <= K::TYI;  // warp-uniform
    float cAX[Q], cAY[Q], mAX[4], mAY[4];
    if (xrow) {
        cdiff(z0, AX, cAX);
        cdiff(z0, AY, cAY);
        mdiff(z0, AX, mAX);
        mdiff(z0, AY, mAY);
    }
    if (upd) {
        float bz[NF], Bz[4];
        const float *c = R(slot_of(z0), row, lane);
        face_parts<Q, 2>(c, c + Q, cAX, cAY, mAX, mAY, cf.kappa, alz, bz, Az, Bz);
        float t[NF];
        direct_face(2, z0 - 1, z0, t);
#pragma unroll
        for (int i = 0; i < NF; i++) fzm[i] = t[i];
    }

    for (int kz = z0; kz < z1; kz++) {
        // ---- P1: fbar+ of plane kz+1 (planes z0 .. z0+1 were made in the prologue) ----
        if (kz > z0) {
            const int pn = kz + 1;
            if (perz || pn < nz) {
                make_phi(pn, US(pn));  // copied by TMA two iterations ago
                ghosts_xy(pn);
            } else if (pn == nz) {
                ghost_z(pn);
            }
            if (__syncthreads_or(!wait_ok)) {
                if constexpr (K::TMA) drain_stages(tid, bars, first, lastp, kz + 4);
                return;
            }
            issue(kz + 4);  // into the stage of plane kz + 1, read above
        }
        const float *cur = R(slot_of(kz), row, lane);

        // ---- P3: x interfaces of plane kz (beta parts exchanged by shuffles) ----
        float Cz[Q], dz[4];
        cdiff(kz, AZ, Cz);
        mdiff(kz, AZ, dz);
        float fxp[NF];
#pragma unroll
        for (int i = 0; i < NF; i++) fxp[i] = 0.0f;
        if (xrow) {  // halo rows own no x interface
            float alx[NF], bex[NF], Ax[4], Bx[4];
            if constexpr (!CARRY) {
                cdiff(kz, AY, cAY);
                mdiff(kz, AY, mAY);
            }
            face_parts<Q, 0>(cur, cur + Q, cAY, Cz, mAY, dz, cf.kappa, alx, bex, Ax, Bx);
            float F[NF], jb[3];
#pragma unroll
            for (int i = 0; i < NF; i++) F[i] = alx[i] + __shfl_down_sync(0xffffffffu, bex[i], 1);
            float drb = Ax[0] + __shfl_down_sync(0xffffffffu, Bx[0], 1);
#pragma unroll
            for (int a = 0; a < 3; a++) jb[a] = Ax[1 + a] + __shfl_down_sync(0xffffffffu, Bx[1 + a], 1);
            float Gb[3] = {0.0f, 0.0f, 0.0f};
            if (FORCE && need_x) faceG(0, gx + 1, gy, kz, Gb);
            if (xwall_tile) {
                // the wall interfaces take step 5 from x_c, the interface that the next lane
                // inward owns (lane + 1 at the low wall, lane - 1 at the high wall); every lane
                // takes part in the exchange
                float Fn[NF], jd[3], ju[3], Gd[3] = {0.0f, 0.0f, 0.0f}, Gu[3] = {0.0f, 0.0f, 0.0f};
                sfor<NF>([&](auto ic) {
                    constexpr int i = ic;
                    if constexpr (Lat<Q>::e(flux_vel<Q>(0, i), 0) > 0) Fn[i] = __shfl_down_sync(0xffffffffu, F[i], 1);
                    else Fn[i] = __shfl_up_sync(0xffffffffu, F[i], 1);
                });
                const float dd = __shfl_down_sync(0xffffffffu, drb, 1), du = __shfl_up_sync(0xffffffffu, drb, 1);
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    jd[a] = __shfl_down_sync(0xffffffffu, jb[a], 1);
                    ju[a] = __shfl_up_sync(0xffffffffu, jb[a], 1);
                    if (FORCE) {
                        Gd[a] = __shfl_down_sync(0xffffffffu, Gb[a], 1);
                        Gu[a] = __shfl_up_sync(0xffffffffu, Gb[a], 1);
                    }
                }
                if (need_x && gx == -1) neq_wall<Q, 0, FORCE, 0>(p, cf, F, drb, jb, Fn, dd, jd, Gd);
                if (need_x && gx == nx - 1) neq_wall<Q, 0, FORCE, 1>(p, cf, F, drb, jb, Fn, du, ju, Gu);
            }
            if (need_x) face_relax<Q, 0, FORCE>(cf, F, drb, jb, Gb, fxp);
        }
        // ---- P4: y parts of plane kz; publish beta_y, B_y; y interfaces ----
        float aly[NF], Ay[4];
        if (ycol) {
            float bey[NF], By[4], Cx[Q], dx[4];
            if (CARRY && xrow) {
#pragma unroll
                for (int k = 0; k < Q; k++) Cx[k] = cAX[k];
#pragma unroll
                for (int i = 0; i < 4; i++) dx[i] = mAX[i];
            } else {
                cdiff(kz, AX, Cx);
                mdiff(kz, AX, dx);
            }
            face_parts<Q, 1>(cur, cur + Q, Cx, Cz, dx, dz, cf.kappa, aly, bey, Ay, By);
            float *b = xb + (row * 32 + lane) * K::BS;
#pragma unroll
            for (int i = 0; i < NF; i++) b[i] = bey[i];
#pragma unroll
            for (int i = 0; i < 4; i++) b[NF + i] = By[i];
        }
        __syncthreads();
        float fyp[NF];
        if (need_y) {
            if (!pery && (gy == -1 || gy == ny - 1)) {
                float t[NF];
                direct_face(1, kz, gy + 1, t);
#pragma unroll
                for (int i = 0; i < NF; i++) fyp[i] = t[i];
            } else {
                const float *nb = xb + ((row + 1) * 32 + lane) * K::BS;
                float F[NF], jb[3];
#pragma unroll
                for (int i = 0; i < NF; i++) F[i] = aly[i] + nb[i];
#pragma unroll
                for (int a = 0; a < 3; a++) jb[a] = Ay[1 + a] + nb[NF + 1 + a];
                float Gb[3] = {0.0f, 0.0f, 0.0f};
                if (FORCE) faceG(1, gx, gy + 1, kz, Gb);
                face_relax<Q, 1, FORCE>(cf, F, Ay[0] + nb[NF], jb, Gb, fyp);
            }
            float *o = xf + (row * 32 + lane) * K::FS;
#pragma unroll
            for (int i = 0; i < NF; i++) o[i] = fyp[i];
        }
        __syncthreads();

        // ---- P2: z parts of plane kz+1 and the z interface kz+1/2 ----
        float alzn[NF], Azn[4], fzp[NF];
        if (xrow) {
            cdiff(kz + 1, AX, cAX);
            cdiff(kz + 1, AY, cAY);
            mdiff(kz + 1, AX, mAX);
            mdiff(kz + 1, AY, mAY);
        }
        if (upd) {
            float bezn[NF], Bzn[4];
            const float *nxt = R(slot_of(kz + 1), row, lane);
            face_parts<Q, 2>(nxt, nxt + Q, cAX, cAY, mAX, mAY, cf.kappa, alzn, bezn, Azn, Bzn);
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

        // ---- P5: steps 8-9, update of cell (gx, gy, kz) ----
        float fxm[NF];
        if (row >= 1 && row <= K::TYI) {
#pragma unroll
            for (int i = 0; i < NF; i++) fxm[i] = __shfl_up_sync(0xffffffffu, fxp[i], 1);
        }
        if (upd) {
            const float *ym = xf + ((row - 1) * 32 + lane) * K::FS;
            const float *u0 = US(kz);
            const int64_t off = (int64_t)kz * p.plane + (int64_t)gy * p.px + gx;
            const CellRandom rnd(seed, off);
            sfor<Q>([&](auto kc) {
                constexpr int k = kc;
                float acc = 0.0f;
                if constexpr (Lat<Q>::e(k, 0) != 0) {
                    constexpr int i = flux_index<Q>(0, k);
                    acc = fmaf((float)Lat<Q>::e(k, 0), fxp[i] - fxm[i], acc);
                }
                if constexpr (Lat<Q>::e(k, 1) != 0) {
                    constexpr int i = flux_index<Q>(1, k);
                    acc = fmaf((float)Lat<Q>::e(k, 1), fyp[i] - ym[i], acc);
                }
                if constexpr (Lat<Q>::e(k, 2) != 0) {
                    constexpr int i = flux_index<Q>(2, k);
                    acc = fmaf((float)Lat<Q>::e(k, 2), fzp[i] - fzm[i], acc);
                }
                // eq. (16): f~(t+dt) = f~+ - dt/|V| flux
                store_state<S>(dst + k * p.dstride + off, fmaf(-cf.two_kappa, acc, u0[k]),
                               sizeof(S) == 2 ? rnd.bits<k>() : 0u);
            });
#pragma unroll
            for (int i = 0; i < NF; i++) { fzm[i] = fzp[i]; alz[i] = alzn[i]; }
#pragma unroll
            for (int i = 0; i < 4; i++) Az[i] = Azn[i];
        }
        // the next P1 overwrites the ring slot of plane kz-1, last read in P3/P4 above and
        // separated from it by the barrier before P5
    }
}

}  // namespace dugks
