// dugks_step3d_ws.cuh -- warp-specialised throughput kernel of the fused DUGKS time step for
// D3Q19 on sm_103a (FP32 arithmetic, F32/BF16/F16 storage): the scheme and readings of
// dugks_step3d.cuh, with the z march split between two groups of warps that run concurrently,
// and the arithmetic done on pairs of opposite velocities.
//
//  * Producer warps (8, one cell column each) make step 1 for plane kz + 2 and
//    beyond: the state of the tile's plane arrives by TMA into one shared-memory stage, each
//    column forms fbar+, its moments and u0 = fbar+ + (fbar+ - f~)/3, then the ghost
//    columns and rows (step 2) and, beyond non-periodic z walls, the ghost planes. Having made
//    plane p they form the x interfaces of plane p - 1 (steps 3-7), which need its x and y
//    neighbours and their own column of planes p - 2 and p.
//  * Consumer warps (8, one cell column each, the 32 x 8 layout of the non-specialised kernel)
//    do the rest of steps 3-9 for plane kz: the y and z interfaces and the update, as
//    dugks_step3d.cuh does them. The split puts about as much work on each group.
//  * The planes pass through a ring of four slots (fbar+ and moments), three u0 slots and two
//    slots of f at the x interfaces. Each
//    ring slot has a "full" mbarrier (every producer thread arrives after its last write of the
//    plane) and an "empty" one (every consumer thread arrives after its last read), so neither
//    group waits on a CTA-wide barrier: the producer runs up to two planes ahead and the
//    step-1 work of one plane overlaps the interface work of another. The consumers' y exchange
//    and the producers' ghost passes use named barriers of their own group.
//
// Pairs. The D3Q19 order puts opposite velocities at k and 18 - k (the rest velocity at 9), so
// the moving velocities form nine pairs (j, 18 - j), j = 0..8, with e_{18-j} = -e_j. Every
// linear step of the scheme treats the two members of a pair with the same operation and
// coefficients of equal size (opposite signs where e enters), so the kernel keeps a pair in one
// float2 and uses the packed FP32 instructions of sm_100 and later (fma/add/mul .f32x2: two
// FP32 operations per instruction, each rounded as its scalar form). Shared memory holds pairs
// side by side, so a pair moves with one 64-bit access; strides of 2 mod 4 words keep those
// accesses free of bank conflicts.
//
// The 512 threads launch with 128 registers each; the producer warpgroups then give registers
// back (setmaxnreg to PROD_REGS) and the consumer warpgroups take them (CONS_REGS): 256 x 96 +
// 256 x 160 = 512 x 128. Every wait on an mbarrier gives up after about two seconds (a device
// flag, then the group leaves together; see tma.cuh).
#pragma once

#include "dugks_step3d.cuh"

namespace dugks {

// D3Q19 opposite pairs and the per-cell layout of the ring.
namespace pr {
__host__ __device__ constexpr int e(int j, int a) { return Lat<19>::e(j, a); }
__host__ __device__ constexpr int nnz(int j) { return (e(j, 0) != 0) + (e(j, 1) != 0) + (e(j, 2) != 0); }
// the p-th pair (0..4) whose velocities cross a face normal to d
__host__ __device__ constexpr int cross(int d, int p) {
    int n = 0, r = -1;
    for (int j = 0; j < 9; j++)
        if (e(j, d) != 0) {
            if (n == p) r = j;
            n++;
        }
    return r;
}
// position of pair j in the crossing list of d
__host__ __device__ constexpr int pos(int d, int j) {
    int n = 0;
    for (int i = 0; i < j; i++) n += e(i, d) != 0;
    return e(j, d) != 0 ? n : -1;
}
// the axis other than d along which pair j has a component (-1: none; D3Q19 has at most one)
__host__ __device__ constexpr int tang(int d, int j) {
    int r = -1;
    for (int a = 2; a >= 0; a--)
        if (a != d && e(j, a) != 0) r = a;
    return r;
}
// Per cell, CS floats: [2j, 2j+1] fbar+ of pair j; [18] the rest velocity; [19] M0;
// [20 + 2a, 21 + 2a] (M_a, M_aa); [26, 27] (M_xy, M_xz); [28, 29] (M_yz, M_xz).
constexpr int CS = 30, REST = 18, M0 = 19, XY = 26, YZ = 28;
__host__ __device__ constexpr int ma(int a) { return 20 + 2 * a; }
// slot of velocity k and of the second moment M_ab
__host__ __device__ constexpr int rslot(int k) { return k < 9 ? 2 * k : (k > 9 ? 2 * (18 - k) + 1 : REST); }
__host__ __device__ constexpr int mslot(int a, int b) {
    return a == b ? 21 + 2 * a : (a + b == 1 ? XY : (a + b == 2 ? XY + 1 : YZ));
}
constexpr bool layout_ok() {
    for (int j = 0; j < 9; j++) {
        if (opposite<19>(j) != 18 - j) return false;
        if (nnz(j) == 0) return false;
    }
    for (int d = 0; d < 3; d++)
        if (cross(d, 4) < 0) return false;
    return nnz(9) == 0;
}
static_assert(layout_ok(), "D3Q19 velocity order without opposite pairs at k, 18 - k");
}  // namespace pr

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void st2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
// a - b, rounded as the scalar difference
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(f2(-1.0f, -1.0f), b, a); }
__device__ __forceinline__ float2 ghost2(float2 a, float2 b) { return f2(ghost_value(a.x, b.x), ghost_value(a.y, b.y)); }

template <int Q, class S>
struct ShapeWS {
    static_assert(Q == 19, "the warp-specialised kernel is written for D3Q19");
    static constexpr int RX = 32, RY = 8, NC = RX * RY;  // cell columns of the tile, halo included
    static constexpr int NPROD = NC, NCONS = NC, NTHREADS = NPROD + NCONS;
    static constexpr int PROD_REGS = 96, CONS_REGS = 160;
    static_assert(NPROD * PROD_REGS + NCONS * CONS_REGS <= NTHREADS * 128, "register split above the launch's");
    static constexpr int TXI = RX - 2, TYI = RY - 2;  // inner columns
    static constexpr int CS = pr::CS;                 // ring floats per cell
    static constexpr int BS = 14;                     // y exchange: beta_y pairs, B_y
    static constexpr int FS = 10;                     // y exchange: f pairs at +y
    static constexpr int UP = 18;                     // u0 pairs of one column and plane
    static constexpr int NSLOT = 4, NU0 = 3;
    static constexpr int NUC = TYI * RX;              // columns that update (rows 1 .. TYI)
    static constexpr int PLANE = RY * RX * CS;
    // ring; beta_y of rows 1..RY-1; f_y of rows 0..RY-2; u0 pairs and rest of rows 1..TYI; f pairs
    // at +x of rows 1..TYI for two planes
    static constexpr size_t FLOATS = (size_t)NSLOT * PLANE + (size_t)(RY - 1) * RX * BS +
                                     (size_t)(RY - 1) * RX * FS + (size_t)NU0 * NUC * UP + (size_t)NU0 * NUC +
                                     (size_t)2 * NUC * FS;
    static_assert(FLOATS % 2 == 0 && PLANE % 2 == 0 && NUC % 2 == 0, "float2 arrays must stay 8-byte aligned");
    static constexpr int BX = 32 + (sizeof(S) == 4 ? 4 : 8);  // TMA box width (start rounded down)
    static constexpr size_t STAGE_BYTES = (size_t)Q * RY * BX * sizeof(S);
    static constexpr size_t STAGE_OFF = FLOATS * 4;  // aligned to 128 bytes at run time
    static constexpr size_t BAR_OFF = STAGE_BYTES;   // from the aligned stage: full[4], empty[4], stage
    static constexpr size_t smem_bytes = STAGE_OFF + 128 + STAGE_BYTES + 9 * 8;
    static_assert(smem_bytes <= 227 * 1024, "warp-specialised tile does not fit");
};

__device__ __forceinline__ void named_bar(int id, int n) { asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory"); }
// Named barrier with an OR over the participating threads' predicates.
__device__ __forceinline__ bool named_bar_or(int id, int n, bool v) {
    uint32_t r;
    asm volatile(
        "{ .reg .pred p, q; setp.ne.u32 p, %1, 0; bar.red.or.pred q, %2, %3, p; selp.u32 %0, 1, 0, q; }\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// Step 1 (eq. (24) with eq. (6)) for one D3Q19 cell on pairs: G[j] = (g~_j, g~_{18-j}),
// g9 the rest velocity, Gh the acceleration / c at t_n (FORCE). Writes fbar+ (F, f9),
// u0 = fbar+ + (fbar+ - g~)/3 (U, u9) and the ten moments of fbar+ in the ring's order
// (mo: M0, M_x, M_y, M_z, M_xx, M_yy, M_zz, M_xy, M_xz, M_yz). The momentum sums are exact
// as in moments<Q, float, true>: heads on the grid of the cell's largest |g| are summed
// without rounding (pair by pair: the head sums of the first and second members, each at
// most five terms, then their difference), tails separately, one rounding at the end. The
// equilibrium pair is geq_pair's, the relaxation relax's, one packed operation per pair.
template <bool FORCE>
__device__ __forceinline__ void step1_pairs(const float2 G[9], float g9, const float Gh[3], const Coef<float> &cf,
                                            float2 F[9], float &f9, float2 U[9], float &u9, float mo[10]) {
    const float2 N1 = f2(-1.0f, -1.0f);
    float2 Rs = G[0];
#pragma unroll
    for (int j = 1; j < 9; j++) Rs = __fadd2_rn(Rs, G[j]);
    const float drho = (Rs.x + Rs.y) + g9;
    float amax = 0.0f;
#pragma unroll
    for (int j = 0; j < 9; j++) amax = fmaxf(amax, fmaxf(fabsf(G[j].x), fabsf(G[j].y)));
    // 1.5 * 2^(E + 5) for amax in [2^E, 2^(E+1)): exponent field + 5, significand 1.5
    const float split = __uint_as_float((__float_as_uint(amax) & 0x7f800000u) + 0x02c00000u);
    const float2 SP = f2(split, split), SN = f2(-split, -split);
    float2 AH[3] = {f2(0.f, 0.f), f2(0.f, 0.f), f2(0.f, 0.f)}, AL[3] = {f2(0.f, 0.f), f2(0.f, 0.f), f2(0.f, 0.f)};
    sfor<9>([&](auto jc) {
        constexpr int j = jc;
        const float2 H = __fadd2_rn(__fadd2_rn(G[j], SP), SN);
        const float2 Lo = sub2(G[j], H);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (pr::e(j, a) > 0) { AH[a] = __fadd2_rn(AH[a], H); AL[a] = __fadd2_rn(AL[a], Lo); }
            if (pr::e(j, a) < 0) { AH[a] = sub2(AH[a], H); AL[a] = sub2(AL[a], Lo); }
        }
    });
    float m[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float lo = AL[a].x - AL[a].y;
        m[a] = __fadd_rn(AH[a].x - AH[a].y, FORCE ? fmaf(Gh[a], cf.wcell * cf.rho0, lo) : lo);
    }
    const float mm = dotD<3, float>(m, m);
    float gm = 0.0f;
    if (FORCE) gm = dotD<3, float>(Gh, m) * cf.inv_rho0;
    const float base = fmaf(-1.5f * cf.inv_rho0, mm, drho);
    const float c45 = 4.5f * cf.inv_rho0;
    const float2 B2 = f2(cf.b1, cf.b1), TH = f2(1.0f / 3.0f, 1.0f / 3.0f);
    sfor<9>([&](auto jc) {
        constexpr int j = jc;
        float em = 0.0f, ge = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (pr::e(j, a) > 0) { em += m[a]; if (FORCE) ge += Gh[a]; }
            if (pr::e(j, a) < 0) { em -= m[a]; if (FORCE) ge -= Gh[a]; }
        }
        const float q = fmaf(c45 * em, em, base);
        const double W = Lat<19>::wt<double>(j);
        const float wh = (float)W, wl = (float)(W - (double)wh);
        const float w3h = (float)(3.0 * W), w3l = (float)(3.0 * W - (double)w3h);
        const float wq = fmaf(wl, q, wh * q);
        const float2 EM = f2(em, em);
        const float2 GEQ = __ffma2_rn(f2(w3h, -w3h), EM, __ffma2_rn(f2(w3l, -w3l), EM, f2(wq, wq)));
        float2 V = __ffma2_rn(B2, sub2(GEQ, G[j]), G[j]);
        if constexpr (FORCE) {
            const float2 FEQ = __ffma2_rn(f2((float)W, (float)W), f2(cf.rho0, cf.rho0), GEQ);
            const float2 SC = __fmul2_rn(f2(3.0f, 3.0f), f2(ge - gm, -ge - gm));
            V = __ffma2_rn(f2(cf.c1, cf.c1), __fmul2_rn(SC, FEQ), V);
        }
        F[j] = V;
        U[j] = __ffma2_rn(TH, sub2(V, G[j]), V);
    });
    {
        const float geq = wmul<19, float>(9, base);
        float v = fmaf(cf.b1, geq - g9, g9);
        if (FORCE) v = fmaf(cf.c1, 3.0f * (0.0f - gm) * fmaf((float)Lat<19>::wt<double>(9), cf.rho0, geq), v);
        f9 = v;
        u9 = fmaf(1.0f / 3.0f, v - g9, v);
    }
    // moments of fbar+: P[a] sums the pairs whose first member has e_a = +1, N[a] those with -1
    // (the second member then counts the other way)
    float2 P[3] = {f2(0.f, 0.f), f2(0.f, 0.f), f2(0.f, 0.f)}, Nn[3] = {f2(0.f, 0.f), f2(0.f, 0.f), f2(0.f, 0.f)};
    float2 S0 = f2(0.f, 0.f), XY = f2(0.f, 0.f), XZ = f2(0.f, 0.f), YZ = f2(0.f, 0.f);
    sfor<9>([&](auto jc) {
        constexpr int j = jc;
        constexpr int ex = pr::e(j, 0), ey = pr::e(j, 1), ez = pr::e(j, 2);
        if constexpr (ex > 0) P[0] = __fadd2_rn(P[0], F[j]);
        if constexpr (ex < 0) Nn[0] = __fadd2_rn(Nn[0], F[j]);
        if constexpr (ex == 0) S0 = __fadd2_rn(S0, F[j]);
        if constexpr (ey > 0) P[1] = __fadd2_rn(P[1], F[j]);
        if constexpr (ey < 0) Nn[1] = __fadd2_rn(Nn[1], F[j]);
        if constexpr (ez > 0) P[2] = __fadd2_rn(P[2], F[j]);
        if constexpr (ez < 0) Nn[2] = __fadd2_rn(Nn[2], F[j]);
        if constexpr (ex * ey > 0) XY = __fadd2_rn(XY, F[j]);
        if constexpr (ex * ey < 0) XY = sub2(XY, F[j]);
        if constexpr (ex * ez > 0) XZ = __fadd2_rn(XZ, F[j]);
        if constexpr (ex * ez < 0) XZ = sub2(XZ, F[j]);
        if constexpr (ey * ez > 0) YZ = __fadd2_rn(YZ, F[j]);
        if constexpr (ey * ez < 0) YZ = sub2(YZ, F[j]);
    });
    float sp[3], sn[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        sp[a] = P[a].x + Nn[a].y;
        sn[a] = P[a].y + Nn[a].x;
    }
    mo[0] = ((S0.x + S0.y) + f9) + (sp[0] + sn[0]);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        mo[1 + a] = sp[a] - sn[a];
        mo[4 + a] = sp[a] + sn[a];
    }
    mo[7] = XY.x + XY.y;
    mo[8] = XZ.x + XZ.y;
    mo[9] = YZ.x + YZ.y;
}

// Steps 3-4 for all 19 velocities at the interface normal to d (reconstruct of
// dugks_step.cuh) from cells in the ring's pair layout; F in velocity order.
template <int d>
__device__ __forceinline__ void reconstruct_pairs(const float *L, const float *R, const float *L1m, const float *R1m,
                                                  const float *L1p, const float *R1p, const float *L2m,
                                                  const float *R2m, const float *L2p, const float *R2p, float kappa,
                                                  float F[19]) {
    constexpr int t1 = d == 0 ? 1 : 0;
    constexpr int t2 = d == 2 ? 1 : 2;
    const float qk = 0.25f * kappa;
    sfor<19>([&](auto kc) {
        constexpr int k = kc;
        constexpr int s = pr::rslot(k);
        const float l = L[s], r = R[s];
        float v = mul_rn(0.5f, l + r);
        if constexpr (Lat<19>::e(k, d) != 0) v = fmaf(-kappa * (float)Lat<19>::e(k, d), r - l, v);
        if constexpr (Lat<19>::e(k, t1) != 0)
            v = fmaf(-qk * (float)Lat<19>::e(k, t1), (L1p[s] + R1p[s]) - (L1m[s] + R1m[s]), v);
        if constexpr (Lat<19>::e(k, t2) != 0)
            v = fmaf(-qk * (float)Lat<19>::e(k, t2), (L2p[s] + R2p[s]) - (L2m[s] + R2m[s]), v);
        F[k] = v;
    });
}

// The direct path of one interface (walls, the chunk's first z interface): all velocities
// reconstructed from the ring (steps 3-4), step 5 at a wall, steps 6-7; interface normal to d
// between the cell (row, lane) at plane pl and the next cell along d, gfd its index along d.
struct Pairs5 {
    float2 v[5];
};
template <bool FORCE>
__device__ __forceinline__ Pairs5 direct_face_ws(const StepParams &p, const Coef<float> &cf, const float *ring, int d,
                                                 int pl, int gfd, int row, int lane, int gx, int gy, int z0, float cth) {
    constexpr int Q = 19, RY = 8, NF = n_flux<19>(0);
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int64_t ncell = (int64_t)nx * ny * nz;
    const bool perx = p.bc[0] == 0, pery = p.bc[2] == 0, perz = p.bc[4] == 0;
    auto slot_of = [&](int pz) { return (pz - (z0 - 1)) & 3; };
    auto ptr = [&](int s, int r, int l) -> const float * { return ring + ((s * RY + r) * 32 + l) * pr::CS; };
    // interface G / c at time t+h between (x,y,z) - e_d and (x,y,z), as in the kernel
    auto faceG = [&](int x, int y, int z, float Gh[3]) {
        int lo[3] = {x, y, z}, hi[3] = {x, y, z};
        const int nd = d == 0 ? nx : (d == 1 ? ny : nz);
        const bool per = d == 0 ? perx : (d == 1 ? pery : perz);
        lo[d] -= 1;
        if (per) { lo[d] = wrap_idx(lo[d], nd); hi[d] = wrap_idx(hi[d], nd); }
        else { lo[d] = max(lo[d], 0); hi[d] = min(hi[d], nd - 1); }
        const int64_t il = (int64_t)lo[0] + (int64_t)nx * ((int64_t)lo[1] + (int64_t)ny * lo[2]);
        const int64_t ih = (int64_t)hi[0] + (int64_t)nx * ((int64_t)hi[1] + (int64_t)ny * hi[2]);
        for (int a = 0; a < 3; a++) {
            float v = p.fg[a];
            if (p.field) v += 0.5f * (__ldg(p.field + a * ncell + il) + __ldg(p.field + a * ncell + ih));
            Gh[a] = v * cth;
        }
    };
    auto rec = [&](int r, int l, int pc, float F[Q]) {
        // interface normal to d whose low cell is (r, l) at plane pc
        const int a = slot_of(pc - 1), b = slot_of(pc), c = slot_of(pc + 1);
        if (d == 0)
            reconstruct_pairs<0>(ptr(b, r, l), ptr(b, r, l + 1), ptr(b, r - 1, l), ptr(b, r - 1, l + 1),
                                 ptr(b, r + 1, l), ptr(b, r + 1, l + 1), ptr(a, r, l), ptr(a, r, l + 1),
                                 ptr(c, r, l), ptr(c, r, l + 1), cf.kappa, F);
        else if (d == 1)
            reconstruct_pairs<1>(ptr(b, r, l), ptr(b, r + 1, l), ptr(b, r, l - 1), ptr(b, r + 1, l - 1),
                                 ptr(b, r, l + 1), ptr(b, r + 1, l + 1), ptr(a, r, l), ptr(a, r + 1, l),
                                 ptr(c, r, l), ptr(c, r + 1, l), cf.kappa, F);
        else
            reconstruct_pairs<2>(ptr(b, r, l), ptr(c, r, l), ptr(b, r, l - 1), ptr(c, r, l - 1),
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
    if (FORCE) faceG(fx, fy, fz, Gb);
    float Fc[Q];
    if (wall) {
        // x_c: the boundary cell's opposite interface, one cell inward (reading R4)
        const int sh = gfd == 0 ? 1 : -1;
        if (d == 0) rec(row, lane + sh, pl, Fc);
        else if (d == 1) rec(row + sh, lane, pl, Fc);
        else rec(row, lane, gfd == 0 ? 0 : nz - 2, Fc);
        if (FORCE) faceG(d == 0 ? gfd + sh : fx, d == 1 ? gfd + sh : fy, d == 2 ? gfd + sh : fz, Gc);
    }
    float o[NF];
    Pairs5 out;
    auto pack = [&](auto dc) {
        constexpr int dd = decltype(dc)::value;
        sfor<5>([&](auto pc) {
            constexpr int j = pr::cross(dd, pc);
            out.v[pc] = f2(o[flux_index<19>(dd, j)], o[flux_index<19>(dd, 18 - j)]);
        });
    };
    if (d == 0) {
        interface_f<Q, 0, float, false>(p, cf, F, Gb, wall, gfd == 0 ? 0 : 1, Fc, Gc, o);
        pack(std::integral_constant<int, 0>{});
    } else if (d == 1) {
        interface_f<Q, 1, float, false>(p, cf, F, Gb, wall, gfd == 0 ? 0 : 1, Fc, Gc, o);
        pack(std::integral_constant<int, 1>{});
    } else {
        interface_f<Q, 2, float, false>(p, cf, F, Gb, wall, gfd == 0 ? 0 : 1, Fc, Gc, o);
        pack(std::integral_constant<int, 2>{});
    }
    return out;
}

template <int Q, class S, bool FORCE>
__global__ void __launch_bounds__(512, 1)
    fused_step3d_ws(const __grid_constant__ StepParams p, const __grid_constant__ CUtensorMap tmap, int zchunk) {
    using K = ShapeWS<Q, S>;
    constexpr int RY = K::RY;
    constexpr int NF = n_flux<Q>(0);
    constexpr int CS = K::CS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(p.nz, z0 + zchunk);
    const int x0 = blockIdx.x * K::TXI, y0 = blockIdx.y * K::TYI;

    float *ring = reinterpret_cast<float *>(smem_raw);  // [NSLOT][RY][32][CS]
    float *xb = ring + K::NSLOT * K::PLANE;            // [rows 1..RY-1][32][BS]: beta_y pairs, B_y
    float *xf = xb + (RY - 1) * 32 * K::BS;            // [rows 0..RY-2][32][FS]: f pairs at +y
    float *u0b = xf + (RY - 1) * 32 * K::FS;           // [NU0][rows 1..TYI][32][UP]
    float *u0r = u0b + K::NU0 * K::NUC * K::UP;        // [NU0][rows 1..TYI][32]: rest velocity
    float *fxb = u0r + K::NU0 * K::NUC;                // [2][rows 1..TYI][32][FS]: f pairs at +x
    unsigned char *stage = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw + K::STAGE_OFF) + 127) & ~(uintptr_t)127);
    uint64_t *full = reinterpret_cast<uint64_t *>(stage + K::BAR_OFF);
    uint64_t *empty = full + 4;
    uint64_t *sbar = full + 8;

    const int tid = threadIdx.x;
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < 4; s++) {
            mbar_init(full + s, K::NPROD);
            mbar_init(empty + s, K::NCONS);
        }
        mbar_init(sbar, 1);
        mbar_fence_init();
    }
    __syncthreads();

    const Coef<float> cf(p);
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int64_t ncell = (int64_t)nx * ny * nz;
    const bool perx = p.bc[0] == 0, pery = p.bc[2] == 0, perz = p.bc[4] == 0;
    const S *src = reinterpret_cast<const S *>(p.src);
    S *dst = reinterpret_cast<S *>(p.dst);
    float ct = p.fcoef[2], cth = p.fcoef[2];
    if (FORCE && p.omega != 0.0) {
        const double tn = ((double)(*p.step_ctr) + (double)p.step_off) * p.dt;
        ct = (float)(cos(p.omega * tn) * p.inv_c);
        cth = (float)(cos(p.omega * (tn + 0.5 * p.dt)) * p.inv_c);
    }
    // planes z0 - 1 .. z1 in order: n = pz - (z0 - 1) selects ring slot n % 4 (phase n / 4) and u0
    // slot n % 3
    auto nidx = [&](int pz) __attribute__((always_inline)) { return pz - (z0 - 1); };
    auto slot_of = [&](int pz) __attribute__((always_inline)) { return nidx(pz) & 3; };
    auto R = [&](int slot, int r, int l) __attribute__((always_inline)) -> float * {
        return ring + ((slot * RY + r) * 32 + l) * CS;
    };
    const bool xwall_tile = !perx && (x0 == 0 || x0 + K::TXI >= nx);
    const bool ywall_tile = !pery && (y0 == 0 || y0 + K::TYI >= ny);

    // the cell column of a thread: producer thread c and consumer thread NPROD + c own column c
    const int lane = tid & 31, row = (tid & (K::NC - 1)) >> 5;
    const int gx = x0 - 1 + lane, gy = y0 - 1 + row;
    const bool xrow = row >= 1 && row <= K::TYI;  // rows that own x interfaces (warp-uniform)
    const float kap = cf.kappa, qk = -0.25f * kap;
    // (1/2 + kappa e, 1/2 - kappa e) of a pair whose first member has e_d = +1 (PK) or -1 (MK);
    // the tangential weight -kappa/4 e_t with e_t = +1 (QP) or -1 (QM) for the first member
    const float2 PK = f2(fmaf(kap, 1.0f, 0.5f), fmaf(kap, -1.0f, 0.5f));
    const float2 MK = f2(PK.y, PK.x);
    const float2 QP = f2(qk, -qk), QM = f2(-qk, qk);
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
    // a crossing-pair array of direction d from velocity-ordered compact values (flux_index)
    // and back
    auto to_pairs = [&](auto dc, const float *Fn, float2 *P2) __attribute__((always_inline)) {
        constexpr int d = decltype(dc)::value;
        sfor<5>([&](auto pc) {
            constexpr int j = pr::cross(d, pc);
            P2[pc] = f2(Fn[flux_index<19>(d, j)], Fn[flux_index<19>(d, 18 - j)]);
        });
    };
    auto from_pairs = [&](auto dc, const float2 *P2, float *Fn) __attribute__((always_inline)) {
        constexpr int d = decltype(dc)::value;
        sfor<5>([&](auto pc) {
            constexpr int j = pr::cross(d, pc);
            Fn[flux_index<19>(d, j)] = P2[pc].x;
            Fn[flux_index<19>(d, 18 - j)] = P2[pc].y;
        });
    };
    constexpr std::integral_constant<int, 0> AX{};
    constexpr std::integral_constant<int, 1> AY{};
    constexpr std::integral_constant<int, 2> AZ{};

    // Central differences of a column's pairs, C[j] for the pairs with components along t and
    // one other axis (a velocity along one axis only has no tangential part), and of its
    // moments: dM[0] of M_t, dM[1 + a] of M_at. lo and hi point at the column's two neighbours
    // along t. In the plane (t = x, y) they are the cell pointer -+ the neighbour's offset:
    // every caller is a row 1..TYI thread, or (along x) a lane 1..TXI thread, so both
    // neighbours lie in the ring.
    auto cdiff = [&](const float *lo, const float *hi, auto tc, float2 C[9]) __attribute__((always_inline)) {
        constexpr int t = decltype(tc)::value;
        sfor<9>([&](auto jc) {
            constexpr int j = jc;
            if constexpr (pr::nnz(j) == 2 && pr::e(j, t) != 0) C[j] = sub2(ld2(hi + 2 * j), ld2(lo + 2 * j));
        });
    };
    auto mdiff = [&](const float *lo, const float *hi, auto tc, float dM[4]) __attribute__((always_inline)) {
        constexpr int t = decltype(tc)::value;
        const float2 d1 = sub2(ld2(hi + pr::ma(t)), ld2(lo + pr::ma(t)));  // (M_t, M_tt)
        dM[0] = d1.x;
        dM[1 + t] = d1.y;
        if constexpr (t == 0) {
            const float2 d2 = sub2(ld2(hi + pr::XY), ld2(lo + pr::XY));  // (M_xy, M_xz)
            dM[2] = d2.x;
            dM[3] = d2.y;
        } else if constexpr (t == 1) {
            dM[1] = ld2(hi + pr::XY).x - ld2(lo + pr::XY).x;  // M_xy
            dM[3] = ld2(hi + pr::YZ).x - ld2(lo + pr::YZ).x;  // M_yz
        } else {
            const float2 d2 = sub2(ld2(hi + pr::YZ), ld2(lo + pr::YZ));  // (M_yz, M_xz)
            dM[2] = d2.x;
            dM[1] = d2.y;
        }
    };
    constexpr int NX1 = CS, NY1 = 32 * CS;  // ring offsets of the x and y neighbours
    // the thread's own column in the ring slot of plane pz
    auto P = [&](int pz) __attribute__((always_inline)) -> const float * {
        return ring + slot_of(pz) * K::PLANE + (row * 32 + lane) * CS;
    };
    // Per-cell parts of the interface normal to d (face_parts of dugks_step3d.cuh on pairs):
    // AL/BE for the five crossing pairs, A = (A0, A1[3]), B likewise. c: the cell in the ring;
    // C1/C2, dM1/dM2: differences along t1 < t2, the tangential axes of d.
    auto parts = [&](auto dc, const float *c, const float2 *C1, const float2 *C2, const float dM1[4],
                     const float dM2[4], float2 AL[5], float2 BE[5], float A[4], float B[4])
                     __attribute__((always_inline)) {
        constexpr int d = decltype(dc)::value;
        constexpr int t1 = d == 0 ? 1 : 0;
        const float2 m0p = ld2(c + pr::REST);
        const float2 mdp = ld2(c + pr::ma(d));
        const float g0 = qk * (dM1[0] + dM2[0]);
        A[0] = fmaf(0.5f, m0p.y, fmaf(kap, mdp.x, g0));
        B[0] = fmaf(0.5f, m0p.y, fmaf(-kap, mdp.x, g0));
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const float g1 = qk * (dM1[1 + a] + dM2[1 + a]);
            const float Ma = ld2(c + pr::ma(a)).x;
            const int ms = pr::mslot(a, d);
            const float2 mp = ld2(c + (ms & ~1));
            const float mad = (ms & 1) ? mp.y : mp.x;
            A[1 + a] = fmaf(0.5f, Ma, fmaf(kap, mad, g1));
            B[1 + a] = fmaf(0.5f, Ma, fmaf(-kap, mad, g1));
        }
        sfor<5>([&](auto pc) {
            constexpr int pp = pc;
            constexpr int j = pr::cross(d, pp);
            constexpr int t = pr::tang(d, j);
            const float2 f = ld2(c + 2 * j);
            const float2 cp = pr::e(j, d) > 0 ? PK : MK, cm = pr::e(j, d) > 0 ? MK : PK;
            if constexpr (t >= 0) {
                const float2 gam = __fmul2_rn(pr::e(j, t) > 0 ? QP : QM, t == t1 ? C1[j] : C2[j]);
                AL[pp] = __ffma2_rn(cp, f, gam);
                BE[pp] = __ffma2_rn(cm, f, gam);
            } else {
                AL[pp] = __fmul2_rn(cp, f);
                BE[pp] = __fmul2_rn(cm, f);
            }
        });
    };
    // Steps 6-7 on pairs (face_relax of dugks_step3d.cuh): F the step-4 values of the crossing
    // pairs, (drho, j) their interface moments; out = F + b7 (geq - F) + c7 S.
    auto relax_face = [&](auto dc, const float2 F[5], float drho, const float j[3], const float Gh[3], float2 out[5])
                          __attribute__((always_inline)) {
        constexpr int d = decltype(dc)::value;
        float mv[3];
#pragma unroll
        for (int a = 0; a < 3; a++) mv[a] = FORCE ? fmaf(Gh[a], cf.wface * cf.rho0, j[a]) : j[a];
        const float mm = dotD<3, float>(mv, mv);
        const float base = fmaf(-1.5f * cf.inv_rho0, mm, drho);
        float gm = 0.0f;
        if (FORCE) gm = dotD<3, float>(Gh, mv) * cf.inv_rho0;
        const float c45 = 4.5f * cf.inv_rho0;
        const float2 OB = f2(1.0f - cf.b7, 1.0f - cf.b7);
        sfor<5>([&](auto pc) {
            constexpr int pp = pc;
            constexpr int jj = pr::cross(d, pp);
            float em = 0.0f, ge = 0.0f;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                if (pr::e(jj, a) > 0) { em += mv[a]; if (FORCE) ge += Gh[a]; }
                if (pr::e(jj, a) < 0) { em -= mv[a]; if (FORCE) ge -= Gh[a]; }
            }
            constexpr float w = Lat<19>::w(jj);
            const float q = fmaf(c45 * em, em, base);
            const float2 X = __ffma2_rn(f2(3.0f, -3.0f), f2(em, em), f2(q, q));  // q +- 3 e.m
            if constexpr (FORCE) {
                const float2 GEQ = __fmul2_rn(f2(w, w), X);
                float2 v = __ffma2_rn(f2(cf.b7, cf.b7), sub2(GEQ, F[pp]), F[pp]);
                const float2 FEQ = __ffma2_rn(f2(w, w), f2(cf.rho0, cf.rho0), GEQ);
                const float c73 = cf.c7 * 3.0f;
                out[pp] = __ffma2_rn(f2(c73 * (ge - gm), c73 * (-ge - gm)), FEQ, v);
            } else {
                // (1 - b7) F + (b7 W) (q +- 3 e.m)
                const float bw = cf.b7 * w;
                out[pp] = __ffma2_rn(f2(bw, bw), X, __fmul2_rn(OB, F[pp]));
            }
        });
    };

    if (tid < K::NPROD) {
        // =============================== producer ===============================
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(K::PROD_REGS));
        // real planes first .. lastp are copied in order into the one stage (phase m & 1 for the
        // m-th); thread 0 issues the next copy once every producer thread has read the stage
        const int first = (!perz && z0 - 1 < 0) ? z0 : z0 - 1;
        const int lastp = (!perz && z1 >= nz) ? nz - 1 : z1;
        constexpr int XA = 16 / (int)sizeof(S);
        const int xs = (x0 - 1 >= 0) ? (x0 - 1) / XA * XA : -XA;
        auto issue = [&](int pz) __attribute__((always_inline)) {
            if (tid == 0 && pz >= first && pz <= lastp) {
                mbar_arrive_expect_tx(sbar, (uint32_t)K::STAGE_BYTES);
                tma_load_4d(stage, &tmap, sbar, xs, y0 - 1, wrap_idx(pz, nz), 0);
            }
        };
        bool ok = true;
        issue(first);
        int cx = gx, cy = gy;
        bool load = true;
        if (gx < 0 || gx >= nx) { if (perx && gx >= -1 && gx <= nx) cx = wrap_idx(gx, nx); else load = false; }
        if (gy < 0 || gy >= ny) { if (pery && gy >= -1 && gy <= ny) cy = wrap_idx(gy, ny); else load = false; }
        const bool boxed = load && cx == gx && cy == gy;
        const bool yreal = (gy >= 0 && gy < ny) || (pery && gy >= -1 && gy <= ny);
        const bool xghost = !perx && (gx == -1 || gx == nx) && yreal;
        const bool yghost = !pery && (gy == -1 || gy == ny) && gx >= -1 && gx <= nx;
        const bool urow = row >= 1 && row <= K::TYI;  // columns whose u0 the consumers read
        int m = 0;  // real planes read from the stage so far
        // step 1 for real plane pz into its ring and u0 slots; false: a wait gave up (every
        // producer thread learns it at the same barrier)
        auto make_plane = [&](int pz) __attribute__((always_inline)) -> bool {
            const int gz = wrap_idx(pz, nz);
            float2 G[9];
            float g9;
            ok = ok && mbar_wait(sbar, (uint32_t)(m & 1));
            m++;
            {
                const S *sb = reinterpret_cast<const S *>(stage) + row * K::BX + ((x0 - 1) - xs + lane);
                if (boxed) {
#pragma unroll
                    for (int j = 0; j < 9; j++)
                        G[j] = f2(stage_value(sb + j * (RY * K::BX)), stage_value(sb + (18 - j) * (RY * K::BX)));
                    g9 = stage_value(sb + 9 * (RY * K::BX));
                } else if (load) {
                    const int64_t off = (int64_t)gz * p.plane + (int64_t)cy * p.px + cx;
#pragma unroll
                    for (int j = 0; j < 9; j++)
                        G[j] = f2((float)Store<S>::ld(src + j * p.dstride + off),
                                  (float)Store<S>::ld(src + (18 - j) * p.dstride + off));
                    g9 = (float)Store<S>::ld(src + 9 * p.dstride + off);
                } else {
#pragma unroll
                    for (int j = 0; j < 9; j++) G[j] = f2(0.0f, 0.0f);
                    g9 = 0.0f;
                }
            }
            // the stage has been read: the next plane may land in it; every producer thread has
            // also finished the previous plane (its rows are visible to the x interfaces)
            if (named_bar_or(1, K::NPROD, !ok)) return false;
            // the next real plane in order
            issue(pz + 1 <= lastp ? pz + 1 : lastp + 1);
            float *o = R(slot_of(pz), row, lane);
            const int us = (nidx(pz) % 3) * K::NUC + (row - 1) * 32 + lane;
            if (!load) {
#pragma unroll
                for (int i = 0; i < CS / 2; i++) st2(o + 2 * i, f2(0.0f, 0.0f));
                return true;
            }
            float Gh[3] = {0.0f, 0.0f, 0.0f};
            if (FORCE) {
                const int64_t ci = (int64_t)cx + (int64_t)nx * ((int64_t)cy + (int64_t)ny * gz);
                cell_G<3, float>(p, ci, ncell, ct, Gh);
            }
            float2 F[9], U[9];
            float f9, u9, mo[10];
            step1_pairs<FORCE>(G, g9, Gh, cf, F, f9, U, u9, mo);
#pragma unroll
            for (int j = 0; j < 9; j++) st2(o + 2 * j, F[j]);
            st2(o + pr::REST, f2(f9, mo[0]));
#pragma unroll
            for (int a = 0; a < 3; a++) st2(o + pr::ma(a), f2(mo[1 + a], mo[4 + a]));
            st2(o + pr::XY, f2(mo[7], mo[8]));
            st2(o + pr::YZ, f2(mo[9], mo[8]));
            if (urow) {
#pragma unroll
                for (int j = 0; j < 9; j++) st2(u0b + us * K::UP + 2 * j, U[j]);
                u0r[us] = u9;
            }
            return true;
        };
        // step 2 (reading R3: ghost = 2 f0 - f1, x then y): fbar+ and, by linearity, its moments
        auto ghosts_xy = [&](int pz) __attribute__((always_inline)) {
            const int sl = slot_of(pz);
            if (xwall_tile) {
                named_bar(1, K::NPROD);
                if (xghost) {
                    const int d1 = gx < 0 ? 1 : -1;
                    float *o = R(sl, row, lane);
                    const float *a = R(sl, row, lane + d1), *b = R(sl, row, lane + 2 * d1);
#pragma unroll
                    for (int i = 0; i < CS / 2; i++) st2(o + 2 * i, ghost2(ld2(a + 2 * i), ld2(b + 2 * i)));
                }
            }
            if (ywall_tile) {
                named_bar(1, K::NPROD);
                if (yghost) {
                    const int d1 = gy < 0 ? 1 : -1;
                    float *o = R(sl, row, lane);
                    const float *a = R(sl, row + d1, lane), *b = R(sl, row + 2 * d1, lane);
#pragma unroll
                    for (int i = 0; i < CS / 2; i++) st2(o + 2 * i, ghost2(ld2(a + 2 * i), ld2(b + 2 * i)));
                }
            }
        };
        // a ghost plane beyond a non-periodic z wall (whole region)
        auto ghost_z = [&](int pz) __attribute__((always_inline)) {
            float *o = R(slot_of(pz), row, lane);
            const float *a = R(slot_of(pz < 0 ? 0 : nz - 1), row, lane);
            const float *b = R(slot_of(pz < 0 ? 1 : nz - 2), row, lane);
#pragma unroll
            for (int i = 0; i < CS / 2; i++) st2(o + 2 * i, ghost2(ld2(a + 2 * i), ld2(b + 2 * i)));
        };
        // x interfaces of plane q (steps 3-7; every plane that the consumers update), for the
        // rows that own them, into +x slot q % 2: beta parts exchanged by shuffles, step 5 at x
        // walls from x_c, the interface that the next lane inward owns
        const bool need_x = xrow && gy >= 0 && gy < ny && lane <= K::TXI && gx >= -1 && gx < nx;
        auto x_faces = [&](int q) __attribute__((always_inline)) {
            if (!xrow) return;  // halo rows own no x interface
            const float *pq = P(q), *pm = P(q - 1), *pp = P(q + 1);
            float2 Cy[9], Cz[9];
            float dy[4], dz[4];
            cdiff(pq - NY1, pq + NY1, AY, Cy);
            cdiff(pm, pp, AZ, Cz);
            mdiff(pq - NY1, pq + NY1, AY, dy);
            mdiff(pm, pp, AZ, dz);
            float2 fxp[5];
#pragma unroll
            for (int i = 0; i < 5; i++) fxp[i] = f2(0.0f, 0.0f);
            float2 alx[5], bex[5];
            float Ax[4], Bx[4];
            parts(AX, pq, Cy, Cz, dy, dz, alx, bex, Ax, Bx);
            float2 F[5];
            float jb[3];
#pragma unroll
            for (int i = 0; i < 5; i++)
                F[i] = __fadd2_rn(alx[i], f2(__shfl_down_sync(0xffffffffu, bex[i].x, 1),
                                             __shfl_down_sync(0xffffffffu, bex[i].y, 1)));
            float drb = Ax[0] + __shfl_down_sync(0xffffffffu, Bx[0], 1);
#pragma unroll
            for (int a = 0; a < 3; a++) jb[a] = Ax[1 + a] + __shfl_down_sync(0xffffffffu, Bx[1 + a], 1);
            float Gb[3] = {0.0f, 0.0f, 0.0f};
            if (FORCE && need_x) faceG(0, gx + 1, gy, q, Gb);
            if (xwall_tile) {
                // the wall interfaces take step 5 from x_c, the interface that the next lane
                // inward owns (lane + 1 at the low wall, lane - 1 at the high wall); every lane
                // takes part in the exchange. The first member of each x pair has e_x = -1.
                float Fv[NF], Fn[NF], jd[3], ju[3], Gd[3] = {0.0f, 0.0f, 0.0f}, Gu[3] = {0.0f, 0.0f, 0.0f};
                float2 Fn2[5];
#pragma unroll
                for (int i = 0; i < 5; i++)
                    Fn2[i] = f2(__shfl_up_sync(0xffffffffu, F[i].x, 1), __shfl_down_sync(0xffffffffu, F[i].y, 1));
                from_pairs(AX, F, Fv);
                from_pairs(AX, Fn2, Fn);
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
                if (need_x && gx == -1) neq_wall<Q, 0, FORCE, 0>(p, cf, Fv, drb, jb, Fn, dd, jd, Gd);
                if (need_x && gx == nx - 1) neq_wall<Q, 0, FORCE, 1>(p, cf, Fv, drb, jb, Fn, du, ju, Gu);
                to_pairs(AX, Fv, F);
            }
            if (need_x) relax_face(AX, F, drb, jb, Gb, fxp);
            float *o = fxb + ((q & 1) * K::NUC + (row - 1) * 32 + lane) * K::FS;
#pragma unroll
            for (int i = 0; i < 5; i++) st2(o + 2 * i, fxp[i]);
        };
        auto leave = [&]() __attribute__((always_inline)) {
            if (tid == 0) mbar_wait(sbar, (uint32_t)(m & 1));  // a copy still in flight: bounded wait
        };

        // prologue: planes z0 - 1 .. z0 + 1 (a ghost plane below z = 0 after the planes it needs)
        for (int pz = z0 - 1; pz <= z0 + 1; pz++) {
            if (!perz && (pz < 0 || pz >= nz)) continue;
            if (!make_plane(pz)) { leave(); return; }
        }
        for (int pz = z0 - 1; pz <= z0 + 1; pz++) {
            if (!perz && (pz < 0 || pz >= nz)) continue;
            ghosts_xy(pz);
        }
        if (named_bar_or(1, K::NPROD, !ok)) { leave(); return; }
        for (int pz = z0 - 1; pz <= z0 + 1; pz++)
            if (!perz && (pz < 0 || pz >= nz)) ghost_z(pz);
        x_faces(z0);  // reads rows of plane z0 (made before the barrier above) and own columns
        for (int pz = z0 - 1; pz <= z0 + 1; pz++) mbar_arrive(full + slot_of(pz));
        // the rest of the chunk, each plane into a slot the consumers have released
        for (int pz = z0 + 2; pz <= z1; pz++) {
            const int n = nidx(pz);
            if (n >= 4) ok = ok && mbar_wait(empty + (n & 3), (uint32_t)(((n >> 2) - 1) & 1));
            if (perz || pz < nz) {
                if (!make_plane(pz)) { leave(); return; }
                ghosts_xy(pz);
            } else {  // pz == nz: the ghost plane above the top wall
                if (named_bar_or(1, K::NPROD, !ok)) { leave(); return; }
                ghost_z(pz);
            }
            // plane pz - 1 was made an iteration ago and is visible since the barrier above; of
            // plane pz the x faces read only the thread's own column
            x_faces(pz - 1);
            mbar_arrive(full + (n & 3));
        }
        return;
    }

    // =============================== consumers ===============================
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(K::CONS_REGS));
    const bool inner = lane >= 1 && lane <= K::TXI && row >= 1 && row <= K::TYI;
    const bool upd = inner && gx < nx && gy < ny;
    const bool ycol = lane >= 1 && lane <= K::TXI && gx >= 0 && gx < nx && gy >= -1 && gy <= ny;
    const bool need_y = ycol && row <= K::TYI && gy < ny;
    uint32_t seed = 0;  // stochastic rounding of 16-bit stores
    if constexpr (sizeof(S) == 2) seed = store_seed(*p.step_ctr + p.step_off);
    auto wait_full = [&](int pz) __attribute__((always_inline)) -> bool {
        const int n = nidx(pz);
        return mbar_wait(full + (n & 3), (uint32_t)((n >> 2) & 1));
    };
    auto release = [&](int pz) __attribute__((always_inline)) {
        if (pz >= z0 - 1) mbar_arrive(empty + slot_of(pz));
    };
    auto cons_bar = [&]() __attribute__((always_inline)) { named_bar(2, K::NCONS); };
    auto cons_bar_or = [&](bool v) __attribute__((always_inline)) { return named_bar_or(2, K::NCONS, v); };
    bool ok = true;
    for (int pz = z0 - 1; pz <= z0 + 1; pz++) ok = ok && wait_full(pz);
    if (cons_bar_or(!ok)) return;

    // carried: alpha_z, A_z of the current plane and f at its -z interface
    float2 alz[5], fzm[5];
    float Az[4];
#pragma unroll
    for (int i = 0; i < 5; i++) alz[i] = fzm[i] = f2(0.0f, 0.0f);
#pragma unroll
    for (int i = 0; i < 4; i++) Az[i] = 0.0f;
    // carried too, by the rows that own x interfaces: the x differences of the current plane,
    // formed with the z parts of the previous iteration and used again by the y parts of this one
    float2 cAX[9];
    float mAX[4];
    if (xrow) {
        const float *c0 = P(z0);
        cdiff(c0 - NX1, c0 + NX1, AX, cAX);
        mdiff(c0 - NX1, c0 + NX1, AX, mAX);
    }
    if (upd) {
        const float *c0 = P(z0);
        float2 bz[5], cAY[9];
        float Bz[4], mAY[4];
        cdiff(c0 - NY1, c0 + NY1, AY, cAY);
        mdiff(c0 - NY1, c0 + NY1, AY, mAY);
        parts(AZ, c0, cAX, cAY, mAX, mAY, alz, bz, Az, Bz);
        const Pairs5 r = direct_face_ws<FORCE>(p, cf, ring, 2, z0 - 1, z0, row, lane, gx, gy, z0, cth);
#pragma unroll
        for (int i = 0; i < 5; i++) fzm[i] = r.v[i];
    }

    for (int kz = z0; kz < z1; kz++) {
        // ---- plane kz+1 (fbar+, moments, ghosts) from the producer warps; planes z0 - 1 .. z0 + 1
        //      were awaited before the loop ----
        if (kz > z0) ok = ok && wait_full(kz + 1);
        const float *cur = P(kz), *prv = P(kz - 1), *nxt = P(kz + 1);
        // the direct paths of this iteration (a y wall row's +y interface, the +z interface below
        // a z wall) first, while the march holds the fewest values: they read only the ring
        float2 fyp[5], fzp[5];
        const bool ydir = need_y && !pery && (gy == -1 || gy == ny - 1);
        const bool zdir = upd && !perz && kz + 1 == nz;
        if (ydir) {
            const Pairs5 r = direct_face_ws<FORCE>(p, cf, ring, 1, kz, gy + 1, row, lane, gx, gy, z0, cth);
#pragma unroll
            for (int i = 0; i < 5; i++) fyp[i] = r.v[i];
        }
        if (zdir) {
            const Pairs5 r = direct_face_ws<FORCE>(p, cf, ring, 2, kz, kz + 1, row, lane, gx, gy, z0, cth);
#pragma unroll
            for (int i = 0; i < 5; i++) fzp[i] = r.v[i];
        }

        float2 Cz[9];
        float dz[4];
        cdiff(prv, nxt, AZ, Cz);
        mdiff(prv, nxt, AZ, dz);
        // ---- P4: y parts of plane kz; publish beta_y, B_y; y interfaces ----
        float2 aly[5];
        float Ay[4];
        if (ycol) {
            float2 bey[5];
            float By[4];
            if (xrow) {
                parts(AY, cur, cAX, Cz, mAX, dz, aly, bey, Ay, By);
            } else {
                float2 Cx[9];
                float dx[4];
                cdiff(cur - NX1, cur + NX1, AX, Cx);
                mdiff(cur - NX1, cur + NX1, AX, dx);
                parts(AY, cur, Cx, Cz, dx, dz, aly, bey, Ay, By);
            }
            if (row >= 1) {
                float *b = xb + ((row - 1) * 32 + lane) * K::BS;
#pragma unroll
                for (int i = 0; i < 5; i++) st2(b + 2 * i, bey[i]);
                st2(b + 10, f2(By[0], By[1]));
                st2(b + 12, f2(By[2], By[3]));
            }
        }
        // ---- P2: z parts of plane kz+1 and the z interface kz+1/2, before the first consumer
        //      barrier: they need nothing from the y exchange, so the y parts and the z
        //      interface form one barrier-free phase of independent chains ----
        float2 alzn[5];
        float Azn[4];
        if (xrow) {
            cdiff(nxt - NX1, nxt + NX1, AX, cAX);
            mdiff(nxt - NX1, nxt + NX1, AX, mAX);
        }
        if (upd) {
            float2 bezn[5], cAY[9];
            float Bzn[4], mAY[4];
            cdiff(nxt - NY1, nxt + NY1, AY, cAY);
            mdiff(nxt - NY1, nxt + NY1, AY, mAY);
            parts(AZ, nxt, cAX, cAY, mAX, mAY, alzn, bezn, Azn, Bzn);
            if (!zdir) {
                float2 F[5];
                float jb[3];
#pragma unroll
                for (int i = 0; i < 5; i++) F[i] = __fadd2_rn(alz[i], bezn[i]);
#pragma unroll
                for (int a = 0; a < 3; a++) jb[a] = Az[1 + a] + Bzn[1 + a];
                float Gb[3] = {0.0f, 0.0f, 0.0f};
                if (FORCE) faceG(2, gx, gy, kz + 1, Gb);
                relax_face(AZ, F, Az[0] + Bzn[0], jb, Gb, fzp);
            }
        }

        // consumer barrier; a wait that gave up makes every consumer leave together
        if (cons_bar_or(!ok)) {
            release(kz - 1);
            return;
        }
        if (need_y) {
            if (!ydir) {
                const float *nb = xb + (row * 32 + lane) * K::BS;  // row + 1's entry
                float2 F[5];
#pragma unroll
                for (int i = 0; i < 5; i++) F[i] = __fadd2_rn(aly[i], ld2(nb + 2 * i));
                const float2 nb0 = ld2(nb + 10), nb1 = ld2(nb + 12);
                const float jb[3] = {Ay[1] + nb0.y, Ay[2] + nb1.x, Ay[3] + nb1.y};
                float Gb[3] = {0.0f, 0.0f, 0.0f};
                if (FORCE) faceG(1, gx, gy + 1, kz, Gb);
                relax_face(AY, F, Ay[0] + nb0.x, jb, Gb, fyp);
            }
            float *o = xf + (row * 32 + lane) * K::FS;
#pragma unroll
            for (int i = 0; i < 5; i++) st2(o + 2 * i, fyp[i]);
        }
        cons_bar();

        // ---- P5: steps 8-9, update of cell (gx, gy, kz) ----
        if (upd) {
            // f at the cell's +x and -x interfaces, from the producer warps
            float2 fxp[5], fxm[5];
            const float *xo = fxb + ((kz & 1) * K::NUC + (row - 1) * 32 + lane) * K::FS;
#pragma unroll
            for (int i = 0; i < 5; i++) {
                fxp[i] = ld2(xo + 2 * i);
                fxm[i] = ld2(xo - K::FS + 2 * i);
            }
            const float *ym = xf + ((row - 1) * 32 + lane) * K::FS;
            const int us = (nidx(kz) % 3) * K::NUC + (row - 1) * 32 + lane;
            const float *u0 = u0b + us * K::UP;
            const int64_t off = (int64_t)kz * p.plane + (int64_t)gy * p.px + gx;
            const CellRandom rnd(seed, off);
            const float2 TK = f2(-cf.two_kappa, -cf.two_kappa);
            sfor<9>([&](auto jc) {
                constexpr int j = jc;
                // flux difference of the pair along each axis it crosses, weighted by (e, -e)
                float2 acc = f2(0.0f, 0.0f);
                if constexpr (pr::e(j, 0) != 0) {
                    constexpr int i = pr::pos(0, j);
                    acc = __fmul2_rn(f2((float)pr::e(j, 0), (float)-pr::e(j, 0)), sub2(fxp[i], fxm[i]));
                }
                if constexpr (pr::e(j, 1) != 0) {
                    constexpr int i = pr::pos(1, j);
                    const float2 dv = sub2(fyp[i], ld2(ym + 2 * i));
                    const float2 ev = f2((float)pr::e(j, 1), (float)-pr::e(j, 1));
                    acc = pr::e(j, 0) != 0 ? __ffma2_rn(ev, dv, acc) : __fmul2_rn(ev, dv);
                }
                if constexpr (pr::e(j, 2) != 0) {
                    constexpr int i = pr::pos(2, j);
                    const float2 dv = sub2(fzp[i], fzm[i]);
                    const float2 ev = f2((float)pr::e(j, 2), (float)-pr::e(j, 2));
                    acc = (pr::e(j, 0) != 0 || pr::e(j, 1) != 0) ? __ffma2_rn(ev, dv, acc) : __fmul2_rn(ev, dv);
                }
                // eq. (16): f~(t+dt) = f~+ - dt/|V| flux
                const float2 v = __ffma2_rn(TK, acc, ld2(u0 + 2 * j));
                store_state_pair<S>(dst + j * p.dstride + off, v.x, dst + (18 - j) * p.dstride + off, v.y,
                                    sizeof(S) == 2 ? rnd.word<j>() : 0u);
            });
            store_state_one<S>(dst + 9 * p.dstride + off, u0r[us], sizeof(S) == 2 ? rnd.word<9>() : 0u);
#pragma unroll
            for (int i = 0; i < 5; i++) { fzm[i] = fzp[i]; alz[i] = alzn[i]; }
#pragma unroll
            for (int i = 0; i < 4; i++) Az[i] = Azn[i];
        }
        // this thread has read the ring slot of plane kz - 1 for the last time
        release(kz - 1);
    }
}

}  // namespace dugks
