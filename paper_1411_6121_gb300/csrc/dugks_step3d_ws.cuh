// dugks_step3d_ws.cuh -- warp-specialised throughput kernel of the fused DUGKS time step for
// D3Q19 on sm_103a (FP32 arithmetic, F32/BF16/F16 storage): the scheme and readings of
// dugks_step3d.cuh, with the z march split between two groups of warps that run concurrently.
//
//  * Producer warps (8, one cell column each) make step 1 for plane kz + 2 and
//    beyond: the state of the tile's plane arrives by TMA into one shared-memory stage, each
//    column forms fbar+, its ten moments and u0 = fbar+ + (fbar+ - f~)/3, then the ghost
//    columns and rows (step 2) and, beyond non-periodic z walls, the ghost planes.
//  * Consumer warps (8, one cell column each, the 32 x 8 layout of the non-specialised kernel)
//    do steps 3-9 for plane kz: the per-cell interface parts, the x, y and z interfaces and the
//    update, exactly as dugks_step3d.cuh does them.
//  * The planes pass through a ring of four slots (fbar+ and moments) and three u0 slots. Each
//    ring slot has a "full" mbarrier (every producer thread arrives after its last write of the
//    plane) and an "empty" one (every consumer thread arrives after its last read), so neither
//    group waits on a CTA-wide barrier: the producer runs up to two planes ahead and the
//    step-1 work of one plane overlaps the interface work of another. The consumers' y exchange
//    and the producers' ghost passes use named barriers of their own group.
// The 512 threads launch with 128 registers each; the producer warpgroups then give registers
// back (setmaxnreg to PROD_REGS) and the consumer warpgroups take them (CONS_REGS): 256 x 72 +
// 256 x 184 = 512 x 128 (the force-free kernels then spill nothing). Every wait on an mbarrier gives up after about two seconds (a device
// flag, then the group leaves together; see tma.cuh).
#pragma once

#include "dugks_step3d.cuh"

namespace dugks {

template <int Q, class S>
struct ShapeWS {
    static constexpr int RX = 32, RY = 8, NC = RX * RY;  // cell columns of the tile, halo included
    static constexpr int NPROD = NC, NCONS = NC, NTHREADS = NPROD + NCONS;
    static constexpr int PROD_REGS = 72, CONS_REGS = 184;
    static_assert(NPROD * PROD_REGS + NCONS * CONS_REGS <= NTHREADS * 128, "register split above the launch's");
    static constexpr int TXI = RX - 2, TYI = RY - 2;  // inner columns
    static constexpr int NF = n_flux<Q>(0);
    static constexpr int NM = 10;
    static constexpr int CS = Q + NM;               // ring floats per cell
    static constexpr int BS = (NF + 4) | 1;         // y exchange: beta_y + B_y
    static constexpr int FS = NF | 1;               // y exchange: f at +y
    static constexpr int US = Q | 1;                // u0 of one column and plane
    static constexpr int NSLOT = 4, NU0 = 3;
    static constexpr int PLANE = RY * RX * CS;
    static constexpr size_t FLOATS = (size_t)NSLOT * PLANE + (size_t)NC * (BS + FS) + (size_t)NU0 * NC * US;
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

template <int Q, class S, bool FORCE>
__global__ void __launch_bounds__(512, 1)
    fused_step3d_ws(const __grid_constant__ StepParams p, const __grid_constant__ CUtensorMap tmap, int zchunk) {
    using K = ShapeWS<Q, S>;
    constexpr int RY = K::RY;
    constexpr int NF = K::NF;
    constexpr int CS = K::CS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(p.nz, z0 + zchunk);
    const int x0 = blockIdx.x * K::TXI, y0 = blockIdx.y * K::TYI;

    float *ring = reinterpret_cast<float *>(smem_raw);  // [NSLOT][RY][32][CS]: fbar+ then moments
    float *xb = ring + K::NSLOT * K::PLANE;            // [RY][32][BS]: beta_y, B_y
    float *xf = xb + K::NC * K::BS;                    // [RY][32][FS]: f at +y
    float *u0b = xf + K::NC * K::FS;                   // [NU0][RY][32][US]
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
        // the column of this thread: c = tid
        struct Col {
            int lane, row, gx, gy, cx, cy;
            bool load, boxed, xghost, yghost;
        };
        constexpr int NCOL = K::NC / K::NPROD;
        Col col[NCOL];
#pragma unroll
        for (int i = 0; i < NCOL; i++) {
            Col &c = col[i];
            const int cc = tid + K::NPROD * i;
            c.lane = cc & 31;
            c.row = cc >> 5;
            c.gx = x0 - 1 + c.lane;
            c.gy = y0 - 1 + c.row;
            c.cx = c.gx;
            c.cy = c.gy;
            c.load = true;
            if (c.gx < 0 || c.gx >= nx) { if (perx && c.gx >= -1 && c.gx <= nx) c.cx = wrap_idx(c.gx, nx); else c.load = false; }
            if (c.gy < 0 || c.gy >= ny) { if (pery && c.gy >= -1 && c.gy <= ny) c.cy = wrap_idx(c.gy, ny); else c.load = false; }
            c.boxed = c.load && c.cx == c.gx && c.cy == c.gy;
            const bool yreal = (c.gy >= 0 && c.gy < ny) || (pery && c.gy >= -1 && c.gy <= ny);
            c.xghost = !perx && (c.gx == -1 || c.gx == nx) && yreal;
            c.yghost = !pery && (c.gy == -1 || c.gy == ny) && c.gx >= -1 && c.gx <= nx;
        }
        int m = 0;  // real planes read from the stage so far
        // step 1 for real plane pz into its ring and u0 slots
        auto make_plane = [&](int pz) __attribute__((always_inline)) {
            const int gz = wrap_idx(pz, nz);
            const int sl = slot_of(pz);
            float g[NCOL][Q];
            ok = ok && mbar_wait(sbar, (uint32_t)(m & 1));
            m++;
#pragma unroll
            for (int i = 0; i < NCOL; i++) {
                const Col &c = col[i];
                const S *sb = reinterpret_cast<const S *>(stage) + c.row * K::BX + ((x0 - 1) - xs + c.lane);
                if (c.boxed) {
#pragma unroll
                    for (int k = 0; k < Q; k++) g[i][k] = stage_value(sb + k * (RY * K::BX));
                } else if (c.load) {
                    const int64_t off = (int64_t)gz * p.plane + (int64_t)c.cy * p.px + c.cx;
#pragma unroll
                    for (int k = 0; k < Q; k++) g[i][k] = (float)Store<S>::ld(src + k * p.dstride + off);
                } else {
#pragma unroll
                    for (int k = 0; k < Q; k++) g[i][k] = 0.0f;
                }
            }
            named_bar(1, K::NPROD);  // the stage has been read: the next plane may land in it
            // the next real plane in order
            issue(pz + 1 <= lastp ? pz + 1 : lastp + 1);
#pragma unroll
            for (int i = 0; i < NCOL; i++) {
                const Col &c = col[i];
                float *o = R(sl, c.row, c.lane);
                float *u0 = u0b + ((nidx(pz) % 3) * K::NC + c.row * 32 + c.lane) * K::US;
                if (!c.load) {
#pragma unroll
                    for (int k = 0; k < CS; k++) o[k] = 0.0f;
                    continue;
                }
                float Gh[3] = {0.0f, 0.0f, 0.0f}, drho, mo3[3];
                if (FORCE) {
                    const int64_t ci = (int64_t)c.cx + (int64_t)nx * ((int64_t)c.cy + (int64_t)ny * gz);
                    cell_G<3, float>(p, ci, ncell, ct, Gh);
                }
                moments<Q, float, true>(g[i], Gh, cf.wcell * cf.rho0, drho, mo3);
                float f[Q];
                relax<Q, float, FORCE>(g[i], drho, mo3, Gh, cf.rho0, cf.inv_rho0, cf.b1, cf.c1, f);
                float mo[10];
                phi_moments<Q>(f, mo);
#pragma unroll
                for (int k = 0; k < Q; k++) {
                    o[k] = f[k];
                    u0[k] = fmaf(1.0f / 3.0f, f[k] - g[i][k], f[k]);
                }
#pragma unroll
                for (int j = 0; j < 10; j++) o[Q + j] = mo[j];
            }
        };
        // step 2 (reading R3: ghost = 2 f0 - f1, x then y): fbar+ and, by linearity, its moments
        auto ghosts_xy = [&](int pz) __attribute__((always_inline)) {
            const int sl = slot_of(pz);
            if (xwall_tile) {
                named_bar(1, K::NPROD);
#pragma unroll
                for (int i = 0; i < NCOL; i++) {
                    const Col &c = col[i];
                    if (!c.xghost) continue;
                    const int d1 = c.gx < 0 ? 1 : -1;
                    float *o = R(sl, c.row, c.lane);
                    const float *a = R(sl, c.row, c.lane + d1), *b = R(sl, c.row, c.lane + 2 * d1);
#pragma unroll
                    for (int k = 0; k < CS; k++) o[k] = ghost_value(a[k], b[k]);
                }
            }
            if (ywall_tile) {
                named_bar(1, K::NPROD);
#pragma unroll
                for (int i = 0; i < NCOL; i++) {
                    const Col &c = col[i];
                    if (!c.yghost) continue;
                    const int d1 = c.gy < 0 ? 1 : -1;
                    float *o = R(sl, c.row, c.lane);
                    const float *a = R(sl, c.row + d1, c.lane), *b = R(sl, c.row + 2 * d1, c.lane);
#pragma unroll
                    for (int k = 0; k < CS; k++) o[k] = ghost_value(a[k], b[k]);
                }
            }
        };
        // a ghost plane beyond a non-periodic z wall (whole region)
        auto ghost_z = [&](int pz) __attribute__((always_inline)) {
#pragma unroll
            for (int i = 0; i < NCOL; i++) {
                const Col &c = col[i];
                float *o = R(slot_of(pz), c.row, c.lane);
                const float *a = R(slot_of(pz < 0 ? 0 : nz - 1), c.row, c.lane);
                const float *b = R(slot_of(pz < 0 ? 1 : nz - 2), c.row, c.lane);
#pragma unroll
                for (int k = 0; k < CS; k++) o[k] = ghost_value(a[k], b[k]);
            }
        };
        auto leave = [&]() __attribute__((always_inline)) {
            if (tid == 0) mbar_wait(sbar, (uint32_t)(m & 1));  // a copy still in flight: bounded wait
        };

        // prologue: planes z0 - 1 .. z0 + 1 (a ghost plane below z = 0 after the planes it needs)
        for (int pz = z0 - 1; pz <= z0 + 1; pz++) {
            if (!perz && (pz < 0 || pz >= nz)) continue;
            make_plane(pz);
        }
        for (int pz = z0 - 1; pz <= z0 + 1; pz++) {
            if (!perz && (pz < 0 || pz >= nz)) continue;
            ghosts_xy(pz);
        }
        if (named_bar_or(1, K::NPROD, !ok)) { leave(); return; }
        for (int pz = z0 - 1; pz <= z0 + 1; pz++)
            if (!perz && (pz < 0 || pz >= nz)) ghost_z(pz);
        for (int pz = z0 - 1; pz <= z0 + 1; pz++) mbar_arrive(full + slot_of(pz));
        // the rest of the chunk, each plane into a slot the consumers have released
        for (int pz = z0 + 2; pz <= z1; pz++) {
            const int n = nidx(pz);
            if (n >= 4) ok = ok && mbar_wait(empty + (n & 3), (uint32_t)(((n >> 2) - 1) & 1));
            if (perz || pz < nz) {
                make_plane(pz);
                ghosts_xy(pz);
            } else if (pz == nz) {
                ghost_z(pz);
            }
            if (named_bar_or(1, K::NPROD, !ok)) { leave(); return; }
            mbar_arrive(full + (n & 3));
        }
        return;
    }

    // =============================== consumers ===============================
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(K::CONS_REGS));
    const int ctid = tid - K::NPROD;
    const int lane = ctid & 31, row = ctid >> 5;
    const int gx = x0 - 1 + lane, gy = y0 - 1 + row;
    const bool inner = lane >= 1 && lane <= K::TXI && row >= 1 && row <= K::TYI;
    const bool upd = inner && gx < nx && gy < ny;
    const bool need_x = row >= 1 && row <= K::TYI && gy >= 0 && gy < ny && lane <= K::TXI && gx >= -1 && gx < nx;
    const bool ycol = lane >= 1 && lane <= K::TXI && gx >= 0 && gx < nx && gy >= -1 && gy <= ny;
    const bool need_y = ycol && row <= K::TYI && gy < ny;
    uint32_t seed = 0;  // stochastic rounding of 16-bit stores
    if constexpr (sizeof(S) == 2) seed = store_seed(*p.step_ctr + p.step_off);
    auto U = [&](int pz) __attribute__((always_inline)) -> float * {
        return u0b + ((nidx(pz) % 3) * K::NC + row * 32 + lane) * K::US;
    };
    auto wait_full = [&](int pz) __attribute__((always_inline)) -> bool {
        const int n = nidx(pz);
        return mbar_wait(full + (n & 3), (uint32_t)((n >> 2) & 1));
    };
    auto release = [&](int pz) __attribute__((always_inline)) {
        if (pz >= z0 - 1) mbar_arrive(empty + slot_of(pz));
    };
    auto cons_bar = [&]() __attribute__((always_inline)) { named_bar(2, K::NCONS); };
    auto cons_bar_or = [&](bool v) __attribute__((always_inline)) { return named_bar_or(2, K::NCONS, v); };
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

    bool ok = true;
    for (int pz = z0 - 1; pz <= z0 + 1; pz++) ok = ok && wait_full(pz);
    if (cons_bar_or(!ok)) return;

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
        // ---- plane kz+1 (fbar+, moments, ghosts) from the producer warps; planes z0 - 1 .. z0 + 1
        //      were awaited before the loop ----
        if (kz > z0) ok = ok && wait_full(kz + 1);
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
        // ---- P2: z parts of plane kz+1 and the z interface kz+1/2, before the first consumer
        //      barrier: they need nothing from the y exchange, so the x interfaces, the y parts
        //      and the z interface form one barrier-free phase of independent chains ----
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

        // consumer barrier; a wait that gave up makes every consumer leave together
        if (cons_bar_or(!ok)) {
            release(kz - 1);
            return;
        }
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
        cons_bar();

        // ---- P5: steps 8-9, update of cell (gx, gy, kz) ----
        float fxm[NF];
        if (row >= 1 && row <= K::TYI) {
#pragma unroll
            for (int i = 0; i < NF; i++) fxm[i] = __shfl_up_sync(0xffffffffu, fxp[i], 1);
        }
        if (upd) {
            const float *ym = xf + ((row - 1) * 32 + lane) * K::FS;
            const float *u0 = U(kz);
            const int64_t off = (int64_t)kz * p.plane + (int64_t)gy * p.px + gx;
            const CellRandom rnd(seed, off);
            float v[Q];
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
                // eq. evolution_equation: f~(t+dt) = f~+ - dt/|V| flux
                v[k] = fmaf(-cf.two_kappa, acc, u0[k]);
            });
            // velocities 2i and 2i+1 share one random word and one rounding instruction
            sfor<Q / 2>([&](auto ic) {
                constexpr int i = ic;
                store_state_pair<S>(dst + (2 * i) * p.dstride + off, v[2 * i], dst + (2 * i + 1) * p.dstride + off,
                                    v[2 * i + 1], sizeof(S) == 2 ? rnd.word<i>() : 0u);
            });
            if constexpr (Q % 2 == 1)
                store_state_one<S>(dst + (Q - 1) * p.dstride + off, v[Q - 1], sizeof(S) == 2 ? rnd.word<Q / 2>() : 0u);
#pragma unroll
            for (int i = 0; i < NF; i++) { fzm[i] = fzp[i]; alz[i] = alzn[i]; }
#pragma unroll
            for (int i = 0; i < 4; i++) Az[i] = Azn[i];
        }
        // this thread has read the ring slot of plane kz - 1 for the last time
        release(kz - 1);
    }
}

}  // namespace dugks
