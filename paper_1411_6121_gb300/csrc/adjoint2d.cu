// adjoint2d.cu -- hand-written discrete adjoint of the 2D (D2Q9) DUGKS step, and the
// checkpointed reverse sweep behind dugks_record / dugks_adjoint.
//
// One step Phi: g~^n -> g~^{n+1} (Appendix steps 1-10 of arXiv 1411.6121 in deviation form,
// as dugks_step.cuh computes it) depends on the acceleration field G(x) and on the wall
// velocities u_w. For lambda' = dL/dg~^{n+1} one reverse step forms
//     lambda = (dPhi/dg~^n)^T lambda',  dL/dG += (dPhi/dG)^T lambda',  dL/du_w += (dPhi/du_w)^T lambda'
// by running the sub-steps backwards in three gather-form kernels:
//   adj_cells_fwd (per cell)       recomputes the cell moments (eq. (27)) and
//                                  fbar+ (step 1, eq. (24));
//   adj_faces_all (per interface)  recomputes steps 3-7 and pulls lambda' back through the
//                                  flux (steps 8-9), the interface relaxation (step 7,
//                                  eq. (20)), the interface moments (step 6) and the
//                                  wall condition (step 5: eq. (32), or eq. (31)), down to the
//                                  adjoint of the step-4 values and of the interface
//                                  acceleration;
//   adj_cells_all (per cell)       transposes the reconstruction (steps 3-4, eq. (23))
//                                  and the ghost extrapolation (step 2), then pulls the
//                                  adjoint of fbar+ back through step 1 and the cell moments
//                                  to g~^n and G; then it makes adj_cells_fwd's work for the
//                                  next reverse step, which leaves adj_cells_fwd to the first
//                                  reverse step of each checkpoint segment.
// The interior of each kernel takes a fast path with compile-time velocities; the band along
// walls, x_c interfaces and periodic seams takes the general path, one item per half-warp with
// one velocity per lane. Every output element is a gather written by one thread, or by one lane
// after a fixed-order butterfly over the velocities (no atomics), so the sweep is bitwise
// reproducible. Arithmetic in the storage type of the handle (float or double). The adjoint
// covers the incompressible model (eq. (6)).
//
// Interfaces: normal to x, (i, j) with i in [0, nx], j in [0, ny), between cells (i-1, j)
// and (i, j), index i + (nx+1) j; normal to y, (i, j) with i in [0, nx), j in [0, ny],
// between (i, j-1) and (i, j), index i + nx j. The forward step evaluates interface 0 and
// interface n of a periodic axis separately (equal values): the first feeds cell 0, the
// second cell n-1, and so they are two interfaces here as well.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "../../include/dugks.h"
#include "dugks_internal.h"
#include "handle.h"

namespace dugks {

namespace {

constexpr int Q = 9;
using L9 = Lat<9>;

template <class T>
struct AdjParams {
    int n[2];                // nx, ny
    int per[2];              // periodic along x / y
    int64_t px, dstride;     // layout of the stored state (row pitch, direction stride)
    int bc[4];               // DUGKS_BC_* of the faces -x, +x, -y, +y
    T mw[4][2];              // wall momentum rho0 u_w / c of a velocity condition
    T drw[4];                // rho_a - rho0 = p_w / RT of a pressure condition
    T drw1[4];               // its oscillating part: + drw1 cos(omega (t_n + h))
    T rho0, inv_rho0, dmw;   // dmw = d m_w / d u_w = rho0 / c
    T b1, c1, b7, c7, kappa, two_kappa, wcell, wface;
    T g[2];                  // uniform acceleration
    const float *field;      // [2][ncell] acceleration field or null
    T ctc, cthc;             // cos(omega t_n) / c and cos(omega (t_n + h)) / c
    T cwh;                   // cos(omega (t_n + h))
    const T *state;          // g~^n (padded layout)
    T *phi;                  // [Q][ncell] fbar+ of the cells
    T *mom;                  // [3][ncell] drho, m_x, m_y of the cells (m in units of c)
    const T *nstate;         // g~^{n-1} for the next reverse step's recompute, or null
    T nctc;                  // cos(omega t_{n-1}) / c
    T *nmom;                 // its cell moments (the other moments buffer)
    const T *lam1;           // lambda' [Q][ncell]
    T *fb[2];                // adjoint of the step-4 values [Q][nface_d]
    T *gb[2];                // adjoint of the interface acceleration Gh [2][nface_d]
    T *lam0;                 // lambda [Q][ncell]
    double *dG;              // [2][ncell] dL/dfield accumulator (null: not wanted)
    double *dW;              // [2 (ny + nx)][2] dL/du_w accumulator per wall interface
};

template <class T>
__device__ __forceinline__ int64_t ncell(const AdjParams<T> &a) {
    return (int64_t)a.n[0] * a.n[1];
}
template <class T>
__device__ __forceinline__ int64_t nface(const AdjParams<T> &a, int d) {
    return d == 0 ? (int64_t)(a.n[0] + 1) * a.n[1] : (int64_t)a.n[0] * (a.n[1] + 1);
}
template <class T>
__device__ __forceinline__ int64_t fidx(const AdjParams<T> &a, int d, int i, int j) {
    return d == 0 ? i + (int64_t)(a.n[0] + 1) * j : i + (int64_t)a.n[0] * j;
}

// ---- step 2: extended positions -1 .. n along one axis (reading R3: ghost = 2 f(0) - f(1)
// at a wall, the periodic image otherwise) ----
// The transpose: positions that cell x contributes to and the weights (at most 3).
template <class T>
__device__ __forceinline__ int ext_users(int x, int n, int per, int c[3], T w[3]) {
    int k = 0;
    c[k] = x; w[k++] = T(1);
    if (per) {
        if (x == n - 1) { c[k] = -1; w[k++] = T(1); }
        if (x == 0) { c[k] = n; w[k++] = T(1); }
    } else {
        if (x == 0) { c[k] = -1; w[k++] = T(2); }
        if (x == 1) { c[k] = -1; w[k++] = T(-1); }
        if (x == n - 1) { c[k] = n; w[k++] = T(2); }
        if (x == n - 2) { c[k] = n; w[k++] = T(-1); }
    }
    return k;
}

// fbar+ at an extended position, branch-free: always two cells per axis (the second with
// weight 0 where the position is a real cell or a periodic image), so every load address is
// known up front and the loads of a reconstruction can all be in flight together.
template <class T>
__device__ __forceinline__ void ext2(int x, int n, int per, int c[2], T w[2]) {
    if (x >= 0 && x < n) { c[0] = x; c[1] = x; w[0] = T(1); w[1] = T(0); }
    else if (per) { c[0] = x < 0 ? x + n : x - n; c[1] = c[0]; w[0] = T(1); w[1] = T(0); }
    else { c[0] = x < 0 ? 0 : n - 1; c[1] = x < 0 ? 1 : n - 2; w[0] = T(2); w[1] = T(-1); }
}
template <class T>
__device__ __forceinline__ T phi_ext(const AdjParams<T> &a, int k, int x, int y) {
    int cx[2], cy[2];
    T wx[2], wy[2];
    ext2<T>(x, a.n[0], a.per[0], cx, wx);
    ext2<T>(y, a.n[1], a.per[1], cy, wy);
    const T *ph = a.phi + k * ncell(a);
    const int64_t r0 = (int64_t)a.n[0] * cy[0], r1 = (int64_t)a.n[0] * cy[1];
    const T p00 = ph[cx[0] + r0], p10 = ph[cx[1] + r0], p01 = ph[cx[0] + r1], p11 = ph[cx[1] + r1];
    return wy[0] * (wx[0] * p00 + wx[1] * p10) + wy[1] * (wx[0] * p01 + wx[1] * p11);
}

// ---- steps 3-4: step-4 value of velocity k at interface (d, i, j) (eq. (23) with the
// step-3 cross points): 1/2 (L + R) - kappa e_d (R - L) - kappa/4 e_t [(L+R)_{t+1} - (L+R)_{t-1}] ----
template <class T>
__device__ __forceinline__ T recon(const AdjParams<T> &a, int d, int i, int j, int k) {
    const int ed = L9::e(k, d), et = L9::e(k, 1 - d);
    const int lx = d == 0 ? i - 1 : i, ly = d == 1 ? j - 1 : j;
    const T l = phi_ext(a, k, lx, ly), r = phi_ext(a, k, i, j);
    T v = T(0.5) * (l + r) - a.kappa * (T)ed * (r - l);
    if (et) {
        const int tx = d == 0 ? 0 : 1, ty = d == 0 ? 1 : 0;
        const T pp = phi_ext(a, k, lx + tx, ly + ty) + phi_ext(a, k, i + tx, j + ty);
        const T pm = phi_ext(a, k, lx - tx, ly - ty) + phi_ext(a, k, i - tx, j - ty);
        v -= T(0.25) * a.kappa * (T)et * (pp - pm);
    }
    return v;
}

// Transpose of recon: d/d fbar+(x, y) of sum over interfaces of fb . F (velocity k).
template <class T>
__device__ __forceinline__ T recon_T(const AdjParams<T> &a, int k, int x, int y) {
    const int ex = L9::e(k, 0), ey = L9::e(k, 1);
    const int64_t n0 = nface(a, 0), n1 = nface(a, 1);
    const T *f0 = a.fb[0] + k * n0, *f1 = a.fb[1] + k * n1;
    // branch-free: the index is clamped into range and the value masked, so the loads do
    // not wait on one another
    auto fx = [&](int i, int j) -> T {
        const bool in = !(i < 0 || i > a.n[0] || j < 0 || j >= a.n[1]);
        const T v = f0[fidx(a, 0, min(max(i, 0), a.n[0]), min(max(j, 0), a.n[1] - 1))];
        return in ? v : T(0);
    };
    auto fy = [&](int i, int j) -> T {
        const bool in = !(i < 0 || i >= a.n[0] || j < 0 || j > a.n[1]);
        const T v = f1[fidx(a, 1, min(max(i, 0), a.n[0] - 1), min(max(j, 0), a.n[1]))];
        return in ? v : T(0);
    };
    const T h = T(0.5), q = T(0.25) * a.kappa;
    // as L of x interface (x+1, y), R of (x, y); as a tangential neighbour of the x
    // interfaces of rows y-1 (their t+1 pair) and y+1 (their t-1 pair)
    T v = (h + a.kappa * ex) * fx(x + 1, y) + (h - a.kappa * ex) * fx(x, y);
    if (ey) v += q * (T)ey * ((fx(x + 1, y + 1) + fx(x, y + 1)) - (fx(x + 1, y - 1) + fx(x, y - 1)));
    // the same for the y interfaces, tangential along x
    v += (h + a.kappa * ey) * fy(x, y + 1) + (h - a.kappa * ey) * fy(x, y);
    if (ex) v += q * (T)ex * ((fy(x + 1, y + 1) + fy(x + 1, y)) - (fy(x - 1, y + 1) + fy(x - 1, y)));
    return v;
}

// ---- equilibrium (eq. (6), deviation form, m = rho0 u / c) and its derivative ----
template <class T>
__device__ __forceinline__ T geq(const AdjParams<T> &a, int k, T dr, const T m[2]) {
    const T em = (T)L9::e(k, 0) * m[0] + (T)L9::e(k, 1) * m[1];
    const T mm = m[0] * m[0] + m[1] * m[1];
    return L9::wt<T>(k) * (dr + T(3) * em + (T(4.5) * em * em - T(1.5) * mm) * a.inv_rho0);
}
template <class T>
__device__ __forceinline__ void geq_dm(const AdjParams<T> &a, int k, const T m[2], T out[2]) {
    const T e0 = (T)L9::e(k, 0), e1 = (T)L9::e(k, 1);
    const T em = e0 * m[0] + e1 * m[1];
    const T W = L9::wt<T>(k);
    out[0] = W * (T(3) * e0 + (T(9) * em * e0 - T(3) * m[0]) * a.inv_rho0);
    out[1] = W * (T(3) * e1 + (T(9) * em * e1 - T(3) * m[1]) * a.inv_rho0);
}

// Moments of a distribution with the force weight w (dt/2 at cells, h/2 at interfaces).
template <class T>
__device__ __forceinline__ void moments2(const AdjParams<T> &a, const T f[Q], const T Gh[2], T w, T &dr, T m[2]) {
    dr = T(0);
    m[0] = m[1] = T(0);
    for (int k = 0; k < Q; k++) {
        dr += f[k];
        m[0] += (T)L9::e(k, 0) * f[k];
        m[1] += (T)L9::e(k, 1) * f[k];
    }
    m[0] += a.rho0 * Gh[0] * w;
    m[1] += a.rho0 * Gh[1] * w;
}

// ---- the general path, velocity-parallel: one half-warp per item of the boundary frame,
// lane k of the half (k < Q) holding velocity k and lanes k >= Q zeros. Sums over the
// velocities are butterflies over the half-warp: every lane ends with the same bits and the
// order is fixed. The two halves of a warp work on different items and may diverge, so the
// shuffles name only their own half. ----
__device__ __forceinline__ int half_lane() { return threadIdx.x & 15; }
template <class T>
__device__ __forceinline__ T wsum(T v) {
    const unsigned m = 0xffffu << (threadIdx.x & 16);
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) v += __shfl_xor_sync(m, v, o, 16);
    return v;
}

// Relaxation P_k = f_k + b (geq_k - f_k) + c S_k with S_k = 3 (Gh.e_k - Gh.m/rho0) f_eq,k
// (steps 1 and 7). Given the weight w = dL/dP_k of one velocity k, its share of dL/d(drho),
// dL/dm and dL/dGh through the moment dependence (the direct part (1 - b) w is left to the
// caller); summed over the velocities by the caller.
template <class T>
__device__ __forceinline__ void relax_T_one(const AdjParams<T> &a, int k, T w, T dr, const T m[2], const T Gh[2],
                                            T b, T c, T &bdr, T bm[2], T bG[2]) {
    const T gm = (Gh[0] * m[0] + Gh[1] * m[1]) * a.inv_rho0;
    const T e0 = (T)L9::e(k, 0), e1 = (T)L9::e(k, 1);
    const T W = L9::wt<T>(k);
    const T s = T(3) * (Gh[0] * e0 + Gh[1] * e1 - gm);
    const T feq = W * a.rho0 + geq(a, k, dr, m);
    T dg[2];
    geq_dm(a, k, m, dg);
    const T coef = b + c * s;  // dP/dgeq
    bdr = w * coef * W;
    bm[0] = w * (coef * dg[0] - c * T(3) * Gh[0] * a.inv_rho0 * feq);
    bm[1] = w * (coef * dg[1] - c * T(3) * Gh[1] * a.inv_rho0 * feq);
    bG[0] = w * c * T(3) * (e0 - m[0] * a.inv_rho0) * feq;
    bG[1] = w * c * T(3) * (e1 - m[1] * a.inv_rho0) * feq;
}

// ---- acceleration at cells and interfaces (reading R2) ----
template <class T>
__device__ __forceinline__ T field_at(const AdjParams<T> &a, int comp, int x, int y) {
    return a.field ? (T)a.field[comp * ncell(a) + x + (int64_t)a.n[0] * y] : T(0);
}
template <class T>
__device__ __forceinline__ void cell_Gh(const AdjParams<T> &a, int x, int y, T Gh[2]) {
    for (int c = 0; c < 2; c++) Gh[c] = (a.g[c] + field_at(a, c, x, y)) * a.ctc;
}
// Cells whose field the interface at position pos along d averages: wrapped on a periodic
// axis, clamped at a wall (the one boundary cell).
template <class T>
__device__ __forceinline__ void face_cells(const AdjParams<T> &a, int d, int pos, int &lo, int &hi) {
    const int nd = a.n[d];
    lo = pos - 1;
    hi = pos;
    if (a.per[d]) {
        if (lo < 0) lo += nd;
        if (hi >= nd) hi -= nd;
    } else {
        if (lo < 0) lo = 0;
        if (hi >= nd) hi = nd - 1;
    }
}
template <class T>
__device__ __forceinline__ void face_Gh(const AdjParams<T> &a, int d, int i, int j, T Gh[2]) {
    int lo, hi;
    face_cells(a, d, d == 0 ? i : j, lo, hi);
    const int lx = d == 0 ? lo : i, ly = d == 1 ? lo : j, hx = d == 0 ? hi : i, hy = d == 1 ? hi : j;
    for (int c = 0; c < 2; c++)
        Gh[c] = (a.g[c] + T(0.5) * (field_at(a, c, lx, ly) + field_at(a, c, hx, hy))) * a.cthc;
}

// ---- forward state of one interface (steps 3-6), one velocity per lane ----
template <class T>
struct FaceLane {
    T F, Fc;               // step-4 value of the lane's velocity (incoming ones replaced at a
                           // wall, step 5) and its value at x_c (wall only)
    T dr, m[2], Gh[2];     // step-6 moments and the interface acceleration
    int wall, side, bb;    // bb: bounce-back wall (eq. (31))
    T drc, mc[2];          // moments at x_c (wall only)
    T ma[2];               // m_a of step 5 (wall only)
};

template <class T>
__device__ __forceinline__ void face_forward_lane(const AdjParams<T> &a, int d, int i, int j, int k, bool act,
                                                  FaceLane<T> &s) {
    const T e0 = (T)L9::e(k, 0), e1 = (T)L9::e(k, 1);
    s.F = act ? recon(a, d, i, j, k) : T(0);
    const int pos = d == 0 ? i : j;
    s.wall = !a.per[d] && (pos == 0 || pos == a.n[d]);
    s.side = pos == 0 ? 0 : 1;
    face_Gh(a, d, i, j, s.Gh);
    s.Fc = T(0);
    s.bb = s.wall && a.bc[2 * d + s.side] == DUGKS_BC_BOUNCE_BACK;
    if (s.bb) {
        // step 5, eq. (31): the incoming velocity takes its opposite's value (lane 8 - k of the
        // half) plus 6 W_k e_k.m_w
        const T Fo = __shfl_sync(0xffffu << (threadIdx.x & 16), s.F, Q - 1 - k, 16);
        const int sgn = s.side == 0 ? -1 : 1;
        const T *mw = a.mw[2 * d + s.side];
        if (act && sgn * L9::e(k, d) < 0) s.F = Fo + T(6) * L9::wt<T>(k) * (e0 * mw[0] + e1 * mw[1]);
    } else if (s.wall) {
        // x_c: the boundary cell's opposite interface (reading R4)
        const int sh = s.side == 0 ? 1 : -1;
        const int ci = d == 0 ? i + sh : i, cj = d == 1 ? j + sh : j;
        s.Fc = act ? recon(a, d, ci, cj, k) : T(0);
        T Ghc[2];
        face_Gh(a, d, ci, cj, Ghc);
        s.drc = wsum(s.Fc);
        s.mc[0] = wsum(e0 * s.Fc) + a.rho0 * Ghc[0] * a.wface;
        s.mc[1] = wsum(e1 * s.Fc) + a.rho0 * Ghc[1] * a.wface;
        const int wid = 2 * d + s.side;
        const bool vel = a.bc[wid] == DUGKS_BC_NEQ_VELOCITY;
        const T dra = vel ? s.drc : a.drw[wid] + a.drw1[wid] * a.cwh;
        s.ma[0] = vel ? a.mw[wid][0] : s.mc[0];
        s.ma[1] = vel ? a.mw[wid][1] : s.mc[1];
        const int sgn = s.side == 0 ? -1 : 1;
        if (act && sgn * L9::e(k, d) < 0) s.F = geq(a, k, dra, s.ma) + s.Fc - geq(a, k, s.drc, s.mc);
    }
    s.dr = wsum(s.F);
    s.m[0] = wsum(e0 * s.F) + a.rho0 * s.Gh[0] * a.wface;
    s.m[1] = wsum(e1 * s.F) + a.rho0 * s.Gh[1] * a.wface;
}

// Adjoint of steps 5-9 at interface (d, i, j) for lambda', velocity k of this lane. Fb:
// dL/d(step-4 value), zero for a velocity the wall replaces; Gb: dL/dGh of the interface
// (the same in every lane). At a wall also what flows to the step-4 value and Gh of x_c
// (Fcb, Gcb) and to the wall velocity (Wb).
template <class T>
__device__ __forceinline__ void face_adjoint_lane(const AdjParams<T> &a, int d, int i, int j, int k, bool act,
                                                  T &Fb, T Gb[2], T &Fcb, T Gcb[2], T Wb[2], int &wall) {
    FaceLane<T> s;
    face_forward_lane(a, d, i, j, k, act, s);
    wall = s.wall;
    const int64_t nc = ncell(a);
    const int pos = d == 0 ? i : j, nd = a.n[d];
    const T e0 = (T)L9::e(k, 0), e1 = (T)L9::e(k, 1);
    // steps 8-9: velocity k of this interface enters the update of its low cell with
    // -2 kappa e_d and of its high cell with +2 kappa e_d
    const bool haslo = pos > 0, hashi = pos < nd;
    const int plo = pos > 0 ? pos - 1 : nd - 1, phi_c = pos < nd ? pos : 0;
    const int64_t clo = d == 0 ? plo + (int64_t)a.n[0] * j : i + (int64_t)a.n[0] * plo;
    const int64_t chi = d == 0 ? phi_c + (int64_t)a.n[0] * j : i + (int64_t)a.n[0] * phi_c;
    const int ed = L9::e(k, d);
    T v = T(0);
    if (act && ed) {
        if (haslo) v -= a.lam1[k * nc + clo];
        if (hashi) v += a.lam1[k * nc + chi];
    }
    const T fbar = a.two_kappa * (T)ed * v;
    // step 7 (eq. (20)) at the step-6 moments, then step 6
    T bdr, bm[2], bG[2];
    relax_T_one(a, k, fbar, s.dr, s.m, s.Gh, a.b7, a.c7, bdr, bm, bG);
    bdr = wsum(bdr);
    bm[0] = wsum(bm[0]);
    bm[1] = wsum(bm[1]);
    Gb[0] = wsum(bG[0]) + a.rho0 * a.wface * bm[0];
    Gb[1] = wsum(bG[1]) + a.rho0 * a.wface * bm[1];
    Fb = act ? (T(1) - a.b7) * fbar + bdr + e0 * bm[0] + e1 * bm[1] : T(0);
    Fcb = T(0);
    Gcb[0] = Gcb[1] = T(0);
    Wb[0] = Wb[1] = T(0);
    if (!wall) return;
    if (s.bb) {
        // step 5, eq. (31): F_k = F_-k + 6 W_k e_k.m_w for incoming k: the weight of an
        // incoming velocity passes to its opposite (lane 8 - k) and to u_w
        const int sgn = s.side == 0 ? -1 : 1;
        const bool incoming = act && sgn * ed < 0;
        const T w = incoming ? Fb : T(0);
        const T back = __shfl_sync(0xffffu << (threadIdx.x & 16), w, Q - 1 - k, 16);
        Fb = (incoming ? T(0) : Fb) + back;
        const T c6 = T(6) * L9::wt<T>(k) * w * a.dmw;
        Wb[0] = wsum(c6 * e0);
        Wb[1] = wsum(c6 * e1);
        return;
    }
    // step 5 (eq. (32)): F_k = geq_k(drho_a, m_a) + Fc_k - geq_k(drho_c, m_c), incoming k.
    // Velocity condition: drho_a = drho_c (the W_k terms cancel), m_a from u_w.
    // Pressure condition: m_a = m_c (the m terms cancel), drho_a fixed.
    const int wid = 2 * d + s.side;
    const bool vel = a.bc[wid] == DUGKS_BC_NEQ_VELOCITY;
    const int sgn = s.side == 0 ? -1 : 1;
    const bool incoming = act && sgn * ed < 0;
    const T w = incoming ? Fb : T(0);
    if (incoming) Fb = T(0);
    Fcb = w;
    T bdrc = T(0), bmc[2] = {T(0), T(0)};
    if (vel) {
        T da[2], dc[2];
        geq_dm(a, k, s.ma, da);
        geq_dm(a, k, s.mc, dc);
        Wb[0] = wsum(w * da[0] * a.dmw);
        Wb[1] = wsum(w * da[1] * a.dmw);
        bmc[0] = -wsum(w * dc[0]);
        bmc[1] = -wsum(w * dc[1]);
    } else {
        bdrc = -wsum(w * L9::wt<T>(k));
    }
    // step 6 at x_c
    if (act) Fcb += bdrc + e0 * bmc[0] + e1 * bmc[1];
    Gcb[0] = a.rho0 * a.wface * bmc[0];
    Gcb[1] = a.rho0 * a.wface * bmc[1];
}

// ---- fast paths: interfaces and cells whose stencils lie inside the domain, away from
// walls and periodic seams (no ghosts, images, NEQ or x_c coupling). Same arithmetic as the
// general path, with compile-time velocities and direct neighbour reads. ----

// relax_T with a compile-time velocity loop; D >= 0 restricts it to the velocities that
// cross an interface normal to axis D (the others have zero weight there).
template <class T, int D>
__device__ __forceinline__ void relax_T_c(const AdjParams<T> &a, const T wk[Q], T dr, const T m[2], const T Gh[2],
                                          T b, T c, T &bdr, T bm[2], T bG[2]) {
    const T gm = (Gh[0] * m[0] + Gh[1] * m[1]) * a.inv_rho0;
    const T mm = m[0] * m[0] + m[1] * m[1];
    sfor<Q>([&](auto kc) {
        constexpr int k = kc;
        constexpr int e0 = L9::e(k, 0), e1 = L9::e(k, 1);
        if constexpr (D < 0 || L9::e(k, D < 0 ? 0 : D) != 0) {
            const T W = L9::wt<T>(k);
            const T em = T(e0) * m[0] + T(e1) * m[1];
            const T s = T(3) * (Gh[0] * T(e0) + Gh[1] * T(e1) - gm);
            const T feq = W * a.rho0 + W * (dr + T(3) * em + (T(4.5) * em * em - T(1.5) * mm) * a.inv_rho0);
            const T w = wk[k];
            const T cw = w * (b + c * s) * W;  // w dP/dgeq times W
            const T fq = w * c * T(3) * feq;
            bdr += cw;
            bm[0] += cw * (T(3) * T(e0) + (T(9) * em * T(e0) - T(3) * m[0]) * a.inv_rho0) - fq * Gh[0] * a.inv_rho0;
            bm[1] += cw * (T(3) * T(e1) + (T(9) * em * T(e1) - T(3) * m[1]) * a.inv_rho0) - fq * Gh[1] * a.inv_rho0;
            bG[0] += fq * (T(e0) - m[0] * a.inv_rho0);
            bG[1] += fq * (T(e1) - m[1] * a.inv_rho0);
        }
    });
}

// The fast regions. Interfaces normal to d: both cells, their tangential neighbours and
// the cells' own interfaces are in the domain without wrapping, and the interface is neither
// a wall nor the x_c of one. Cells: every interface of the stencil transposed in adj_cells
// is in the domain and the cell feeds no ghost or periodic image. Everything else (a frame
// along the boundary) takes the general path.
struct Rect {
    int W, H;            // index space W x H
    int x0, x1, y0, y1;  // fast rectangle, inclusive (empty when x0 > x1 or y0 > y1)
};
__host__ __device__ inline Rect face_rect(int d, int nx, int ny, int perx, int pery) {
    if (d == 0) {
        const int m = perx ? 1 : 2;
        return Rect{nx + 1, ny, m, nx - m, 1, ny - 2};
    }
    const int m = pery ? 1 : 2;
    return Rect{nx, ny + 1, 1, nx - 2, m, ny - m};
}
__host__ __device__ inline Rect cell_rect(int nx, int ny, int perx, int pery) {
    const int mx = perx ? 1 : 2, my = pery ? 1 : 2;
    return Rect{nx, ny, mx, nx - 1 - mx, my, ny - 1 - my};
}
__host__ __device__ inline bool rect_empty(const Rect &r) { return r.x0 > r.x1 || r.y0 > r.y1; }
__host__ __device__ inline int64_t rect_count(const Rect &r) {
    return rect_empty(r) ? 0 : (int64_t)(r.x1 - r.x0 + 1) * (r.y1 - r.y0 + 1);
}
__host__ __device__ inline int64_t frame_count(const Rect &r) { return (int64_t)r.W * r.H - rect_count(r); }
// The t-th element (row-major) of the index space outside the fast rectangle.
__device__ inline void frame_at(const Rect &r, int64_t t, int &x, int &y) {
    if (rect_empty(r)) {
        x = (int)(t % r.W);
        y = (int)(t / r.W);
        return;
    }
    const int64_t below = (int64_t)r.y0 * r.W, above = (int64_t)(r.H - 1 - r.y1) * r.W;
    if (t < below) {
        x = (int)(t % r.W);
        y = (int)(t / r.W);
    } else if (t < below + above) {
        t -= below;
        x = (int)(t % r.W);
        y = r.y1 + 1 + (int)(t / r.W);
    } else {
        t -= below + above;
        const int side = r.x0 + (r.W - 1 - r.x1);  // frame columns of a middle row
        y = r.y0 + (int)(t / side);
        const int c = (int)(t % side);
        x = c < r.x0 ? c : r.x1 + 1 + (c - r.x0);
    }
}

template <class T, int d>
__device__ __forceinline__ void face_fast(const AdjParams<T> &a, int i, int j, int64_t f, int64_t nf) {
    const int nx = a.n[0];
    const int64_t nc = ncell(a);
    const int64_t cR = i + (int64_t)nx * j;
    const int64_t cL = d == 0 ? cR - 1 : cR - nx;
    const int64_t ts = d == 0 ? nx : 1;  // step to the tangential neighbour
    T F[Q];
    sfor<Q>([&](auto kc) {
        constexpr int k = kc;
        constexpr int ed = L9::e(k, d), et = L9::e(k, 1 - d);
        const T *ph = a.phi + k * nc;
        const T l = ph[cL], r = ph[cR];
        T v = T(0.5) * (l + r);
        if constexpr (ed != 0) v -= a.kappa * T(ed) * (r - l);
        if constexpr (et != 0) v -= T(0.25) * a.kappa * T(et) * ((ph[cL + ts] + ph[cR + ts]) - (ph[cL - ts] + ph[cR - ts]));
        F[k] = v;
    });
    T Gh[2];
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const T fl = a.field ? T(0.5) * ((T)a.field[c * nc + cL] + (T)a.field[c * nc + cR]) : T(0);
        Gh[c] = (a.g[c] + fl) * a.cthc;
    }
    T dr, m[2];
    moments2(a, F, Gh, a.wface, dr, m);
    T fbar[Q];
    sfor<Q>([&](auto kc) {
        constexpr int k = kc;
        constexpr int ed = L9::e(k, d);
        if constexpr (ed != 0) fbar[k] = a.two_kappa * T(ed) * (a.lam1[k * nc + cR] - a.lam1[k * nc + cL]);
        else fbar[k] = T(0);
    });
    T bdr = T(0), bm[2] = {T(0), T(0)}, Gb[2] = {T(0), T(0)};
    relax_T_c<T, d>(a, fbar, dr, m, Gh, a.b7, a.c7, bdr, bm, Gb);
    T *fb = a.fb[d];
    sfor<Q>([&](auto kc) {
        constexpr int k = kc;
        fb[k * nf + f] = (T(1) - a.b7) * fbar[k] + bdr + T(L9::e(k, 0)) * bm[0] + T(L9::e(k, 1)) * bm[1];
    });
    a.gb[d][f] = Gb[0] + a.rho0 * a.wface * bm[0];
    a.gb[d][nf + f] = Gb[1] + a.rho0 * a.wface * bm[1];
}

template <class T>
__device__ __forceinline__ void cell_fast(const AdjParams<T> &a, int x, int y, int64_t c) {
    const int nx = a.n[0];
    const int64_t nc = ncell(a), n0 = nface(a, 0), n1 = nface(a, 1);
    const int64_t ix = x + (int64_t)(nx + 1) * y;  // x interface (x, y): the cell's -x interface
    const int64_t iy = x + (int64_t)nx * y;        // y interface (x, y): the cell's -y interface
    const int64_t sx = nx + 1, sy = nx;            // row strides of the interface arrays
    const T h = T(0.5), q = T(0.25) * a.kappa;
    T pb[Q];
    sfor<Q>([&](auto kc) {
        constexpr int k = kc;
        constexpr int ex = L9::e(k, 0), ey = L9::e(k, 1);
        const T *f0 = a.fb[0] + k * n0, *f1 = a.fb[1] + k * n1;
        T v = T(4) / T(3) * a.lam1[k * nc + c];
        v += (h + a.kappa * T(ex)) * f0[ix + 1] + (h - a.kappa * T(ex)) * f0[ix];
        if constexpr (ey != 0) v += q * T(ey) * ((f0[ix + 1 + sx] + f0[ix + sx]) - (f0[ix + 1 - sx] + f0[ix - sx]));
        v += (h + a.kappa * T(ey)) * f1[iy + sy] + (h - a.kappa * T(ey)) * f1[iy];
        if constexpr (ex != 0) v += q * T(ex) * ((f1[iy + 1 + sy] + f1[iy + 1]) - (f1[iy - 1 + sy] + f1[iy - 1]));
        pb[k] = v;
    });
    const T dr = a.mom[c];
    const T m[2] = {a.mom[nc + c], a.mom[2 * nc + c]};
    T Gh[2];
    cell_Gh(a, x, y, Gh);
    T bdr = T(0), bm[2] = {T(0), T(0)}, bG[2] = {T(0), T(0)};
    relax_T_c<T, -1>(a, pb, dr, m, Gh, a.b1, a.c1, bdr, bm, bG);
    sfor<Q>([&](auto kc) {
        constexpr int k = kc;
        a.lam0[k * nc + c] = -a.lam1[k * nc + c] / T(3) + (T(1) - a.b1) * pb[k] + bdr + T(L9::e(k, 0)) * bm[0] +
                             T(L9::e(k, 1)) * bm[1];
    });
    if (a.dG) {
#pragma unroll
        for (int comp = 0; comp < 2; comp++) {
            const T fs = T(0.5) * (a.gb[0][comp * n0 + ix] + a.gb[0][comp * n0 + ix + 1]) +
                         T(0.5) * (a.gb[1][comp * n1 + iy] + a.gb[1][comp * n1 + iy + sy]);
            a.dG[comp * nc + c] += (double)((bG[comp] + a.rho0 * a.wcell * bm[comp]) * a.ctc + fs * a.cthc);
        }
    }
}

// ---- kernels ----
// fbar+ (step 1, eq. (24)) and the moments (eq. (27)) of cell c of `state` into
// a.phi and `mom`, with ctc = cos(omega t) / c at that state's time. Not inlined: the
// recompute kernel and the cells kernel that carries the next step's recompute run the same
// code, so the sweep's bits do not depend on which of them computed a step.
template <class T>
__device__ __noinline__ void fwd_cell(const AdjParams<T> &a, const T *state, T ctc, T *mom, int64_t c) {
    const int64_t nc = ncell(a);
    const int x = (int)(c % a.n[0]), y = (int)(c / a.n[0]);
    T g[Q], Gh[2], dr, m[2];
#pragma unroll
    for (int k = 0; k < Q; k++) g[k] = state[k * a.dstride + (int64_t)y * a.px + x];
#pragma unroll
    for (int comp = 0; comp < 2; comp++) Gh[comp] = (a.g[comp] + field_at(a, comp, x, y)) * ctc;
    moments2(a, g, Gh, a.wcell, dr, m);
    const T gm = (Gh[0] * m[0] + Gh[1] * m[1]) * a.inv_rho0;
#pragma unroll
    for (int k = 0; k < Q; k++) {
        const T q = geq(a, k, dr, m);
        const T s = T(3) * (Gh[0] * (T)L9::e(k, 0) + Gh[1] * (T)L9::e(k, 1) - gm);
        a.phi[k * nc + c] = g[k] + a.b1 * (q - g[k]) + a.c1 * s * (L9::wt<T>(k) * a.rho0 + q);
    }
    mom[c] = dr;
    mom[nc + c] = m[0];
    mom[2 * nc + c] = m[1];
}

template <class T>
__global__ void __launch_bounds__(256) adj_cells_fwd(const AdjParams<T> a) {
    const int64_t nc = ncell(a);
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x)
        fwd_cell(a, a.state, a.ctc, a.mom, c);
}

// The t-th interface of the frame of both axes (walls: NEQ and dL/du_w; x_c interfaces;
// periodic seams), one velocity per lane of the calling half-warp.
template <class T>
__device__ __noinline__ void faces_frame_item(const AdjParams<T> &a, int64_t t) {
    const Rect r0 = face_rect(0, a.n[0], a.n[1], a.per[0], a.per[1]);
    const Rect r1 = face_rect(1, a.n[0], a.n[1], a.per[0], a.per[1]);
    const int64_t c0 = frame_count(r0);
    const int lane = half_lane();
    const bool act = lane < Q;
    const int k = act ? lane : 0;
    const int d = t < c0 ? 0 : 1;
    int i, j;
    frame_at(d == 0 ? r0 : r1, d == 0 ? t : t - c0, i, j);
    const int64_t f = fidx(a, d, i, j);
    const int pos = d == 0 ? i : j, nd = a.n[d];
    T Fb, Gb[2], Fcb, Gcb[2], Wb[2];
    int wall;
    face_adjoint_lane(a, d, i, j, k, act, Fb, Gb, Fcb, Gcb, Wb, wall);
    const int wbc = a.bc[2 * d + (pos == 0 ? 0 : 1)];
    if (wall && a.dW && lane == 0 && (wbc == DUGKS_BC_NEQ_VELOCITY || wbc == DUGKS_BC_BOUNCE_BACK)) {
        const int64_t slot = d == 0 ? (pos == 0 ? 0 : a.n[1]) + j : 2 * (int64_t)a.n[1] + (pos == 0 ? 0 : a.n[0]) + i;
        a.dW[2 * slot] += (double)Wb[0];
        a.dW[2 * slot + 1] += (double)Wb[1];
    }
    // this interface is x_c of the wall interface at 0 (pos == 1) and/or at nd (pos == nd - 1)
    if (!a.per[d]) {
        for (int sd = 0; sd < 2; sd++) {
            if (pos != (sd == 0 ? 1 : nd - 1)) continue;
            const int wp = sd == 0 ? 0 : nd;
            T wFb, wGb[2], wFcb, wGcb[2], wWb[2];
            int ww;
            face_adjoint_lane(a, d, d == 0 ? wp : i, d == 1 ? wp : j, k, act, wFb, wGb, wFcb, wGcb, wWb, ww);
            Fb += wFcb;
            Gb[0] += wGcb[0];
            Gb[1] += wGcb[1];
        }
    }
    T *fb = a.fb[d], *gb = a.gb[d];
    const int64_t nf = nface(a, d);
    if (act) fb[k * nf + f] = Fb;
    if (lane == 0) {
        gb[f] = Gb[0];
        gb[nf + f] = Gb[1];
    }
}

// Every interface of both axes in one launch of 128-thread blocks: the frame blocks first
// (eight frame interfaces per block, one per half-warp), then 32 x 4 tiles of the interior
// rectangle of x interfaces (nt0 tiles, tx0 per row), then those of y interfaces (tx1 per row).
template <class T>
__global__ void __launch_bounds__(128, 6) adj_faces_all(const AdjParams<T> a, int64_t nframe, int nfb, int nt0,
                                                         int tx0, int tx1) {
    if ((int)blockIdx.x < nfb) {
        const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 4;
        if (t < nframe) faces_frame_item(a, t);
        return;
    }
    int b = (int)blockIdx.x - nfb;
    const int d = b < nt0 ? 0 : 1;
    if (d) b -= nt0;
    const int tx = d ? tx1 : tx0;
    const Rect r = face_rect(d, a.n[0], a.n[1], a.per[0], a.per[1]);
    const int i = r.x0 + (b % tx) * 32 + (threadIdx.x & 31), j = r.y0 + (b / tx) * 4 + (threadIdx.x >> 5);
    if (i > r.x1 || j > r.y1) return;
    const int64_t f = fidx(a, d, i, j);
    if (d == 0) face_fast<T, 0>(a, i, j, f, nface(a, 0));
    else face_fast<T, 1>(a, i, j, f, nface(a, 1));
}

// dL/dGh summed over the interfaces whose acceleration averages cell (x, y), with the
// averaging weights (1/2 per side; the clamped wall interface takes the cell twice).
template <class T>
__device__ __forceinline__ T face_G_T(const AdjParams<T> &a, int comp, int x, int y) {
    T s = T(0);
    for (int d = 0; d < 2; d++) {
        const int pc = d == 0 ? x : y, nd = a.n[d];
        int cand[4], nc = 0;
        cand[nc++] = pc;
        cand[nc++] = pc + 1;
        if (a.per[d] && nd > 1) {  // the interfaces across the periodic seam
            if (pc == nd - 1) cand[nc++] = 0;
            if (pc == 0) cand[nc++] = nd;
        }
        const int64_t nf = nface(a, d);
        for (int u = 0; u < nc; u++) {
            int lo, hi;
            face_cells(a, d, cand[u], lo, hi);
            const T w = (lo == pc ? T(0.5) : T(0)) + (hi == pc ? T(0.5) : T(0));
            if (w != T(0)) {
                const int i = d == 0 ? cand[u] : x, j = d == 1 ? cand[u] : y;
                s += w * a.gb[d][comp * nf + fidx(a, d, i, j)];
            }
        }
    }
    return s;
}

// The t-th frame cell (cells whose stencil meets a wall ghost, a periodic image or a
// wall-clamped interface acceleration), one velocity per lane of the calling half-warp.
template <class T>
__device__ __noinline__ void cells_frame_item(const AdjParams<T> &a, int64_t t) {
    const int64_t nc = ncell(a);
    const Rect r = cell_rect(a.n[0], a.n[1], a.per[0], a.per[1]);
    const int lane = half_lane();
    const bool act = lane < Q;
    const int k = act ? lane : 0;
    int x, y;
    frame_at(r, t, x, y);
    const int64_t c = x + (int64_t)a.n[0] * y;
    int ux[3], uy[3];
    T wx[3], wy[3];
    const int nux = ext_users<T>(x, a.n[0], a.per[0], ux, wx);
    const int nuy = ext_users<T>(y, a.n[1], a.per[1], uy, wy);
    // adjoint of fbar+ of this cell: eq. (25) (4/3 fbar+) and every interface value
    // reconstructed from it, directly or through a ghost / periodic image
    const T l1 = act ? a.lam1[k * nc + c] : T(0);
    T pb = T(0);
    if (act) {
        T v = T(4) / T(3) * l1;
        for (int p = 0; p < nux; p++)
            for (int q = 0; q < nuy; q++) v += wx[p] * wy[q] * recon_T(a, k, ux[p], uy[q]);
        pb = v;
    }
    // step 1 (eq. (24)) and the cell moments (eq. (27))
    const T dr = a.mom[c];
    const T m[2] = {a.mom[nc + c], a.mom[2 * nc + c]};
    T Gh[2];
    cell_Gh(a, x, y, Gh);
    T bdr, bm[2], bG[2];
    relax_T_one(a, k, pb, dr, m, Gh, a.b1, a.c1, bdr, bm, bG);
    bdr = wsum(bdr);
    bm[0] = wsum(bm[0]);
    bm[1] = wsum(bm[1]);
    bG[0] = wsum(bG[0]);
    bG[1] = wsum(bG[1]);
    if (act)
        a.lam0[k * nc + c] = -l1 / T(3) + (T(1) - a.b1) * pb + bdr + (T)L9::e(k, 0) * bm[0] + (T)L9::e(k, 1) * bm[1];
    if (a.dG && lane < 2) {
        const int comp = lane;
        const T sv = (bG[comp] + a.rho0 * a.wcell * bm[comp]) * a.ctc + face_G_T(a, comp, x, y) * a.cthc;
        a.dG[comp * nc + c] += (double)sv;
    }
}

// All cells in one launch of 128-thread blocks: frame blocks first (a half-warp per frame cell),
// then 32 x 4 tiles of the fast rectangle (tx x ty blocks).
// With a.nstate set, the blocks then recompute the next reverse step's fbar+ and moments,
// one cell per thread, the interior tiles first (the frame blocks are the longest): this
// step's interfaces no longer read a.phi, and each cell's moments go to the other buffer, so
// no block reads what another overwrites.
template <class T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 7 : 5) adj_cells_all(const AdjParams<T> a, int nfb, int tx, int ty) {
    const Rect r = cell_rect(a.n[0], a.n[1], a.per[0], a.per[1]);
    if ((int)blockIdx.x < nfb) {  // eight frame cells per block, one per half-warp
        const int64_t t = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 4);
        if (t < frame_count(r)) cells_frame_item(a, t);
    } else {
        const int b = blockIdx.x - nfb;
        const int x = r.x0 + (b % tx) * 32 + (threadIdx.x & 31), y = r.y0 + (b / tx) * 4 + (threadIdx.x >> 5);
        if (x <= r.x1 && y <= r.y1) cell_fast(a, x, y, x + (int64_t)a.n[0] * y);
    }
    if (a.nstate) {
        const int64_t nc = ncell(a);
        const int nb = (int)gridDim.x, bi = (int)blockIdx.x;
        const int rb = bi >= nfb ? bi - nfb : bi + (nb - nfb);  // tiles take blocks 0 .. nb - nfb - 1
        for (int64_t c = rb * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)nb * blockDim.x)
            fwd_cell(a, a.nstate, a.nctc, a.nmom, c);
    }
}

// Loss seed from dL/d(moments) [3][ncell] (p, u_x, u_y as dugks_moments returns them):
// p = RT sum g~, u = c/rho0 sum e g~ + G cos(omega t) dt/2 (eq. (27)).
template <class T>
__global__ void adj_seed(const AdjParams<T> a, const float *dLdm, T rt, T c_over_rho0, double gdt) {
    const int64_t nc = ncell(a);
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        const T gp = (T)dLdm[c], gu0 = (T)dLdm[nc + c], gu1 = (T)dLdm[2 * nc + c];
        for (int k = 0; k < Q; k++)
            a.lam0[k * nc + c] = rt * gp + c_over_rho0 * ((T)L9::e(k, 0) * gu0 + (T)L9::e(k, 1) * gu1);
        if (a.dG) {
            a.dG[c] += (double)gu0 * gdt;
            a.dG[nc + c] += (double)gu1 * gdt;
        }
    }
}

// dL/du_w per face [6][3] from the per-wall-interface slots (-x: ny, +x: ny, -y: nx, +y: nx
// slots of 2 components), each sum in slot order (deterministic); zero for the faces that
// are not velocity walls.
__global__ void adj_wall_sum(const double *slots, double *out, int nx, int ny, int vx0, int vx1, int vy0, int vy1) {
    const int t = threadIdx.x;  // face * 3 + component
    if (t >= 18) return;
    const int f = t / 3, comp = t % 3;
    const int vel[4] = {vx0, vx1, vy0, vy1};
    double s = 0.0;
    if (f < 4 && comp < 2 && vel[f]) {
        const int first = f == 0 ? 0 : f == 1 ? ny : f == 2 ? 2 * ny : 2 * ny + nx;
        const int count = f < 2 ? ny : nx;
        for (int i = 0; i < count; i++) s += slots[2 * (first + i) + comp];
    }
    out[t] = s;
}

__global__ void adj_to_float(const double *src, float *dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

// Face types whose wall velocity enters the step (and so has a gradient).
static int moving_wall(int type) { return type == DUGKS_BC_NEQ_VELOCITY || type == DUGKS_BC_BOUNCE_BACK; }

int blocks_for(int64_t n, int threads) {
    const int64_t b = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 1 << 20));
}

// Work buffers carved from one allocation (element size es, 256-byte aligned pieces).
struct AdjBufs {
    void *phi, *mom[2], *fb[2], *gb[2], *lam[2];
};

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

size_t scratch_bytes(int64_t nx, int64_t ny, size_t es) {
    const int64_t nc = nx * ny, n0 = (nx + 1) * ny, n1 = nx * (ny + 1);
    return al256(es * Q * nc) + 2 * al256(es * 3 * nc) + al256(es * Q * n0) + al256(es * Q * n1) + al256(es * 2 * n0) +
           al256(es * 2 * n1) + 2 * al256(es * Q * nc);
}

AdjBufs carve(void *base, int64_t nx, int64_t ny, size_t es) {
    const int64_t nc = nx * ny, n0 = (nx + 1) * ny, n1 = nx * (ny + 1);
    char *p = (char *)base;
    AdjBufs B;
    B.phi = p; p += al256(es * Q * nc);
    B.mom[0] = p; p += al256(es * 3 * nc);
    B.mom[1] = p; p += al256(es * 3 * nc);
    B.fb[0] = p; p += al256(es * Q * n0);
    B.fb[1] = p; p += al256(es * Q * n1);
    B.gb[0] = p; p += al256(es * 2 * n0);
    B.gb[1] = p; p += al256(es * 2 * n1);
    B.lam[0] = p; p += al256(es * Q * nc);
    B.lam[1] = p;
    return B;
}

template <class T>
AdjParams<T> base_params(const dugks_t h, const AdjBufs &B) {
    AdjParams<T> a;
    memset(&a, 0, sizeof a);
    const StepParams p = handle_params(h);
    a.n[0] = (int)h->nx;
    a.n[1] = (int)h->ny;
    a.per[0] = h->bcs.face[0].type == DUGKS_BC_PERIODIC;
    a.per[1] = h->bcs.face[2].type == DUGKS_BC_PERIODIC;
    a.px = p.px;
    a.dstride = p.dstride;
    for (int w = 0; w < 4; w++) {
        a.bc[w] = p.bc[w];
        a.mw[w][0] = (T)(p.bc_u[w][0] * p.rho0 * p.inv_c);
        a.mw[w][1] = (T)(p.bc_u[w][1] * p.rho0 * p.inv_c);
        a.drw[w] = (T)p.bc_drho[w];
        a.drw1[w] = (T)p.bc_drho1[w];
    }
    a.rho0 = (T)p.rho0;
    a.inv_rho0 = (T)(1.0 / p.rho0);
    a.dmw = (T)(p.rho0 * p.inv_c);
    a.b1 = (T)p.b1;
    a.c1 = (T)p.c1;
    a.b7 = (T)p.b7;
    a.c7 = (T)p.c7;
    a.kappa = (T)p.kappa;
    a.two_kappa = (T)p.two_kappa;
    a.wcell = (T)p.wcell;
    a.wface = (T)p.wface;
    a.g[0] = (T)p.g[0];
    a.g[1] = (T)p.g[1];
    a.field = p.field;
    a.phi = (T *)B.phi;
    a.mom = (T *)B.mom[0];
    for (int d = 0; d < 2; d++) {
        a.fb[d] = (T *)B.fb[d];
        a.gb[d] = (T *)B.gb[d];
    }
    a.dG = h->tape.dG;
    a.dW = h->tape.dW;
    return a;
}

// cos(omega t) / c at the time t of a state, as the recompute of that state uses it.
template <class T>
T force_factor(const dugks_t h, double t) {
    return (T)(cos(h->force.omega * t) * (1.0 / h->c));
}

// One reverse step at the state g~^n held in `state` (t_n = tn): lambda' in lam1 -> lam0,
// with the cell moments of g~^n in `mom`. Launches: the cell recompute unless the previous
// reverse step's cells kernel made it (have_fwd), all interfaces (frame blocks first), and
// all cells (frame blocks first), which also recompute g~^{n-1} = `next` (at time tnext) into
// a.phi and `nmom` when `next` is given.
template <class T>
cudaError_t reverse_step(AdjParams<T> a, const dugks_t h, const void *state, double tn, const void *lam1,
                         void *lam0, void *mom, bool have_fwd, const void *next, double tnext, void *nmom,
                         int64_t *launches) {
    const double om = h->force.omega, inv_c = 1.0 / h->c;
    a.ctc = force_factor<T>(h, tn);
    a.cthc = (T)(cos(om * (tn + 0.5 * h->dt)) * inv_c);
    a.cwh = (T)cos(om * (tn + 0.5 * h->dt));
    a.state = (const T *)state;
    a.lam1 = (const T *)lam1;
    a.lam0 = (T *)lam0;
    a.mom = (T *)mom;
    a.nstate = (const T *)next;
    a.nmom = (T *)nmom;
    a.nctc = next ? force_factor<T>(h, tnext) : T(0);
    cudaStream_t st = h->stream;
    const int nx = (int)h->nx, ny = (int)h->ny;
    const int64_t nc = h->ncell;
    int64_t n = 0;
    if (!have_fwd) {
        adj_cells_fwd<T><<<blocks_for(nc, 256), 256, 0, st>>>(a);
        n++;
    }
    {
        const Rect r0 = face_rect(0, nx, ny, a.per[0], a.per[1]), r1 = face_rect(1, nx, ny, a.per[0], a.per[1]);
        const int64_t nframe = frame_count(r0) + frame_count(r1);
        const int nfb = (int)((nframe + 7) / 8);
        const int tx0 = rect_empty(r0) ? 0 : (r0.x1 - r0.x0 + 32) / 32, ty0 = rect_empty(r0) ? 0 : (r0.y1 - r0.y0 + 4) / 4;
        const int tx1 = rect_empty(r1) ? 0 : (r1.x1 - r1.x0 + 32) / 32, ty1 = rect_empty(r1) ? 0 : (r1.y1 - r1.y0 + 4) / 4;
        const int nb = nfb + tx0 * ty0 + tx1 * ty1;
        if (nb > 0) {
            adj_faces_all<T><<<nb, 128, 0, st>>>(a, nframe, nfb, tx0 * ty0, tx0, tx1);
            n++;
        }
    }
    {
        const Rect rc = cell_rect(nx, ny, a.per[0], a.per[1]);
        const int tx = rect_empty(rc) ? 0 : (rc.x1 - rc.x0 + 32) / 32, ty = rect_empty(rc) ? 0 : (rc.y1 - rc.y0 + 4) / 4;
        const int nfb = (int)((frame_count(rc) + 7) / 8);
        const int nb = nfb + tx * ty;
        if (nb > 0) {
            adj_cells_all<T><<<nb, 128, 0, st>>>(a, nfb, tx, ty);
            n++;
        }
    }
    *launches += n;
    return cudaGetLastError();
}

// The work of one checkpoint segment of `len` steps whose first state is in seg[0] (copied
// from the checkpoint) and whose clock starts at `start`: recompute the states into
// seg[1 .. len-1], then the reverse steps len-1 .. 0 with lambda ping-ponging from
// lam[cur]. Returns the number of launches through *launches.
template <class T>
cudaError_t enqueue_segment(dugks_t h, const AdjParams<T> &a, const AdjBufs &B, int64_t start, int64_t len, int cur,
                            int64_t *launches) {
    AdjointTape &t = h->tape;
    for (int64_t j = 1; j < len; j++) {
        StepParams p = handle_params(h);
        p.src = t.seg[(size_t)j - 1];
        p.dst = t.seg[(size_t)j];
        p.step_ctr = t.zero;
        p.step_off = (int)(t.step0 + start + j - 1);
        cudaError_t e = handle_launch_step(h, p);
        if (e != cudaSuccess) return e;
        (*launches)++;
    }
    // step j's cell moments are in mom[j & 1]; each cells kernel but the segment's last also
    // recomputes step j - 1
    for (int64_t j = len - 1; j >= 0; j--) {
        const double tn = (double)(t.step0 + start + j) * h->dt;
        const double tprev = (double)(t.step0 + start + j - 1) * h->dt;
        cudaError_t e = reverse_step<T>(a, h, t.seg[(size_t)j], tn, B.lam[cur], B.lam[cur ^ 1], B.mom[j & 1],
                                        j < len - 1, j > 0 ? t.seg[(size_t)j - 1] : nullptr, tprev,
                                        B.mom[(j - 1) & 1], launches);
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    return cudaSuccess;
}

template <class T>
int enqueue_adjoint(dugks_t h, const float *dL_dmom, float *dL_dfield, void *dL_dstate0) {
    AdjointTape &t = h->tape;
    const size_t es = sizeof(T);
    const AdjBufs B = carve(t.scratch, h->nx, h->ny, es);
    const int64_t nc = h->ncell;
    const int64_t nwall = 2 * (h->nx + h->ny);
    cudaStream_t st = h->stream;
    cudaError_t e = cudaMemsetAsync(t.dG, 0, sizeof(double) * 2 * nc, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(t.dW, 0, sizeof(double) * 2 * nwall, st);
    if (e != cudaSuccess) return handle_fail(h, DUGKS_E_CUDA, "adjoint: %s", cudaGetErrorString(e));
    AdjParams<T> a = base_params<T>(h, B);
    {  // seed at the end of the rollout
        const double tend = (double)(t.step0 + t.steps) * h->dt;
        AdjParams<T> s = a;
        s.lam0 = (T *)B.lam[0];
        adj_seed<T><<<blocks_for(nc, 256), 256, 0, st>>>(s, dL_dmom, (T)h->rt, (T)(h->c / h->rho0),
                                                          cos(h->force.omega * tend) * 0.5 * h->dt);
        h->launches++;
    }
    int cur = 0;
    const int64_t every = t.every;
    const int64_t nseg = (t.steps + every - 1) / every;
    // With a time-independent acceleration every segment of the same length and starting
    // parity is the same sequence of launches on the same buffers: capture it once as a
    // CUDA graph and replay it per segment.
    const bool graphs = h->use_graph && h->force.omega == 0.0 && nseg >= 3;
    // What a captured segment bakes in besides its length and parity: the forward step's and
    // the adjoint's parameter records (with omega = 0 neither depends on the segment's
    // time), the segment state buffers and the kernel selection. A graph of an earlier call
    // is reused while all of these are unchanged (its work has completed: the caller's
    // stream was synchronised before this call).
    std::vector<unsigned char> sig;
    if (graphs) {
        StepParams p0 = handle_params(h);
        p0.src = p0.dst = nullptr;
        p0.step_ctr = t.zero;
        auto put = [&](const void *q, size_t n) {
            const unsigned char *c = (const unsigned char *)q;
            sig.insert(sig.end(), c, c + n);
        };
        put(&p0, sizeof p0);
        put(&a, sizeof a);
        const int sel[4] = {h->kernel, h->tile_x, h->tile_y, h->store};
        put(sel, sizeof sel);
        for (void *q : t.seg) put(&q, sizeof q);
    }
    int rc = DUGKS_OK;
    for (int64_t sg = nseg - 1; sg >= 0 && rc == DUGKS_OK; sg--) {
        const int64_t start = sg * every;
        const int64_t len = std::min<int64_t>(every, t.steps - start);
        e = cudaMemcpyAsync(t.seg[0], t.ckpt[(size_t)sg], h->state_bytes, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) { rc = handle_fail(h, DUGKS_E_CUDA, "adjoint: %s", cudaGetErrorString(e)); break; }
        int64_t nl = 0;
        if (graphs) {
            AdjointTape::SegGraph *hit = nullptr;
            for (auto &gr : t.graphs)
                if (gr.len == len && gr.cur == cur) hit = &gr;
            if (hit && hit->sig != sig) {  // captured with other buffers or parameters
                cudaGraphExecDestroy(hit->exec);
                *hit = t.graphs.back();
                t.graphs.pop_back();
                hit = nullptr;
            }
            if (!hit) {
                cudaGraph_t g;
                e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    cudaError_t e2 = enqueue_segment<T>(h, a, B, start, len, cur, &nl);
                    e = cudaStreamEndCapture(st, &g);
                    if (e2 != cudaSuccess) e = e2;
                }
                cudaGraphExec_t ge = nullptr;
                if (e == cudaSuccess) {
                    e = cudaGraphInstantiate(&ge, g, 0);
                    cudaGraphDestroy(g);
                }
                if (e != cudaSuccess) { rc = handle_fail(h, DUGKS_E_CUDA, "adjoint graph: %s", cudaGetErrorString(e)); break; }
                t.graphs.push_back(AdjointTape::SegGraph{len, cur, sig, ge, nl});
                hit = &t.graphs.back();
            }
            nl = hit->launches;
            e = cudaGraphLaunch(hit->exec, st);
        } else {
            e = enqueue_segment<T>(h, a, B, start, len, cur, &nl);
        }
        if (e != cudaSuccess) { rc = handle_fail(h, DUGKS_E_CUDA, "adjoint step: %s", cudaGetErrorString(e)); break; }
        h->launches += nl;
        if (len & 1) cur ^= 1;
    }
    if (rc != DUGKS_OK) {
        cudaStreamSynchronize(st);
        return rc;
    }
    if (dL_dfield) {
        adj_to_float<<<blocks_for(2 * nc, 256), 256, 0, st>>>(t.dG, dL_dfield, 2 * nc);
        h->launches++;
    }
    if (dL_dstate0) {
        e = cudaMemcpyAsync(dL_dstate0, B.lam[cur], es * Q * nc, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return handle_fail(h, DUGKS_E_CUDA, "adjoint: %s", cudaGetErrorString(e));
    }
    adj_wall_sum<<<1, 32, 0, st>>>(t.dW, t.dW_face, (int)h->nx, (int)h->ny,
                                   moving_wall(h->bcs.face[0].type), moving_wall(h->bcs.face[1].type),
                                   moving_wall(h->bcs.face[2].type), moving_wall(h->bcs.face[3].type));
    h->launches++;
    e = cudaMemcpyAsync(t.h_wall, t.dW_face, sizeof(double) * 18, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return handle_fail(h, DUGKS_E_CUDA, "adjoint: %s", cudaGetErrorString(e));
    return DUGKS_OK;
}

}  // namespace

void adjoint_release(dugks_t h) {
    AdjointTape &t = h->tape;
    for (void *p : t.ckpt) cudaFree(p);
    for (void *p : t.seg) cudaFree(p);
    t.ckpt.clear();
    t.seg.clear();
    cudaFree(t.scratch);
    cudaFree(t.dG);
    cudaFree(t.dW);
    cudaFree(t.zero);
    cudaFree(t.dW_face);
    if (t.h_wall) cudaFreeHost(t.h_wall);
    for (auto &gr : t.graphs) cudaGraphExecDestroy(gr.exec);
    t.graphs.clear();
    t.scratch = nullptr;
    t.dG = t.dW = t.dW_face = t.h_wall = nullptr;
    t.zero = nullptr;
    t.steps = 0;
}

}  // namespace dugks

using namespace dugks;

static int check_adjoint_support(dugks_t h) {
    if (h->q != DUGKS_D2Q9 || h->dim != 2)
        return handle_fail(h, DUGKS_E_UNSUPPORTED, "record/adjoint: built for D2Q9 only");
    if (h->store != DUGKS_STORE_F32 && h->store != DUGKS_STORE_F64)
        return handle_fail(h, DUGKS_E_UNSUPPORTED, "record/adjoint: F32 or F64 storage only");
    if (h->model != DUGKS_MODEL_INCOMPRESSIBLE)
        return handle_fail(h, DUGKS_E_UNSUPPORTED, "record/adjoint: the incompressible model only");
    if (h->d_metric) return handle_fail(h, DUGKS_E_UNSUPPORTED, "record/adjoint: uniform meshes only");
    return DUGKS_OK;
}

extern "C" int dugks_record(dugks_t h, int64_t nsteps, int32_t every) {
    if (!h) return DUGKS_E_INVAL;
    if (nsteps < 1 || every < 1) return handle_fail(h, DUGKS_E_INVAL, "record: nsteps and every must be >= 1");
    int rc = check_adjoint_support(h);
    if (rc != DUGKS_OK) return rc;
    if (h->step + nsteps > 2147483647LL) return handle_fail(h, DUGKS_E_INVAL, "record: step index past 2^31 - 1");
    AdjointTape &t = h->tape;
    t.steps = 0;
    // an earlier asynchronous adjoint may still read the buffers reused below
    cudaError_t es0 = cudaStreamSynchronize(h->stream);
    if (es0 != cudaSuccess) return handle_fail(h, DUGKS_E_CUDA, "record: %s", cudaGetErrorString(es0));
    const int64_t nseg = (nsteps + every - 1) / every;
    const int64_t nbuf = std::min<int64_t>(every, nsteps);  // seg[0] receives the checkpoint
    cudaError_t e = cudaSuccess;
    auto resize = [&](std::vector<void *> &v, int64_t count) {
        while ((int64_t)v.size() > count) {
            cudaFree(v.back());
            v.pop_back();
        }
        while (e == cudaSuccess && (int64_t)v.size() < count) {
            void *p = nullptr;
            e = cudaMalloc(&p, h->state_bytes);
            if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, h->state_bytes, h->stream);  // zero padding columns
            if (e == cudaSuccess) v.push_back(p);
            else cudaFree(p);
        }
    };
    resize(t.ckpt, nseg);
    resize(t.seg, nbuf);
    const size_t es = h->store == DUGKS_STORE_F64 ? 8 : 4;
    if (e == cudaSuccess && !t.scratch) {
        t.scratch_bytes = scratch_bytes(h->nx, h->ny, es);
        e = cudaMalloc(&t.scratch, t.scratch_bytes);
        if (e == cudaSuccess) e = cudaMalloc((void **)&t.dG, sizeof(double) * 2 * h->ncell);
        if (e == cudaSuccess) e = cudaMalloc((void **)&t.dW, sizeof(double) * 4 * (h->nx + h->ny));
        if (e == cudaSuccess) e = cudaMalloc((void **)&t.zero, sizeof(long long));
        if (e == cudaSuccess) e = cudaMalloc((void **)&t.dW_face, sizeof(double) * 18);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&t.h_wall, sizeof(double) * 18);
        if (e == cudaSuccess) e = cudaMemsetAsync(t.zero, 0, sizeof(long long), h->stream);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        adjoint_release(h);
        return handle_fail(h, e == cudaErrorMemoryAllocation ? DUGKS_E_NOMEM : DUGKS_E_CUDA, "record: %s",
                           cudaGetErrorString(e));
    }
    t.step0 = h->step;
    t.every = every;
    for (int64_t s = 0; s < nseg; s++) {
        e = cudaMemcpyAsync(t.ckpt[(size_t)s], h->buf[h->cur], h->state_bytes, cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) return handle_fail(h, DUGKS_E_CUDA, "record: %s", cudaGetErrorString(e));
        rc = dugks_step(h, std::min<int64_t>(every, nsteps - s * every));
        if (rc != DUGKS_OK) return rc;
    }
    t.steps = nsteps;
    return DUGKS_OK;
}

static int adjoint_enqueue_checked(dugks_t h, const float *dL_dmom, float *dL_dfield, void *dL_dstate0) {
    if (!h || !dL_dmom) return DUGKS_E_INVAL;
    int rc = check_adjoint_support(h);
    if (rc != DUGKS_OK) return rc;
    if (h->tape.steps < 1) return handle_fail(h, DUGKS_E_INVAL, "adjoint: no recorded rollout (call dugks_record)");
    // the previous call's graphs and buffers are reused: its work must have completed
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return handle_fail(h, DUGKS_E_CUDA, "adjoint: %s", cudaGetErrorString(e));
    return h->store == DUGKS_STORE_F64 ? enqueue_adjoint<double>(h, dL_dmom, dL_dfield, dL_dstate0)
                                       : enqueue_adjoint<float>(h, dL_dmom, dL_dfield, dL_dstate0);
}

extern "C" int dugks_adjoint_async(dugks_t h, const float *dL_dmom, float *dL_dfield, void *dL_dstate0) {
    return adjoint_enqueue_checked(h, dL_dmom, dL_dfield, dL_dstate0);
}

extern "C" int dugks_adjoint_wall(dugks_t h, double *dL_dwall) {
    if (!h || !dL_dwall) return DUGKS_E_INVAL;
    if (!h->tape.h_wall) return handle_fail(h, DUGKS_E_INVAL, "adjoint_wall: no adjoint has run");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return handle_fail(h, DUGKS_E_CUDA, "adjoint_wall: %s", cudaGetErrorString(e));
    for (int i = 0; i < 18; i++) dL_dwall[i] = h->tape.h_wall[i];
    return DUGKS_OK;
}

extern "C" int dugks_adjoint(dugks_t h, const float *dL_dmom, float *dL_dfield, double *dL_dwall,
                             void *dL_dstate0) {
    int rc = adjoint_enqueue_checked(h, dL_dmom, dL_dfield, dL_dstate0);
    if (rc != DUGKS_OK) return rc;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return handle_fail(h, DUGKS_E_CUDA, "adjoint: %s", cudaGetErrorString(e));
    if (dL_dwall)
        for (int i = 0; i < 18; i++) dL_dwall[i] = h->tape.h_wall[i];
    return DUGKS_OK;
}
