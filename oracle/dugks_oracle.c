/*
 * dugks_oracle.c -- FP64 CPU oracle of the incompressible discrete unified gas kinetic
 * scheme (DUGKS) with force term: Wu, Shi, Chai and Wang, "Discrete unified gas kinetic
 * scheme with force term for incompressible fluid flows" (arXiv 1411.6121).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE. This is the plain, slow reference that the CUDA
 * path is checked against. Only the test suite, the smoke check and the CPU-baseline /
 * reference legs of the benchmark load it. It shares no code, header, table or helper
 * with the CUDA library, and the CUDA library never loads it.
 *
 * What it computes: one time step is the Appendix algorithm (steps 1-10), in that order,
 * on explicit arrays for the Appendix's point sets
 *     X_c  cell centres              -> F_c (holds f~ between steps), fc (holds fbar+)
 *     X_cg ghost cells               -> fc (the extended cell array, one layer per side)
 *     X_b  interface midpoints       -> fb (fbar+ interpolated), Fb (fbar, then f)
 *     X_bc interface cross points    -> fbc (fbar+ interpolated)
 * in double precision with round-to-nearest and no blocking, fusion or reordering beyond
 * what the Appendix writes. Where the paper leaves a choice open, the reading taken is
 * stated at the function that makes it (readings R1..R9 below).
 *
 * Readings of the paper, each a choice where the paper is silent, ambiguous or garbled:
 *  R1  tau = nu / RT (Sec. 2.1 introduces tau but relates it to nu nowhere; this is the
 *      Chapman-Enskog viscosity of the BGK model with sound speed^2 = RT).
 *  R2  G(x, t) = (g + field(x)) cos(omega t). At a cell centre G is the cell's value; at
 *      an interior or periodic interface it is the mean of the two adjacent cells; at a
 *      wall interface it is the value of the one adjacent cell. Cell quantities at t_n use
 *      G(t_n); interface quantities at t_n + h use G(t_n + h).
 *  R3  Step 2 ("extrapolation from several points"): linear, ghost = 2 f_0 - f_1 along the
 *      wall normal, applied axis by axis (x, then y, then z) over the already-extended
 *      range of the earlier axes, which fills edge and corner ghosts. Periodic axes fill
 *      their ghost layer with the periodic image.
 *  R4  NEQ boundary (Sec. 2.4, eq. (32)): x_c is the midpoint of the boundary cell's
 *      interface opposite the wall; (rho_c, u_c) are the step-6 moments of the step-4
 *      value there. Velocity condition: u_a = u_w, rho_a = rho_c. Pressure condition:
 *      rho_a = rho0 + p_w / RT, u_a = u_c. Applied, as the Appendix's step 5 says, to
 *      fbar before step 7, only for xi . n < 0 (n the outward normal of the domain), with
 *      the equilibrium of eq. (6).
 *  R5  Step 3 cross points: the mean of the 4 cells that share the cross point (the
 *      vertex in 2D, the edge midpoint in 3D). Step 4 tangential gradients difference the
 *      two cross points on the interface; the normal gradient differences the two cells.
 *  R6  The cell moments entering step 1 are those of the current F (eq. (27),
 *      i.e. step 10 of the previous step, or of the initial F at the first step).
 *  R7  Initial state: F = f_eq(rho0 + p/RT, u) of eq. (6) (the paper initialises "the
 *      equilibrium distribution" from the fields), with no force correction.
 *  R8  D3Q19 (not in the paper, which uses D3Q27) is the D3Q27 set of Sec. 2.3 with its 8
 *      corner velocities removed and the standard weights 1/3, 1/18, 1/36; it has the
 *      same moments up to fourth order, which is all eq. (6) uses.
 *  R9  Pressure p = (rho - rho0) RT (the paper initialises rho = rho0 + p/RT).
 *  R14 Bounce-back (Sec. 2.4, eq. (31)) is applied, like NEQ, to fbar at the wall interface
 *      in the Appendix's step 5: for xi_k . n < 0, fbar_k = fbar_(-k) + 2 rho_w W_k
 *      xi_k . u_w / RT, with the opposite velocity's step-4 value at the same interface
 *      and rho_w = rho0 (the incompressible limit the paper names).
 *  R16 The original DUGKS (the comparison model of Sec. 2.1 and 2.2, model = 1): eq. (5)
 *      in place of eq. (6) everywhere f_eq appears (step 1, the NEQ equilibria, step 7,
 *      the force term S, the initial state), with rho u = sum xi f~ + rho G dt/2 at cells
 *      and the same with h at interfaces; the incompressible model is model = 0.
 *  R17 Oscillating wall pressure (the pressure-driven Womersley flow of Sec. 3.3): a
 *      pressure wall holds p_w(t) = p + p_amp cos(omega t), with the force's omega, and the
 *      NEQ pressure condition takes it at the interface time t_n + h.
 *  R18 Non-uniform mesh (Sec. 3.4, the tanh mesh): the mesh is given by its interface
 *      coordinates per axis; cell centres are the midpoints of their two interfaces. Step 3
 *      interpolates linearly in each axis between the two centres around the interface
 *      (bilinearly at cross points), step 4 divides the normal difference by the centre
 *      distance and the tangential one by the interface length, step 2 extrapolates
 *      linearly through the two boundary centres to the ghost centre (the boundary
 *      centre mirrored in the wall; periodic ghosts sit one period away), the interface G
 *      is interpolated like fbar+, and step 8 uses each cell's interface areas and volume.
 *      On a uniform mesh every one of these reduces to the uniform formula.
 *
 * Complex-step build: compiled with -DORACLE_COMPLEX_STEP the same code runs on
 * double _Complex values. The scheme only adds, subtracts and multiplies state values, so
 * Im(Phi(x + i eps v)) / eps is the exact directional derivative J v to rounding: this
 * is the oracle's derivative, used to check the hand-written adjoint of the CUDA path.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef ORACLE_COMPLEX_STEP
#include <complex.h>
typedef double _Complex real;
#define RE(x) creal(x)
#define IM(x) cimag(x)
#else
typedef double real;
#define RE(x) (x)
#define IM(x) (0.0 * (x))
#endif

void oracle_destroy(void *p);

#define BC_PERIODIC 0
#define BC_NEQ_VELOCITY 1
#define BC_NEQ_PRESSURE 2
#define BC_BOUNCE_BACK 3

/* Plain configuration record (mirrored by ctypes in oracle.py). */
typedef struct {
    int dim;          /* 2 or 3 */
    int q;            /* 9 (D2Q9), 19 (D3Q19), 27 (D3Q27) */
    int nx, ny, nz;   /* cells per axis (nz = 1 in 2D) */
    double dx;        /* uniform grid spacing, Delta x = Delta y = Delta z */
    double rt;        /* RT */
    double rho0;      /* reference density rho_0 */
    double nu;        /* kinematic viscosity */
    double dt;        /* time step Delta t */
    double g[3];      /* uniform part of the acceleration G */
    double omega;     /* G(x,t) = (g + field(x)) cos(omega t) */
    int bc_type[6];   /* faces -x,+x,-y,+y,-z,+z */
    double bc_u[6][3];/* wall velocity u_w (velocity condition) */
    double bc_p[6];   /* wall pressure p_w (pressure condition) */
    int model;        /* 0: the incompressible model (eq. (6), eq. (27));
                         1: the original DUGKS (eq. (5), rho u = sum xi f~ + rho G dt/2) */
    double bc_p_amp[6];/* pressure condition: p_w(t) = bc_p + bc_p_amp cos(omega t) */
    const double *faces[3]; /* non-uniform mesh (reading R18): the n+1 interface
                               coordinates per axis, or NULL for uniform spacing dx */
} oracle_config;

typedef struct {
    oracle_config cfg;
    int D, Q;
    int n[3];           /* cells per axis; n[2] = 1 in 2D */
    int e[27][3];       /* lattice unit vectors, xi_k = c e_k */
    double W[27];
    double c, tau, h;
    long ncell;
    long next;          /* cells of the extended array X_c u X_cg */
    int en[3];          /* extended extents */
    int eo[3];          /* extended offsets (1 per side on used axes) */
    long nface[3];
    long ncross[3];     /* pairs (0,1), (0,2), (1,2) */
    real *F;            /* X_c: f~ [ncell][Q] */
    real *fc;           /* X_c u X_cg: fbar+ [next][Q] */
    real *fb[3];        /* X_b per normal axis: fbar+ [nface][Q] */
    real *Fb[3];        /* X_b per normal axis: fbar(t+h) then f(t+h) [nface][Q] */
    real *rhob[3];      /* X_b moments */
    real *ub[3];        /* [nface][3] */
    real *fbc[3];       /* X_bc per axis pair */
    real *m;            /* micro-flux [ncell][Q] */
    real *field;        /* [3][ncell] acceleration field (zero where absent) */
    real wall_u[6][3];  /* u_w per face; real-typed so it can carry a complex step */
    double t;
    long step;
    int nonuni;         /* the mesh is given by its interface coordinates */
    double *xf[3];      /* interface coordinates, n+1 per axis */
    double *xc[3];      /* centres, extended: xc[a][i + 1] for i = -1 .. n (ghosts included) */
} ostate;

/* ---------------------------------------------------------------------------------
 * Discrete velocities (Sec. 2.3). D1Q3: xi = sqrt(3RT){-1,0,1}, W = {1/6,2/3,1/6}.
 * The paper prints W = 1/3 for the two moving D1Q3 velocities, which does not sum to
 * one; its own D2Q9 and D3Q27 weights are the tensor products of {1/6, 2/3, 1/6}
 * (e.g. 1/36 = 1/6 * 1/6, 4/9 = 2/3 * 2/3), so the tensor product uses those.
 * Index order: the paper's (x slowest, then y, then z), i.e. k = 9(ex+1)+3(ey+1)+(ez+1)
 * in 3D and k = 3(ex+1)+(ey+1) in 2D.
 * --------------------------------------------------------------------------------- */
static void build_lattice(ostate *s)
{
    static const double w1[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
    int q = 0;
    if (s->Q == 9) {
        for (int a = -1; a <= 1; a++)
            for (int b = -1; b <= 1; b++) {
                s->e[q][0] = a; s->e[q][1] = b; s->e[q][2] = 0;
                s->W[q] = w1[a + 1] * w1[b + 1];
                q++;
            }
    } else if (s->Q == 27) {
        for (int a = -1; a <= 1; a++)
            for (int b = -1; b <= 1; b++)
                for (int g = -1; g <= 1; g++) {
                    s->e[q][0] = a; s->e[q][1] = b; s->e[q][2] = g;
                    s->W[q] = w1[a + 1] * w1[b + 1] * w1[g + 1];
                    q++;
                }
    } else { /* Q == 19, reading R8 */
        for (int a = -1; a <= 1; a++)
            for (int b = -1; b <= 1; b++)
                for (int g = -1; g <= 1; g++) {
                    int nz = (a != 0) + (b != 0) + (g != 0);
                    if (nz == 3) continue;
                    s->e[q][0] = a; s->e[q][1] = b; s->e[q][2] = g;
                    s->W[q] = nz == 0 ? 1.0 / 3.0 : (nz == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
                    q++;
                }
    }
}

/* ---------------------------------------------------------------------------------
 * Equilibrium of the incompressible model, eq. (6):
 *   f_eq_k = W_k { rho + rho0 [ xi_k.u/RT + (xi_k.u)^2/(2 RT^2) - |u|^2/(2RT) ] }.
 * --------------------------------------------------------------------------------- */
static real feq(const ostate *s, int k, real rho, const real u[3])
{
    const double rt = s->cfg.rt, rho0 = s->cfg.rho0;
    real xu = 0, uu = 0;
    for (int a = 0; a < 3; a++) {
        xu += s->c * s->e[k][a] * u[a];
        uu += u[a] * u[a];
    }
    const real bracket = xu / rt + xu * xu / (2.0 * rt * rt) - uu / (2.0 * rt);
    /* the original DUGKS (reading R16), eq. (5): W_k rho [1 + bracket] */
    if (s->cfg.model == 1) return s->W[k] * rho * (1.0 + bracket);
    return s->W[k] * (rho + rho0 * bracket);
}

/* Force term, eq. (9): S_k = G.(xi_k - u)/RT f_eq_k (with f_eq of eq. (6)). */
static real source(const ostate *s, int k, const real G[3], const real u[3], real fe)
{
    real gx = 0;
    for (int a = 0; a < 3; a++) gx += G[a] * (s->c * s->e[k][a] - u[a]);
    return gx / s->cfg.rt * fe;
}

/* Index of the velocity opposite to k. */
static int opposite(const ostate *s, int k)
{
    for (int j = 0; j < s->Q; j++)
        if (s->e[j][0] == -s->e[k][0] && s->e[j][1] == -s->e[k][1] && s->e[j][2] == -s->e[k][2]) return j;
    return k;
}

/* Macroscopic variables, eq. (27) (cell, weight dt/2) and the Appendix's step 6
 * (interface, weight h/2): rho = sum_k f_k, rho0 u = sum_k xi_k f_k + rho0 G w. The original
 * DUGKS (reading R16) divides by and weights the force with rho instead:
 * rho u = sum_k xi_k f_k + rho G w. */
static void moments(const ostate *s, const real *f, const real G[3], double w, real *rho,
                    real u[3])
{
    real r = 0, j[3] = {0, 0, 0};
    for (int k = 0; k < s->Q; k++) {
        r += f[k];
        for (int a = 0; a < 3; a++) j[a] += s->c * s->e[k][a] * f[k];
    }
    *rho = r;
    const real rd = s->cfg.model == 1 ? r : (real)s->cfg.rho0;
    for (int a = 0; a < 3; a++) u[a] = (j[a] + rd * G[a] * w) / rd;
}

/* ------------------------------- indexing --------------------------------------- */
static long cell_index(const ostate *s, const int x[3])
{
    return x[0] + (long)s->n[0] * (x[1] + (long)s->n[1] * x[2]);
}

static long ext_index(const ostate *s, const int x[3])
{
    return (x[0] + s->eo[0]) + (long)s->en[0] * ((x[1] + s->eo[1]) + (long)s->en[1] * (x[2] + s->eo[2]));
}

/* X_b normal to axis d: position x[d] in 0..n[d] (interface between cells x[d]-1 and
 * x[d]); other coordinates are cell indices. */
static long face_index(const ostate *s, int d, const int x[3])
{
    int ex[3];
    for (int a = 0; a < 3; a++) ex[a] = s->n[a] + (a == d);
    return x[0] + (long)ex[0] * (x[1] + (long)ex[1] * x[2]);
}

/* X_bc for the axis pair p = (a,b) in {(0,1),(0,2),(1,2)}: x[a], x[b] in 0..n (cross
 * point between cells x-1 and x on both axes); the third coordinate is a cell index. */
static void pair_axes(int p, int *a, int *b)
{
    *a = (p == 2) ? 1 : 0;
    *b = (p == 0) ? 1 : 2;
}

static long cross_index(const ostate *s, int p, const int x[3])
{
    int a, b, ex[3];
    pair_axes(p, &a, &b);
    for (int i = 0; i < 3; i++) ex[i] = s->n[i] + (i == a || i == b);
    return x[0] + (long)ex[0] * (x[1] + (long)ex[1] * x[2]);
}

static int pair_of(int a, int b)
{
    if (a > b) { int t = a; a = b; b = t; }
    return (a == 0 && b == 1) ? 0 : (a == 0 ? 1 : 2);
}

/* Acceleration at a cell centre and time t (reading R2). */
static void G_cell(const ostate *s, long ci, double t, real G[3])
{
    const double ct = cos(s->cfg.omega * t);
    for (int a = 0; a < 3; a++) G[a] = (s->cfg.g[a] + s->field[a * s->ncell + ci]) * ct;
}

/* ---- non-uniform mesh metrics (reading R18) ---- */
/* Interpolation weight of the high cell at interface i of axis a (centres i-1, i). */
static double wface(const ostate *s, int a, int i)
{
    const double *c = s->xc[a] + 1;
    return (s->xf[a][i] - c[i - 1]) / (c[i] - c[i - 1]);
}
/* 1 / (distance of the two centres across interface i of axis a). */
static double inv_dc(const ostate *s, int a, int i)
{
    const double *c = s->xc[a] + 1;
    return 1.0 / (c[i] - c[i - 1]);
}
/* Width of cell i along axis a. */
static double width(const ostate *s, int a, int i) { return s->xf[a][i + 1] - s->xf[a][i]; }

/* Acceleration at the interface x (normal axis d) and time t (reading R2). */
static void G_face(const ostate *s, int d, const int x[3], double t, real G[3])
{
    int lo[3] = {x[0], x[1], x[2]}, hi[3] = {x[0], x[1], x[2]};
    const int nd = s->n[d];
    const int periodic = s->cfg.bc_type[2 * d] == BC_PERIODIC;
    real Gl[3], Gh[3];
    lo[d] = x[d] - 1;
    hi[d] = x[d];
    if (periodic) {
        lo[d] = (lo[d] + nd) % nd;
        hi[d] = hi[d] % nd;
    } else if (x[d] == 0) {
        lo[d] = 0;
    } else if (x[d] == nd) {
        hi[d] = nd - 1;
    }
    G_cell(s, cell_index(s, lo), t, Gl);
    G_cell(s, cell_index(s, hi), t, Gh);
    if (s->nonuni && lo[d] != hi[d]) { /* linear interpolation to the interface (R18) */
        const double w = wface(s, d, x[d]);
        for (int a = 0; a < 3; a++) G[a] = (1.0 - w) * Gl[a] + w * Gh[a];
        return;
    }
    for (int a = 0; a < 3; a++) G[a] = 0.5 * (Gl[a] + Gh[a]);
}

/* --------------------------------------------------------------------------------
 * One time step t_n -> t_n + dt: the Appendix algorithm, steps 1 to 10.
 * -------------------------------------------------------------------------------- */
static void step_once(ostate *s)
{
    const int Q = s->Q, D = s->D;
    const double tau = s->tau, dt = s->cfg.dt, h = s->h, dx = s->cfg.dx;
    const double rho0 = s->cfg.rho0;
    const double t = s->t;
    int x[3];

    /* Step 1: fbar+ at X_c from eq. (24):
     *   fbar+ = (2tau-h)/(2tau+dt) f~ + 3h/(2tau+dt) f_eq + 3 tau h/(2tau+dt) S,
     * with rho, u the moments of f~ (eq. (27), reading R6). */
    const double a1 = (2 * tau - h) / (2 * tau + dt);
    const double b1 = 3 * h / (2 * tau + dt);
    const double c1 = 3 * tau * h / (2 * tau + dt);
    for (x[2] = 0; x[2] < s->n[2]; x[2]++)
        for (x[1] = 0; x[1] < s->n[1]; x[1]++)
            for (x[0] = 0; x[0] < s->n[0]; x[0]++) {
                const long ci = cell_index(s, x);
                const real *F = s->F + ci * Q;
                real *f = s->fc + ext_index(s, x) * Q;
                real G[3], rho, u[3];
                G_cell(s, ci, t, G);
                moments(s, F, G, 0.5 * dt, &rho, u);
                for (int k = 0; k < Q; k++) {
                    real fe = feq(s, k, rho, u);
                    f[k] = a1 * F[k] + b1 * fe + c1 * source(s, k, G, u, fe);
                }
            }

    /* Step 2: fbar+ at the ghost points X_cg (reading R3). Axis by axis; axes before d
     * run over their extended range, axes after d over the interior. */
    for (int d = 0; d < D; d++) {
        int lo[3], hi[3];
        for (int a = 0; a < 3; a++) {
            lo[a] = (a < d && a < D) ? -1 : 0;
            hi[a] = (a < d && a < D) ? s->n[a] : s->n[a] - 1;
        }
        const int nd = s->n[d];
        const int periodic = s->cfg.bc_type[2 * d] == BC_PERIODIC;
        for (int side = 0; side < 2; side++) {
            lo[d] = hi[d] = side == 0 ? -1 : nd;
            for (x[2] = lo[2]; x[2] <= hi[2]; x[2]++)
                for (x[1] = lo[1]; x[1] <= hi[1]; x[1]++)
                    for (x[0] = lo[0]; x[0] <= hi[0]; x[0]++) {
                        int y0[3] = {x[0], x[1], x[2]}, y1[3] = {x[0], x[1], x[2]};
                        real *g = s->fc + ext_index(s, x) * Q;
                        if (periodic) {
                            y0[d] = side == 0 ? nd - 1 : 0;
                            const real *f0 = s->fc + ext_index(s, y0) * Q;
                            for (int k = 0; k < Q; k++) g[k] = f0[k];
                        } else {
                            y0[d] = side == 0 ? 0 : nd - 1;
                            y1[d] = side == 0 ? 1 : nd - 2;
                            const real *f0 = s->fc + ext_index(s, y0) * Q;
                            const real *f1 = s->fc + ext_index(s, y1) * Q;
                            if (s->nonuni) { /* linear through the two centres to the ghost (R18) */
                                const double *c = s->xc[d] + 1;
                                const int i0 = y0[d], i1 = y1[d], ig = x[d];
                                const double eg = (c[ig] - c[i0]) / (c[i1] - c[i0]);
                                for (int k = 0; k < Q; k++) g[k] = f0[k] + eg * (f1[k] - f0[k]);
                            } else {
                                for (int k = 0; k < Q; k++) g[k] = 2.0 * f0[k] - f1[k];
                            }
                        }
                    }
        }
    }

    /* Step 3: fbar+ at X_b and X_bc by centre interpolation (reading R5). */
    for (int d = 0; d < D; d++) {
        for (x[2] = 0; x[2] < s->n[2] + (d == 2); x[2]++)
            for (x[1] = 0; x[1] < s->n[1] + (d == 1); x[1]++)
                for (x[0] = 0; x[0] < s->n[0] + (d == 0); x[0]++) {
                    int l[3] = {x[0], x[1], x[2]};
                    l[d] -= 1;
                    const real *fl = s->fc + ext_index(s, l) * Q;
                    const real *fr = s->fc + ext_index(s, x) * Q;
                    real *fb = s->fb[d] + face_index(s, d, x) * Q;
                    if (s->nonuni) {
                        const double w = wface(s, d, x[d]);
                        for (int k = 0; k < Q; k++) fb[k] = (1.0 - w) * fl[k] + w * fr[k];
                    } else {
                        for (int k = 0; k < Q; k++) fb[k] = 0.5 * (fl[k] + fr[k]);
                    }
                }
    }
    for (int p = 0; p < (D == 3 ? 3 : 1); p++) {
        int a, b;
        pair_axes(p, &a, &b);
        for (x[2] = 0; x[2] < s->n[2] + (a == 2 || b == 2); x[2]++)
            for (x[1] = 0; x[1] < s->n[1] + (a == 1 || b == 1); x[1]++)
                for (x[0] = 0; x[0] < s->n[0] + (a == 0 || b == 0); x[0]++) {
                    real *fbc = s->fbc[p] + cross_index(s, p, x) * Q;
                    int y[3];
                    for (int k = 0; k < Q; k++) fbc[k] = 0;
                    for (int da = -1; da <= 0; da++)
                        for (int db = -1; db <= 0; db++) {
                            y[0] = x[0]; y[1] = x[1]; y[2] = x[2];
                            y[a] += da;
                            y[b] += db;
                            const real *f = s->fc + ext_index(s, y) * Q;
                            double wt = 0.25;
                            if (s->nonuni) { /* bilinear in the two axes (R18) */
                                const double wa = wface(s, a, x[a]), wb = wface(s, b, x[b]);
                                wt = (da == 0 ? wa : 1.0 - wa) * (db == 0 ? wb : 1.0 - wb);
                            }
                            for (int k = 0; k < Q; k++) fbc[k] += wt * f[k];
                        }
                }
    }

    /* Step 4: fbar(x_b, t+h) = fbar+(x_b) - h xi . sigma_b (eq. (23)). Normal
     * component of sigma_b: difference of the two cells; tangential components:
     * difference of the two cross points on the interface (reading R5). */
    for (int d = 0; d < D; d++) {
        for (x[2] = 0; x[2] < s->n[2] + (d == 2); x[2]++)
            for (x[1] = 0; x[1] < s->n[1] + (d == 1); x[1]++)
                for (x[0] = 0; x[0] < s->n[0] + (d == 0); x[0]++) {
                    const long fi = face_index(s, d, x);
                    const real *fb = s->fb[d] + fi * Q;
                    real *Fb = s->Fb[d] + fi * Q;
                    int l[3] = {x[0], x[1], x[2]};
                    l[d] -= 1;
                    const real *fl = s->fc + ext_index(s, l) * Q;
                    const real *fr = s->fc + ext_index(s, x) * Q;
                    const real *cm[3] = {0, 0, 0}, *cp[3] = {0, 0, 0};
                    for (int tdir = 0; tdir < D; tdir++) {
                        if (tdir == d) continue;
                        int y[3] = {x[0], x[1], x[2]};
                        const int p = pair_of(d, tdir);
                        cm[tdir] = s->fbc[p] + cross_index(s, p, y) * Q;
                        y[tdir] += 1;
                        cp[tdir] = s->fbc[p] + cross_index(s, p, y) * Q;
                    }
                    for (int k = 0; k < Q; k++) {
                        real sigma[3] = {0, 0, 0};
                        if (s->nonuni) {
                            sigma[d] = (fr[k] - fl[k]) * inv_dc(s, d, x[d]);
                            for (int tdir = 0; tdir < D; tdir++)
                                if (tdir != d) sigma[tdir] = (cp[tdir][k] - cm[tdir][k]) / width(s, tdir, x[tdir]);
                        } else {
                            sigma[d] = (fr[k] - fl[k]) / dx;
                            for (int tdir = 0; tdir < D; tdir++)
                                if (tdir != d) sigma[tdir] = (cp[tdir][k] - cm[tdir][k]) / dx;
                        }
                        real xs = 0;
                        for (int a = 0; a < D; a++) xs += s->c * s->e[k][a] * sigma[a];
                        Fb[k] = fb[k] - h * xs;
                    }
                }
    }

    /* Step 5: boundary processing of fbar at the wall interfaces: NEQ, eq. (32)
     * (reading R4), or bounce-back, eq. (31) (reading R14). */
    for (int d = 0; d < D; d++) {
        if (s->cfg.bc_type[2 * d] == BC_PERIODIC) continue;
        for (int side = 0; side < 2; side++) {
            const int wall = 2 * d + side;
            const int type = s->cfg.bc_type[wall];
            const int nsign = side == 0 ? -1 : 1;       /* outward normal n = nsign e_d */
            int lo[3] = {0, 0, 0}, hi[3];
            for (int a = 0; a < 3; a++) hi[a] = s->n[a] - 1;
            lo[d] = hi[d] = side == 0 ? 0 : s->n[d];
            for (x[2] = lo[2]; x[2] <= hi[2]; x[2]++)
                for (x[1] = lo[1]; x[1] <= hi[1]; x[1]++)
                    for (x[0] = lo[0]; x[0] <= hi[0]; x[0]++) {
                        if (type == BC_BOUNCE_BACK) {
                            real *Fw = s->Fb[d] + face_index(s, d, x) * Q;
                            for (int k = 0; k < Q; k++) {
                                if (nsign * s->e[k][d] >= 0) continue; /* only xi.n < 0 */
                                real xu = 0;
                                for (int a = 0; a < 3; a++) xu += s->c * s->e[k][a] * s->wall_u[wall][a];
                                Fw[k] = Fw[opposite(s, k)] + 2.0 * rho0 * s->W[k] * xu / s->cfg.rt;
                            }
                            continue;
                        }
                        int xc[3] = {x[0], x[1], x[2]};
                        xc[d] = side == 0 ? 1 : s->n[d] - 1;
                        const real *Fc = s->Fb[d] + face_index(s, d, xc) * Q;
                        real *Fw = s->Fb[d] + face_index(s, d, x) * Q;
                        real Gc[3], rhoc, uc[3], rhoa, ua[3];
                        G_face(s, d, xc, t + h, Gc);
                        moments(s, Fc, Gc, 0.5 * h, &rhoc, uc);
                        if (type == BC_NEQ_VELOCITY) {
                            rhoa = rhoc;
                            for (int a = 0; a < 3; a++) ua[a] = s->wall_u[wall][a];
                        } else {
                            /* the wall pressure at the interface time t + h */
                            const double pw = s->cfg.bc_p[wall] + s->cfg.bc_p_amp[wall] * cos(s->cfg.omega * (t + h));
                            rhoa = rho0 + pw / s->cfg.rt;
                            for (int a = 0; a < 3; a++) ua[a] = uc[a];
                        }
                        for (int k = 0; k < Q; k++) {
                            if (nsign * s->e[k][d] >= 0) continue; /* only xi.n < 0 */
                            Fw[k] = feq(s, k, rhoa, ua) + (Fc[k] - feq(s, k, rhoc, uc));
                        }
                    }
        }
    }

    /* Step 6: rho, u at X_b (weight h/2 on G). Step 7: the original distribution at the
     * interface, eq. (20) solved for f:
     *   f = 2tau/(2tau+h) fbar + h/(2tau+h) f_eq + tau h/(2tau+h) S. */
    const double a7 = 2 * tau / (2 * tau + h);
    const double b7 = h / (2 * tau + h);
    const double c7 = tau * h / (2 * tau + h);
    for (int d = 0; d < D; d++) {
        for (x[2] = 0; x[2] < s->n[2] + (d == 2); x[2]++)
            for (x[1] = 0; x[1] < s->n[1] + (d == 1); x[1]++)
                for (x[0] = 0; x[0] < s->n[0] + (d == 0); x[0]++) {
                    const long fi = face_index(s, d, x);
                    real G[3];
                    G_face(s, d, x, t + h, G);
                    moments(s, s->Fb[d] + fi * Q, G, 0.5 * h, &s->rhob[d][fi], s->ub[d] + 3 * fi);
                }
        for (x[2] = 0; x[2] < s->n[2] + (d == 2); x[2]++)
            for (x[1] = 0; x[1] < s->n[1] + (d == 1); x[1]++)
                for (x[0] = 0; x[0] < s->n[0] + (d == 0); x[0]++) {
                    const long fi = face_index(s, d, x);
                    real *Fb = s->Fb[d] + fi * Q;
                    const real *u = s->ub[d] + 3 * fi;
                    real G[3];
                    G_face(s, d, x, t + h, G);
                    for (int k = 0; k < Q; k++) {
                        real fe = feq(s, k, s->rhob[d][fi], u);
                        Fb[k] = a7 * Fb[k] + b7 * fe + c7 * source(s, k, G, u, fe);
                    }
                }
    }

    /* Step 8: micro-flux m = sum over the cell's interfaces of (xi.n_j) f(x_j) s_j
     * (eq. (13)); on the uniform mesh s_j = dx^(D-1), on a non-uniform one the cell's
     * extent across the other axes (R18). */
    const double area = D == 3 ? dx * dx : dx;
    const double vol = D == 3 ? dx * dx * dx : dx * dx;
    for (x[2] = 0; x[2] < s->n[2]; x[2]++)
        for (x[1] = 0; x[1] < s->n[1]; x[1]++)
            for (x[0] = 0; x[0] < s->n[0]; x[0]++) {
                real *m = s->m + cell_index(s, x) * Q;
                for (int k = 0; k < Q; k++) m[k] = 0;
                double cvol = vol;
                if (s->nonuni) {
                    cvol = 1.0;
                    for (int a = 0; a < D; a++) cvol *= width(s, a, x[a]);
                }
                for (int d = 0; d < D; d++) {
                    int xp[3] = {x[0], x[1], x[2]};
                    xp[d] += 1;
                    const real *fm = s->Fb[d] + face_index(s, d, x) * Q;  /* n = -e_d */
                    const real *fp = s->Fb[d] + face_index(s, d, xp) * Q; /* n = +e_d */
                    /* interface area s_j: the cell's extent across the other axes */
                    const double ar = s->nonuni ? cvol / width(s, d, x[d]) : area;
                    for (int k = 0; k < Q; k++) {
                        const double xn = s->c * s->e[k][d];
                        m[k] += xn * fp[k] * ar - xn * fm[k] * ar;
                    }
                }
            }

    /* Step 9: f~+ = 4/3 fbar+ - 1/3 f~ (eq. (25)), then
     * f~(t+dt) = f~+ - dt/|V| m (eq. (16)). */
    for (x[2] = 0; x[2] < s->n[2]; x[2]++)
        for (x[1] = 0; x[1] < s->n[1]; x[1]++)
            for (x[0] = 0; x[0] < s->n[0]; x[0]++) {
                const long ci = cell_index(s, x);
                real *F = s->F + ci * Q;
                const real *f = s->fc + ext_index(s, x) * Q;
                const real *m = s->m + ci * Q;
                double cvol = vol;
                if (s->nonuni) {
                    cvol = 1.0;
                    for (int a = 0; a < D; a++) cvol *= width(s, a, x[a]);
                }
                for (int k = 0; k < Q; k++) {
                    real ftp = 4.0 / 3.0 * f[k] - 1.0 / 3.0 * F[k];
                    F[k] = ftp - dt / cvol * m[k];
                }
            }

    /* Step 10 (moments of the new F) is evaluated on demand by moments(). */
    s->step += 1;
    s->t = s->cfg.dt * (double)s->step;
}

/* ------------------------------- public API ------------------------------------- */

static int check_config(const oracle_config *c)
{
    if (!(c->dim == 2 || c->dim == 3)) return -1;
    if (c->dim == 2 && c->q != 9) return -1;
    if (c->dim == 3 && !(c->q == 19 || c->q == 27)) return -1;
    if (c->nx < 1 || c->ny < 1 || c->nz < 1) return -1;
    if (c->dim == 2 && c->nz != 1) return -1;
    if (!(c->dx > 0 && c->rt > 0 && c->rho0 > 0 && c->nu > 0 && c->dt > 0)) return -1;
    if (!(c->model == 0 || c->model == 1)) return -1;
    const int n[3] = {c->nx, c->ny, c->nz};
    for (int d = 0; d < c->dim; d++) {
        const int lo = c->bc_type[2 * d], hi = c->bc_type[2 * d + 1];
        if ((lo == BC_PERIODIC) != (hi == BC_PERIODIC)) return -1;
        if (lo < 0 || lo > 3 || hi < 0 || hi > 3) return -1;
        if (lo != BC_PERIODIC && n[d] < 2) return -1;
    }
    return 0;
}

void *oracle_create(const oracle_config *cfg)
{
    if (!cfg || check_config(cfg) != 0) return NULL;
    ostate *s = (ostate *)calloc(1, sizeof(ostate));
    if (!s) return NULL;
    s->cfg = *cfg;
    s->D = cfg->dim;
    s->Q = cfg->q;
    s->n[0] = cfg->nx; s->n[1] = cfg->ny; s->n[2] = cfg->dim == 3 ? cfg->nz : 1;
    build_lattice(s);
    s->c = sqrt(3.0 * cfg->rt);         /* xi = sqrt(3RT) e (Sec. 2.3) */
    s->tau = cfg->nu / cfg->rt;         /* reading R1 */
    s->h = 0.5 * cfg->dt;               /* h = dt/2 (Sec. 2.2) */
    s->ncell = (long)s->n[0] * s->n[1] * s->n[2];
    for (int a = 0; a < 3; a++) {
        s->eo[a] = a < s->D ? 1 : 0;
        s->en[a] = s->n[a] + 2 * s->eo[a];
    }
    s->next = (long)s->en[0] * s->en[1] * s->en[2];
    const int Q = s->Q;
    s->F = (real *)calloc((size_t)s->ncell * Q, sizeof(real));
    s->fc = (real *)calloc((size_t)s->next * Q, sizeof(real));
    s->m = (real *)calloc((size_t)s->ncell * Q, sizeof(real));
    s->field = (real *)calloc((size_t)3 * s->ncell, sizeof(real));
    int ok = s->F && s->fc && s->m && s->field;
    for (int d = 0; d < s->D; d++) {
        long nf = 1;
        for (int a = 0; a < 3; a++) nf *= s->n[a] + (a == d);
        s->nface[d] = nf;
        s->fb[d] = (real *)calloc((size_t)nf * Q, sizeof(real));
        s->Fb[d] = (real *)calloc((size_t)nf * Q, sizeof(real));
        s->rhob[d] = (real *)calloc((size_t)nf, sizeof(real));
        s->ub[d] = (real *)calloc((size_t)nf * 3, sizeof(real));
        ok = ok && s->fb[d] && s->Fb[d] && s->rhob[d] && s->ub[d];
    }
    for (int p = 0; p < (s->D == 3 ? 3 : 1); p++) {
        int a, b;
        long nc = 1;
        pair_axes(p, &a, &b);
        for (int i = 0; i < 3; i++) nc *= s->n[i] + (i == a || i == b);
        s->ncross[p] = nc;
        s->fbc[p] = (real *)calloc((size_t)nc * Q, sizeof(real));
        ok = ok && s->fbc[p];
    }
    for (int w = 0; w < 6; w++)
        for (int a = 0; a < 3; a++) s->wall_u[w][a] = cfg->bc_u[w][a];
    /* non-uniform mesh (reading R18): interface coordinates and extended centres */
    for (int a = 0; a < s->D; a++) s->nonuni |= cfg->faces[a] != NULL;
    for (int a = 0; ok && s->nonuni && a < s->D; a++) {
        const int n = s->n[a];
        s->xf[a] = (double *)calloc((size_t)n + 1, sizeof(double));
        s->xc[a] = (double *)calloc((size_t)n + 2, sizeof(double));
        ok = s->xf[a] && s->xc[a];
        if (!ok) break;
        for (int i = 0; i <= n; i++) s->xf[a][i] = cfg->faces[a] ? cfg->faces[a][i] : i * cfg->dx;
        for (int i = 0; i < n; i++) {
            if (!(s->xf[a][i + 1] > s->xf[a][i])) ok = 0;
            s->xc[a][i + 1] = 0.5 * (s->xf[a][i] + s->xf[a][i + 1]);
        }
        if (!ok) break;
        if (cfg->bc_type[2 * a] == BC_PERIODIC) { /* images one period away */
            const double L = s->xf[a][n] - s->xf[a][0];
            s->xc[a][0] = s->xc[a][n] - L;
            s->xc[a][n + 1] = s->xc[a][1] + L;
        } else { /* boundary centres mirrored in the walls */
            s->xc[a][0] = 2.0 * s->xf[a][0] - s->xc[a][1];
            s->xc[a][n + 1] = 2.0 * s->xf[a][n] - s->xc[a][n];
        }
    }
    if (!ok) {
        oracle_destroy(s);
        return NULL;
    }
    return s;
}

void oracle_destroy(void *p)
{
    ostate *s = (ostate *)p;
    if (!s) return;
    free(s->F); free(s->fc); free(s->m); free(s->field);
    for (int d = 0; d < 3; d++) {
        free(s->fb[d]); free(s->Fb[d]); free(s->rhob[d]); free(s->ub[d]); free(s->fbc[d]);
        free(s->xf[d]); free(s->xc[d]);
    }
    free(s);
}

/* Lattice table: e[Q][3] (integers, xi = sqrt(3RT) e) and W[Q]. */
int oracle_lattice(void *p, int *e, double *W)
{
    ostate *s = (ostate *)p;
    for (int k = 0; k < s->Q; k++) {
        for (int a = 0; a < 3; a++) e[3 * k + a] = s->e[k][a];
        W[k] = s->W[k];
    }
    return s->Q;
}

/* Per-cell acceleration field [dim][ncell] (x fastest); NULL clears it. */
int oracle_set_field(void *p, const double *field)
{
    ostate *s = (ostate *)p;
    for (int a = 0; a < 3; a++)
        for (long i = 0; i < s->ncell; i++)
            s->field[a * s->ncell + i] = (field && a < s->D) ? field[a * s->ncell + i] : 0.0;
    return 0;
}

/* Initial state, reading R7: f~ = f_eq(rho0 + p/RT, u) (eq. (6)). p: [ncell] or NULL
 * (zero); u: [dim][ncell] or NULL (rest). Resets the clock to t = 0. */
int oracle_init(void *p, const double *pres, const double *vel)
{
    ostate *s = (ostate *)p;
    for (long i = 0; i < s->ncell; i++) {
        real rho = s->cfg.rho0 + (pres ? pres[i] / s->cfg.rt : 0.0);
        real u[3] = {0, 0, 0};
        for (int a = 0; a < s->D; a++) u[a] = vel ? vel[a * s->ncell + i] : 0.0;
        for (int k = 0; k < s->Q; k++) s->F[i * s->Q + k] = feq(s, k, rho, u);
    }
    s->step = 0;
    s->t = 0.0;
    return 0;
}

int oracle_step(void *p, long nsteps)
{
    ostate *s = (ostate *)p;
    for (long i = 0; i < nsteps; i++) step_once(s);
    return 0;
}

double oracle_time(void *p) { return ((ostate *)p)->t; }
long oracle_step_count(void *p) { return ((ostate *)p)->step; }

/* Moments of the current state (eq. (27) with G(t)): out[(dim+1)][ncell] =
 * p = (rho - rho0) RT (reading R9), then u_x, u_y[, u_z]. out_im: imaginary parts (the
 * complex-step derivative direction), may be NULL. */
int oracle_moments(void *p, double *out, double *out_im)
{
    ostate *s = (ostate *)p;
    int x[3];
    for (x[2] = 0; x[2] < s->n[2]; x[2]++)
        for (x[1] = 0; x[1] < s->n[1]; x[1]++)
            for (x[0] = 0; x[0] < s->n[0]; x[0]++) {
                const long ci = cell_index(s, x);
                real G[3], rho, u[3];
                G_cell(s, ci, s->t, G);
                moments(s, s->F + ci * s->Q, G, 0.5 * s->cfg.dt, &rho, u);
                real pr = (rho - s->cfg.rho0) * s->cfg.rt;
                out[ci] = RE(pr);
                if (out_im) out_im[ci] = IM(pr);
                for (int a = 0; a < s->D; a++) {
                    out[(a + 1) * s->ncell + ci] = RE(u[a]);
                    if (out_im) out_im[(a + 1) * s->ncell + ci] = IM(u[a]);
                }
            }
    return 0;
}

/* State f~ as [Q][ncell] (direction-major, x fastest) real parts and imaginary parts. */
int oracle_get_state(void *p, double *re, double *im)
{
    ostate *s = (ostate *)p;
    for (long i = 0; i < s->ncell; i++)
        for (int k = 0; k < s->Q; k++) {
            re[k * s->ncell + i] = RE(s->F[i * s->Q + k]);
            if (im) im[k * s->ncell + i] = IM(s->F[i * s->Q + k]);
        }
    return 0;
}

int oracle_set_state(void *p, const double *re, const double *im, double t, long step)
{
    ostate *s = (ostate *)p;
    (void)im;
    for (long i = 0; i < s->ncell; i++)
        for (int k = 0; k < s->Q; k++) {
            real v = re[k * s->ncell + i];
#ifdef ORACLE_COMPLEX_STEP
            if (im) v += I * im[k * s->ncell + i];
#endif
            s->F[i * s->Q + k] = v;
        }
    s->t = t;
    s->step = step;
    return 0;
}

#ifdef ORACLE_COMPLEX_STEP
/* Complex-step directions on the inputs the adjoint differentiates: the per-cell
 * acceleration field ([dim][ncell]) and the wall velocities ([6][3]). */
int oracle_set_field_im(void *p, const double *im)
{
    ostate *s = (ostate *)p;
    for (int a = 0; a < s->D; a++)
        for (long i = 0; i < s->ncell; i++)
            s->field[a * s->ncell + i] = RE(s->field[a * s->ncell + i]) + I * (im ? im[a * s->ncell + i] : 0.0);
    return 0;
}

int oracle_set_wall_u_im(void *p, const double *im)
{
    ostate *s = (ostate *)p;
    for (int w = 0; w < 6; w++)
        for (int a = 0; a < 3; a++) s->wall_u[w][a] = s->cfg.bc_u[w][a] + I * (im ? im[3 * w + a] : 0.0);
    return 0;
}
#endif

/* Conservation sums over X_c of the current state: out[0] = sum rho, out[1+a] = sum
 * rho0 u_a with u from eq. (27) (per cell, no volume factor). */
int oracle_sums(void *p, double *out)
{
    ostate *s = (ostate *)p;
    double r = 0, j[3] = {0, 0, 0};
    for (long i = 0; i < s->ncell; i++) {
        real G[3], rho, u[3];
        G_cell(s, i, s->t, G);
        moments(s, s->F + i * s->Q, G, 0.5 * s->cfg.dt, &rho, u);
        r += RE(rho);
        for (int a = 0; a < 3; a++) j[a] += RE(s->cfg.rho0 * u[a]);
    }
    out[0] = r;
    for (int a = 0; a < s->D; a++) out[1 + a] = j[a];
    return 0;
}

/* Relative L2 change between two velocity fields (the steady-state criterion of Sec.
 * 3.1): sqrt(sum |u_new - u_old|^2) / sqrt(sum |u_new|^2); fields [dim][n]. */
double oracle_rel_change(const double *u_new, const double *u_old, long n, int dim)
{
    double num = 0, den = 0;
    for (int a = 0; a < dim; a++)
        for (long i = 0; i < n; i++) {
            const double dlt = u_new[a * n + i] - u_old[a * n + i];
            num += dlt * dlt;
            den += u_new[a * n + i] * u_new[a * n + i];
        }
    return den > 0 ? sqrt(num) / sqrt(den) : (num > 0 ? INFINITY : 0.0);
}

/* L2 relative global error E(phi) of Sec. 3.1 (phi = u, a vector with ncomp components
 * stored [ncomp][n], or p with ncomp = 1). */
double oracle_l2_error(const double *phi, const double *ref, long n, int ncomp)
{
    double num = 0, den = 0;
    for (int a = 0; a < ncomp; a++)
        for (long i = 0; i < n; i++) {
            const double dlt = phi[a * n + i] - ref[a * n + i];
            num += dlt * dlt;
            den += ref[a * n + i] * ref[a * n + i];
        }
    return sqrt(num) / sqrt(den);
}
