/*
 * dugks.h -- C ABI of the GB300 (sm_103a) hot path of the incompressible discrete unified
 * gas kinetic scheme (DUGKS) with force term of Wu, Shi, Chai and Wang (arXiv 1411.6121).
 *
 * One handle (dugks_t) owns one simulation on one CUDA device: the cell-averaged
 * distribution f~ of the paper (Sec. 2.2, eq. (16)) on a uniform Cartesian
 * mesh with the D2Q9 or D3Q19 (or D3Q27) velocity set, and everything the time step needs.
 * Every entry point returns DUGKS_OK (0) or a negative DUGKS_E_* code; none throws,
 * aborts or exits. dugks_last_error() gives a one-line reason for the last failure on a
 * handle (or, with a NULL handle, for the last failed dugks_create in this thread).
 *
 * Conventions
 *  - Cells are indexed x fastest: cell (i, j, k) is i + nx*(j + ny*k). Field arrays
 *    passed in or out are "component-major": component a of cell n is at a*ncell + n.
 *  - Lattice units are not assumed: dx, RT, rho0, nu and dt are given explicitly. The
 *    particle speed is c = sqrt(3 RT) (Sec. 2.3), the relaxation time tau = nu / RT.
 *  - Boundary faces are ordered -x, +x, -y, +y, -z, +z. A periodic face must be paired
 *    with a periodic opposite face. A wall axis needs at least 2 cells.
 *  - Work is enqueued on the handle's CUDA stream (opts.stream, or a non-blocking stream
 *    the handle creates when NULL) and runs asynchronously unless the entry point says
 *    otherwise.
 *  - Device memory is owned by the handle and released by dugks_destroy. Caller buffers
 *    are never retained after a call returns.
 */
#ifndef DUGKS_H
#define DUGKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------------------- */
#define DUGKS_OK 0
#define DUGKS_E_INVAL (-1)       /* bad argument (NULL, size, combination)              */
#define DUGKS_E_CFL (-2)         /* dt > dx / sqrt(3RT): CFL number above one (Sec. 3)  */
#define DUGKS_E_NOMEM (-3)       /* device or host allocation failed                    */
#define DUGKS_E_CUDA (-4)        /* a CUDA runtime call failed                          */
#define DUGKS_E_UNSTABLE (-5)    /* non-finite moments found by the FP64 reduction      */
#define DUGKS_E_TIMEOUT (-6)     /* dugks_sync ran past its time limit                  */
#define DUGKS_E_UNSUPPORTED (-7) /* lattice/storage/dimension combination not built     */

/* ---- enumerations ---------------------------------------------------------------- */
/* Velocity sets (Sec. 2.3): D2Q9 and D3Q27 are the paper's tensor-product sets; D3Q19 is
 * D3Q27 without its 8 corner velocities (weights 1/3, 1/18, 1/36). Index order is the
 * paper's: x component slowest. */
#define DUGKS_D2Q9 9
#define DUGKS_D3Q19 19
#define DUGKS_D3Q27 27

/* Storage of f~ in device memory. The stored quantity is the deviation from the rest
 * equilibrium, g~ = f~ - W_k rho0 (exact algebra: every linear step of the scheme has
 * coefficients summing to one or zero). F32, BF16 and F16 storage use FP32 arithmetic;
 * F64 storage uses FP64 arithmetic throughout. BF16 stores g~ and F16 stores g~ * 2^12 (the
 * exact scale keeps small deviations out of FP16's subnormal range), both with unbiased
 * stochastic rounding (random bits from a hash of the address and the step), which keeps
 * slowly varying values from accumulating a rounding bias or losing small increments.
 * dugks_get_state / dugks_set_state move these raw stored values. */
#define DUGKS_STORE_F32 0
#define DUGKS_STORE_BF16 1
#define DUGKS_STORE_F16 2
#define DUGKS_STORE_F64 3

/* Boundary conditions of Sec. 2.4 applied at a domain face. */
#define DUGKS_BC_PERIODIC 0
#define DUGKS_BC_NEQ_VELOCITY 1 /* eq. (32), velocity condition: u_a = u_w, rho_a = rho(x_c)  */
#define DUGKS_BC_NEQ_PRESSURE 2 /* eq. (32), pressure condition: rho_a = rho0 + p_w/RT, u_a = u(x_c) */
#define DUGKS_BC_BOUNCE_BACK 3  /* eq. (31): fbar_k = fbar_-k + 2 rho0 W_k xi_k.u_w / RT for xi.n < 0
                                   (rho_w = rho0), at the wall interface before step 6        */

/* Equilibrium models (Sec. 2.1-2.2). The incompressible model is the paper's: eq. (6) with
 * rho0 u = sum xi f~ + rho0 G dt/2 (eq. (27)). The original DUGKS, the model it is
 * compared against, uses eq. (5) with rho u = sum xi f~ + rho G dt/2. */
#define DUGKS_MODEL_INCOMPRESSIBLE 0
#define DUGKS_MODEL_ORIGINAL 1

/* ---- parameter records ----------------------------------------------------------- */
typedef struct {
    int32_t dim;     /* 2 or 3 */
    int64_t nx, ny;  /* cells per axis */
    int64_t nz;      /* 1 in 2D */
    double dx;       /* uniform spacing, dx = dy = dz */
    const double *faces[3]; /* optional non-uniform mesh (Sec. 3.4's tanh mesh, which
                               Sec. 3.5 also uses for the cube; 2D and 3D, the reference
                               kernel, no adjoint or batch): HOST arrays of the n+1
                               interface coordinates of x, y (and z in 3D), copied at
                               creation; NULL (default) means uniform spacing dx along that
                               axis. F32 or F64 storage; 16-bit storage: the handle is not
                               created (DUGKS_E_UNSUPPORTED); coordinates that do not
                               increase, or faces[2] in 2D: DUGKS_E_INVAL. The time step
                               must satisfy dt <= min width / sqrt(3RT) (DUGKS_E_CFL). */
} dugks_mesh;

typedef struct {
    int32_t type;    /* DUGKS_BC_* */
    double u[3];     /* wall velocity u_w (velocity condition, bounce-back) */
    double p;        /* wall pressure p_w = (rho_w - rho0) RT (pressure condition) */
    double p_amp;    /* pressure condition: p_w(t) = p + p_amp cos(omega t), with the omega of
                        the force record (0: steady)                               */
} dugks_face_bc;

typedef struct {
    dugks_face_bc face[6]; /* -x, +x, -y, +y, -z, +z */
} dugks_boundaries;

/* Acceleration G(x, t) = (g + field(x)) * cos(omega t) of eq. (9) (Sec. 2.2). field is a
 * DEVICE pointer to [dim][ncell] floats or NULL; the handle reads it during every step, so
 * it must stay valid (and may be rewritten between steps) until it is replaced by
 * dugks_set_force_field or the handle is destroyed. */
typedef struct {
    double g[3];
    double omega;
    const float *field;
} dugks_force;

typedef struct {
    double rt;              /* RT (default 1/3: lattice units with c = 1)            */
    double rho0;            /* reference density rho0 (default 1)                    */
    int32_t store;          /* DUGKS_STORE_* (default F32)                           */
    void *stream;           /* cudaStream_t to run on (default NULL: own stream)     */
    int32_t use_graph;      /* 1: dugks_step replays a captured CUDA graph (default) */
    int32_t tile_x, tile_y; /* 0: default tile. Throughput kernels (kernel 0, F32/BF16/F16
                               storage): tile_y = thread-block rows (D2Q9: 4, 8 or 16;
                               D3Q19: 8 or 10; D3Q27: 8; default 8), tile_x ignored.
                               Reference
                               kernel: tile_x x tile_y = 32x8 or 16x8                   */
    int32_t kernel;         /* 0: fastest kernel built for the case (default);
                               1: the reference fused kernel (any lattice/storage)     */
    int32_t model;          /* DUGKS_MODEL_INCOMPRESSIBLE (default) or DUGKS_MODEL_ORIGINAL
                               (runs on the reference kernel; no adjoint, no batch)    */
} dugks_opts;

typedef struct dugks_s *dugks_t;

/* Fill *opts with the defaults listed above. */
int dugks_opts_default(dugks_opts *opts);

/* Create a simulation (Sec. 2.2 and Sec. 3): validates the mesh, boundaries and
 * dt <= dx / sqrt(3RT) (the CFL condition of Sec. 3; DUGKS_E_CFL otherwise), allocates the
 * state on the current CUDA device and initialises it to the rest state f~ = W rho0.
 * lattice: DUGKS_D2Q9 (dim 2) or DUGKS_D3Q19 / DUGKS_D3Q27 (dim 3). nu > 0, dt > 0.
 * force, bcs: required (use DUGKS_BC_PERIODIC everywhere for a periodic box).
 * opts: NULL for defaults. On success *out receives the handle. */
int dugks_create(const dugks_mesh *mesh, int32_t lattice, double nu, double dt,
                 const dugks_force *force, const dugks_boundaries *bcs,
                 const dugks_opts *opts, dugks_t *out);

/* Initial state as in Sec. 3 ("the equilibrium distribution is initialised by"):
 * f~ = f_eq(rho0 + p/RT, u) of eq. (6), computed on the device. p: HOST [ncell] doubles
 * or NULL (p = 0); u: HOST [dim][ncell] doubles or NULL (rest). Resets the clock to t = 0.
 * Synchronous. */
int dugks_init(dugks_t h, const double *p, const double *u);

/* Advance n >= 0 time steps (the Appendix algorithm, steps 1-10, one fused kernel launch
 * per step). Asynchronous; returns after enqueueing. */
int dugks_step(dugks_t h, int64_t n);

/* Macroscopic fields of the current state (eq. (27) with G(t)):
 * out[0][n] = p = (rho - rho0) RT, out[1+a][n] = u_a, i.e. [dim+1][ncell] floats.
 * out_is_device: 1 if out is device memory, 0 for host memory (pinned or pageable).
 * Synchronous. */
int dugks_moments(dugks_t h, float *out, int32_t out_is_device);

/* FP64 reductions of the current state (the steady-state criterion of Sec. 3.1 and the
 * conservation totals): out[0] = ||u - u_prev||_2 / ||u||_2 where u_prev is the velocity
 * field at the previous dugks_residual call (or at dugks_init; +inf before any), then
 * stores u as the new u_prev; out[1] = sum rho; out[2+a] = sum rho0 u_a (sum rho u_a in the
 * original model; per cell, no volume factor). out: HOST array of dim+2 doubles. Returns DUGKS_E_UNSTABLE if any sum
 * is not finite. Synchronous. */
int dugks_residual(dugks_t h, double *out);

/* Raw state for checkpoint/restart: g~ = f~ - W rho0 in the storage type, laid out
 * [Q][nz][ny][nx] (unpadded). dugks_state_bytes gives the size. buf_is_device as above.
 * The clock (time, step count) is part of the handle, see dugks_get_clock. Synchronous. */
int dugks_state_bytes(dugks_t h, size_t *bytes);
int dugks_get_state(dugks_t h, void *buf, size_t bytes, int32_t buf_is_device);
int dugks_set_state(dugks_t h, const void *buf, size_t bytes, int32_t buf_is_device);
int dugks_get_clock(dugks_t h, int64_t *step, double *time);
int dugks_set_clock(dugks_t h, int64_t step);

/* Replace the per-cell acceleration field (device [dim][ncell] floats, or NULL). */
int dugks_set_force_field(dugks_t h, const float *field);

/* Replace the wall velocities u and wall pressures p of the boundaries given at creation.
 * The face types must be unchanged (DUGKS_E_INVAL otherwise). Takes effect at the next step. */
int dugks_set_boundaries(dugks_t h, const dugks_boundaries *bcs);

/* Wait for the handle's stream, polling for at most timeout_s seconds (<= 0: no limit).
 * DUGKS_E_TIMEOUT if the work has not finished by then (the work keeps running), or if a
 * 3D step found that a state copy into shared memory did not land within two seconds (that
 * CTA left its step undone; the state is then invalid). */
int dugks_sync(dugks_t h, double timeout_s);

/* Number of kernel launches the handle enqueued since creation (diagnostics). */
int64_t dugks_launch_count(dugks_t h);

const char *dugks_last_error(dugks_t h);
void dugks_destroy(dugks_t h);

/* ---- differentiation: checkpointed adjoint of the step (D2Q9, F32 or F64 storage) -------
 * The paper has no adjoint; these two calls give the gradient of a loss of the final
 * moments with respect to the acceleration field, the wall velocities and the initial state,
 * through the exact discrete adjoint of the step (Appendix steps 1-10, transposed step by
 * step in the handle's arithmetic type).
 *
 * dugks_record runs nsteps steps from the current state, exactly as dugks_step does, and
 * keeps a device copy of the state every `every` steps (ceil(nsteps/every) state buffers plus
 * `every` buffers for the reverse sweep, owned by the handle and reused by later calls). The
 * handle's clock advances by nsteps. A new record replaces the previous one.
 *
 * dugks_adjoint takes dL_dmom = dL/d(moments at the end of the recorded rollout), a DEVICE
 * [3][ncell] float array in the layout of dugks_moments (p, u_x, u_y), and runs the reverse
 * sweep: for each checkpoint segment, last first, it recomputes the segment's states from its
 * checkpoint and applies the transposed step to them in reverse order. Outputs (each may be
 * NULL when not wanted):
 *   dL_dfield  DEVICE [2][ncell] floats: dL/d(acceleration field) (the per-cell G of
 *              dugks_force, whether or not a field is set), overwritten;
 *   dL_dwall   HOST [6][3] doubles: dL/d(u of each face) for velocity walls, zero elsewhere;
 *   dL_dstate0 DEVICE [Q][ncell] values of the storage type: dL/d(state at the start of the
 *              rollout), unpadded layout as dugks_get_state.
 * The acceleration, wall velocities and viscosity must be those of the recorded rollout.
 * Synchronous. DUGKS_E_UNSUPPORTED for 3D lattices or BF16/F16 storage; DUGKS_E_INVAL
 * without a recorded rollout. Memory: (ceil(nsteps/every) + every) x the state size plus
 * about 7 state sizes of work buffers. With use_graph, a time-independent acceleration and
 * at least 3 segments, each segment's work is captured once as a CUDA graph and kept by the
 * handle across calls (and across records of the same length) while the buffers and
 * parameters it was captured with are unchanged; a later call with any of them changed
 * captures again. */
int dugks_record(dugks_t h, int64_t nsteps, int32_t every);
int dugks_adjoint(dugks_t h, const float *dL_dmom, float *dL_dfield, double *dL_dwall, void *dL_dstate0);
/* Asynchronous form of dugks_adjoint for running the reverse sweeps of several handles
 * concurrently on their streams: enqueues the same work and returns; dL_dfield and
 * dL_dstate0 are complete once the handle's stream is (dugks_sync). dugks_adjoint_wall waits
 * for the stream and writes the wall-velocity gradient [6][3] of the last adjoint to HOST
 * memory. dugks_adjoint_async first waits for any earlier work of the handle. */
int dugks_adjoint_async(dugks_t h, const float *dL_dmom, float *dL_dfield, void *dL_dstate0);
int dugks_adjoint_wall(dugks_t h, double *dL_dwall);

/* ---- batched form: many independent 2D instances ---------------------------------------
 * A batch advances `count` independent D2Q9 instances (each its own mesh, viscosity,
 * acceleration and boundaries; shared dt, RT, rho0 and storage from opts) together: one time
 * step of the whole batch is one persistent kernel launch over a work list of (instance,
 * tile) items, largest instances first, and dugks_batch_step replays n such launches as one
 * captured CUDA graph. The per-instance scheme is exactly that of dugks_step (Appendix
 * steps 1-10 of the paper). meshes/nu/forces/bcs: HOST arrays of `count` records (a force
 * field pointer, if any, is a DEVICE [2][ncell] float array read at every step). opts may
 * be NULL; opts->tile_x/tile_y pick the tile: 30x2, 30x6 or 30x14 inner cells of the throughput
 * kernel (32 x 4, 8 or 16 threads; F32/BF16/F16), or 32x8, 16x8, 32x4 or 64x4 of the reference
 * kernel; default 30x6.
 * Errors as for the single-instance calls; dugks_batch_last_error(b) gives the reason
 * (NULL b: the last failed dugks_batch_create in this thread). */
typedef struct dugks_batch_s *dugks_batch_t;
int dugks_batch_create(int32_t count, const dugks_mesh *meshes, const double *nu, double dt,
                       const dugks_force *forces, const dugks_boundaries *bcs, const dugks_opts *opts,
                       dugks_batch_t *out);
/* Initial state of instance i (as dugks_init: f~ = f_eq(rho0 + p/RT, u), HOST fields or NULL). */
int dugks_batch_init(dugks_batch_t b, int32_t i, const double *p, const double *u);
/* Advance every instance by n steps (asynchronous). */
int dugks_batch_step(dugks_batch_t b, int64_t n);
/* Moments of instance i: [3][ncell_i] floats (p, u_x, u_y); synchronous. */
int dugks_batch_moments(dugks_batch_t b, int32_t i, float *out, int32_t out_is_device);
/* Autotuner: times each built tile shape (best of three interleaved 16-step trials) on a copy
 * of the batch state (the state and clock are restored), keeps the fastest and caches the
 * choice per (instance sizes, storage, SM count) for the process. Writes the chosen tile to
 * tile_x/tile_y (may be NULL). */
int dugks_batch_tune(dugks_batch_t b, int32_t *tile_x, int32_t *tile_y);
int dugks_batch_sync(dugks_batch_t b);
int64_t dugks_batch_launch_count(dugks_batch_t b);
const char *dugks_batch_last_error(dugks_batch_t b);
void dugks_batch_destroy(dugks_batch_t b);

/* Allocation-free FP64 residual and conservation totals (the paper has no counterpart; this
 * is a library facility). Same reduction, on the same number of blocks in the same order,
 * and the same outputs as dugks_residual for a state of the incompressible model (the
 * default, DUGKS_MODEL_INCOMPRESSIBLE; the original model's velocity divides by the local
 * density, which this call does not do). It serves callers that cannot call cudaMalloc:
 * hosts whose own allocator already owns the device memory, and loops that must not take
 * cudaMalloc's implicit device synchronisation. Nothing is allocated: the partial sums go to
 * a fixed 256 KB array in device memory that the library reserves on every GPU that loads
 * it, held until the process exits. The call copies its sums to host memory and synchronises
 * `stream` before it returns, so it cannot be called while that stream is being captured
 * into a CUDA graph.
 *   state:  DEVICE pointer to g~ = f~ - W rho0 in the storage type `store`, unpadded layout
 *           [Q][nz][ny][nx] (what dugks_get_state writes with buf_is_device = 1).
 *   nx, ny, nz, lattice: the mesh and velocity set (nz = 1 and DUGKS_D2Q9 in 2D).
 *   rt, rho0: RT and rho0 of the simulation.
 *   shift:  HOST [3] doubles or NULL: the uniform part of the velocity shift of eq.
 *           (27), G(t) dt/2 (u = c/rho0 sum_k e_k g~_k + shift).
 *   shift_field: DEVICE [dim][ncell] floats or NULL: the per-cell part of that shift.
 *   uprev:  DEVICE [dim][ncell] doubles owned by the caller: the velocity of the previous
 *           call, read when have_prev != 0 and overwritten with the current velocity.
 *   out:    HOST [dim+2] doubles: out[0] = ||u - uprev||/||u|| (+inf when have_prev == 0),
 *           out[1] = sum rho, out[2+a] = sum rho0 u_a.
 *   stream: cudaStream_t (NULL: legacy stream); the call synchronises it before returning.
 * Limit: at most 16,777,216 cells (256^3; 4096 partial-sum blocks of at most 4096 cells);
 * larger meshes return DUGKS_E_INVAL with the limit in dugks_last_error(NULL). The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current) and caches it. Every call on a device shares the one array: calls that
 * overlap on the GPU (from several streams or threads) race and give wrong sums. Each call
 * rewrites every partial it reads, so nothing has to be cleared between calls. Errors:
 * DUGKS_E_INVAL, DUGKS_E_CUDA, DUGKS_E_UNSTABLE (non-finite sums); the reason is in
 * dugks_last_error(NULL). */
int dugks_residual_static(int32_t lattice, int32_t store, const void *state, int64_t nx, int64_t ny, int64_t nz,
                          double rt, double rho0, const double *shift, const float *shift_field, double *uprev,
                          int32_t have_prev, double *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* DUGKS_H */
