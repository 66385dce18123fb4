// handle.h -- the simulation handle behind dugks_t, shared by the host translation units
// that implement the C ABI (api.cu, adjoint2d.cu).
#pragma once

#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/dugks.h"
#include "dugks_internal.h"

namespace dugks {

// Checkpoints of a recorded rollout (dugks_record) and the buffers of its adjoint sweep.
struct AdjointTape {
    int64_t steps = 0;           // recorded steps (0: nothing recorded)
    int64_t step0 = 0;           // clock step at the start of the rollout
    int every = 0;               // checkpoint interval
    std::vector<void *> ckpt;    // padded state at step0 + s * every, s = 0 .. nseg - 1
    std::vector<void *> seg;     // every padded states of the segment being reversed (seg[0]: its checkpoint)
    void *scratch = nullptr;     // adjoint work buffers (adjoint_carve)
    size_t scratch_bytes = 0;
    double *dG = nullptr;        // [2][ncell] dL/dfield accumulator
    double *dW = nullptr;        // [nwall][2] dL/du_w per wall interface
    long long *zero = nullptr;   // device counter fixed at 0 (recompute clock)
    double *dW_face = nullptr;   // [6][3] dL/du_w per face (device), reduced in fixed order
    double *h_wall = nullptr;    // [6][3] pinned copy of dW_face
    // Captured reverse-sweep segments, kept across calls: one per (segment length, lambda
    // parity), valid while every pointer and value that the capture baked in is unchanged
    // (sig holds them: the step and adjoint parameter records, the segment buffers, the
    // kernel and tile selection).
    struct SegGraph {
        int64_t len;
        int cur;
        std::vector<unsigned char> sig;
        cudaGraphExec_t exec;
        int64_t launches;
    };
    std::vector<SegGraph> graphs;
};

}  // namespace dugks

struct dugks_s {
    int dim, q, store;
    int64_t nx, ny, nz, px, ncell;
    double dx, nu, dt, rt, rho0, c, tau;
    dugks_force force;
    dugks_boundaries bcs;
    cudaStream_t stream;
    int use_graph, tile_x, tile_y;
    int kernel;            // 0: throughput kernel where built, 1: reference kernel
    int model;             // DUGKS_MODEL_*
    double *d_metric;      // non-uniform mesh metrics (device; NULL: uniform), see StepParams
    double eg[3][2];       // its ghost extrapolation coefficients
    int64_t metric_off[3]; // offset of each axis' block in d_metric
    int ry3d;              // CTA rows of the 3D throughput kernel
    int own_stream;
    size_t esize;          // bytes per stored element
    size_t state_bytes;    // padded device bytes of one buffer
    void *buf[2];
    int cur;               // index of the buffer that holds the current state
    long long *d_step;     // device step counter
    int64_t step;          // host mirror of the step counter
    double *d_uprev;       // [dim][ncell] velocity at the previous residual
    int have_prev;
    double *d_partials;
    int res_blocks;
    double *d_res;         // 8 doubles
    float *d_mom;          // moments staging for host outputs (allocated on first use)
    double *h_res;         // pinned 8 doubles
    int64_t launches;
    std::map<std::pair<int64_t, int>, cudaGraphExec_t> graphs;
    std::string err;
    dugks::AdjointTape tape;  // recorded rollout for dugks_adjoint (adjoint2d.cu)
};

namespace dugks {
// Records a message on h (or for dugks_last_error(NULL) when h is NULL); returns code.
int handle_fail(dugks_t h, int code, const char *fmt, ...);
// Step parameters of the handle (source: current buffer, destination: the other one).
StepParams handle_params(const dugks_t h);
// Launches one step with the handle's kernel choice on the handle's stream.
cudaError_t handle_launch_step(dugks_t h, StepParams &p);
// Frees the adjoint tape (adjoint2d.cu).
void adjoint_release(dugks_t h);
}  // namespace dugks
