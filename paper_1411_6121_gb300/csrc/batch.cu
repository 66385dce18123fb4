// batch.cu -- many independent 2D (D2Q9) DUGKS instances advanced together.
//
// Every instance keeps its own mesh, viscosity, acceleration and boundaries; they share the
// time step, RT, rho0 and the storage type. One time step of the whole batch is one
// persistent launch (fused_step_batch) that walks a work list of (instance, tile) items,
// largest instances first; dugks_batch_step replays n such launches as a captured CUDA
// graph. The tile body is that of the D2Q9 throughput kernel (dugks_step2d.cuh) or of the
// reference kernel (dugks_step.cuh); the tile comes from a timing autotuner
// (dugks_batch_tune) whose choice is cached per (instance sizes, storage, SM count).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/dugks.h"
#include "dugks_internal.h"
#include "dugks_step.cuh"

using namespace dugks;

struct dugks_batch_s {
    int count = 0, store = 0, tx = 32, ty = 8;
    double dt = 0, rt = 0, rho0 = 0, c = 0;
    std::vector<dugks_mesh> mesh;
    std::vector<double> nu;
    std::vector<dugks_force> force;
    std::vector<dugks_boundaries> bcs;
    std::vector<int64_t> off;  // element offset of each instance in a state buffer
    std::vector<int64_t> px;
    int64_t elems = 0;         // elements of one state buffer (all instances)
    size_t esize = 4;
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;
    StepParams *d_params = nullptr;  // [2 * count]
    int4 *d_items = nullptr;
    int nitems = 0, items_cap = 0;
    long long *d_step = nullptr;
    int64_t step = 0;
    bool timedep = false;
    bool anyforce = false;  // some instance has an acceleration (uniform or field)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int grid = 0;
    int64_t launches = 0;
    std::map<std::pair<int64_t, int>, cudaGraphExec_t> graphs;
    std::string err;
};

namespace {

int bfail(dugks_batch_t b, int code, const char *fmt, ...) {
    char m[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(m, sizeof m, fmt, ap);
    va_end(ap);
    if (b) b->err = m;
    else set_null_handle_error(m);
    return code;
}

#define BTRY(b, call)                                                                                        \
    do {                                                                                                     \
        cudaError_t e_ = (call);                                                                             \
        if (e_ != cudaSuccess) return bfail((b), DUGKS_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

template <int TX, int TY, class S>
cudaError_t launch_batch_t(const dugks_batch_t b, int parity) {
    using K = StepShape<9, TX, TY, typename Arith<S>::T>;
    static int configured_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(fused_step_batch<9, S, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)K::smem_bytes);
        if (e != cudaSuccess) return e;
        configured_dev = dev;
    }
    fused_step_batch<9, S, TX, TY><<<b->grid, TX * TY, K::smem_bytes, b->stream>>>(b->d_params, b->d_items,
                                                                                   b->nitems, parity);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_batch_s(const dugks_batch_t b, int parity) {
    if (b->tx == 32 && b->ty == 8) return launch_batch_t<32, 8, S>(b, parity);
    if (b->tx == 16 && b->ty == 8) return launch_batch_t<16, 8, S>(b, parity);
    if (b->tx == 32 && b->ty == 4) return launch_batch_t<32, 4, S>(b, parity);
    if (b->tx == 64 && b->ty == 4) return launch_batch_t<64, 4, S>(b, parity);
    return cudaErrorNotSupported;
}

cudaError_t launch_batch(const dugks_batch_t b, int parity) {
    // throughput tiles: 30 x (ry - 2) inner cells (dugks_step2d.cuh)
    if (b->tx == 30) {
        const int ry = b->ty + 2;
        return launch_step2d_batch(b->d_params, b->d_items, b->nitems, parity, b->store, ry, b->anyforce, b->stream);
    }
    switch (b->store) {
        case DUGKS_STORE_F32: return launch_batch_s<float>(b, parity);
        case DUGKS_STORE_BF16: return launch_batch_s<__nv_bfloat16>(b, parity);
        case DUGKS_STORE_F16: return launch_batch_s<__half>(b, parity);
    }
    return cudaErrorNotSupported;
}

bool tile_supported(int tx, int ty) {
    return (tx == 32 && ty == 8) || (tx == 16 && ty == 8) || (tx == 32 && ty == 4) || (tx == 64 && ty == 4) ||
           (tx == 30 && (ty == 2 || ty == 6 || ty == 14));
}

StepParams instance_params(const dugks_batch_t b, int i, int parity) {
    StepParams p;
    memset(&p, 0, sizeof p);
    const dugks_mesh &m = b->mesh[i];
    p.nx = (int)m.nx;
    p.ny = (int)m.ny;
    p.nz = 1;
    p.px = b->px[i];
    p.plane = p.px * m.ny;
    p.dstride = p.plane;
    const double tau = b->nu[i] / b->rt, dt = b->dt, hh = 0.5 * dt;
    p.rho0 = b->rho0;
    p.inv_c = 1.0 / b->c;
    p.a1 = (2 * tau - hh) / (2 * tau + dt);
    p.b1 = 3 * hh / (2 * tau + dt);
    p.c1 = 3 * tau * hh / (2 * tau + dt);
    p.a7 = 2 * tau / (2 * tau + hh);
    p.b7 = hh / (2 * tau + hh);
    p.c7 = tau * hh / (2 * tau + hh);
    p.kappa = hh * b->c / m.dx;
    p.two_kappa = dt * b->c / m.dx;
    p.c_over_rho0 = b->c / b->rho0;
    p.wcell = 0.5 * dt;
    p.wface = 0.5 * hh;
    for (int a = 0; a < 3; a++) p.g[a] = b->force[i].g[a];
    p.field = b->force[i].field;
    p.omega = b->force[i].omega;
    p.dt = dt;
    p.step_ctr = b->d_step;
    p.step_off = 0;
    for (int w = 0; w < 6; w++) {
        p.bc[w] = b->bcs[i].face[w].type;
        for (int a = 0; a < 3; a++) p.bc_u[w][a] = b->bcs[i].face[w].u[a];
        p.bc_drho[w] = b->bcs[i].face[w].p / b->rt;
        p.bc_drho1[w] = b->bcs[i].face[w].p_amp / b->rt;
    }
    finish_step_params(p);
    const char *b0 = static_cast<const char *>(b->buf[parity]) + b->off[i] * b->esize;
    char *b1 = static_cast<char *>(b->buf[parity ^ 1]) + b->off[i] * b->esize;
    p.src = b0;
    p.dst = b1;
    return p;
}

// Work list for the tile shape (tx, ty): every tile of every instance, largest instances
// first so that the persistent CTAs end together.
int build_items(dugks_batch_t b) {
    std::vector<int> order(b->count);
    for (int i = 0; i < b->count; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return b->mesh[a].nx * b->mesh[a].ny > b->mesh[c].nx * b->mesh[c].ny;
    });
    std::vector<int4> items;
    for (int i : order) {
        const dugks_mesh &m = b->mesh[i];
        for (int64_t y = 0; y < m.ny; y += b->ty)
            for (int64_t x = 0; x < m.nx; x += b->tx) items.push_back(make_int4(i, (int)x, (int)y, 0));
    }
    if ((int)items.size() > b->items_cap) {
        cudaFree(b->d_items);
        b->d_items = nullptr;
        BTRY(b, cudaMalloc((void **)&b->d_items, sizeof(int4) * items.size()));
        b->items_cap = (int)items.size();
    }
    BTRY(b, cudaMemcpyAsync(b->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, b->stream));
    BTRY(b, cudaStreamSynchronize(b->stream));
    b->nitems = (int)items.size();
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // persistent grid: resident CTAs (up to 8 per SM), never more than the items
    const int per_sm = std::max(1, std::min(8, 2048 / (b->tx * b->ty)));
    b->grid = std::max(1, std::min(b->nitems, sms * per_sm));
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    return DUGKS_OK;
}

int enqueue_steps(dugks_batch_t b, int64_t n, int cur) {
    for (int64_t s = 0; s < n; s++) {
        cudaError_t e = launch_batch(b, cur);
        if (e != cudaSuccess) return bfail(b, DUGKS_E_CUDA, "batch launch: %s", cudaGetErrorString(e));
        if (b->timedep) {
            e = launch_advance(b->d_step, 1, b->stream);
            if (e != cudaSuccess) return bfail(b, DUGKS_E_CUDA, "advance: %s", cudaGetErrorString(e));
        }
        cur ^= 1;
    }
    return DUGKS_OK;
}

std::mutex g_tune_mutex;
std::map<std::tuple<int64_t, int64_t, int, int>, std::pair<int, int>> g_tune_cache;

}  // namespace

extern "C" {

int dugks_batch_create(int32_t count, const dugks_mesh *meshes, const double *nu, double dt,
                       const dugks_force *forces, const dugks_boundaries *bcs, const dugks_opts *opts,
                       dugks_batch_t *out) {
    if (!out) return bfail(nullptr, DUGKS_E_INVAL, "out is NULL");
    *out = nullptr;
    if (count < 1 || !meshes || !nu || !forces || !bcs) return bfail(nullptr, DUGKS_E_INVAL, "bad batch arguments");
    dugks_opts o;
    dugks_opts_default(&o);
    if (opts) o = *opts;
    if (o.store < 0 || o.store > 2) return bfail(nullptr, DUGKS_E_UNSUPPORTED, "batch storage must be F32/BF16/F16");
    if (!(o.rt > 0) || !(o.rho0 > 0) || !(dt > 0)) return bfail(nullptr, DUGKS_E_INVAL, "RT, rho0, dt must be positive");
    const double c = sqrt(3.0 * o.rt);
    for (int i = 0; i < count; i++) {
        const dugks_mesh &m = meshes[i];
        if (m.faces[0] || m.faces[1] || m.faces[2])
            return bfail(nullptr, DUGKS_E_UNSUPPORTED, "instance %d: the batch takes uniform meshes", i);
        if (m.dim != 2 || m.nz != 1 || m.nx < 1 || m.ny < 1 || m.nx > (1 << 30) || m.ny > (1 << 30) || !(m.dx > 0) ||
            !(nu[i] > 0))
            return bfail(nullptr, DUGKS_E_INVAL, "instance %d: bad 2D mesh or viscosity", i);
        if (dt > m.dx / c * (1.0 + 1e-12))
            return bfail(nullptr, DUGKS_E_CFL, "instance %d: dt exceeds dx/sqrt(3RT)", i);
        const int64_t n[2] = {m.nx, m.ny};
        for (int d = 0; d < 2; d++) {
            const int lo = bcs[i].face[2 * d].type, hi = bcs[i].face[2 * d + 1].type;
            if (lo < 0 || lo > 3 || hi < 0 || hi > 3 || ((lo == 0) != (hi == 0)) || (lo != 0 && n[d] < 2))
                return bfail(nullptr, DUGKS_E_INVAL, "instance %d: bad boundaries on axis %d", i, d);
        }
    }
    if (o.model != DUGKS_MODEL_INCOMPRESSIBLE)
        return bfail(nullptr, DUGKS_E_UNSUPPORTED, "the batch runs the incompressible model only");
    int tx = o.tile_x ? o.tile_x : 30, ty = o.tile_y ? o.tile_y : 6;  // default: the throughput tile
    if (!tile_supported(tx, ty)) return bfail(nullptr, DUGKS_E_UNSUPPORTED, "batch tile %dx%d not built", tx, ty);
    dugks_batch_t b = new (std::nothrow) dugks_batch_s();
    if (!b) return bfail(nullptr, DUGKS_E_NOMEM, "host allocation failed");
    b->count = count;
    b->store = o.store;
    b->tx = tx;
    b->ty = ty;
    b->dt = dt;
    b->rt = o.rt;
    b->rho0 = o.rho0;
    b->c = c;
    b->esize = o.store == DUGKS_STORE_F32 ? 4 : 2;
    b->mesh.assign(meshes, meshes + count);
    b->nu.assign(nu, nu + count);
    b->force.assign(forces, forces + count);
    b->bcs.assign(bcs, bcs + count);
    for (int i = 0; i < count; i++) {
        b->px.push_back((meshes[i].nx + 63) / 64 * 64);  // rows start on 256-byte boundaries
        b->off.push_back(b->elems);
        b->elems += 9 * b->px.back() * meshes[i].ny;
        if (forces[i].omega != 0.0) b->timedep = true;
        if (forces[i].field || forces[i].g[0] != 0.0 || forces[i].g[1] != 0.0) b->anyforce = true;
    }
    // the device clock also seeds the stochastic rounding of 16-bit stores
    if (o.store == DUGKS_STORE_BF16 || o.store == DUGKS_STORE_F16) b->timedep = true;
    b->stream = (cudaStream_t)o.stream;
    cudaError_t e = cudaSuccess;
    if (!b->stream) {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = true;
    }
    const size_t bytes = (size_t)b->elems * b->esize;
    if (e == cudaSuccess) e = cudaMalloc(&b->buf[0], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->buf[1], bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_params, sizeof(StepParams) * 2 * count);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_step, sizeof(long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->buf[0], 0, bytes, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->buf[1], 0, bytes, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_step, 0, sizeof(long long), b->stream);
    if (e != cudaSuccess) {
        const int rc = bfail(nullptr, e == cudaErrorMemoryAllocation ? DUGKS_E_NOMEM : DUGKS_E_CUDA, "batch create: %s",
                             cudaGetErrorString(e));
        cudaGetLastError();
        dugks_batch_destroy(b);
        return rc;
    }
    std::vector<StepParams> ps(2 * count);
    for (int i = 0; i < count; i++)
        for (int par = 0; par < 2; par++) ps[2 * i + par] = instance_params(b, i, par);
    e = cudaMemcpyAsync(b->d_params, ps.data(), sizeof(StepParams) * ps.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    int rc = e == cudaSuccess ? build_items(b) : bfail(b, DUGKS_E_CUDA, "params: %s", cudaGetErrorString(e));
    if (rc != DUGKS_OK) {
        set_null_handle_error(b->err.c_str());
        dugks_batch_destroy(b);
        return rc;
    }
    *out = b;
    return DUGKS_OK;
}

void dugks_batch_destroy(dugks_batch_t b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    cudaFree(b->buf[0]);
    cudaFree(b->buf[1]);
    cudaFree(b->d_params);
    cudaFree(b->d_items);
    cudaFree(b->d_step);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char *dugks_batch_last_error(dugks_batch_t b) { return b ? b->err.c_str() : dugks_last_error(nullptr); }

int dugks_batch_init(dugks_batch_t b, int32_t i, const double *pres, const double *vel) {
    if (!b || i < 0 || i >= b->count) return DUGKS_E_INVAL;
    const dugks_mesh &m = b->mesh[i];
    const int64_t ncell = m.nx * m.ny;
    double *dp = nullptr, *du = nullptr;
    if (pres) {
        BTRY(b, cudaMalloc((void **)&dp, sizeof(double) * ncell));
        BTRY(b, cudaMemcpyAsync(dp, pres, sizeof(double) * ncell, cudaMemcpyHostToDevice, b->stream));
    }
    if (vel) {
        BTRY(b, cudaMalloc((void **)&du, sizeof(double) * 2 * ncell));
        BTRY(b, cudaMemcpyAsync(du, vel, sizeof(double) * 2 * ncell, cudaMemcpyHostToDevice, b->stream));
    }
    StepParams p = instance_params(b, i, b->cur);
    p.dst = const_cast<void *>(p.src);
    cudaError_t e = launch_init(9, b->store, p, dp, du, b->rt, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(dp);
    cudaFree(du);
    if (e != cudaSuccess) return bfail(b, DUGKS_E_CUDA, "batch init: %s", cudaGetErrorString(e));
    return DUGKS_OK;
}

int dugks_batch_step(dugks_batch_t b, int64_t n) {
    if (!b || n < 0) return DUGKS_E_INVAL;
    const int64_t chunk = 256;
    while (n > 0) {
        const int64_t m = std::min(n, chunk);
        if (m >= 4) {
            auto key = std::make_pair(m, b->cur);
            auto it = b->graphs.find(key);
            if (it == b->graphs.end()) {
                cudaGraph_t g;
                BTRY(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
                const int rc = enqueue_steps(b, m, b->cur);
                cudaError_t e = cudaStreamEndCapture(b->stream, &g);
                if (rc != DUGKS_OK) return rc;
                if (e != cudaSuccess) return bfail(b, DUGKS_E_CUDA, "capture: %s", cudaGetErrorString(e));
                cudaGraphExec_t ge;
                e = cudaGraphInstantiate(&ge, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return bfail(b, DUGKS_E_CUDA, "instantiate: %s", cudaGetErrorString(e));
                it = b->graphs.emplace(key, ge).first;
            }
            BTRY(b, cudaGraphLaunch(it->second, b->stream));
        } else {
            const int rc = enqueue_steps(b, m, b->cur);
            if (rc != DUGKS_OK) return rc;
        }
        b->launches += m * (b->timedep ? 2 : 1);
        if (m & 1) b->cur ^= 1;
        b->step += m;
        n -= m;
    }
    return DUGKS_OK;
}

int dugks_batch_moments(dugks_batch_t b, int32_t i, float *out, int32_t out_is_device) {
    if (!b || i < 0 || i >= b->count || !out) return DUGKS_E_INVAL;
    const dugks_mesh &m = b->mesh[i];
    const size_t bytes = sizeof(float) * 3 * m.nx * m.ny;
    float *d = out;
    if (!out_is_device) BTRY(b, cudaMalloc((void **)&d, bytes));
    StepParams p = instance_params(b, i, b->cur);
    cudaError_t e = launch_moments(9, b->store, p, b->step * b->dt, b->rt, d, b->stream);
    if (e == cudaSuccess && !out_is_device) e = cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (!out_is_device) cudaFree(d);
    if (e != cudaSuccess) return bfail(b, DUGKS_E_CUDA, "batch moments: %s", cudaGetErrorString(e));
    return DUGKS_OK;
}

int dugks_batch_sync(dugks_batch_t b) {
    if (!b) return DUGKS_E_INVAL;
    BTRY(b, cudaStreamSynchronize(b->stream));
    return DUGKS_OK;
}

int64_t dugks_batch_launch_count(dugks_batch_t b) { return b ? b->launches : 0; }

int dugks_batch_tune(dugks_batch_t b, int32_t *tile_x, int32_t *tile_y) {
    if (!b) return DUGKS_E_INVAL;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t cells = 0, maxn = 0;
    for (const auto &m : b->mesh) {
        cells += m.nx * m.ny;
        maxn = std::max<int64_t>(maxn, m.nx * m.ny);
    }
    const auto key = std::make_tuple(cells, maxn * 1000003 + b->count, b->store, sms);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            b->tx = it->second.first;
            b->ty = it->second.second;
            const int rc = build_items(b);
            if (rc != DUGKS_OK) return rc;
            if (tile_x) *tile_x = b->tx;
            if (tile_y) *tile_y = b->ty;
            return DUGKS_OK;
        }
    }
    // time every candidate on a copy of the state (the batch's own state is restored)
    const size_t bytes = (size_t)b->elems * b->esize;
    void *save = nullptr;
    long long clock = 0;
    BTRY(b, cudaMalloc(&save, bytes));
    BTRY(b, cudaMemcpyAsync(save, b->buf[b->cur], bytes, cudaMemcpyDeviceToDevice, b->stream));
    BTRY(b, cudaMemcpyAsync(&clock, b->d_step, sizeof clock, cudaMemcpyDeviceToHost, b->stream));
    BTRY(b, cudaStreamSynchronize(b->stream));
    constexpr int NC = 7, REPS = 3, STEPS = 16;
    const int cand[NC][2] = {{30, 6}, {30, 14}, {30, 2}, {32, 8}, {16, 8}, {32, 4}, {64, 4}};
    // every candidate timed REPS times, interleaved (clock or neighbour changes hit all of
    // them alike); each keeps its fastest trial
    float tbest[NC];
    for (int c = 0; c < NC; c++) tbest[c] = 1e30f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int rep = 0; rep < REPS; rep++) {
        for (int c = 0; c < NC; c++) {
            b->tx = cand[c][0];
            b->ty = cand[c][1];
            int rc = build_items(b);
            if (rc == DUGKS_OK) rc = enqueue_steps(b, 2, b->cur);  // warm-up (and first-use configuration)
            if (rc != DUGKS_OK) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                cudaFree(save);
                return rc;
            }
            cudaEventRecord(e0, b->stream);
            rc = enqueue_steps(b, STEPS, b->cur);
            cudaEventRecord(e1, b->stream);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rc == DUGKS_OK && ms < tbest[c]) tbest[c] = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int bx = cand[0][0], by = cand[0][1];
    float best = tbest[0];
    for (int c = 1; c < NC; c++)
        if (tbest[c] < best) {
            best = tbest[c];
            bx = cand[c][0];
            by = cand[c][1];
        }
    BTRY(b, cudaMemcpyAsync(b->buf[b->cur], save, bytes, cudaMemcpyDeviceToDevice, b->stream));
    BTRY(b, cudaMemcpyAsync(b->d_step, &clock, sizeof clock, cudaMemcpyHostToDevice, b->stream));
    BTRY(b, cudaStreamSynchronize(b->stream));
    cudaFree(save);
    b->tx = bx;
    b->ty = by;
    const int rc = build_items(b);
    if (rc != DUGKS_OK) return rc;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = std::make_pair(bx, by);
    }
    if (tile_x) *tile_x = bx;
    if (tile_y) *tile_y = by;
    return DUGKS_OK;
}

}  // extern "C"
