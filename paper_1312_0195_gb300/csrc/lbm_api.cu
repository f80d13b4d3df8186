// lbm_api.cu -- the C ABI of include/lbm.h for grids: validation, ownership,
// CUDA-graph replay of the fused step, residual checks and field read-back.
#include "lbm_internal.h"

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

namespace lbm {

static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static thread_local std::string t_err;

lbm_status fail(lbm_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return s;
}

#define LBM_CUDA(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            cudaGetLastError();                                                             \
            return lbm::fail(e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,      \
                             "%s failed: %s", #call, cudaGetErrorString(e_));               \
        }                                                                                   \
    } while (0)

// Device pointer test without touching the memory.
bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static bool finite(double v) { return std::isfinite(v); }

lbm_status validate_params(const lbm_params *p)
{
    if (!p) return fail(LBM_EINVAL, "params is NULL");
    if (p->nx < 1 || p->ny < 1) return fail(LBM_EINVAL, "nx, ny must be >= 1 (got %d, %d)", p->nx, p->ny);
    if ((int64_t)p->nx * p->ny > (int64_t)1 << 31)
        return fail(LBM_EINVAL, "nx * ny must be <= 2^31 cells");
    if (!finite(p->tau) || p->tau < 0.5) return fail(LBM_EINVAL, "tau must be finite and >= 0.5 (got %g)", p->tau);
    if (!finite(p->nu)) return fail(LBM_EINVAL, "nu must be finite");
    if (!finite(p->eps) || p->eps < 0.0) return fail(LBM_EINVAL, "eps must be finite and >= 0 (got %g)", p->eps);
    if (!finite(p->gx) || !finite(p->gy)) return fail(LBM_EINVAL, "gx, gy must be finite");
    if (p->bc != LBM_BC_PERIODIC && p->bc != LBM_BC_WALLS_Y) return fail(LBM_EINVAL, "unknown bc %d", p->bc);
    if (p->storage != LBM_F32 && p->storage != LBM_F16 && p->storage != LBM_F64)
        return fail(LBM_EINVAL, "unknown storage %d", p->storage);
    if (!finite(p->scale) || p->scale < 0.0) return fail(LBM_EINVAL, "scale must be finite and >= 0");
    if (p->force_model != 0 && p->force_model != 1) return fail(LBM_EINVAL, "unknown force_model %d", p->force_model);
    if (p->scale > 0.0) {
        int ex2;
        double m = std::frexp(p->scale, &ex2);
        if (m != 0.5) return fail(LBM_EINVAL, "scale must be a power of two (got %g)", p->scale);
    }
    return LBM_OK;
}

double effective_nu(const lbm_params *p) { return p->nu < 0.0 ? (p->tau - 0.5) / 3.0 : p->nu; }

size_t storage_bytes(int storage) { return storage == LBM_F64 ? 8 : (storage == LBM_F16 ? 2 : 4); }

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int sm_count(int dev)
{
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        n = 1;
    }
    return n < 1 ? 1 : n;
}

}  // namespace lbm

using namespace lbm;

struct lbm_grid {
    lbm_params p;
    double nu = 0, S = 1;
    int dev = 0;
    int coef_mode = COEF_SCALAR;
    bool has_g = false;
    cudaStream_t stream = nullptr;   // user's stream
    cudaStream_t cap = nullptr;      // private stream used only for graph capture
    int64_t plane = 0;
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;                     // buf[cur] = post-collision state of the last step
    void *coef = nullptr;
    void *gfield = nullptr;
    double *partials = nullptr;
    double *result = nullptr;        // device [4]
    unsigned *flags = nullptr;       // device [2]: error bits, max finite kappa bits
    double *h_result = nullptr;      // pinned [4]
    GridLaunch L{};
    int64_t t = 0;
    std::map<std::tuple<int, int, int>, std::pair<cudaGraphExec_t, int>> graphs;
};

namespace lbm {

// Fills the step / moment argument blocks for one launch of grid g reading src.
template <typename T, typename CT>
static StepArgs<T, CT> make_args(const lbm_grid *g, const void *src, void *dst)
{
    StepArgs<T, CT> a;
    a.nx = g->p.nx;
    a.ny = g->p.ny;
    a.plane = g->plane;
    a.omega = (CT)(1.0 / g->p.tau);
    a.two_tau = (CT)(2.0 * g->p.tau);
    a.one_m_two_tau = (CT)(1.0 - 2.0 * g->p.tau);
    a.half_eps = (CT)(0.5 * g->p.eps);
    a.gx = (CT)g->p.gx;
    a.gy = (CT)g->p.gy;
    a.rho0 = (CT)g->S;
    a.guo = g->p.force_model == 1 ? 1 : 0;
    a.guo_c = (CT)(6.0 * (1.0 - 1.0 / (2.0 * g->p.tau)));
    a.src = static_cast<const T *>(src);
    a.dst = static_cast<T *>(dst);
    a.coef = static_cast<const CT *>(g->coef);
    a.gfield = static_cast<const CT *>(g->gfield);
    return a;
}

static cudaError_t enqueue_step(const lbm_grid *g, int src_idx, cudaStream_t st)
{
    const void *src = g->buf[src_idx];
    void *dst = g->buf[1 - src_idx];
    const bool walls = g->p.bc == LBM_BC_WALLS_Y;
    switch (g->p.storage) {
    case LBM_F32: {
        auto a = make_args<float, float>(g, src, dst);
        return launch_step(LBM_F32, g->coef_mode, g->has_g, walls, &a, g->L, st);
    }
    case LBM_F16: {
        auto a = make_args<__half, float>(g, src, dst);
        return launch_step(LBM_F16, g->coef_mode, g->has_g, walls, &a, g->L, st);
    }
    default: {
        auto a = make_args<double, double>(g, src, dst);
        return launch_step(LBM_F64, g->coef_mode, g->has_g, walls, &a, g->L, st);
    }
    }
}

// Moment pass over buf[cur_idx] (and buf[prev_idx] when prev_idx >= 0).
static cudaError_t enqueue_moments(const lbm_grid *g, int cur_idx, int prev_idx, float *rho, float *u, float *v,
                                   cudaStream_t st)
{
    const bool walls = g->p.bc == LBM_BC_WALLS_Y;
    const void *prev = prev_idx >= 0 ? g->buf[prev_idx] : nullptr;
    switch (g->p.storage) {
    case LBM_F32: {
        MomArgs<float, float> m{make_args<float, float>(g, g->buf[cur_idx], nullptr),
                                static_cast<const float *>(prev), 1.0f, rho, u, v, g->partials};
        return launch_moments(LBM_F32, g->coef_mode, g->has_g, walls, &m, g->L, st);
    }
    case LBM_F16: {
        MomArgs<__half, float> m{make_args<__half, float>(g, g->buf[cur_idx], nullptr),
                                 static_cast<const __half *>(prev), (float)(1.0 / g->S), rho, u, v, g->partials};
        return launch_moments(LBM_F16, g->coef_mode, g->has_g, walls, &m, g->L, st);
    }
    default: {
        MomArgs<double, double> m{make_args<double, double>(g, g->buf[cur_idx], nullptr),
                                  static_cast<const double *>(prev), 1.0, rho, u, v, g->partials};
        return launch_moments(LBM_F64, g->coef_mode, g->has_g, walls, &m, g->L, st);
    }
    }
}

// Graph of n fused steps starting from buf[parity], optionally followed by the
// residual pass (moments of the last two states, reduction, copy to pinned host).
static lbm_status get_graph(lbm_grid *g, int n, int parity, int check, cudaGraphExec_t *out, int *nk)
{
    auto key = std::make_tuple(n, parity, check);
    auto it = g->graphs.find(key);
    if (it != g->graphs.end()) {
        *out = it->second.first;
        *nk = it->second.second;
        return LBM_OK;
    }
    cudaGraph_t graph = nullptr;
    LBM_CUDA(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    int idx = parity, kernels = 0;
    for (int i = 0; i < n && err == cudaSuccess; ++i) {
        err = enqueue_step(g, idx, g->cap);
        idx = 1 - idx;
        ++kernels;
    }
    if (check && err == cudaSuccess) {
        err = enqueue_moments(g, idx, 1 - idx, nullptr, nullptr, nullptr, g->cap);
        if (err == cudaSuccess) err = launch_reduce_partials(g->partials, g->L.mom_blocks, g->result, g->cap);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(g->h_result, g->result, 4 * sizeof(double), cudaMemcpyDeviceToHost, g->cap);
        kernels += 2;
    }
    cudaError_t e2 = cudaStreamEndCapture(g->cap, &graph);
    if (err != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(LBM_ECUDA, "graph capture failed: %s",
                    cudaGetErrorString(err != cudaSuccess ? err : e2));
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e3));
    }
    g->graphs[key] = {exec, kernels};
    *out = exec;
    *nk = kernels;
    return LBM_OK;
}

// ---------------------------------------------------------------- autotuner
// Picks the fused step's launch shape (threads per block, resident blocks per SM,
// cells per thread) by timing candidates on the grid itself right after
// creation, then resets the state to rest. The choice is cached per lattice
// shape and variant for the whole process. Results do not depend on the launch
// shape (every cell's arithmetic and every reduction order are fixed), so
// tuning never changes answers. LBM_AUTOTUNE=0 disables it.
struct TuneKey {
    int nx, ny, storage, coef, gf, walls;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(nx, ny, storage, coef, gf, walls) < std::tie(o.nx, o.ny, o.storage, o.coef, o.gf, o.walls);
    }
};
static std::map<TuneKey, GridLaunch> g_tuned;
static std::mutex g_tune_mu;

static lbm_status autotune(lbm_grid *g)
{
    const char *env = std::getenv("LBM_AUTOTUNE");
    if (env && env[0] == '0') return LBM_OK;
    if (std::getenv("LBM_STEP_VEC")) return LBM_OK;      // a variant was chosen explicitly
    const int64_t n = (int64_t)g->p.nx * g->p.ny;
    if (n < ((int64_t)1 << 20)) return LBM_OK;      // small lattices are launch-bound: keep the default
    const bool walls = g->p.bc == LBM_BC_WALLS_Y;
    const TuneKey key{g->p.nx, g->p.ny, g->p.storage, g->coef_mode, g->has_g, walls};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            g->L.step_blocks = it->second.step_blocks;
            g->L.step_threads = it->second.step_threads;
            g->L.step_vec = it->second.step_vec;
            return LBM_OK;
        }
    }
    const int sms = sm_count(g->dev);
    // cells-per-thread candidates: the default for this storage and row length, then the other
    // built packs (FP32: 8; FP16: 4 and 2, fewer registers and more resident warps)
    const int dvec = step_vec(g->p.storage, g->p.nx);
    int vecs[3] = {dvec, 0, 0};
    int nvec = 1;
    const int others[2] = {g->p.storage == LBM_F32 ? 8 : (g->p.storage == LBM_F16 ? 4 : 0),
                           g->p.storage == LBM_F16 ? 2 : 0};
    for (int o : others)
        if (o && o != dvec && step_vec_ok(g->p.storage, g->p.nx, o)) vecs[nvec++] = o;
    GridLaunch best = g->L;
    float best_ms = -1.0f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LBM_CUDA(cudaEventCreate(&e0));
    LBM_CUDA(cudaEventCreate(&e1));
    const int warm = 2, timed = 8;
    for (int vi = 0; vi < nvec; ++vi) {
        const int vec = vecs[vi];
        for (int threads : {128, 256, 512}) {
            const int occ = step_blocks_per_sm(g->p.storage, g->coef_mode, g->has_g, walls, g->p.nx, threads, vec);
            const int64_t chunks = n / vec;
            const int64_t want = (chunks + threads - 1) / threads;
            for (int bpsm : {occ, occ > 1 ? occ / 2 : 0}) {
                if (bpsm < 1) continue;
                const int64_t cap = (int64_t)sms * bpsm;
                GridLaunch L = g->L;
                L.step_threads = threads;
                L.step_vec = vec;
                L.step_blocks = (int)(want < cap ? want : cap);
                g->L = L;
                cudaError_t err = cudaSuccess;
                for (int i = 0; i < warm && err == cudaSuccess; ++i) { err = enqueue_step(g, g->cur, g->stream); g->cur ^= 1; }
                cudaEventRecord(e0, g->stream);
                for (int i = 0; i < timed && err == cudaSuccess; ++i) { err = enqueue_step(g, g->cur, g->stream); g->cur ^= 1; }
                cudaEventRecord(e1, g->stream);
                count_launches(warm + timed);
                if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                float ms = 0.0f;
                if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
                if (err != cudaSuccess) {
                    cudaGetLastError();
                    continue;
                }
                if (best_ms < 0.0f || ms < best_ms) {
                    best_ms = ms;
                    best = L;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g->L.step_blocks = best.step_blocks;
    g->L.step_threads = best.step_threads;
    g->L.step_vec = best.step_vec;
    // back to rest: zero deviations in both buffers
    const size_t bytes = 9 * g->plane * storage_bytes(g->p.storage);
    LBM_CUDA(cudaMemsetAsync(g->buf[0], 0, bytes, g->stream));
    LBM_CUDA(cudaMemsetAsync(g->buf[1], 0, bytes, g->stream));
    LBM_CUDA(cudaStreamSynchronize(g->stream));
    g->cur = 0;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = g->L;
    return LBM_OK;
}

static void free_grid(lbm_grid *g)
{
    if (!g) return;
    for (auto &kv : g->graphs) cudaGraphExecDestroy(kv.second.first);
    g->graphs.clear();
    cudaFree(g->buf[0]);
    cudaFree(g->buf[1]);
    cudaFree(g->coef);
    cudaFree(g->gfield);
    cudaFree(g->partials);
    cudaFree(g->result);
    cudaFree(g->flags);
    if (g->h_result) cudaFreeHost(g->h_result);
    if (g->cap) cudaStreamDestroy(g->cap);
    cudaGetLastError();
    delete g;
}

// Shared by lbm_grid_create (scalar kappa) and the coarse run (tensor K*).
// kstar_scale multiplies K* before the coefficient is formed.
lbm_status grid_create_impl(const lbm_params *p, const float *kappa_dev, const double *kstar_dev,
                            double kstar_scale, const float *g_field_dev, void *cuda_stream, lbm_grid **out)
{
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    lbm_status s = validate_params(p);
    if (s != LBM_OK) return s;
    if (kappa_dev && !is_device_ptr(kappa_dev)) return fail(LBM_EINVAL, "kappa_dev is not a device pointer");
    if (kstar_dev && !is_device_ptr(kstar_dev)) return fail(LBM_EINVAL, "keff_dev is not a device pointer");
    if (!kappa_dev && !kstar_dev) return fail(LBM_EINVAL, "kappa_dev is NULL");
    if (g_field_dev && !is_device_ptr(g_field_dev)) return fail(LBM_EINVAL, "g_field_dev is not a device pointer");

    lbm_grid *g = new lbm_grid();
    g->p = *p;
    g->nu = effective_nu(p);
    g->coef_mode = kstar_dev ? COEF_TENSOR : COEF_SCALAR;
    g->has_g = g_field_dev != nullptr;
    g->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaGetDevice(&g->dev) != cudaSuccess) {
        cudaGetLastError();
        delete g;
        return fail(LBM_ECUDA, "no CUDA device");
    }
    const int64_t n = (int64_t)p->nx * p->ny;
    g->plane = (n + 63) / 64 * 64;
    const size_t sb = storage_bytes(p->storage);
    const size_t cb = p->storage == LBM_F64 ? 8 : 4;
    const int ncoef = kstar_dev ? 4 : 1;

    auto bail = [&](lbm_status st) { free_grid(g); return st; };
#define LBM_GRID_CUDA(call)                                                                 \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            cudaGetLastError();                                                             \
            return bail(fail(e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,      \
                             "%s failed: %s", #call, cudaGetErrorString(e_)));              \
        }                                                                                   \
    } while (0)

    // launch shapes: persistent step grid, fixed moment grid (fixed reduction order)
    const int sms = sm_count(g->dev);
    const int vec = step_vec(p->storage, p->nx);
    const int64_t chunks = n / vec;
    g->L.step_threads = 256;
    g->L.step_vec = 0;
    const int64_t want = (chunks + g->L.step_threads - 1) / g->L.step_threads;
    const int64_t cap = (int64_t)sms * step_blocks_per_sm(p->storage, g->coef_mode, g->has_g,
                                                          p->bc == LBM_BC_WALLS_Y, p->nx, g->L.step_threads);
    g->L.step_blocks = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
    // LBM_STEP_VEC=v selects another built cells-per-thread variant of the step (the arithmetic per
    // cell is the same in every variant) and turns the autotuner off for this grid
    if (const char *ev = std::getenv("LBM_STEP_VEC")) {
        const int v = std::atoi(ev);
        if (step_vec_ok(p->storage, p->nx, v)) {
            g->L.step_vec = v;
            const int64_t w2 = (n / v + g->L.step_threads - 1) / g->L.step_threads;
            const int64_t c2 = (int64_t)sms * step_blocks_per_sm(p->storage, g->coef_mode, g->has_g,
                                                                 p->bc == LBM_BC_WALLS_Y, p->nx, g->L.step_threads, v);
            g->L.step_blocks = (int)(w2 < c2 ? (w2 < 1 ? 1 : w2) : c2);
        }
    }
    g->L.mom_threads = 256;
    const int64_t mwant = (chunks + 255) / 256;
    const int64_t mcap = (int64_t)sms * 2;   // 128 registers: two 256-thread blocks per SM
    g->L.mom_blocks = (int)(mwant < mcap ? (mwant < 1 ? 1 : mwant) : mcap);

    LBM_GRID_CUDA(cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking));
    LBM_GRID_CUDA(cudaMalloc(&g->buf[0], 9 * g->plane * sb));
    LBM_GRID_CUDA(cudaMalloc(&g->buf[1], 9 * g->plane * sb));
    LBM_GRID_CUDA(cudaMalloc(&g->coef, ncoef * g->plane * cb));
    if (g->has_g) LBM_GRID_CUDA(cudaMalloc(&g->gfield, 2 * g->plane * cb));
    LBM_GRID_CUDA(cudaMalloc(&g->partials, 4 * sizeof(double) * g->L.mom_blocks));
    LBM_GRID_CUDA(cudaMalloc(&g->result, 4 * sizeof(double)));
    LBM_GRID_CUDA(cudaMalloc(&g->flags, 2 * sizeof(unsigned)));
    LBM_GRID_CUDA(cudaMallocHost(&g->h_result, 8 * sizeof(double)));

    cudaStream_t st = g->stream;
    // rest state: deviations are zero in both buffers (state of step -1 and -2)
    LBM_GRID_CUDA(cudaMemsetAsync(g->buf[0], 0, 9 * g->plane * sb, st));
    LBM_GRID_CUDA(cudaMemsetAsync(g->buf[1], 0, 9 * g->plane * sb, st));
    LBM_GRID_CUDA(cudaMemsetAsync(g->coef, 0, ncoef * g->plane * cb, st));
    LBM_GRID_CUDA(cudaMemsetAsync(g->flags, 0, 2 * sizeof(unsigned), st));
    if (kstar_dev) {
        // The coarse run passes a K* already divided by r^2 when kstar_scale != 1.
        LBM_GRID_CUDA(launch_coef_tensor(p->storage, kstar_dev, g->coef, n, g->plane,
                                         0.5 * p->eps * g->nu / kstar_scale, g->flags, st));
        count_launches(1);
    } else {
        LBM_GRID_CUDA(launch_coef_scalar(p->storage, kappa_dev, g->coef, n, g->plane, p->eps * g->nu, g->flags,
                                         g->flags + 1, st));
        count_launches(1);
    }
    if (g->has_g) {
        LBM_GRID_CUDA(launch_copy_force(p->storage, g_field_dev, g->gfield, n, g->plane, 1.0, st));
        count_launches(1);
    }
    unsigned hflags[2] = {0, 0};
    LBM_GRID_CUDA(cudaMemcpyAsync(hflags, g->flags, sizeof hflags, cudaMemcpyDeviceToHost, st));
    LBM_GRID_CUDA(cudaStreamSynchronize(st));
    if (hflags[0] & 1u) return bail(fail(LBM_EINVAL, kstar_dev ? "K* has non-finite entries"
                                                                 : "kappa has negative or NaN entries"));
    if (hflags[0] & 2u) return bail(fail(LBM_EINVAL, "K* + (eps nu / 2) I is singular in some cell"));

    if (p->storage == LBM_F16) {
        if (p->scale > 0.0) {
            g->S = p->scale;
        } else {
            // Largest deviation ~ w_1 * 3 * |u|, |u| <~ kappa_max |G| / nu; aim that at 2^12
            // (headroom of 16x below the FP16 maximum for transients and pressure).
            float kmax;
            std::memcpy(&kmax, &hflags[1], sizeof kmax);
            double gmag = std::fabs(p->gx) + std::fabs(p->gy);
            double umax = (g->nu > 0.0 && kmax > 0.0f) ? (double)kmax * gmag / g->nu : gmag * 1e3;
            if (!(umax > 0.0)) umax = 1e-3;
            if (umax > 0.1) umax = 0.1;
            int e2 = (int)std::floor(std::log2(4096.0 / umax));
            if (e2 > 60) e2 = 60;
            if (e2 < 0) e2 = 0;
            g->S = std::ldexp(1.0, e2);
        }
    }
    s = autotune(g);
    if (s != LBM_OK) return bail(s);
    *out = g;
    return LBM_OK;
#undef LBM_GRID_CUDA
}

}  // namespace lbm

extern "C" {

const char *lbm_last_error(void) { return lbm::t_err.c_str(); }

int64_t lbm_launch_count(void) { return lbm::g_launches.load(); }

lbm_status lbm_grid_create(const lbm_params *p, const float *kappa_dev, const float *g_field_dev, void *cuda_stream,
                           lbm_grid **out)
{
    if (!kappa_dev) {
        if (out) *out = nullptr;
        lbm_status s = validate_params(p);
        return s != LBM_OK ? s : fail(LBM_EINVAL, "kappa_dev is NULL");
    }
    return grid_create_impl(p, kappa_dev, nullptr, 1.0, g_field_dev, cuda_stream, out);
}

lbm_status lbm_grid_destroy(lbm_grid *g)
{
    if (!g) return LBM_OK;
    DeviceGuard dg(g->dev);
    cudaStreamSynchronize(g->stream);
    cudaGetLastError();
    free_grid(g);
    return LBM_OK;
}

lbm_status lbm_step(lbm_grid *g, int64_t max_steps, double tol_rel, int32_t check_every, int64_t *steps_done,
                    double *residual)
{
    if (steps_done) *steps_done = 0;
    if (residual) *residual = -1.0;
    if (!g) return fail(LBM_EINVAL, "grid is NULL");
    if (max_steps < 0) return fail(LBM_EINVAL, "max_steps must be >= 0");
    if (check_every < 0) return fail(LBM_EINVAL, "check_every must be >= 0");
    if (!std::isfinite(tol_rel)) return fail(LBM_EINVAL, "tol_rel must be finite");
    if (tol_rel > 0.0 && check_every == 0) return fail(LBM_EINVAL, "tol_rel > 0 needs check_every > 0");
    DeviceGuard dg(g->dev);
    const int CHUNK = 1024;
    int64_t left = max_steps, done = 0;
    double resid = -1.0;
    bool converged = false, checked = false;
    while (left > 0) {
        int64_t n = left < CHUNK ? left : CHUNK;
        int check = 0;
        if (check_every > 0) {
            const int64_t to_next = check_every - (g->t % check_every);
            if (to_next <= n) {
                n = to_next;
                check = 1;
            }
        }
        cudaGraphExec_t ex = nullptr;
        int nk = 0;
        lbm_status s = get_graph(g, (int)n, g->cur, check, &ex, &nk);
        if (s != LBM_OK) return s;
        LBM_CUDA(cudaGraphLaunch(ex, g->stream));
        count_launches(nk);
        g->t += n;
        done += n;
        left -= n;
        if (n & 1) g->cur = 1 - g->cur;
        if (check) {
            checked = true;
            if (tol_rel > 0.0) {      // the stop test needs the value now; otherwise read it at the end
                LBM_CUDA(cudaStreamSynchronize(g->stream));
                const double dmax = g->h_result[0], umax = g->h_result[1];
                resid = umax > 0.0 ? dmax / umax : dmax;
                if (resid <= tol_rel) {
                    converged = true;
                    break;
                }
            }
        }
    }
    LBM_CUDA(cudaStreamSynchronize(g->stream));
    if (checked && tol_rel <= 0.0) {
        const double dmax = g->h_result[0], umax = g->h_result[1];
        resid = umax > 0.0 ? dmax / umax : dmax;
    }
    if (steps_done) *steps_done = done;
    if (residual) *residual = resid;
    if (tol_rel > 0.0 && !converged)
        return fail(LBM_ENOTCONV, "residual %.3e above tolerance %.3e after %lld steps", resid, tol_rel,
                    (long long)done);
    return LBM_OK;
}

lbm_status lbm_get_fields(lbm_grid *g, float *rho_dev, float *u_dev, float *v_dev)
{
    if (!g) return fail(LBM_EINVAL, "grid is NULL");
    if ((rho_dev && !is_device_ptr(rho_dev)) || (u_dev && !is_device_ptr(u_dev)) || (v_dev && !is_device_ptr(v_dev)))
        return fail(LBM_EINVAL, "field outputs must be device pointers");
    DeviceGuard dg(g->dev);
    LBM_CUDA(enqueue_moments(g, g->cur, -1, rho_dev, u_dev, v_dev, g->stream));
    count_launches(1);
    LBM_CUDA(cudaStreamSynchronize(g->stream));
    return LBM_OK;
}

lbm_status lbm_mean_velocity(lbm_grid *g, double out_mean_uv[2])
{
    if (!g || !out_mean_uv) return fail(LBM_EINVAL, "grid or output is NULL");
    DeviceGuard dg(g->dev);
    LBM_CUDA(enqueue_moments(g, g->cur, -1, nullptr, nullptr, nullptr, g->stream));
    LBM_CUDA(launch_reduce_partials(g->partials, g->L.mom_blocks, g->result, g->stream));
    count_launches(2);
    LBM_CUDA(cudaMemcpyAsync(g->h_result, g->result, 4 * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    LBM_CUDA(cudaStreamSynchronize(g->stream));
    const double n = (double)g->p.nx * g->p.ny;
    out_mean_uv[0] = g->h_result[2] / n;
    out_mean_uv[1] = g->h_result[3] / n;
    return LBM_OK;
}

int64_t lbm_grid_steps(const lbm_grid *g) { return g ? g->t : -1; }

int64_t lbm_grid_state_bytes(const lbm_grid *g)
{
    return g ? CKPT_HEADER_BYTES + (int64_t)(2 * 9 * g->plane * storage_bytes(g->p.storage)) : -1;
}

}  // extern "C"

namespace lbm {

// The header a checkpoint of grid g carries (and a loaded one must match).
static CkptHeader grid_header(const lbm_grid *g)
{
    CkptHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, "LBM2CKPT", 8);
    h.version = 1;
    h.storage = g->p.storage;
    h.nx = g->p.nx;
    h.ny = g->p.ny;
    h.nz = 1;
    h.scale = g->S;
    const double d[5] = {g->p.tau, g->nu, g->p.eps, g->p.gx, g->p.gy};
    const int32_t i[4] = {g->p.bc, g->p.force_model, g->coef_mode, g->has_g ? 1 : 0};
    h.params_hash = fnv1a(i, sizeof i, fnv1a(d, sizeof d));
    h.steps = g->t;
    return h;
}

}  // namespace lbm

extern "C" {

lbm_status lbm_grid_save_state(lbm_grid *g, void *state_dev, int64_t nbytes, int64_t *steps)
{
    if (!g || !state_dev) return fail(LBM_EINVAL, "grid or state is NULL");
    if (nbytes != lbm_grid_state_bytes(g))
        return fail(LBM_EINVAL, "state buffer holds %lld bytes, the grid's state is %lld", (long long)nbytes,
                    (long long)lbm_grid_state_bytes(g));
    if (!is_device_ptr(state_dev)) return fail(LBM_EINVAL, "state_dev is not a device pointer");
    DeviceGuard dg(g->dev);
    const size_t half = 9 * g->plane * storage_bytes(g->p.storage);
    const CkptHeader h = grid_header(g);
    char *dst = static_cast<char *>(state_dev);
    LBM_CUDA(cudaMemcpyAsync(dst, &h, sizeof h, cudaMemcpyHostToDevice, g->stream));
    LBM_CUDA(cudaMemcpyAsync(dst + CKPT_HEADER_BYTES, g->buf[g->cur], half, cudaMemcpyDeviceToDevice, g->stream));
    LBM_CUDA(cudaMemcpyAsync(dst + CKPT_HEADER_BYTES + half, g->buf[1 - g->cur], half, cudaMemcpyDeviceToDevice,
                             g->stream));
    LBM_CUDA(cudaStreamSynchronize(g->stream));
    if (steps) *steps = g->t;
    return LBM_OK;
}

lbm_status lbm_grid_load_state(lbm_grid *g, const void *state_dev, int64_t nbytes, int64_t steps)
{
    if (!g || !state_dev) return fail(LBM_EINVAL, "grid or state is NULL");
    if (steps < 0) return fail(LBM_EINVAL, "steps must be >= 0");
    if (nbytes != lbm_grid_state_bytes(g))
        return fail(LBM_EINVAL, "state buffer holds %lld bytes, the grid's state is %lld", (long long)nbytes,
                    (long long)lbm_grid_state_bytes(g));
    if (!is_device_ptr(state_dev)) return fail(LBM_EINVAL, "state_dev is not a device pointer");
    DeviceGuard dg(g->dev);
    CkptHeader saved;
    LBM_CUDA(cudaMemcpyAsync(&saved, state_dev, sizeof saved, cudaMemcpyDeviceToHost, g->stream));
    LBM_CUDA(cudaStreamSynchronize(g->stream));
    const CkptHeader mine = grid_header(g);
    if (std::memcmp(saved.magic, mine.magic, 8) || saved.version != mine.version || saved.storage != mine.storage ||
        saved.nx != mine.nx || saved.ny != mine.ny || saved.nz != mine.nz || saved.scale != mine.scale ||
        saved.params_hash != mine.params_hash)
        return fail(LBM_EINVAL, "the state was saved by a grid of another size, storage, scale or parameter set");
    const size_t half = 9 * g->plane * storage_bytes(g->p.storage);
    const char *src = static_cast<const char *>(state_dev);
    LBM_CUDA(cudaMemcpyAsync(g->buf[g->cur], src + CKPT_HEADER_BYTES, half, cudaMemcpyDeviceToDevice, g->stream));
    LBM_CUDA(cudaMemcpyAsync(g->buf[1 - g->cur], src + CKPT_HEADER_BYTES + half, half, cudaMemcpyDeviceToDevice,
                             g->stream));
    LBM_CUDA(cudaStreamSynchronize(g->stream));
    g->t = steps;
    return LBM_OK;
}

double lbm_grid_scale(const lbm_grid *g) { return g ? g->S : 0.0; }

}  // extern "C"
