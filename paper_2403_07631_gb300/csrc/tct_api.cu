// tct_api.cu -- the C ABI of libtct: argument checks, workspace layout,
// per-call constants and the launch sequence.  See include/tct.h.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <atomic>

#include "tct_internal.cuh"

namespace tct {

namespace {
size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t cnt, start, partial, zs, scratch, bucket_l, bcur, long_count, long_cells, zkeys, upre, ubits,
        stats, queue, falls, total;
};

Layout layout(const tct_grid &g, int64_t n_points) {
    const size_t m = (size_t)g.W * (size_t)g.H;
    const size_t nb = (m + kScanTile - 1) / kScanTile;
    Layout L;
    size_t o = 0;
    L.cnt = o; o = align_up(o + 4 * m);
    L.bcur = o; o = align_up(o + 4 * (size_t)(n_points > 0 ? n_buckets_max((int64_t)m) : 0));
    L.long_count = o; o = align_up(o + 8);
    L.start = o; o = align_up(o + 4 * (m + 1));
    L.partial = o; o = align_up(o + 4 * (nb + 1));
    L.zs = o; o = align_up(o + 4 * (size_t)(n_points > 0 ? n_points : 0));
    L.scratch = o; o = align_up(o + 4 * (size_t)(n_points > 0 ? n_points : 0));
    L.bucket_l = o; o = align_up(o + 2 * (size_t)(n_points > 0 ? n_points : 0));
    L.long_cells = o; o = align_up(o + 4 * (n_points > 0 ? m : 0));
    L.zkeys = o; o = align_up(o + 4 * 2);
    L.upre = o; o = align_up(o + 4 * (TCT_MAX_SLICES + 1));
    L.ubits = o; o = align_up(o + 16 * (TCT_MAX_SLICES + 1));
    L.stats = o; o = align_up(o + sizeof(tct_stats));
    L.queue = o; o = align_up(o + 8);
    L.falls = o; o = align_up(o + 4);
    L.total = o;
    return L;
}

bool grid_ok(const tct_grid *g) {
    if (!g) return false;
    if (!(g->res > 0.0f) || !isfinite(g->res)) return false;
    if (!(g->d_s > 0.0f) || !isfinite(g->d_s)) return false;
    if (!isfinite(g->x0) || !isfinite(g->y0) || !isfinite(g->z_min)) return false;
    if (g->W < 1 || g->H < 1) return false;
    if ((int64_t)g->W * g->H > ((int64_t)1 << 30)) return false;
    if (g->n_slices < 1) return false;
    return true;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? TCT_OK : TCT_ERR_CUDA; }

double round6(double x) { return nearbyint(x * 1e6) / 1e6; }

// Eq. 6 in cell units; a zero safe margin leaves the step function K = [d <= D_inf].
double inflation_weight(double d, double d_inf_cells, double d_sm_cells) {
    if (d_sm_cells <= 0.0) return d <= d_inf_cells ? 1.0 : 0.0;
    double v = 1.0 - (d - d_inf_cells) / d_sm_cells;
    return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
}
std::atomic<int64_t> g_launches{0};

// Per-phase events of the profiling hook (tct_timing_enable / _read).
struct Timing {
    bool on = false;
    bool created = false;
    bool valid = false;
    bool marks_ok = false;       // every event of the current call was recorded
    int device = -1;             // the device the events belong to
    cudaEvent_t ev[4];
};
thread_local Timing g_timing;

// Records phase event i of a timed call.  A call on another device than the
// events' is not timed; a record that fails leaves the call untimed and its
// error is cleared here (the launch errors before it were already taken).
void mark(int i, cudaStream_t s) {
    if (!g_timing.on || !g_timing.created) return;
    if (i == 0) g_timing.marks_ok = true;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != g_timing.device ||
        cudaEventRecord(g_timing.ev[i], s) != cudaSuccess) {
        g_timing.marks_ok = false;
        cudaGetLastError();
    }
}
}  // namespace

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

Workspace carve(void *base, const tct_grid &g, int64_t n_points) {
    const Layout L = layout(g, n_points);
    char *b = static_cast<char *>(base);
    Workspace w;
    w.cnt = reinterpret_cast<int32_t *>(b + L.cnt);
    w.start = reinterpret_cast<int32_t *>(b + L.start);
    w.partial = reinterpret_cast<int32_t *>(b + L.partial);
    w.zs = reinterpret_cast<float *>(b + L.zs);
    w.scratch = reinterpret_cast<float *>(b + L.scratch);
    w.bucket_l = reinterpret_cast<uint16_t *>(b + L.bucket_l);
    w.bcur = reinterpret_cast<int32_t *>(b + L.bcur);
    w.long_count = reinterpret_cast<int32_t *>(b + L.long_count);
    w.long_cells = reinterpret_cast<int32_t *>(b + L.long_cells);
    w.zkeys = reinterpret_cast<int32_t *>(b + L.zkeys);
    w.upre = reinterpret_cast<int32_t *>(b + L.upre);
    w.ubits = reinterpret_cast<uint32_t *>(b + L.ubits);
    w.stats = reinterpret_cast<tct_stats *>(b + L.stats);
    w.queue = reinterpret_cast<int32_t *>(b + L.queue);
    w.falls = reinterpret_cast<int32_t *>(b + L.falls);
    w.bytes = L.total;
    return w;
}

int make_eval_consts(const tct_grid &g, const tct_params &p, EvalConsts *c) {
    const float vals[] = {p.d_min, p.d_ref, p.theta_b, p.theta_s, p.theta_p, p.c_b,
                          p.alpha_d, p.alpha_b, p.alpha_s, p.d_inf, p.d_sm};
    for (float v : vals)
        if (!isfinite(v)) return TCT_ERR_INVALID_ARG;
    if (!(p.theta_s > 0.0f) || !(p.theta_b > 0.0f) || !(p.c_b > 0.0f) || p.d_inf < 0.0f)
        return TCT_ERR_INVALID_ARG;
    // the scaling factors are non-negative (Table I); -0 is folded to +0
    if (p.alpha_d < 0.0f || p.alpha_b < 0.0f || p.alpha_s < 0.0f) return TCT_ERR_INVALID_ARG;
    if (p.patch_radius < 0) return TCT_ERR_INVALID_ARG;
    if (p.patch_radius > TCT_MAX_PATCH_RADIUS) return TCT_ERR_UNSUPPORTED;
    if (g.d_s > p.d_min && !(p.flags & TCT_ALLOW_COARSE)) return TCT_ERR_COVERAGE;
    memset(c, 0, sizeof(*c));
    c->d_min = p.d_min;
    c->d_ref = p.d_ref;
    c->theta_b = p.theta_b;
    c->theta_s = p.theta_s;
    c->c_b = p.c_b;
    c->alpha_d = p.alpha_d + 0.0f;
    c->alpha_b = p.alpha_b + 0.0f;
    c->alpha_s = p.alpha_s + 0.0f;
    c->inv2r = (float)(1.0 / (2.0 * (double)g.res));
    c->inv_ts = (float)(1.0 / (double)p.theta_s);
    c->inv_tb = (float)(1.0 / (double)p.theta_b);
    c->patch_radius = p.patch_radius;
    c->flags = p.flags;
    // p_s > theta_p  <=>  count > theta_p * n  <=>  count > floor(theta_p * n);
    // the product of a float and a small integer is exact in double
    const int n_patch = (2 * p.patch_radius + 1) * (2 * p.patch_radius + 1) - 1;
    double thr = floor((double)p.theta_p * (double)n_patch);
    if (thr < -1.0) thr = -1.0;
    if (thr > (double)n_patch) thr = (double)n_patch;
    c->count_thresh = n_patch > 0 ? (int32_t)thr : 0x7fffffff;
    // Eq. 6 in cells: D_inf = d_inf / r_g, D_sm = (d_sm - r_g) / r_g, rounded to
    // 6 decimals so that distances that are whole cells stay whole
    const double dinf = round6((double)p.d_inf / (double)g.res);
    const double dsm = round6(((double)p.d_sm - (double)g.res) / (double)g.res);
    int rk = 0;
    while (rk <= TCT_MAX_KERNEL_RADIUS && inflation_weight(rk + 1, dinf, dsm) > 0.0) ++rk;
    if (rk > TCT_MAX_KERNEL_RADIUS) return TCT_ERR_UNSUPPORTED;
    c->rk = rk;
    const int side = 2 * rk + 1;
    for (int n = -rk; n <= rk; ++n)
        for (int m = -rk; m <= rk; ++m)
            c->K[(n + rk) * side + (m + rk)] =
                (float)inflation_weight(sqrt((double)(m * m + n * n)), dinf, dsm);
    return TCT_OK;
}

}  // namespace tct

using namespace tct;

extern "C" {

const char *tct_status_string(int status) {
    switch (status) {
        case TCT_OK: return "ok";
        case TCT_ERR_INVALID_ARG: return "invalid argument";
        case TCT_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
        case TCT_ERR_COVERAGE: return "slice interval d_s exceeds d_min (set TCT_ALLOW_COARSE to accept)";
        case TCT_ERR_UNSUPPORTED: return "beyond a documented limit";
        case TCT_ERR_CUDA: return "CUDA error";
        default: return "unknown status";
    }
}

int tct_version(void) { return 10000; }

int tct_get_status(const tct_stats *d_stats, int32_t *h_status, tct_stream stream) {
    if (!d_stats || !h_status) return TCT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(h_status, &d_stats->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return TCT_ERR_CUDA;
    return TCT_OK;
}

void tct_params_default(tct_params *p) {
    if (!p) return;
    p->d_min = 0.50f;
    p->d_ref = 0.65f;
    p->theta_b = 1.70f;
    p->theta_s = 0.36f;
    p->theta_p = 0.20f;
    p->c_b = 50.0f;
    p->alpha_d = 20.0f;
    p->alpha_b = 20.0f;
    p->alpha_s = 15.0f;
    p->d_inf = 0.2f;
    p->d_sm = 0.4f;
    p->patch_radius = 2;
    p->flags = 0;
}

int tct_plan_grid(const float *b, float res, float d_s, tct_grid *out) {
    if (!b || !out || !(res > 0.0f) || !(d_s > 0.0f)) return TCT_ERR_INVALID_ARG;
    for (int a = 0; a < 6; ++a)
        if (!isfinite(b[a])) return TCT_ERR_INVALID_ARG;
    if (b[3] < b[0] || b[4] < b[1] || b[5] < b[2]) return TCT_ERR_INVALID_ARG;
    tct_grid g;
    memset(&g, 0, sizeof(g));
    g.x0 = b[0];
    g.y0 = b[1];
    g.res = res;
    volatile float du = b[3] - g.x0, dv = b[4] - g.y0;   // float32 operations
    volatile float u = du / res, v = dv / res;
    if (u >= 1e9f || v >= 1e9f) return TCT_ERR_UNSUPPORTED;
    g.W = (int32_t)floorf(u) + 1;
    g.H = (int32_t)floorf(v) + 1;
    g.d_s = d_s;
    g.z_min = b[2];
    g.flags = 0;
    g.n_slices = 0;
    for (int n = 1; n <= TCT_MAX_SLICES; ++n) {
        if (fmaf((float)n, d_s, g.z_min) >= b[5]) { g.n_slices = n; break; }
    }
    if (g.n_slices == 0) return TCT_ERR_UNSUPPORTED;
    *out = g;
    return TCT_OK;
}

size_t tct_workspace_bytes(const tct_grid *grid, int64_t n_points, const tct_params *params) {
    (void)params;
    if (!grid_ok(grid) || n_points < 0 || n_points > TCT_MAX_POINTS) return 0;
    return layout(*grid, n_points).total;
}

int tct_bounds(const float *d_xyz, int64_t n, int32_t stride, float *d_out6, tct_stats *d_stats,
               tct_stream stream) {
    if (!d_out6 || (stride != 3 && stride != 4) || n < 0 || n > TCT_MAX_POINTS) return TCT_ERR_INVALID_ARG;
    if (n > 0 && !d_xyz) return TCT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (d_stats) {
        cudaError_t e = cudaMemsetAsync(d_stats, 0, sizeof(tct_stats), s);
        if (e != cudaSuccess) return TCT_ERR_CUDA;
    }
    // the reduction runs on ordered-int keys held in d_out6 itself
    return cuda_status(launch_bounds(d_xyz, n, stride, d_out6, d_stats, s));
}

int tct_build(const float *d_xyz, int64_t n, int32_t stride, const tct_grid *grid, void *d_ws,
              size_t ws_bytes, float *d_ground, float *d_ceil, tct_stats *d_stats,
              tct_stream stream) {
    if (!grid_ok(grid) || grid->n_slices > TCT_MAX_SLICES) return grid && grid->n_slices > TCT_MAX_SLICES ? TCT_ERR_UNSUPPORTED : TCT_ERR_INVALID_ARG;
    if ((stride != 3 && stride != 4) || n < 0 || n > TCT_MAX_POINTS) return TCT_ERR_INVALID_ARG;
    if ((n > 0 && !d_xyz) || !d_ws || !d_ground || !d_ceil) return TCT_ERR_INVALID_ARG;
    if (ws_bytes < tct_workspace_bytes(grid, n, nullptr)) return TCT_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    const Workspace ws = carve(d_ws, *grid, n);
    tct_stats *st = d_stats ? d_stats : ws.stats;    // zeroed by the partition's first launch
    mark(0, s);
    cudaError_t e = launch_partition(d_xyz, n, stride, *grid, ws, st, s);
    mark(1, s);
    if (e == cudaSuccess) e = launch_elevations(*grid, ws, d_ground, d_ceil, s);
    mark(2, s);
    mark(3, s);
    g_timing.valid = g_timing.on && g_timing.marks_ok && e == cudaSuccess;
    return cuda_status(e);
}

int tct_evaluate(const tct_grid *grid, const tct_params *params, const float *d_ground,
                 const float *d_ceil, void *d_ws, size_t ws_bytes, float *d_cost, uint8_t *d_mask,
                 uint8_t *d_keep, float *d_aux, tct_stats *d_stats, tct_stream stream) {
    if (!grid_ok(grid) || !params) return TCT_ERR_INVALID_ARG;
    if (grid->n_slices > TCT_MAX_SLICES) return TCT_ERR_UNSUPPORTED;
    if (!d_ground || !d_ceil || !d_ws || !d_cost || !d_mask || !d_keep) return TCT_ERR_INVALID_ARG;
    if (ws_bytes < tct_workspace_bytes(grid, 0, params)) return TCT_ERR_WORKSPACE_TOO_SMALL;
    EvalConsts c;
    int rc = make_eval_consts(*grid, *params, &c);
    if (rc != TCT_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const Workspace ws = carve(d_ws, *grid, 0);
    tct_stats *st = d_stats ? d_stats : ws.stats;
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(tct_stats), s);
    mark(0, s);
    mark(1, s);
    if (e == cudaSuccess)
        e = launch_stack(*grid, c, nullptr, nullptr, d_ground, d_ceil, nullptr, nullptr, d_cost,
                         d_mask, d_aux, ws.upre, ws.ubits, st, s, TCT_TILE_AUTO, ws.queue,
                         ws.falls);
    mark(2, s);
    if (e == cudaSuccess) e = launch_chain(grid->n_slices, ws.upre, ws.ubits, params->flags, d_keep, st, s);
    mark(3, s);
    g_timing.valid = g_timing.on && g_timing.marks_ok && e == cudaSuccess;
    return cuda_status(e);
}

int tct_build_evaluate(const float *d_xyz, int64_t n, int32_t stride, const tct_grid *grid,
                       const tct_params *params, void *d_ws, size_t ws_bytes, float *d_ground,
                       float *d_ceil, float *d_cost, uint8_t *d_mask, uint8_t *d_keep,
                       tct_stats *d_stats, tct_stream stream) {
    if (!grid_ok(grid) || !params) return TCT_ERR_INVALID_ARG;
    if (grid->n_slices > TCT_MAX_SLICES) return TCT_ERR_UNSUPPORTED;
    if ((stride != 3 && stride != 4) || n < 0 || n > TCT_MAX_POINTS) return TCT_ERR_INVALID_ARG;
    if ((n > 0 && !d_xyz) || !d_ws || !d_ground || !d_ceil || !d_cost || !d_mask || !d_keep)
        return TCT_ERR_INVALID_ARG;
    if (ws_bytes < tct_workspace_bytes(grid, n, params)) return TCT_ERR_WORKSPACE_TOO_SMALL;
    EvalConsts c;
    int rc = make_eval_consts(*grid, *params, &c);
    if (rc != TCT_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const Workspace ws = carve(d_ws, *grid, n);
    tct_stats *st = d_stats ? d_stats : ws.stats;    // zeroed by the partition's first launch
    mark(0, s);
    cudaError_t e = launch_partition(d_xyz, n, stride, *grid, ws, st, s);
    mark(1, s);
    bool chained = false;       // the slice stack's last CTA ran the chain
    if (e == cudaSuccess)
        e = launch_stack(*grid, c, &ws, ws.zkeys, nullptr, nullptr, d_ground, d_ceil, d_cost,
                         d_mask, nullptr, ws.upre, ws.ubits, st, s, TCT_TILE_AUTO, nullptr,
                         nullptr, d_keep, &chained);
    mark(2, s);
    if (e == cudaSuccess && !chained)
        e = launch_chain(grid->n_slices, ws.upre, ws.ubits, params->flags, d_keep, st, s);
    mark(3, s);
    g_timing.valid = g_timing.on && g_timing.marks_ok && e == cudaSuccess;
    return cuda_status(e);
}

int tct_build_evaluate_host(tct_host_io *io, int64_t n, int32_t stride, const tct_grid *grid,
                            const tct_params *params, void *d_ws, size_t ws_bytes, float *d_xyz,
                            float *d_ground, float *d_ceil, float *d_cost, uint8_t *d_mask,
                            uint8_t *d_keep, tct_stats *d_stats, tct_stream stream) {
    if (!io || !grid_ok(grid) || !d_xyz || (n > 0 && !io->h_xyz)) return TCT_ERR_INVALID_ARG;
    if ((stride != 3 && stride != 4) || n < 0 || n > TCT_MAX_POINTS) return TCT_ERR_INVALID_ARG;
    const bool kept_only = (io->flags & TCT_HOST_KEPT_ONLY) != 0;
    if (kept_only && !io->h_keep) return TCT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (n > 0 && cudaMemcpyAsync(d_xyz, io->h_xyz, sizeof(float) * (size_t)n * stride,
                                 cudaMemcpyHostToDevice, s) != cudaSuccess)
        return TCT_ERR_CUDA;
    int rc = tct_build_evaluate(d_xyz, n, stride, grid, params, d_ws, ws_bytes, d_ground, d_ceil,
                                d_cost, d_mask, d_keep, d_stats, stream);
    if (rc != TCT_OK) return rc;
    const int N = grid->n_slices;
    const size_t hw = (size_t)grid->W * grid->H;
    // the layers with a host destination: (device, host, bytes per cell)
    struct Layer { const void *d; void *h; size_t es; } layers[4] = {
        {d_ground, io->h_ground, 4}, {d_ceil, io->h_ceil, 4}, {d_cost, io->h_cost, 4},
        {d_mask, io->h_mask, 1}};
    cudaError_t e = cudaSuccess;
    if (io->h_keep)
        e = cudaMemcpyAsync(io->h_keep, d_keep, (size_t)N, cudaMemcpyDeviceToHost, s);
    if (!kept_only) {
        for (const Layer &L : layers)
            if (L.h && e == cudaSuccess)
                e = cudaMemcpyAsync(L.h, L.d, L.es * hw * N, cudaMemcpyDeviceToHost, s);
        io->n_kept = N;
        return e == cudaSuccess ? TCT_OK : TCT_ERR_CUDA;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int m = 0;
    for (int k = 0; k < N && e == cudaSuccess; ++k) {
        if (!io->h_keep[k]) continue;
        for (const Layer &L : layers)
            if (L.h && e == cudaSuccess)
                e = cudaMemcpyAsync(static_cast<uint8_t *>(L.h) + L.es * hw * m,
                                    static_cast<const uint8_t *>(L.d) + L.es * hw * k, L.es * hw,
                                    cudaMemcpyDeviceToHost, s);
        ++m;
    }
    io->n_kept = m;
    return e == cudaSuccess ? TCT_OK : TCT_ERR_CUDA;
}

int tct_timing_enable(int on) {
    if (on && !g_timing.created) {
        if (cudaGetDevice(&g_timing.device) != cudaSuccess) return TCT_ERR_CUDA;
        for (int i = 0; i < 4; ++i)
            if (cudaEventCreate(&g_timing.ev[i]) != cudaSuccess) return TCT_ERR_CUDA;
        g_timing.created = true;
    }
    g_timing.on = on != 0;
    g_timing.valid = false;
    return TCT_OK;
}

int tct_timing_read(float *ms, int cap) {
    if (!ms || cap < 0) return TCT_ERR_INVALID_ARG;
    if (!g_timing.valid) return TCT_ERR_INVALID_ARG;
    if (cudaEventSynchronize(g_timing.ev[3]) != cudaSuccess) return TCT_ERR_CUDA;
    int w = 0;
    for (int i = 0; i < 3 && w < cap; ++i, ++w)
        if (cudaEventElapsedTime(&ms[i], g_timing.ev[i], g_timing.ev[i + 1]) != cudaSuccess)
            return TCT_ERR_CUDA;
    return w;
}

int64_t tct_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
