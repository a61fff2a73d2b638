// tct_batch.cu -- many maps per call: tct_build_evaluate_batched and its
// autotuner.  The maps' cells and heights are concatenated in one workspace;
// one launch of each point pass serves every cloud, one persistent launch of
// the slice stack serves every tile of every map, and one launch runs every
// map's simplification chain.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "tct_internal.cuh"

namespace tct {
namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct BatchLayout {
    size_t cnt, start, partial, zs, scratch, bucket_l, bcur, long_count, long_cells, queue;
    size_t zkeys, upre, ubits, stats, total;
    int64_t cells, points;
};

BatchLayout batch_layout(const tct_map *maps, int n_maps) {
    BatchLayout L;
    int64_t cells = 0, points = 0;
    for (int i = 0; i < n_maps; ++i) {
        cells += (int64_t)maps[i].grid.W * maps[i].grid.H;
        points += maps[i].n;
    }
    L.cells = cells;
    L.points = points;
    const size_t nb = (size_t)((cells + kScanTile - 1) / kScanTile);
    size_t o = 0;
    L.cnt = o; o = align256(o + 4 * (size_t)cells);
    L.bcur = o; o = align256(o + 4 * (size_t)n_buckets_max(cells));
    L.long_count = o; o = align256(o + 8);
    L.start = o; o = align256(o + 4 * ((size_t)cells + 1));
    L.partial = o; o = align256(o + 4 * (nb + 1));
    L.zs = o; o = align256(o + 4 * (size_t)points);
    L.scratch = o; o = align256(o + 4 * (size_t)points);
    L.bucket_l = o; o = align256(o + 2 * (size_t)points);
    L.long_cells = o; o = align256(o + 4 * (size_t)cells);
    L.queue = o; o = align256(o + 4);
    L.zkeys = o; o = align256(o + 8 * (size_t)n_maps);
    L.upre = o; o = align256(o + 4 * (TCT_MAX_SLICES + 1) * (size_t)n_maps);
    L.ubits = o; o = align256(o + 16 * (TCT_MAX_SLICES + 1) * (size_t)n_maps);
    L.stats = o; o = align256(o + sizeof(tct_stats) * (size_t)n_maps);
    L.total = o;
    return L;
}

// Per-map pointers of the small per-batch kernels.
struct BatchSmall {
    int32_t n_maps;
    int32_t *queue;
    struct {
        int32_t *zkeys, *upre;
        uint32_t *ubits;
        tct_stats *stats;
        uint8_t *keep;
        int64_t n_points;
        int32_t n_slices;
        uint32_t flags;
    } m[TCT_MAX_BATCH];
};

// Zero each map's statistics and uniqueness matrix, seed its z bounds, reset the queue.
__global__ void k_batch_init(const __grid_constant__ BatchSmall b) {
    const auto &m = b.m[blockIdx.x];
    uint32_t *st = reinterpret_cast<uint32_t *>(m.stats);
    for (int i = threadIdx.x; i < (int)(sizeof(tct_stats) / 4); i += blockDim.x) st[i] = 0;
    for (int i = threadIdx.x; i <= TCT_MAX_SLICES; i += blockDim.x) {
        m.upre[i] = 0;
        m.ubits[4 * i] = m.ubits[4 * i + 1] = m.ubits[4 * i + 2] = m.ubits[4 * i + 3] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        m.zkeys[0] = float_key(INFINITY);
        m.zkeys[1] = float_key(-INFINITY);
        m.stats->n_points = m.n_points;
        m.stats->n_slices = m.n_slices;
        if (blockIdx.x == 0) *b.queue = 0;
    }
}

// Each block runs one map's chain (Sec. III-C) and copies its z bounds.
__global__ void k_batch_chain(const __grid_constant__ BatchSmall b) {
    const auto &m = b.m[blockIdx.x];
    __shared__ int32_t s_pre[TCT_MAX_SLICES + 1];
    __shared__ uint32_t s_bits[4 * (TCT_MAX_SLICES + 1)];
    const int N = m.n_slices;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        s_pre[k] = m.upre[k];
        for (int w = 0; w < 4; ++w) s_bits[4 * k + w] = m.ubits[4 * k + w];
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    m.stats->n_kept = chain_walk(N, s_pre, s_bits, m.flags, m.keep);
    m.stats->z_min = key_float(m.zkeys[0]);
    m.stats->z_max = key_float(m.zkeys[1]);
}

int check_batch(const tct_map *maps, int n_maps, const tct_params *params, EvalConsts *c) {
    if (!maps || !params || n_maps < 1) return TCT_ERR_INVALID_ARG;
    if (n_maps > TCT_MAX_BATCH) return TCT_ERR_UNSUPPORTED;
    int64_t cells = 0, points = 0;
    for (int i = 0; i < n_maps; ++i) {
        const tct_map &m = maps[i];
        if (tct_workspace_bytes(&m.grid, m.n, params) == 0) return TCT_ERR_INVALID_ARG;
        if (m.grid.n_slices > TCT_MAX_SLICES) return TCT_ERR_UNSUPPORTED;
        if ((m.stride != 3 && m.stride != 4) || (m.n > 0 && !m.d_xyz)) return TCT_ERR_INVALID_ARG;
        if (!m.d_ground || !m.d_ceil || !m.d_cost || !m.d_mask || !m.d_keep) return TCT_ERR_INVALID_ARG;
        cells += (int64_t)m.grid.W * m.grid.H;
        points += m.n;
    }
    if (cells >= ((int64_t)1 << 31) || points >= ((int64_t)1 << 31)) return TCT_ERR_UNSUPPORTED;
    for (int i = 0; i < n_maps; ++i) {
        const int rc = make_eval_consts(maps[i].grid, *params, c);
        if (rc != TCT_OK) return rc;
    }
    return TCT_OK;
}

int run_batch(const tct_map *maps, int n_maps, const tct_params *params, const tct_tuning &tn,
              const EvalConsts &c, void *d_ws, cudaStream_t s) {
    const BatchLayout L = batch_layout(maps, n_maps);
    char *base = static_cast<char *>(d_ws);
    Workspace ws;
    memset(&ws, 0, sizeof(ws));
    ws.cnt = reinterpret_cast<int32_t *>(base + L.cnt);
    ws.start = reinterpret_cast<int32_t *>(base + L.start);
    ws.partial = reinterpret_cast<int32_t *>(base + L.partial);
    ws.zs = reinterpret_cast<float *>(base + L.zs);
    ws.scratch = reinterpret_cast<float *>(base + L.scratch);
    ws.bucket_l = reinterpret_cast<uint16_t *>(base + L.bucket_l);
    ws.bcur = reinterpret_cast<int32_t *>(base + L.bcur);
    ws.long_count = reinterpret_cast<int32_t *>(base + L.long_count);
    ws.long_cells = reinterpret_cast<int32_t *>(base + L.long_cells);
    int32_t *queue = reinterpret_cast<int32_t *>(base + L.queue);
    int32_t *zkeys = reinterpret_cast<int32_t *>(base + L.zkeys);
    int32_t *upre = reinterpret_cast<int32_t *>(base + L.upre);
    uint32_t *ubits = reinterpret_cast<uint32_t *>(base + L.ubits);
    tct_stats *stats = reinterpret_cast<tct_stats *>(base + L.stats);

    BatchSmall small;
    memset(&small, 0, sizeof(small));
    small.n_maps = n_maps;
    small.queue = queue;
    std::vector<BatchPointsIn> pin(n_maps);
    std::vector<StackArgs> sargs(n_maps);
    int64_t cell_off = 0;
    for (int i = 0; i < n_maps; ++i) {
        const tct_map &m = maps[i];
        auto &sm = small.m[i];
        sm.zkeys = zkeys + 2 * i;
        sm.upre = upre + (TCT_MAX_SLICES + 1) * i;
        sm.ubits = ubits + 4 * (TCT_MAX_SLICES + 1) * i;
        sm.stats = m.d_stats ? m.d_stats : stats + i;
        sm.keep = m.d_keep;
        sm.n_points = m.n;
        sm.n_slices = m.grid.n_slices;
        sm.flags = params->flags;
        pin[i] = BatchPointsIn{m.d_xyz, m.n, m.stride, m.grid, cell_off, sm.zkeys, sm.stats};
        StackArgs &a = sargs[i];
        memset(&a, 0, sizeof(a));
        a.W = m.grid.W;
        a.H = m.grid.H;
        a.N = m.grid.n_slices;
        a.d_s = m.grid.d_s;
        a.z_min = m.grid.z_min;
        a.zmin_from_data = (m.grid.flags & TCT_GRID_ZMIN_FROM_DATA) ? 1 : 0;
        a.zkeys = sm.zkeys;
        a.start = ws.start + cell_off;
        a.zs = ws.zs;
        a.ground = m.d_ground;
        a.ceil = m.d_ceil;
        a.cost = m.d_cost;
        a.mask = m.d_mask;
        a.upre = sm.upre;
        a.ubits = sm.ubits;
        a.stats = sm.stats;
        cell_off += (int64_t)m.grid.W * m.grid.H;
    }
    // the persistent kernel takes the largest maps first
    std::vector<int> order(n_maps);
    for (int i = 0; i < n_maps; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const double cx = (double)sargs[x].W * sargs[x].H * sargs[x].N;
        const double cy = (double)sargs[y].W * sargs[y].H * sargs[y].N;
        return cx > cy;
    });
    std::vector<StackArgs> sorted(n_maps);
    for (int i = 0; i < n_maps; ++i) sorted[i] = sargs[order[i]];

    k_batch_init<<<n_maps, 256, 0, s>>>(small);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_partition_batched(pin.data(), n_maps, tn.points_per_block, L.cells, ws, s);
    // one persistent launch when every map shares the window (one r_g) and an
    // instance has its radii; otherwise map after map, each with its own
    // constants, on the incremental kernel where it has the radii and on the
    // generic one where not (as the single-map path does)
    bool shared = true;
    for (int i = 0; i < n_maps; ++i) {
        shared = shared && maps[i].grid.res == maps[0].grid.res &&
                 inc_supported(c, maps[i].grid.n_slices);
        sorted[i].c = c;
    }
    int tile = tn.tile;
    if (shared) {
        if (tile == TCT_TILE_AUTO) tile = choose_tile(c, n_maps, sorted.data(), 2);
        if (e == cudaSuccess)
            e = launch_stack_batched(c, n_maps, sorted.data(), queue, tile, tn.ctas_per_sm, s);
    } else {
        for (int i = 0; i < n_maps && e == cudaSuccess; ++i) {
            StackArgs a = sorted[i];
            const tct_map &m = maps[order[i]];
            if (make_eval_consts(m.grid, *params, &a.c) != TCT_OK) return TCT_ERR_INVALID_ARG;
            if (inc_supported(a.c, a.N)) {
                const int t = tn.tile == TCT_TILE_AUTO ? choose_tile(a.c, 1, &a, 2) : tn.tile;
                e = cudaMemsetAsync(queue, 0, sizeof(int32_t), s);
                if (e == cudaSuccess) e = launch_stack_batched(a.c, 1, &a, queue, t, tn.ctas_per_sm, s);
            } else {
                e = launch_stack_generic(a, s);
            }
        }
    }
    if (e == cudaSuccess) {
        k_batch_chain<<<n_maps, 128, 0, s>>>(small);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaErrorNotSupported) return TCT_ERR_UNSUPPORTED;
    return e == cudaSuccess ? TCT_OK : TCT_ERR_CUDA;
}

tct_tuning default_tuning() {
    tct_tuning t;
    t.tile = TCT_TILE_AUTO;
    t.ctas_per_sm = 0;
    t.points_per_block = 4096;
    t.reserved = 0;
    return t;
}

// The construction alone for a batch: one thread per cell of all maps walks
// the slices with the monotone pointer (as tct_build does for one map).
struct ElevBatch {
    int32_t n_maps;
    int64_t cell_start[TCT_MAX_BATCH + 1];   // first cell of each map in the concatenation
    struct {
        int32_t N, zmin_from_data;
        float d_s, z_min;
        const int32_t *zkeys;
        float *ground, *ceil;
    } m[TCT_MAX_BATCH];
};

__global__ void __launch_bounds__(256)
k_elevations_batched(const __grid_constant__ ElevBatch b, const int32_t *__restrict__ start,
                     const float *__restrict__ zs) {
    const int64_t total = b.cell_start[b.n_maps];
    for (int64_t gc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gc < total;
         gc += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = b.n_maps - 1;           // the map holding cell gc
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (b.cell_start[mid] <= gc) lo = mid;
            else hi = mid - 1;
        }
        const auto &m = b.m[lo];
        const int64_t c = gc - b.cell_start[lo];
        const int64_t hw = b.cell_start[lo + 1] - b.cell_start[lo];
        float z_min = m.z_min;
        if (m.zmin_from_data) {
            z_min = key_float(m.zkeys[0]);
            if (!isfinite(z_min)) z_min = 0.0f;
        }
        int32_t p = start[gc];
        const int32_t e = start[gc + 1];
        float zg = -INFINITY;
        float zc = p < e ? zs[p] : INFINITY;
        for (int k = 0; k < m.N; ++k) {
            const float h = __fmaf_rn((float)(k + 1), m.d_s, z_min);
            while (zc <= h) {
                zg = zc;
                ++p;
                zc = p < e ? zs[p] : INFINITY;
            }
            __stcs(&m.ground[(int64_t)k * hw + c], zg);
            __stcs(&m.ceil[(int64_t)k * hw + c], zc);
        }
    }
}

// z bounds of each map into its statistics (the construction-only batch).
__global__ void k_batch_bounds(const __grid_constant__ BatchSmall b) {
    const auto &m = b.m[blockIdx.x];
    if (threadIdx.x == 0) {
        m.stats->z_min = key_float(m.zkeys[0]);
        m.stats->z_max = key_float(m.zkeys[1]);
    }
}

int run_build_batch(const tct_map *maps, int n_maps, int points_per_block, void *d_ws,
                    cudaStream_t s) {
    const BatchLayout L = batch_layout(maps, n_maps);
    char *base = static_cast<char *>(d_ws);
    Workspace ws;
    memset(&ws, 0, sizeof(ws));
    ws.cnt = reinterpret_cast<int32_t *>(base + L.cnt);
    ws.start = reinterpret_cast<int32_t *>(base + L.start);
    ws.partial = reinterpret_cast<int32_t *>(base + L.partial);
    ws.zs = reinterpret_cast<float *>(base + L.zs);
    ws.scratch = reinterpret_cast<float *>(base + L.scratch);
    ws.bucket_l = reinterpret_cast<uint16_t *>(base + L.bucket_l);
    ws.bcur = reinterpret_cast<int32_t *>(base + L.bcur);
    ws.long_count = reinterpret_cast<int32_t *>(base + L.long_count);
    ws.long_cells = reinterpret_cast<int32_t *>(base + L.long_cells);
    int32_t *zkeys = reinterpret_cast<int32_t *>(base + L.zkeys);
    tct_stats *stats = reinterpret_cast<tct_stats *>(base + L.stats);
    BatchSmall small;
    memset(&small, 0, sizeof(small));
    small.n_maps = n_maps;
    small.queue = reinterpret_cast<int32_t *>(base + L.queue);
    ElevBatch eb;
    memset(&eb, 0, sizeof(eb));
    eb.n_maps = n_maps;
    std::vector<BatchPointsIn> pin(n_maps);
    int64_t cell_off = 0;
    for (int i = 0; i < n_maps; ++i) {
        const tct_map &m = maps[i];
        auto &sm = small.m[i];
        sm.zkeys = zkeys + 2 * i;
        sm.upre = reinterpret_cast<int32_t *>(base + L.upre) + (TCT_MAX_SLICES + 1) * i;
        sm.ubits = reinterpret_cast<uint32_t *>(base + L.ubits) + 4 * (TCT_MAX_SLICES + 1) * i;
        sm.stats = m.d_stats ? m.d_stats : stats + i;
        sm.n_points = m.n;
        sm.n_slices = m.grid.n_slices;
        pin[i] = BatchPointsIn{m.d_xyz, m.n, m.stride, m.grid, cell_off, sm.zkeys, sm.stats};
        eb.cell_start[i] = cell_off;
        eb.m[i].N = m.grid.n_slices;
        eb.m[i].zmin_from_data = (m.grid.flags & TCT_GRID_ZMIN_FROM_DATA) ? 1 : 0;
        eb.m[i].d_s = m.grid.d_s;
        eb.m[i].z_min = m.grid.z_min;
        eb.m[i].zkeys = sm.zkeys;
        eb.m[i].ground = m.d_ground;
        eb.m[i].ceil = m.d_ceil;
        cell_off += (int64_t)m.grid.W * m.grid.H;
    }
    eb.cell_start[n_maps] = cell_off;
    k_batch_init<<<n_maps, 256, 0, s>>>(small);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_partition_batched(pin.data(), n_maps, points_per_block, L.cells, ws, s);
    if (e == cudaSuccess) {
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int64_t blocks = (cell_off + 255) / 256;
        if (blocks > 8 * (int64_t)sms) blocks = 8 * (int64_t)sms;
        if (blocks < 1) blocks = 1;
        k_elevations_batched<<<(unsigned)blocks, 256, 0, s>>>(eb, ws.start, ws.zs);
        k_batch_bounds<<<n_maps, 32, 0, s>>>(small);
        count_launches(2);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? TCT_OK : TCT_ERR_CUDA;
}

}  // namespace
}  // namespace tct

using namespace tct;

extern "C" int tct_build_batched(const tct_map *h_maps, int32_t n_maps, const tct_tuning *tuning,
                                 void *d_ws, size_t ws_bytes, tct_stream stream) {
    if (!h_maps || n_maps < 1 || !d_ws) return TCT_ERR_INVALID_ARG;
    if (n_maps > TCT_MAX_BATCH) return TCT_ERR_UNSUPPORTED;
    int64_t cells = 0, points = 0;
    for (int i = 0; i < n_maps; ++i) {
        const tct_map &m = h_maps[i];
        if (tct_workspace_bytes(&m.grid, m.n, nullptr) == 0) return TCT_ERR_INVALID_ARG;
        if (m.grid.n_slices > TCT_MAX_SLICES) return TCT_ERR_UNSUPPORTED;
        if ((m.stride != 3 && m.stride != 4) || (m.n > 0 && !m.d_xyz)) return TCT_ERR_INVALID_ARG;
        if (!m.d_ground || !m.d_ceil) return TCT_ERR_INVALID_ARG;
        cells += (int64_t)m.grid.W * m.grid.H;
        points += m.n;
    }
    if (cells >= ((int64_t)1 << 31) || points >= ((int64_t)1 << 31)) return TCT_ERR_UNSUPPORTED;
    if (ws_bytes < batch_layout(h_maps, n_maps).total) return TCT_ERR_WORKSPACE_TOO_SMALL;
    const int ppb = tuning ? tuning->points_per_block : default_tuning().points_per_block;
    if (ppb < 4 || ppb % 4) return TCT_ERR_INVALID_ARG;
    return run_build_batch(h_maps, n_maps, ppb, d_ws, (cudaStream_t)stream);
}

extern "C" size_t tct_workspace_bytes_evaluate_batched(const tct_map *h_maps, int32_t n_maps,
                                                       const tct_params *params) {
    if (!h_maps || n_maps < 1 || n_maps > TCT_MAX_BATCH) return 0;
    size_t most = 0;
    for (int i = 0; i < n_maps; ++i) {
        const size_t b = tct_workspace_bytes(&h_maps[i].grid, 0, params);
        if (b == 0) return 0;
        most = std::max(most, b);
    }
    return most;
}

extern "C" int tct_evaluate_batched(const tct_map *h_maps, int32_t n_maps, const tct_params *params,
                                    void *d_ws, size_t ws_bytes, tct_stream stream) {
    if (!h_maps || n_maps < 1 || !params || !d_ws) return TCT_ERR_INVALID_ARG;
    if (n_maps > TCT_MAX_BATCH) return TCT_ERR_UNSUPPORTED;
    const size_t need = tct_workspace_bytes_evaluate_batched(h_maps, n_maps, params);
    if (need == 0) return TCT_ERR_INVALID_ARG;
    if (ws_bytes < need) return TCT_ERR_WORKSPACE_TOO_SMALL;
    for (int i = 0; i < n_maps; ++i) {
        const tct_map &m = h_maps[i];
        const int rc = tct_evaluate(&m.grid, params, m.d_ground, m.d_ceil, d_ws, ws_bytes, m.d_cost,
                                    m.d_mask, m.d_keep, nullptr, m.d_stats, stream);
        if (rc != TCT_OK) return rc;
    }
    return TCT_OK;
}

extern "C" size_t tct_workspace_bytes_batched(const tct_map *h_maps, int32_t n_maps,
                                              const tct_params *params) {
    (void)params;
    if (!h_maps || n_maps < 1 || n_maps > TCT_MAX_BATCH) return 0;
    for (int i = 0; i < n_maps; ++i)
        if (tct_workspace_bytes(&h_maps[i].grid, h_maps[i].n, params) == 0) return 0;
    return batch_layout(h_maps, n_maps).total;
}

extern "C" int tct_build_evaluate_batched(const tct_map *h_maps, int32_t n_maps,
                                          const tct_params *params, const tct_tuning *tuning,
                                          void *d_ws, size_t ws_bytes, tct_stream stream) {
    EvalConsts c;
    int rc = check_batch(h_maps, n_maps, params, &c);
    if (rc != TCT_OK) return rc;
    if (!d_ws) return TCT_ERR_INVALID_ARG;
    if (ws_bytes < batch_layout(h_maps, n_maps).total) return TCT_ERR_WORKSPACE_TOO_SMALL;
    tct_tuning tn = tuning ? *tuning : default_tuning();
    if (tn.points_per_block < 4 || tn.points_per_block % 4) return TCT_ERR_INVALID_ARG;
    if (tn.tile != TCT_TILE_AUTO && tn.tile != TCT_TILE_64 && tn.tile != TCT_TILE_32 &&
        tn.tile != TCT_TILE_64x56 && tn.tile != TCT_TILE_64x40 && tn.tile != TCT_TILE_128x56)
        return TCT_ERR_INVALID_ARG;
    return run_batch(h_maps, n_maps, params, tn, c, d_ws, (cudaStream_t)stream);
}

extern "C" int tct_autotune_batched(const tct_map *h_maps, int32_t n_maps,
                                    const tct_params *params, void *d_ws, size_t ws_bytes,
                                    tct_stream stream, tct_tuning *out) {
    EvalConsts c;
    int rc = check_batch(h_maps, n_maps, params, &c);
    if (rc != TCT_OK) return rc;
    if (!d_ws || !out) return TCT_ERR_INVALID_ARG;
    if (ws_bytes < batch_layout(h_maps, n_maps).total) return TCT_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return TCT_ERR_CUDA;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return TCT_ERR_CUDA; }
    const int tiles[] = {TCT_TILE_64, TCT_TILE_64x56, TCT_TILE_64x40, TCT_TILE_128x56, TCT_TILE_32};
    const int ctas[] = {0, 1};
    const int ppb[] = {2048, 8192};
    float best = INFINITY;
    tct_tuning chosen = default_tuning();
    rc = TCT_OK;
    for (int ti : tiles)
        for (int ci : ctas)
            for (int pi : ppb) {
                tct_tuning t = default_tuning();
                t.tile = ti;
                t.ctas_per_sm = ci;
                t.points_per_block = pi;
                float ms = 0.0f;
                for (int rep = 0; rep < 2 && rc == TCT_OK; ++rep) {   // warm, then timed
                    cudaEventRecord(a, s);
                    rc = run_batch(h_maps, n_maps, params, t, c, d_ws, s);
                    cudaEventRecord(b, s);
                    if (cudaEventSynchronize(b) != cudaSuccess) rc = TCT_ERR_CUDA;
                    if (rc == TCT_OK) cudaEventElapsedTime(&ms, a, b);
                }
                if (rc != TCT_OK) break;
                if (ms < best) { best = ms; chosen = t; }
            }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc != TCT_OK) return rc;
    *out = chosen;
    return TCT_OK;
}
