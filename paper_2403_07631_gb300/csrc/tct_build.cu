// tct_build.cu -- tomogram construction kernels (Sec. III-A, the construction part of Alg. 1).
//
// The cloud is partitioned by cell with a counting sort:
//   count    one pass over the points: rasterise, per-cell histogram with
//            L2 atomics, bounds of z (block-reduced ordered-int atomics),
//            dropped / non-finite counts;
//   scan     exclusive prefix of the histogram (two small kernels);
//   bucket   second pass over the points: each z, with its cell's place in
//            its bucket of kBucket consecutive cells, is appended to the
//            bucket's range of a staging array (the range of zs the bucket's
//            cells occupy), one cursor atomic per warp when the warp's points
//            share a bucket;
//   sort     one block per bucket places the heights by cell and sorts the
//            short segments in shared memory and writes the bucket back in
//            one coalesced sweep; longer segments go to a warp (up to 256
//            heights) or a block (beyond) in global memory.
// A sorted segment answers every plane with one monotone pointer: the ground
// of plane h is the last z <= h, the ceiling the first z > h.  The fused
// per-tile evaluation (tct_stack.cu) consumes the segments directly;
// k_elevations below writes the two layers for tct_build alone.
#include <cuda_runtime.h>
#include <math.h>

#include "tct_internal.cuh"

namespace tct {
namespace {

constexpr int kThreads = 256;

struct GridDev {
    float x0, y0, res, Wf, Hf;
    int32_t W, H;
};

GridDev grid_dev(const tct_grid &g) {
    return GridDev{g.x0, g.y0, g.res, (float)g.W, (float)g.H, g.W, g.H};
}

// Alg. 1 "rasterize": cell = (floor(fl32(fl32(y-y0)/r)), floor(fl32(fl32(x-x0)/r))).
__device__ __forceinline__ int cell_of(const GridDev &g, float x, float y) {
    const float u = __fdiv_rn(__fsub_rn(x, g.x0), g.res);
    const float v = __fdiv_rn(__fsub_rn(y, g.y0), g.res);
    if (!(u >= 0.0f && u < g.Wf && v >= 0.0f && v < g.Hf)) return -1;
    return __float2int_rd(v) * g.W + __float2int_rd(u);
}

__device__ __forceinline__ bool finite3(float x, float y, float z) {
    return isfinite(x) && isfinite(y) && isfinite(z);
}

__device__ __forceinline__ float fold_zero(float z) { return z == 0.0f ? 0.0f : z; }

// Loads the 4 consecutive points of group `grp` (points 4*grp .. 4*grp+3).
// The vector path needs the base 16-byte aligned; n is checked by the caller.
__device__ __forceinline__ void load4(const float *__restrict__ xyz, int stride, int64_t grp,
                                      float (&p)[4][3]) {
    if (stride == 3) {
        const float4 *v = reinterpret_cast<const float4 *>(xyz) + 3 * grp;
        const float4 a = __ldg(v), b = __ldg(v + 1), c = __ldg(v + 2);
        p[0][0] = a.x; p[0][1] = a.y; p[0][2] = a.z;
        p[1][0] = a.w; p[1][1] = b.x; p[1][2] = b.y;
        p[2][0] = b.z; p[2][1] = b.w; p[2][2] = c.x;
        p[3][0] = c.y; p[3][1] = c.z; p[3][2] = c.w;
    } else {
        const float4 *v = reinterpret_cast<const float4 *>(xyz) + 4 * grp;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 a = __ldg(v + q);
            p[q][0] = a.x; p[q][1] = a.y; p[q][2] = a.z;
        }
    }
}

__device__ __forceinline__ void load1(const float *__restrict__ xyz, int stride, int64_t i,
                                      float (&p)[3]) {
    const float *q = xyz + i * stride;
    p[0] = __ldg(q); p[1] = __ldg(q + 1); p[2] = __ldg(q + 2);
}

// Per-block accumulation of the statistics every pass over the points keeps.
struct PointTally {
    int32_t zlo, zhi;            // ordered-int keys
    unsigned long long dropped, nonfinite;
    __device__ void init() {
        zlo = float_key(INFINITY);
        zhi = float_key(-INFINITY);
        dropped = nonfinite = 0;
    }
};

__device__ void flush_tally(PointTally t, int32_t *zkeys, tct_stats *stats, bool with_z) {
    __shared__ int32_t s_lo[kThreads / 32], s_hi[kThreads / 32];
    __shared__ unsigned long long s_d[kThreads / 32], s_n[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    t.zlo = __reduce_min_sync(0xffffffffu, t.zlo);
    t.zhi = __reduce_max_sync(0xffffffffu, t.zhi);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t.dropped += __shfl_xor_sync(0xffffffffu, t.dropped, o);
        t.nonfinite += __shfl_xor_sync(0xffffffffu, t.nonfinite, o);
    }
    if (lane == 0) { s_lo[warp] = t.zlo; s_hi[warp] = t.zhi; s_d[warp] = t.dropped; s_n[warp] = t.nonfinite; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t lo = s_lo[0], hi = s_hi[0];
        unsigned long long d = s_d[0], nf = s_n[0];
        for (int w = 1; w < kThreads / 32; ++w) {
            lo = min(lo, s_lo[w]); hi = max(hi, s_hi[w]); d += s_d[w]; nf += s_n[w];
        }
        if (with_z) {
            atomicMin(&zkeys[0], lo);
            atomicMax(&zkeys[1], hi);
        }
        if (d) atomicAdd(reinterpret_cast<unsigned long long *>(&stats->n_dropped), d);
        if (nf) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&stats->n_nonfinite), nf);
            atomicOr(&stats->status, TCT_DEV_NONFINITE);
        }
    }
}

// Warp-aggregated update of a per-cell counter: lanes of the warp that hit the
// same cell are served by one atomic; returns this lane's slot (0-based rank
// among the lanes of its group, plus the counter value the group saw).
// Per-cell counter update; returns this point's slot.  (A warp-aggregated
// form with __match_any_sync was measured slower: in stratified and
// spatially sorted clouds the 32 points of a warp fall in 32 distinct cells,
// so the match only adds work.)
template <bool kSubtract>
__device__ __forceinline__ int32_t cell_slot(int32_t *ctr, int64_t cell) {
    return kSubtract ? atomicSub(&ctr[cell], 1) - 1 : atomicAdd(&ctr[cell], 1);
}

__global__ void __launch_bounds__(kThreads)
k_bounds(const float *__restrict__ xyz, int64_t n, int stride, int32_t *keys6,
         tct_stats *stats) {
    // keys6: ordered-int min x, y, z then max x, y, z
    int32_t lo[3], hi[3];
    unsigned long long bad = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) { lo[a] = float_key(INFINITY); hi[a] = float_key(-INFINITY); }
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += nthreads) {
        float p[3];
        load1(xyz, stride, i, p);
        if (!finite3(p[0], p[1], p[2])) { ++bad; continue; }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int32_t k = float_key(fold_zero(p[a]));
            lo[a] = min(lo[a], k); hi[a] = max(hi[a], k);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = __reduce_min_sync(0xffffffffu, lo[a]);
        hi[a] = __reduce_max_sync(0xffffffffu, hi[a]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) { atomicMin(&keys6[a], lo[a]); atomicMax(&keys6[3 + a], hi[a]); }
        if (bad && stats) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&stats->n_nonfinite), bad);
            atomicOr(&stats->status, TCT_DEV_NONFINITE);
        }
    }
}

__global__ void k_bounds_init(int32_t *keys6, tct_stats *stats, int64_t n) {
    if (threadIdx.x < 3) {
        keys6[threadIdx.x] = float_key(INFINITY);
        keys6[3 + threadIdx.x] = float_key(-INFINITY);
    }
    if (threadIdx.x == 0 && stats) stats->n_points = n;
}

// Converts the ordered-int keys held in out6 back to floats, in place.
__global__ void k_bounds_finish(float *out6, tct_stats *stats) {
    const int t = threadIdx.x;
    int32_t k = 0;
    if (t < 6) k = reinterpret_cast<const int32_t *>(out6)[t];
    __syncwarp();
    if (t < 6) out6[t] = key_float(k);
    if (t == 2 && stats) stats->z_min = key_float(k);
    if (t == 5 && stats) stats->z_max = key_float(k);
}

// One point of a map in pass 1: counted in its cell, bounds and tallies.
__device__ __forceinline__ void count_point(float x, float y, float z, const GridDev &g,
                                            int64_t cell_off, int32_t *__restrict__ cnt,
                                            PointTally &t) {
    if (!finite3(x, y, z)) {
        ++t.nonfinite;
        return;
    }
    z = fold_zero(z);
    const int32_t k = float_key(z);
    t.zlo = min(t.zlo, k);
    t.zhi = max(t.zhi, k);
    const int cell = cell_of(g, x, y);
    if (cell < 0) {
        ++t.dropped;
        return;
    }
    cell_slot<false>(cnt, cell_off + cell);
}

// U points of each lane in pass 2.  Called by every active lane of the warp
// at once (gc < 0: no point).  The points that share the bucket of the
// warp's first valid point (most of them: the points of a scan line fall in
// consecutive cells) append their height and their cell's place in the
// bucket to the bucket's range of the staging arrays, with one atomic for
// all of them; the bucket sort later fills their cells' segments from the
// bottom.  Any other point (a cloud in no particular order) takes a slot
// from the top of its own cell's segment with an atomic on that cell's
// count, which few other points share, and is written to zs directly.
template <int U>
__device__ __forceinline__ void bucket_points(const int64_t (&gc)[U], const float (&z)[U],
                                              const int32_t *__restrict__ start,
                                              int32_t *__restrict__ cnt,
                                              int32_t *__restrict__ bcur, float *__restrict__ bz,
                                              uint16_t *__restrict__ bl, float *__restrict__ zs,
                                              int blog) {
    const uint32_t act = __activemask();
    const int lane = threadIdx.x & 31;
    uint32_t vm[U];
    int first = -1;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        vm[u] = __ballot_sync(act, gc[u] >= 0);
        if (first < 0 && vm[u]) first = u;
    }
    if (first < 0) return;
    const int src = __ffs(vm[first]) - 1;
    int64_t mine = -1;
#pragma unroll
    for (int u = 0; u < U; ++u)
        if (u == first) mine = gc[u];
    const int64_t b0 = __shfl_sync(act, mine, src) >> blog;
    const int32_t pos0 = start[b0 << blog];              // issued before the atomics
    uint32_t sm[U];
    int n0 = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        sm[u] = __ballot_sync(act, gc[u] >= 0 && (gc[u] >> blog) == b0);
        n0 += __popc(sm[u]);
    }
    int32_t base = 0;
    if (lane == src) base = atomicAdd(&bcur[b0], n0);
    // the other points: all their slot atomics, then their segment starts
    int32_t dslot[U], dpos[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
        dslot[u] = gc[u] >= 0 && !((sm[u] >> lane) & 1u) ? atomicSub(&cnt[gc[u]], 1) - 1 : -1;
#pragma unroll
    for (int u = 0; u < U; ++u) dpos[u] = dslot[u] >= 0 ? start[gc[u]] + dslot[u] : 0;
    base = __shfl_sync(act, base, src);
    const uint32_t lt = (1u << lane) - 1u;
    int run = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if ((sm[u] >> lane) & 1u) {
            const int64_t pos = (int64_t)pos0 + base + run + __popc(sm[u] & lt);
            bz[pos] = z[u];
            bl[pos] = (uint16_t)(gc[u] & ((1 << blog) - 1));
        } else if (dslot[u] >= 0) {
            zs[dpos[u]] = z[u];
        }
        run += __popc(sm[u]);
    }
}

__device__ __forceinline__ int64_t point_cell(float x, float y, const GridDev &g, int64_t cell_off) {
    if (!finite3(x, y, 0.0f)) return -1;
    const int cell = cell_of(g, x, y);
    return cell < 0 ? -1 : cell_off + cell;
}

// Points [p0, p1) of one map, thread `tid` of `nthreads`: groups of four
// with vector loads where the base allows, the ragged ends one by one.  Pass
// 1 (kBucketPass false) counts, pass 2 buckets.
template <bool kBucketPass>
__device__ __forceinline__ void visit_range(const float *__restrict__ xyz, int stride, bool vec,
                                            int64_t p0, int64_t p1, int64_t tid, int64_t nthreads,
                                            const GridDev &g, int64_t cell_off,
                                            int32_t *__restrict__ cnt,
                                            const int32_t *__restrict__ start,
                                            int32_t *__restrict__ bcur, float *__restrict__ bz,
                                            uint16_t *__restrict__ bl, float *__restrict__ zs,
                                            int blog, PointTally &t) {
    auto one = [&](float x, float y, float z) {
        if (kBucketPass) {
            const int64_t gc[1] = {finite3(x, y, z) ? point_cell(x, y, g, cell_off) : -1};
            const float zz[1] = {fold_zero(z)};
            bucket_points<1>(gc, zz, start, cnt, bcur, bz, bl, zs, blog);
        } else {
            count_point(x, y, z, g, cell_off, cnt, t);
        }
    };
    int64_t q0 = 0, q1 = 0;
    if (vec) {
        q0 = (p0 + 3) / 4;
        q1 = p1 / 4;
        if (q1 < q0) q1 = q0;
    }
    // two groups of four points a thread per round, their loads issued together
    for (int64_t qq = q0 + tid; qq < q1; qq += 2 * nthreads) {
        float pp[2][4][3];
        load4(xyz, stride, qq, pp[0]);
        const bool two = qq + nthreads < q1;
        if (two) load4(xyz, stride, qq + nthreads, pp[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
        if (h == 1 && !two) break;
        float (&p)[4][3] = pp[h];
        if (kBucketPass) {
            int64_t gc[4];
            float zz[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                gc[u] = finite3(p[u][0], p[u][1], p[u][2]) ? point_cell(p[u][0], p[u][1], g, cell_off)
                                                            : -1;
                zz[u] = fold_zero(p[u][2]);
            }
            bucket_points<4>(gc, zz, start, cnt, bcur, bz, bl, zs, blog);
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) one(p[u][0], p[u][1], p[u][2]);
        }
        }
    }
    const int64_t a1 = vec ? min(4 * q0, p1) : p1;
    for (int64_t i = p0 + tid; i < a1; i += nthreads) {
        float p[3];
        load1(xyz, stride, i, p);
        one(p[0], p[1], p[2]);
    }
    if (vec) {
        for (int64_t i = max(4 * q1, p0) + tid; i < p1; i += nthreads) {
            float p[3];
            load1(xyz, stride, i, p);
            one(p[0], p[1], p[2]);
        }
    }
}

// Pass 1 of one map: histogram of points per cell, z bounds and tallies.
__global__ void __launch_bounds__(kThreads)
k_count(const float *__restrict__ xyz, int64_t n, int stride, bool vec, GridDev g,
        int32_t *__restrict__ cnt, int32_t *zkeys, tct_stats *stats) {
    PointTally t;
    t.init();
    visit_range<false>(xyz, stride, vec, 0, n, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                       (int64_t)gridDim.x * blockDim.x, g, 0, cnt, nullptr, nullptr, nullptr,
                       nullptr, nullptr, 0, t);
    flush_tally(t, zkeys, stats, true);
}

// Pass 2 of one map.
__global__ void __launch_bounds__(kThreads)
k_bucket(const float *__restrict__ xyz, int64_t n, int stride, bool vec, GridDev g,
         int32_t *__restrict__ cnt, const int32_t *__restrict__ start, int32_t *__restrict__ bcur,
         float *__restrict__ bz, uint16_t *__restrict__ bl, float *__restrict__ zs, int blog) {
    PointTally t;
    t.init();
    visit_range<true>(xyz, stride, vec, 0, n, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                      (int64_t)gridDim.x * blockDim.x, g, 0, cnt, start, bcur, bz, bl, zs, blog, t);
}

// Both passes over a batch: block b serves one chunk of one map's points.
struct PointMap {
    const float *xyz;
    int64_t n;
    int32_t stride, vec;
    GridDev g;
    int64_t cell_off;            // first cell of the map in the concatenated arrays
    int32_t *zkeys;
    tct_stats *stats;
    int32_t block_start;         // first block of the map
};

struct PointBatch {
    int32_t n_maps;
    int32_t chunk;               // points per block, a multiple of 4
    PointMap maps[TCT_MAX_BATCH];
};

__device__ __forceinline__ int batch_map_of_block(const PointBatch &b) {
    int m = 0;
    while (m + 1 < b.n_maps && b.maps[m + 1].block_start <= (int)blockIdx.x) ++m;
    return m;
}

__global__ void __launch_bounds__(kThreads)
k_count_batched(const __grid_constant__ PointBatch b, int32_t *__restrict__ cnt) {
    const PointMap &m = b.maps[batch_map_of_block(b)];
    const int64_t p0 = (int64_t)((int)blockIdx.x - m.block_start) * b.chunk;
    const int64_t p1 = min(m.n, p0 + b.chunk);
    PointTally t;
    t.init();
    visit_range<false>(m.xyz, m.stride, m.vec != 0, p0, p1, threadIdx.x, blockDim.x, m.g,
                       m.cell_off, cnt, nullptr, nullptr, nullptr, nullptr, nullptr, 0, t);
    flush_tally(t, m.zkeys, m.stats, true);
}

__global__ void __launch_bounds__(kThreads)
k_bucket_batched(const __grid_constant__ PointBatch b, int32_t *__restrict__ cnt,
                 const int32_t *__restrict__ start, int32_t *__restrict__ bcur,
                 float *__restrict__ bz, uint16_t *__restrict__ bl, float *__restrict__ zs,
                 int blog) {
    const PointMap &m = b.maps[batch_map_of_block(b)];
    const int64_t p0 = (int64_t)((int)blockIdx.x - m.block_start) * b.chunk;
    const int64_t p1 = min(m.n, p0 + b.chunk);
    PointTally t;
    t.init();
    visit_range<true>(m.xyz, m.stride, m.vec != 0, p0, p1, threadIdx.x, blockDim.x, m.g,
                      m.cell_off, cnt, start, bcur, bz, bl, zs, blog, t);
}

// Exclusive scan of cnt[0, m) into start[0, m], in tiles of kScanTile.
constexpr int kPerThread = kScanTile / kThreads;   // 16

__global__ void __launch_bounds__(kThreads)
k_scan_reduce(const int32_t *__restrict__ cnt, int64_t m, int32_t *__restrict__ partial) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kPerThread;
    int32_t s = 0;
#pragma unroll
    for (int q = 0; q < kPerThread; ++q)
        if (base + q < m) s += cnt[base + q];
    s = __reduce_add_sync(0xffffffffu, s);
    __shared__ int32_t ws[kThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += ws[w];
        partial[blockIdx.x] = t;
    }
}

// The down sweep: each block adds up the sums of the blocks before it (its
// threads each take a strided share of them), scans its own cells and writes
// their starts; the last block writes the total.  Block 0 also turns the z
// bounds of the count pass into the statistics' floats (zkeys and stats may
// be NULL).
__global__ void __launch_bounds__(kThreads)
k_scan_down(const int32_t *__restrict__ cnt, int64_t m, const int32_t *__restrict__ partial,
            int32_t *__restrict__ start, int nb, const int32_t *zkeys, tct_stats *stats) {
    __shared__ int32_t ws[kThreads / 32];
    __shared__ int32_t s_pre;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t pre = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += kThreads) pre += partial[b];
    pre = __reduce_add_sync(0xffffffffu, pre);
    if (lane == 0) ws[warp] = pre;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += ws[w];
        s_pre = t;
        if (blockIdx.x == 0 && zkeys && stats) {
            stats->z_min = key_float(zkeys[0]);
            stats->z_max = key_float(zkeys[1]);
        }
    }
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kPerThread;
    int32_t v[kPerThread];
    int32_t s = 0;
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) {
        v[q] = base + q < m ? cnt[base + q] : 0;
        s += v[q];
    }
    int32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    int32_t off = s_pre + x - s;
    for (int w = 0; w < warp; ++w) off += ws[w];
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) {
        if (base + q < m) start[base + q] = off;
        off += v[q];
    }
    if (blockIdx.x == nb - 1 && threadIdx.x == kThreads - 1) start[m] = off;
}

// Exclusive scan of ws.cnt[0, m) into ws.start[0, m]; returns the launches.
int launch_scan(const Workspace &ws, int64_t m, const int32_t *zkeys, tct_stats *stats,
                cudaStream_t s) {
    const int nb = (int)((m + kScanTile - 1) / kScanTile);
    k_scan_reduce<<<nb, kThreads, 0, s>>>(ws.cnt, m, ws.partial);
    k_scan_down<<<nb, kThreads, 0, s>>>(ws.cnt, m, ws.partial, ws.start, nb, zkeys, stats);
    return 2;
}

// Sort each cell's segment ascending.  Segments of up to 16 heights are
// sorted in registers by a bitonic network (padded with +inf); segments of
// up to kWarpSort heights are queued for the warp sort of k_sort_queued (from
// the front of long_cells, counted in long_count[0]), longer ones for its
// block sort (from the back, counted in long_count[1]).
constexpr int kWarpSort = 256;
template <int L>
__device__ __forceinline__ void bitonic_sort(float (&v)[L]) {
#pragma unroll
    for (int size = 2; size <= L; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
#pragma unroll
            for (int i = 0; i < L; ++i) {
                const int jx = i ^ stride;
                if (jx > i) {
                    const bool up = (i & size) == 0;
                    const float a = v[i], b = v[jx];
                    const float lo = fminf(a, b), hi = fmaxf(a, b);
                    v[i] = up ? lo : hi;
                    v[jx] = up ? hi : lo;
                }
            }
        }
    }
}

template <int L>
__device__ __forceinline__ void sort_segment(float *__restrict__ zs, int32_t s, int32_t n) {
    float v[L];
#pragma unroll
    for (int i = 0; i < L; ++i) v[i] = i < n ? zs[s + i] : INFINITY;
    bitonic_sort<L>(v);
#pragma unroll
    for (int i = 0; i < L; ++i)
        if (i < n) zs[s + i] = v[i];
}

// Pass 3: one block per bucket of 2^blog cells.  The bucket's staged
// heights sit in the staging arrays at the start of the range of zs its
// cells occupy; the heights written directly already fill the top of their
// cells' segments in zs.  The block reads the range of zs into shared
// memory, places each staged height at its cell's next slot from the bottom
// (shared-memory cursors), sorts segments of up to 16 heights in registers
// and writes the range back.  When the bucket holds more than kBucketStage
// heights the same happens in global memory.  Segments of 17 .. kWarpSort
// heights are queued for the warp sort of k_sort_queued (from the front of
// long_cells, counted in long_count[0]), longer ones for its block sort (from
// the back, long_count[1]); a block takes its places in each queue with one
// atomic.
constexpr int kBucketStage = 8192;

// Sorts a segment of up to 16 heights in place; returns 0, or 1 for a
// segment the warp sort takes (17 .. kWarpSort heights), 2 for the block sort.
__device__ __forceinline__ int sort_short(float *seg, int32_t n) {
    if (n <= 1) return 0;
    if (n <= 4) sort_segment<4>(seg, 0, n);
    else if (n <= 8) sort_segment<8>(seg, 0, n);
    else if (n <= 16) sort_segment<16>(seg, 0, n);
    else return n <= kWarpSort ? 1 : 2;
    return 0;
}

__global__ void __launch_bounds__(kThreads)
k_bucket_sort(const int32_t *__restrict__ start, int64_t m, const int32_t *__restrict__ bcur,
              const float *__restrict__ bz, const uint16_t *__restrict__ bl,
              float *__restrict__ zs, int32_t *__restrict__ long_count,
              int32_t *__restrict__ long_cells, int blog) {
    __shared__ int32_t s_off[kBucket + 1];
    __shared__ int32_t s_cur[kBucket];
    __shared__ float s_z[kBucketStage];
    __shared__ uint16_t s_q[kBucket];            // long segments from the front, huge from the back
    __shared__ int32_t s_n[2], s_base[2];
    const int tid = threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.x << blog;
    const int ncell = (int)min((int64_t)1 << blog, m - c0);
    const int32_t z0 = start[c0];
    const int32_t staged = bcur[blockIdx.x];
    for (int l = tid; l <= ncell; l += kThreads) s_off[l] = start[c0 + l] - z0;
    for (int l = tid; l < ncell; l += kThreads) s_cur[l] = 0;
    if (tid < 2) s_n[tid] = 0;
    __syncthreads();
    const int32_t nb = s_off[ncell];
    if (nb == 0) return;
    const bool staged_in_smem = nb <= kBucketStage;
    float *seg0 = staged_in_smem ? s_z : zs + z0;
    if (staged_in_smem) {
        if (staged < nb)
            for (int32_t i = tid; i < nb; i += kThreads) s_z[i] = zs[z0 + i];
        __syncthreads();
    }
    for (int32_t i = tid; i < staged; i += kThreads) {
        const int l = bl[z0 + i];
        seg0[s_off[l] + atomicAdd(&s_cur[l], 1)] = bz[z0 + i];
    }
    __syncthreads();
    for (int l = tid; l < ncell; l += kThreads) {
        const int cls = sort_short(seg0 + s_off[l], s_off[l + 1] - s_off[l]);
        if (cls == 1) s_q[atomicAdd(&s_n[0], 1)] = (uint16_t)l;
        else if (cls == 2) s_q[ncell - 1 - atomicAdd(&s_n[1], 1)] = (uint16_t)l;
    }
    __syncthreads();
    // the block's long segments join the queues with one atomic each
    if (tid == 0) {
        s_base[0] = s_n[0] ? atomicAdd(long_count, s_n[0]) : 0;
        s_base[1] = s_n[1] ? atomicAdd(long_count + 1, s_n[1]) : 0;
    }
    __syncthreads();
    for (int i = tid; i < s_n[0]; i += kThreads) long_cells[s_base[0] + i] = (int32_t)(c0 + s_q[i]);
    for (int i = tid; i < s_n[1]; i += kThreads)
        long_cells[m - 1 - (s_base[1] + i)] = (int32_t)(c0 + s_q[ncell - 1 - i]);
    if (staged_in_smem)
        for (int32_t i = tid; i < nb; i += kThreads) zs[z0 + i] = s_z[i];
}

// Bitonic network over 32 * EPL heights held by one warp: element e * 32 +
// lane in v[e] of that lane.  Partners 32 or more apart sit in the same
// lane's registers; nearer ones are exchanged by shuffles.
template <int EPL>
__device__ __forceinline__ void warp_bitonic(float (&v)[EPL], int lane) {
    constexpr int L = 32 * EPL;
#pragma unroll
    for (int size = 2; size <= L; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {
#pragma unroll
                for (int e = 0; e < EPL; ++e) {
                    const int f = e ^ (stride >> 5);
                    if (f > e) {
                        const bool up = ((e * 32) & size) == 0;
                        const float a = v[e], b = v[f];
                        const float lo = fminf(a, b), hi = fmaxf(a, b);
                        v[e] = up ? lo : hi;
                        v[f] = up ? hi : lo;
                    }
                }
            } else {
                const bool lower = (lane & stride) == 0;
#pragma unroll
                for (int e = 0; e < EPL; ++e) {
                    const float y = __shfl_xor_sync(0xffffffffu, v[e], stride);
                    const bool up = ((e * 32 + lane) & size) == 0;
                    v[e] = lower == up ? fminf(v[e], y) : fmaxf(v[e], y);
                }
            }
        }
    }
}

// One segment of n <= 32 * EPL heights sorted by one warp in registers
// (coalesced loads and stores, padded with +inf).
template <int EPL>
__device__ __forceinline__ void warp_sort_segment(float *__restrict__ zs, int32_t s, int32_t n,
                                                  int lane) {
    float v[EPL];
#pragma unroll
    for (int e = 0; e < EPL; ++e) v[e] = e * 32 + lane < n ? zs[s + e * 32 + lane] : INFINITY;
    warp_bitonic<EPL>(v, lane);
#pragma unroll
    for (int e = 0; e < EPL; ++e)
        if (e * 32 + lane < n) zs[s + e * 32 + lane] = v[e];
}

// One block per huge segment (more than kWarpSort heights).  Up to kHugeStage
// heights are sorted by a bitonic network in shared memory (padded with
// +inf), a barrier between its steps.  Longer segments (a cloud that puts
// most of its points in one cell: invalid returns written as the origin, a
// dense pole) are cut into chunks of kHugeStage heights, each sorted the
// same way in place, and the sorted runs are then merged pairwise, doubling
// their length per pass, between the segment and its copy in global scratch:
// every height finds its output position from its index in its own run and
// a binary search in the partner run (strictly smaller heights of the right
// run before it, equal or smaller ones of the left run before a right one),
// so a pass costs O(n log n) and the whole sort O(n log^2 n).
constexpr int kHugeThreads = 512;
constexpr int kHugeStage = 8192;

// Sorts buf[0, L) ascending, L a power of two; called by the whole block.
__device__ void block_bitonic(float *buf, int L) {
    const int tid = threadIdx.x;
    for (int size = 2; size <= L; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            // pair k compares i = 2 stride (k / stride) + k % stride with i + stride
            for (int k = tid; k < L / 2; k += kHugeThreads) {
                const int i = 2 * stride * (k / stride) + k % stride, jx = i + stride;
                const float x = buf[i], y = buf[jx];
                const bool up = (i & size) == 0;
                if ((x > y) == up) { buf[i] = y; buf[jx] = x; }
            }
            __syncthreads();
        }
    }
}

// Sorts the n heights at seg (global memory) through buf; whole block.
__device__ void block_sort_chunk(float *__restrict__ seg, int32_t n, float *buf) {
    const int tid = threadIdx.x;
    int L = 2 * kWarpSort;
    while (L < n) L <<= 1;
    for (int i = tid; i < L; i += kHugeThreads) buf[i] = i < n ? seg[i] : INFINITY;
    __syncthreads();
    block_bitonic(buf, L);
    for (int i = tid; i < n; i += kHugeThreads) seg[i] = buf[i];
    __syncthreads();
}

// Both queues in one launch: the blocks take the block-sort segments (from
// the back of long_cells) in turn first, then their warps take the segments of
// 17 .. kWarpSort heights (from the front), each sorted in a warp's registers.
__global__ void __launch_bounds__(kHugeThreads, 3)
k_sort_queued(const int32_t *__restrict__ start, float *__restrict__ zs,
              float *__restrict__ scratch, const int32_t *__restrict__ long_count,
              const int32_t *__restrict__ long_cells, int64_t m) {
    __shared__ float buf[kHugeStage];
    const int tid = threadIdx.x;
    const int total = long_count[1];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int32_t c = long_cells[m - 1 - t];
        const int32_t s = start[c], n = start[c + 1] - s;
        if (n <= kHugeStage) {
            block_sort_chunk(zs + s, n, buf);
            continue;
        }
        for (int64_t c0 = 0; c0 < n; c0 += kHugeStage)
            block_sort_chunk(zs + s + c0, (int32_t)min((int64_t)kHugeStage, (int64_t)n - c0), buf);
        float *src = zs + s, *dst = scratch + s;
        for (int64_t w = kHugeStage; w < n; w *= 2) {
            for (int64_t i = tid; i < n; i += kHugeThreads) {
                const int64_t run = i / w, a0 = (run & ~(int64_t)1) * w;
                const int64_t a1 = min(a0 + w, (int64_t)n), b1 = min(a0 + 2 * w, (int64_t)n);
                const float x = src[i];
                int64_t lo, hi, pos;
                if ((run & 1) == 0) {
                    lo = a1; hi = b1;                       // right run: heights < x
                    while (lo < hi) {
                        const int64_t mid = (lo + hi) >> 1;
                        if (src[mid] < x) lo = mid + 1; else hi = mid;
                    }
                    pos = i + (lo - a1);
                } else {
                    lo = a0; hi = a1;                       // left run: heights <= x
                    while (lo < hi) {
                        const int64_t mid = (lo + hi) >> 1;
                        if (src[mid] <= x) lo = mid + 1; else hi = mid;
                    }
                    pos = a0 + (i - a1) + (lo - a0);
                }
                dst[pos] = x;
            }
            __syncthreads();
            float *tmp = src; src = dst; dst = tmp;
        }
        if (src != zs + s) {
            for (int64_t i = tid; i < n; i += kHugeThreads) zs[s + i] = src[i];
            __syncthreads();
        }
    }
    const int lane = tid & 31, wib = tid >> 5;
    constexpr int kWarps = kHugeThreads / 32;
    const int n_long = long_count[0];
    for (int t = blockIdx.x * kWarps + wib; t < n_long; t += gridDim.x * kWarps) {
        const int32_t c = long_cells[t];
        const int32_t s = start[c], n = start[c + 1] - s;
        if (n <= 32) warp_sort_segment<1>(zs, s, n, lane);
        else if (n <= 64) warp_sort_segment<2>(zs, s, n, lane);
        else if (n <= 128) warp_sort_segment<4>(zs, s, n, lane);
        else warp_sort_segment<8>(zs, s, n, lane);
    }
}

// Blocks of the long-segment sorts: a resident wave (three blocks per SM).
int sm_count() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// The statistics block starts from zero (the partition's passes add to it),
// then takes the call's sizes; the z bounds start empty.  The slice stack's
// uniqueness rows, tile queue and count of finished CTAs of the same
// workspace are cleared here too, a launch ahead of their use.
__global__ void k_partition_init(int32_t *zkeys, tct_stats *stats, int64_t n, int32_t n_slices,
                                 int32_t *upre, uint32_t *ubits, int32_t *queue) {
    int32_t *w = reinterpret_cast<int32_t *>(stats);
    for (int i = threadIdx.x; i < (int)(sizeof(tct_stats) / sizeof(int32_t)); i += blockDim.x)
        w[i] = 0;
    for (int i = threadIdx.x; i <= TCT_MAX_SLICES; i += blockDim.x) upre[i] = 0;
    for (int i = threadIdx.x; i < 4 * (TCT_MAX_SLICES + 1); i += blockDim.x) ubits[i] = 0;
    if (threadIdx.x == 0) queue[0] = queue[1] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        zkeys[0] = float_key(INFINITY);
        zkeys[1] = float_key(-INFINITY);
        stats->n_points = n;
        stats->n_slices = n_slices;
    }
}


// tct_build alone: thread per cell walks the slices with the monotone pointer.
__global__ void __launch_bounds__(kThreads)
k_elevations(const int32_t *__restrict__ start, const float *__restrict__ zs, int64_t m,
             int n_slices, float d_s, float z_min_given, bool zmin_from_data,
             const int32_t *__restrict__ zkeys, float *__restrict__ ground,
             float *__restrict__ ceil) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    float z_min = z_min_given;
    if (zmin_from_data) {
        z_min = key_float(zkeys[0]);
        if (!isfinite(z_min)) z_min = 0.0f;
    }
    int32_t p = start[c];
    const int32_t e = start[c + 1];
    float zg = -INFINITY;
    float zc = p < e ? zs[p] : INFINITY;
    for (int k = 0; k < n_slices; ++k) {
        const float h = __fmaf_rn((float)(k + 1), d_s, z_min);
        while (zc <= h) {
            zg = zc;
            ++p;
            zc = p < e ? zs[p] : INFINITY;
        }
        __stcs(&ground[(int64_t)k * m + c], zg);
        __stcs(&ceil[(int64_t)k * m + c], zc);
    }
}

int grid_blocks(int64_t work_items, int per_block) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t b = (work_items + per_block - 1) / per_block;
    int64_t cap = (int64_t)sms * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

cudaError_t launch_bounds(const float *xyz, int64_t n, int stride, float *out6, tct_stats *stats,
                          cudaStream_t s) {
    int32_t *keys6 = reinterpret_cast<int32_t *>(out6);
    k_bounds_init<<<1, 32, 0, s>>>(keys6, stats, n);
    if (n > 0) k_bounds<<<grid_blocks(n, kThreads * 4), kThreads, 0, s>>>(xyz, n, stride, keys6, stats);
    k_bounds_finish<<<1, 32, 0, s>>>(out6, stats);
    count_launches(n > 0 ? 3 : 2);
    return cudaGetLastError();
}

cudaError_t launch_partition(const float *xyz, int64_t n, int stride, const tct_grid &g,
                             const Workspace &ws, tct_stats *stats, cudaStream_t s) {
    const int64_t m = (int64_t)g.W * g.H;
    const GridDev gd = grid_dev(g);
    const bool vec = (reinterpret_cast<uintptr_t>(xyz) & 15u) == 0;
    // the cell counts, bucket cursors and long-segment counts lie back to back
    cudaError_t e = cudaMemsetAsync(ws.cnt, 0,
                                    reinterpret_cast<char *>(ws.long_count + 2) -
                                        reinterpret_cast<char *>(ws.cnt), s);
    if (e != cudaSuccess) return e;
    k_partition_init<<<1, 256, 0, s>>>(ws.zkeys, stats, n, g.n_slices, ws.upre, ws.ubits,
                                       ws.queue);
    const int64_t work = vec ? n / 4 + 1 : n;
    if (n > 0)
        k_count<<<grid_blocks(work, kThreads), kThreads, 0, s>>>(xyz, n, stride, vec, gd, ws.cnt,
                                                                 ws.zkeys, stats);
    const int scan_launches = launch_scan(ws, m, ws.zkeys, stats, s);
    if (n > 0) {
        const int blog = bucket_log(m, sm_count());
        k_bucket<<<grid_blocks(work, kThreads), kThreads, 0, s>>>(xyz, n, stride, vec, gd, ws.cnt,
                                                                  ws.start, ws.bcur, ws.scratch,
                                                                  ws.bucket_l, ws.zs, blog);
        const unsigned nbk = (unsigned)((m + (1 << blog) - 1) >> blog);
        k_bucket_sort<<<nbk, kThreads, 0, s>>>(ws.start, m, ws.bcur, ws.scratch, ws.bucket_l, ws.zs,
                                               ws.long_count, ws.long_cells, blog);
        k_sort_queued<<<3 * sm_count(), kHugeThreads, 0, s>>>(ws.start, ws.zs, ws.scratch,
                                                              ws.long_count, ws.long_cells, m);
    }
    count_launches((n > 0 ? 5 : 1) + scan_launches);
    return cudaGetLastError();
}

cudaError_t launch_partition_batched(const BatchPointsIn *maps, int n_maps, int chunk,
                                     int64_t total_cells, const Workspace &ws, cudaStream_t s) {
    if (n_maps < 1 || n_maps > TCT_MAX_BATCH || chunk < 4 || chunk % 4) return cudaErrorInvalidValue;
    PointBatch b;
    b.n_maps = n_maps;
    b.chunk = chunk;
    int64_t blocks = 0;
    for (int i = 0; i < n_maps; ++i) {
        PointMap &m = b.maps[i];
        m.xyz = maps[i].xyz;
        m.n = maps[i].n;
        m.stride = maps[i].stride;
        m.vec = (reinterpret_cast<uintptr_t>(maps[i].xyz) & 15u) == 0 ? 1 : 0;
        m.g = grid_dev(maps[i].grid);
        m.cell_off = maps[i].cell_off;
        m.zkeys = maps[i].zkeys;
        m.stats = maps[i].stats;
        m.block_start = (int32_t)blocks;
        blocks += (maps[i].n + chunk - 1) / chunk;
    }
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    const int64_t m = total_cells;
    cudaError_t e = cudaMemsetAsync(ws.cnt, 0,
                                    reinterpret_cast<char *>(ws.long_count + 2) -
                                        reinterpret_cast<char *>(ws.cnt), s);
    if (e != cudaSuccess) return e;
    int launches = 1;   // the long-segment sorts
    if (blocks > 0) {
        k_count_batched<<<(unsigned)blocks, kThreads, 0, s>>>(b, ws.cnt);
        ++launches;
    }
    launches += launch_scan(ws, m, nullptr, nullptr, s);
    if (blocks > 0) {
        const int blog = bucket_log(m, sm_count());
        k_bucket_batched<<<(unsigned)blocks, kThreads, 0, s>>>(b, ws.cnt, ws.start, ws.bcur,
                                                               ws.scratch, ws.bucket_l, ws.zs,
                                                               blog);
        const unsigned nbk = (unsigned)((m + (1 << blog) - 1) >> blog);
        k_bucket_sort<<<nbk, kThreads, 0, s>>>(ws.start, m, ws.bcur, ws.scratch, ws.bucket_l, ws.zs,
                                               ws.long_count, ws.long_cells, blog);
        launches += 2;
    }
    k_sort_queued<<<3 * sm_count(), kHugeThreads, 0, s>>>(ws.start, ws.zs, ws.scratch,
                                                          ws.long_count, ws.long_cells, m);
    count_launches(launches);
    return cudaGetLastError();
}

cudaError_t launch_elevations(const tct_grid &g, const Workspace &ws, float *ground, float *ceil,
                              cudaStream_t s) {
    const int64_t m = (int64_t)g.W * g.H;
    k_elevations<<<(unsigned)((m + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        ws.start, ws.zs, m, g.n_slices, g.d_s, g.z_min, (g.flags & TCT_GRID_ZMIN_FROM_DATA) != 0,
        ws.zkeys, ground, ceil);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace tct
