// tct_internal.cuh -- private declarations shared by the libtct translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tct.h"

namespace tct {

constexpr int kMaxK = 2 * TCT_MAX_KERNEL_RADIUS + 1;

// Order-preserving map between float and int32 (non-NaN floats): a < b as
// floats iff key(a) < key(b) as signed ints.
__host__ __device__ __forceinline__ int32_t float_key(float f) {
#ifdef __CUDA_ARCH__
    int32_t i = __float_as_int(f);
#else
    union { float f; int32_t i; } u; u.f = f; int32_t i = u.i;
#endif
    return i ^ ((i >> 31) & 0x7fffffff);
}
__host__ __device__ __forceinline__ float key_float(int32_t k) {
    int32_t i = k ^ ((k >> 31) & 0x7fffffff);
#ifdef __CUDA_ARCH__
    return __int_as_float(i);
#else
    union { float f; int32_t i; } u; u.i = i; return u.f;
#endif
}

#ifdef __CUDACC__
// The chain of Sec. III-C: slice k is kept when it is unique against the last
// kept slice (uniqueness row p + 1: below pre[k], or its bit in bits[4 k ..]),
// an end slice also with TCT_KEEP_ENDS.  One thread; returns the slices kept.
__device__ __forceinline__ int chain_walk(int n_slices, const int32_t *pre, const uint32_t *bits,
                                          uint32_t flags, uint8_t *keep) {
    int p = -1, kept = 0;
    for (int k = 0; k < n_slices; ++k) {
        const int row = p + 1;
        bool u = row < pre[k] || ((bits[4 * k + (row >> 5)] >> (row & 31)) & 1u);
        if ((flags & TCT_KEEP_ENDS) && (k == 0 || k == n_slices - 1)) u = true;
        keep[k] = u ? 1 : 0;
        if (u) { p = k; ++kept; }
    }
    return kept;
}
#endif

// Workspace carved from the caller's buffer; offsets are 256-byte aligned.
struct Workspace {
    int32_t *cnt;       // [HW]   points per cell (zero between builds)
    int32_t *start;     // [HW+1] exclusive prefix of cnt
    int32_t *partial;   // [n_scan_blocks + 1]
    float *zs;          // [P]    point heights grouped by cell, sorted per cell
    float *scratch;     // [P]    heights by bucket before the bucket sort; later the
                        //        copy of very long segments while they are sorted
    uint16_t *bucket_l; // [P]    each bucketed height's cell within its bucket
    int32_t *bcur;      // [HW / kBucket + 1] fill level of each bucket (zero between builds)
    int32_t *long_count;  // [2]  cells queued for the warp sort, for the block sort
    int32_t *long_cells;  // [HW] their indices (warp sort from the front, block sort from the back)
    int32_t *zkeys;     // [2]    ordered-int min / max z of the finite points
    int32_t *upre;      // [128]  per slice: bits [0, upre) of the uniqueness row set
    uint32_t *ubits;    // [128][4] per slice: further uniqueness bits
    tct_stats *stats;   // fallback stats block when the caller passes none
    int32_t *queue;     // [2]    tile queue of the persistent slice-stack kernel, and its
                        //        count of finished CTAs (the last one runs the chain)
    int32_t *falls;     // [1]    set when a given ground layer falls from a slice to the next
    size_t bytes;
};

constexpr int kScanTile = 4096;   // cells per scan block
// Buckets of the partition: 2^bucket_log consecutive cells, 64 .. 1024,
// the largest that still gives each SM at least four buckets to sort.
constexpr int kBucketLogMin = 6, kBucketLogMax = 10;
constexpr int kBucket = 1 << kBucketLogMax;   // the largest bucket
inline int bucket_log(int64_t cells, int sms) {
    int lg = kBucketLogMin;
    while (lg < kBucketLogMax && (cells >> (lg + 1)) >= 4 * (int64_t)sms) ++lg;
    return lg;
}
// Bucket cursors the workspace holds: enough for the smallest buckets.
inline int64_t n_buckets_max(int64_t cells) {
    return (cells + (1 << kBucketLogMin) - 1) >> kBucketLogMin;
}

Workspace carve(void *base, const tct_grid &g, int64_t n_points);

// Inflation kernel and per-call constants of Sec. III-B in float32.
struct EvalConsts {
    float d_min, d_ref, theta_b, theta_s, c_b, alpha_d, alpha_b, alpha_s;
    float inv2r;        // 1 / (2 r_g)
    float inv_ts;       // 1 / theta_s
    float inv_tb;       // 1 / theta_b
    int32_t patch_radius;
    int32_t count_thresh;   // p_s > theta_p  <=>  gentle count > count_thresh
    int32_t rk;             // inflation window radius
    uint32_t flags;
    float K[kMaxK * kMaxK]; // weights, row-major (n, m), (2 rk + 1)^2 used
};

int make_eval_consts(const tct_grid &g, const tct_params &p, EvalConsts *c);

// Host-side count of kernel launches (tct_launch_count).
void count_launches(int n);

// Arguments of the slice-stack kernels (tct_stack.cu, tct_stack_inc.cu).
struct StackArgs {
    int32_t W, H, N;
    float d_s, z_min;
    int32_t zmin_from_data;
    const int32_t *zkeys;        // ordered-int z bounds from the count pass
    const int32_t *start;        // per-cell segments (build path)
    const float *zs;
    const float *gin, *cin;      // given layers (evaluate path)
    int32_t *falls;              // set by the kernel when a given ground falls
    uint8_t *keep;               // with done: the chain runs in the stack kernel's last CTA
    int32_t *done;               // finished CTAs (zero at launch)
    int32_t split;               // slice ranges per tile (0 or 1: one; single-map build path)
    float *ground, *ceil, *cost, *aux;
    uint8_t *mask;
    int32_t *upre;
    uint32_t *ubits;
    tct_stats *stats;
    EvalConsts c;
};

// launchers (tct_build.cu)
cudaError_t launch_bounds(const float *xyz, int64_t n, int stride, float *out6,
                          tct_stats *stats, cudaStream_t s);
cudaError_t launch_partition(const float *xyz, int64_t n, int stride, const tct_grid &g,
                             const Workspace &ws, tct_stats *stats, cudaStream_t s);
// Batches: the maps' cells are concatenated (map i starts at cell_off), so one
// scan over all of them gives every point's position in the shared zs.
struct BatchPointsIn {
    const float *xyz;
    int64_t n;
    int32_t stride;
    tct_grid grid;
    int64_t cell_off;
    int32_t *zkeys;      // initialised by the caller
    tct_stats *stats;    // zeroed by the caller
};
cudaError_t launch_partition_batched(const BatchPointsIn *maps, int n_maps, int chunk,
                                     int64_t total_cells, const Workspace &ws, cudaStream_t s);
cudaError_t launch_elevations(const tct_grid &g, const Workspace &ws, float *ground,
                              float *ceil, cudaStream_t s);

// launchers (tct_stack.cu)
// tile: TCT_TILE_AUTO or one of the TCT_TILE_* shapes.
// lists: the workspace launch_partition has just filled (its first launch
// also cleared that workspace's uniqueness rows and tile queue).
// Given layers (lists NULL) run the incremental kernel too when it supports
// the radii and no aux output is asked for; queue and falls are then that
// call's tile queue and falling-ground flag.
// keep: with lists, the keep flags the incremental kernel's last CTA writes
// by the chain of Sec. III-C; *chained tells whether it did (otherwise the
// caller launches the chain).
cudaError_t launch_stack(const tct_grid &g, const EvalConsts &c, const Workspace *lists,
                         const int32_t *zkeys, const float *gin, const float *cin,
                         float *ground, float *ceil, float *cost, uint8_t *mask, float *aux,
                         int32_t *upre, uint32_t *ubits, tct_stats *stats, cudaStream_t s,
                         int tile = TCT_TILE_AUTO, int32_t *queue = nullptr,
                         int32_t *falls = nullptr, uint8_t *keep = nullptr,
                         bool *chained = nullptr);
// The incremental kernel for the build path; returns cudaErrorNotSupported
// when no instance matches the window radii (the caller then falls back).
// tile: one of the TCT_TILE_* shapes.
bool inc_supported(const EvalConsts &c, int n_slices);
cudaError_t launch_stack_inc(const StackArgs &a, int32_t *queue, int tile, cudaStream_t s);
// One persistent launch over the tiles of n_maps maps (largest first);
// queue must be zero when the launch starts.
// The automatic tile shape of the incremental stack: 32 x 32 when the 64 x 64
// tiles of all maps number fewer than small_tiles64 per SM, otherwise the
// shape with the least work per SM over whole waves of resident CTAs.
int choose_tile(const EvalConsts &c, int n_maps, const StackArgs *maps, int64_t small_tiles64);
cudaError_t launch_stack_batched(const EvalConsts &c, int n_maps, const StackArgs *maps,
                                 int32_t *queue, int tile, int ctas_per_sm, cudaStream_t s);
// The generic (any window radius) slice stack for one map of the build path;
// the map's uniqueness rows must be zero and a.c its constants.
cudaError_t launch_stack_generic(const StackArgs &a, cudaStream_t s);
cudaError_t launch_chain(int n_slices, const int32_t *upre, const uint32_t *ubits,
                         uint32_t flags, uint8_t *keep, tct_stats *stats, cudaStream_t s);

}  // namespace tct
