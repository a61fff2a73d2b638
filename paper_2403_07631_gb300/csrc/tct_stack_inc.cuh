// tct_stack_inc.cuh -- the build-path slice stack, incremental over slices.
//
// Same computation as k_stack in tct_stack.cu (Sec. III-B Eq. 1-6 per slice,
// the uniqueness bits of Sec. III-C), specialised for compile-time window
// radii and organised around one observation: consecutive tomogram slices
// differ only where the plane passed a point (the redundancy Sec. III-C
// removes afterwards).  The CTA keeps, in shared memory, the state of every
// stage for its tile (64 x 64, 64 x 56, 64 x 40 or 128 x 56 cells with strips
// of 8 rows, or 32 x 32 cells with strips of 2 rows for small maps) and the
// halo and,
// slice after slice,
//   1. lists the cells whose next height the plane passed and advances their
//      pointers into the sorted z segments, the list spread over all threads;
//      per-row bit words mark the cells whose ground or ceiling changed;
//   2. recomputes the gentle flags (Eq. 2) only in 32-column row blocks whose
//      ground stencil changed (found one lane per block, listed, then taken
//      by all warps in turn);
//   3. recomputes c^init (Eq. 1, 3-5) only in the row blocks where one of its
//      inputs changed (listed the same way), marking the cells whose value
//      changed;
//   4. re-inflates (Eq. 6) a warp's 32-column strip only when a c^init in its
//      window changed, otherwise keeps the previous c^T (bit-identical
//      inputs give bit-identical results; when few strips changed, their
//      halves are spread over all warps), and accumulates the uniqueness
//      bits, reading earlier costs back only for cells whose run holds a
//      higher cost than the current one,
// and writes all four layers of every slice.  Work follows the changes,
// while the writes of every slice's layers (the algorithmic bytes) are
// always done.  Given layers (tct_evaluate) take the place of step 1: each
// slice's ground and ceiling of the region are read and compared with the
// previous slice's, and only cost and mask are written.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "tct_internal.cuh"

namespace tct {
namespace inc {

constexpr uint32_t kSat = 0xffffu;   // saturated 16-bit pointer offset

// Tile of TW x TH cells: TW/32 column halves x TH/KS strips of 32 x KS
// cells, one warp each (a thread holds KS cells of one column).
template <int RK, int RP, int TW, int TH, int KS>
struct Geo {
    static_assert(TW % 32 == 0 && TH % KS == 0 && KS % 2 == 0 && KS <= 8, "tile made of 32 x KS strips");
    static constexpr int NHALF = TW / 32;
    static constexpr int NW = NHALF * (TH / KS);
    static_assert(NW <= 32, "one bit per warp in the inflation mask");
    static constexpr int NT = 32 * NW;
    static constexpr int HE = RK + RP + 1;
    static constexpr int EW = TW + 2 * HE, EH = TH + 2 * HE;      // elevation region
    static constexpr int NE = EW * EH;
    static constexpr int GW = EW - 2, GH = EH - 2;                // gentle region
    static constexpr int CW = TW + 2 * RK, CH = TH + 2 * RK;      // c^init region
    static constexpr int EWW = (EW + 31) / 32 + 1;                // change words per row (+pad)
    static constexpr int GWW = (GW + 31) / 32 + 1;                // gentle words per row (+pad)
    static constexpr int CWW = (CW + 31) / 32 + 1;                // c^init change words (+pad)
    static constexpr int GPASS = (GW + 31) / 32, CPASS = (CW + 31) / 32;
    static constexpr int WORDS = 4 * EH * EWW + 2 * GH * GWW + CH * CWW;
    static_assert(NE < 65536, "16-bit indices of the elevation region");
    static_assert(NE % 4 == 0, "the elevation region is read four cells at a time");
    static constexpr size_t smem_bytes() {
        // state, change words, 16-bit pointer offsets, 16-bit list of the
        // cells a plane passed
        return sizeof(float) * (2 * NE + CW * CH) + sizeof(uint32_t) * WORDS +
               2 * (((sizeof(uint16_t) * NE + 15) / 16) * 16);
    }
};

// Shared state of the per-slice counters, kept in static shared memory.
struct SliceCounters {
    int32_t nlist[3];                  // cells a plane passed, slice k in nlist[k % 3]
    int32_t nwork[2];                  // dirty row blocks: gentle flags, c^init
    uint32_t infl;                     // warps whose strip is re-inflated this slice
    int32_t upre[TCT_MAX_SLICES + 1];
    int32_t valid[TCT_MAX_SLICES + 1];
    int32_t trav[TCT_MAX_SLICES + 1];
};

__device__ __forceinline__ float max3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Index of the first height greater than z in the sorted segment [s, e).
__device__ __forceinline__ int32_t upper_bound(const float *__restrict__ zs, int32_t s, int32_t e,
                                               float z) {
    while (s < e) {
        const int32_t m = s + ((e - s) >> 1);
        if (zs[m] <= z) s = m + 1;
        else e = m;
    }
    return s;
}

// Eq. 6 for NQ cells of one column: acc[q] = max over the window of K * c^init
// for the cell of row q, where row0 points at the cell's column (less R_K) in
// the first of the NQ + 2 R_K c^init rows it reads, CW floats apart.  Every
// c^init row is loaded once, folded into pair maxima max(c(j-d), c(j+d)),
// weighted and reduced with the three-input max.
template <int RK, int NQ, int CW>
__device__ __forceinline__ void inflate_column(const float *row0, const EvalConsts &c,
                                               float (&acc)[NQ]) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0f;
    // wide windows (R_K > 8) keep the row loop rolled: the full unrolling of
    // a 25 x 25 window costs minutes of compilation
#pragma unroll(RK <= 8 ? NQ + 2 * RK : 1)
    for (int rr = 0; rr < NQ + 2 * RK; ++rr) {
        const float *row = row0 + rr * CW;
        float P[RK + 1];
        P[0] = row[RK];
#pragma unroll
        for (int d = 1; d <= RK; ++d) P[d] = fmaxf(row[RK - d], row[RK + d]);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int n = rr - RK - q;       // row offset of this row for cell q
            if (n < -RK || n > RK) continue;
            const int an = n < 0 ? -n : n;
            const float *Kr = c.K + (an + RK) * (2 * RK + 1) + RK;
            // the disc d^2 < (RK+1)^2 holds every positive weight
#pragma unroll
            for (int d = 0; d <= RK; d += 2) {
                if (d * d + an * an >= (RK + 1) * (RK + 1)) break;
                const float t0 = Kr[d] * P[d];
                const float t1 = (d + 1 <= RK && (d + 1) * (d + 1) + an * an < (RK + 1) * (RK + 1))
                                     ? Kr[d + 1] * P[d + 1] : 0.0f;
                acc[q] = max3(acc[q], t0, t1);
            }
        }
    }
}

// The per-map fields the incremental slice stack reads and writes.
struct IncMap {
    int32_t W, H, N;
    float d_s, z_min;
    int32_t zmin_from_data;
    const int32_t *zkeys;        // ordered-int z bounds from the count pass
    const int32_t *start;        // per-cell segments
    const float *zs;
    const float *gin, *cin;      // given layers instead of segments (evaluate alone)
    int32_t *falls;              // set when a given ground falls from one slice to the next
    float *ground, *ceil, *cost;
    uint8_t *mask;
    int32_t *upre;
    uint32_t *ubits;
    tct_stats *stats;
    uint8_t *keep;               // keep flags the last CTA writes (with BatchArgs::done)
};

// One tile (TW x TH cells at tx0, ty0) of one map over its slices
// [k_begin, k_end), by one CTA of Geo::NT threads.  smem is the dynamic buffer
// of smem_bytes(); the caller synchronises before the buffer is used for
// another tile.  The first slice of the range is computed in full (as slice 0
// always is), so a range may start anywhere; the uniqueness rows are
// accumulated only when uniq is set (the whole slice range), otherwise they
// are left to a pass over the finished layers.
template <int RK, int RP, int TW, int TH, int KS>
__device__ __forceinline__ void stack_tile(const IncMap &a, const EvalConsts &c, int tx0, int ty0,
                                           unsigned char *smem, SliceCounters &counters,
                                           int k_begin, int k_end, bool uniq) {
    using G = Geo<RK, RP, TW, TH, KS>;
    constexpr int kStrip = KS;             // rows of a thread's inflation strip
    constexpr int kNT = G::NT, kNW = G::NW;
    int32_t *s_upre = counters.upre, *s_valid = counters.valid, *s_trav = counters.trav;

    float *sEG = reinterpret_cast<float *>(smem);          // ground (state)
    float *sZC = sEG + G::NE;                                // next z = ceiling (state)
    float *sCI = sZC + G::NE;                                // c^init (state)
    uint32_t *sChgG0 = reinterpret_cast<uint32_t *>(sCI + G::CW * G::CH);   // ground changed, 2 buffers
    uint32_t *sChgC0 = sChgG0 + 2 * G::EH * G::EWW;          // ceiling changed, 2 buffers
    uint32_t *sGB = sChgC0 + 2 * G::EH * G::EWW;             // gentle bits (state)
    uint32_t *sGChg = sGB + G::GH * G::GWW;
    uint32_t *sCIChg = sGChg + G::GH * G::GWW;
    uint16_t *sOff = reinterpret_cast<uint16_t *>(sCIChg + G::CH * G::CWW);
    uint16_t *sList = sOff + ((sizeof(uint16_t) * G::NE + 15) / 16) * 8;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t HW = (int64_t)a.W * a.H;
    const float ts2 = c.theta_s * c.theta_s;   // m^grad < theta_s  <=>  m^2 < theta_s^2
    const float inv_ts2 = c.inv_ts * c.inv_ts;
    // the columns a 32-wide block or strip reads, as masks of its own change
    // word (Lo) and of the next one (Hi)
    static_assert(RP + 2 < 32 && 2 * RP < 32 && 2 * RK < 32, "windows span two change words");
    constexpr uint32_t kGrndLo = ~0u << RP, kGrndHi = (1u << (RP + 2)) - 1u;
    constexpr uint32_t kCeilLo = ~0u << (RP + 1), kCeilHi = (1u << (RP + 1)) - 1u;
    constexpr uint32_t kGentHi = (1u << (2 * RP)) - 1u;
    constexpr uint32_t kWinHi = (1u << (2 * RK)) - 1u;

    const bool given = a.gin != nullptr;
    if (tid < 3) counters.nlist[tid] = 0;
    if (tid == 0) counters.infl = 0;
    for (int i = tid; i <= TCT_MAX_SLICES; i += kNT) {
        s_upre[i] = 0;
        s_valid[i] = 0;
        s_trav[i] = 0;
    }
    for (int i = tid; i < G::WORDS; i += kNT) sChgG0[i] = 0;
    // each cell's lowest height; four cells a thread at a time, so that their
    // segment and height loads are in flight together
    constexpr int kInit = 4;
    for (int e0 = tid; e0 < G::NE; e0 += kInit * kNT) {
        int32_t b[kInit], end[kInit];
#pragma unroll
        for (int u = 0; u < kInit; ++u) {
            const int e = e0 + u * kNT;
            const int r = e / G::EW, s = e - r * G::EW;
            const int i = ty0 - G::HE + r, j = tx0 - G::HE + s;
            b[u] = end[u] = 0;
            if (!given && e < G::NE && i >= 0 && i < a.H && j >= 0 && j < a.W) {
                const int64_t cell = (int64_t)i * a.W + j;
                b[u] = a.start[cell];
                end[u] = a.start[cell + 1];
            }
        }
        float zc[kInit];
#pragma unroll
        for (int u = 0; u < kInit; ++u) zc[u] = b[u] < end[u] ? a.zs[b[u]] : INFINITY;
#pragma unroll
        for (int u = 0; u < kInit; ++u) {
            const int e = e0 + u * kNT;
            if (e < G::NE) {
                sEG[e] = -INFINITY;
                sZC[e] = zc[u];
                sOff[e] = 0;
            }
        }
    }
    float z_min = a.z_min;
    if (a.zmin_from_data) {
        z_min = key_float(a.zkeys[0]);
        if (!isfinite(z_min)) z_min = 0.0f;
    }

    // ---- per-thread state of its strip: 8 cells in one column ----
    const int half = warp % G::NHALF, strip = warp / G::NHALF;
    const int ts = 32 * half + lane;           // tile column
    const int tr0 = kStrip * strip;            // first tile row of the strip
    const int j_out = tx0 + ts;
    float cT[kStrip];
    uint32_t run_lo = 0, run_hi = 0;           // run starts, one byte per cell
    uint32_t validbits = 0, travbits = 0;
    int wvalid = 0, wtrav = 0;
    // the strip's cells inside the map, one bit per row
    const int rows_in = a.H - (ty0 + tr0);
    const uint32_t inmap = j_out >= a.W || rows_in <= 0 ? 0u
                           : (rows_in >= kStrip ? (1u << kStrip) - 1u : (1u << rows_in) - 1u);
#pragma unroll
    for (int q = 0; q < kStrip; ++q) cT[q] = 0.0f;
    auto run_get = [&](int q) -> int {
        return q < 4 ? (run_lo >> (8 * q)) & 0xffu : (run_hi >> (8 * (q - 4))) & 0xffu;
    };
    // per cell, an upper bound of c^T over its run before the current slice,
    // fp16 rounded up (never below the true maximum), kept while the flag
    // below is clear; with the flag it decides whether a cell can set a bit
    // of U(p, k-1) for p in its run; cells that cannot skip the walk
    uint32_t rmax[kStrip / 2];
#pragma unroll
    for (int q = 0; q < kStrip / 2; ++q) rmax[q] = 0xfc00fc00u;
    // per cell, exactly: no earlier cost of the run exceeds the current one
    // (constant and rising costs keep it; only then is the rounded bound needed)
    uint32_t runle = 0xffu;
    auto rmax_get = [&](int q) -> float {
        const unsigned short hb = (unsigned short)(rmax[q >> 1] >> (16 * (q & 1)));
        return __half2float(__ushort_as_half(hb));
    };
    auto rmax_set = [&](int q, unsigned short hb) {
        const int sh = 16 * (q & 1);
        rmax[q >> 1] = (rmax[q >> 1] & ~(0xffffu << sh)) | ((uint32_t)hb << sh);
    };
    auto run_set = [&](int q, int v) {
        if (q < 4) run_lo = (run_lo & ~(0xffu << (8 * q))) | ((uint32_t)v << (8 * q));
        else run_hi = (run_hi & ~(0xffu << (8 * (q - 4)))) | ((uint32_t)v << (8 * (q - 4)));
    };
    // U(p, kk) |= [c^T_kk < c^T_p] for p in the equal-ground run [r0, kk) of
    // each cell of the strip in `walk` (cT holds slice kk).  The earlier
    // slices' costs are read back from the output, four slices at a time, so
    // that the loads of a cell overlap; the bits gather in
    // registers and leave with one atomic per word and warp.  Called by the
    // whole warp.
    auto mark_run = [&](uint32_t walk, int kk) {
        if (!__any_sync(0xffffffffu, walk != 0)) return;
        uint32_t u0 = 0, u1 = 0, u2 = 0, u3 = 0;
        int lo = kk;
#pragma unroll
        for (int q = 0; q < kStrip; ++q)
            if ((walk >> q) & 1u) lo = min(lo, run_get(q));
        const int64_t cell0 = (int64_t)(ty0 + tr0) * a.W + j_out;
        for (int p = lo; p < kk; p += 4) {
#pragma unroll
            for (int q = 0; q < kStrip; ++q) {
                if (!((walk >> q) & 1u)) continue;
                const int r0 = run_get(q);
                const int64_t cell = cell0 + (int64_t)q * a.W;
                float cp[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    cp[u] = (p + u >= r0 && p + u < kk) ? a.cost[(int64_t)(p + u) * HW + cell]
                                                        : -INFINITY;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int bit = p + u + 1, w = bit >> 5;
                    const uint32_t m = cT[q] < cp[u] ? 1u << (bit & 31) : 0u;
                    u0 |= w == 0 ? m : 0u;
                    u1 |= w == 1 ? m : 0u;
                    u2 |= w == 2 ? m : 0u;
                    u3 |= w == 3 ? m : 0u;
                }
            }
        }
        u0 = __reduce_or_sync(0xffffffffu, u0);
        u1 = __reduce_or_sync(0xffffffffu, u1);
        u2 = __reduce_or_sync(0xffffffffu, u2);
        u3 = __reduce_or_sync(0xffffffffu, u3);
        if (lane == 0) {
            uint32_t *ub = a.ubits + 4 * kk;
            if (u0) atomicOr(ub + 0, u0);
            if (u1) atomicOr(ub + 1, u1);
            if (u2) atomicOr(ub + 2, u2);
            if (u3) atomicOr(ub + 3, u3);
        }
    };
    __syncthreads();

    for (int k = k_begin; k < k_end; ++k) {
        const bool first = k == k_begin;
        const float h = __fmaf_rn((float)(k + 1), a.d_s, z_min);
        uint32_t *sChgG = sChgG0 + (k & 1) * G::EH * G::EWW;
        uint32_t *sChgC = sChgC0 + (k & 1) * G::EH * G::EWW;

        // ---- 1. grounds and ceilings: advance the pointers past h ----
        // 1a. list the cells whose next height the plane passed: four cells a
        //     thread (one 16-byte load), one shared counter add per warp
        // three counters in turn: the next slice's is cleared here, where the
        // last reader of its previous use (two slices back) has passed the
        // previous barrier, and before this slice's barrier, past which the
        // next slice's listing may start (a quiet slice has no other barrier)
        int32_t *nlist = &counters.nlist[k % 3];
        if (tid == 0) {
            counters.nwork[0] = counters.nwork[1] = 0;   // read before the last barrier
            counters.nlist[(k + 1) % 3] = 0;
        }
        int n_pass;
        if (given) {
            // given layers: this slice's ground and ceiling of the region,
            // compared bit for bit with the previous slice's; four cells a
            // thread at a time, so that their loads are in flight together
            int moved = 0;
            const float *gk = a.gin + (int64_t)k * HW, *ck = a.cin + (int64_t)k * HW;
            constexpr int kLoad = 4;
            for (int e0 = tid; e0 < G::NE; e0 += kLoad * kNT) {
                float g[kLoad], cz[kLoad];
#pragma unroll
                for (int u = 0; u < kLoad; ++u) {
                    const int e = e0 + u * kNT;
                    const int r = e / G::EW, s = e - r * G::EW;
                    const int i = ty0 - G::HE + r, j = tx0 - G::HE + s;
                    g[u] = -INFINITY;
                    cz[u] = INFINITY;
                    if (e < G::NE && i >= 0 && i < a.H && j >= 0 && j < a.W) {
                        const int64_t cell = (int64_t)i * a.W + j;
                        g[u] = gk[cell];
                        cz[u] = ck[cell];
                    }
                }
#pragma unroll
                for (int u = 0; u < kLoad; ++u) {
                    const int e = e0 + u * kNT;
                    if (e >= G::NE) break;
                    const int r = e / G::EW, s = e - r * G::EW;
                    const float g0 = sEG[e], c0 = sZC[e];
                    const bool gch = __float_as_uint(g[u]) != __float_as_uint(g0);
                    const bool cch = __float_as_uint(cz[u]) != __float_as_uint(c0);
                    if (gch || cch) {
                        moved = 1;
                        sEG[e] = g[u];
                        sZC[e] = cz[u];
                        const uint32_t bit = 1u << (s & 31);
                        if (gch) atomicOr(&sChgG[r * G::EWW + (s >> 5)], bit);
                        if (cch) atomicOr(&sChgC[r * G::EWW + (s >> 5)], bit);
                        // a ground of the tile that falls: the run-based
                        // uniqueness bits below assume grounds never fall
                        if (g[u] < g0 && r >= G::HE && r < G::HE + TH && s >= G::HE && s < G::HE + TW)
                            *a.falls = 1;
                    }
                }
            }
            n_pass = __syncthreads_or(moved);
            if (tid == 0) counters.infl = 0;   // last read before this barrier
        } else {
        for (int base = 0; base < G::NE / 4; base += kNT) {
            const int e4 = base + tid;
            float4 z = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
            if (e4 < G::NE / 4) z = reinterpret_cast<const float4 *>(sZC)[e4];
            const bool p0 = z.x <= h, p1 = z.y <= h, p2 = z.z <= h, p3 = z.w <= h;
            if (__any_sync(0xffffffffu, p0 || p1 || p2 || p3)) {
                const uint32_t m0 = __ballot_sync(0xffffffffu, p0), m1 = __ballot_sync(0xffffffffu, p1);
                const uint32_t m2 = __ballot_sync(0xffffffffu, p2), m3 = __ballot_sync(0xffffffffu, p3);
                const uint32_t lt = (1u << lane) - 1u;
                const int n0 = __popc(m0), n01 = n0 + __popc(m1), n012 = n01 + __popc(m2);
                int at = 0;
                if (lane == 0) at = atomicAdd(nlist, n012 + __popc(m3));
                at = __shfl_sync(0xffffffffu, at, 0);
                const int e = 4 * e4;
                if (p0) sList[at + __popc(m0 & lt)] = (uint16_t)e;
                if (p1) sList[at + n0 + __popc(m1 & lt)] = (uint16_t)(e + 1);
                if (p2) sList[at + n01 + __popc(m2 & lt)] = (uint16_t)(e + 2);
                if (p3) sList[at + n012 + __popc(m3 & lt)] = (uint16_t)(e + 3);
            }
        }
        __syncthreads();
        if (tid == 0) counters.infl = 0;   // last read before this barrier
        n_pass = *nlist;
        }
        // A quiet slice (no plane passed a height of the region) changes no
        // ground, ceiling, gentle flag, c^init or c^T: it only writes the
        // layers again, with no uniqueness bit (Eq. 9 fails against an
        // identical slice) and the counts of the slice before.
        const bool quiet = !first && n_pass == 0;
        // 1b. advance the listed cells, spread evenly over the threads; each
        //     round reads the next four heights of the segment at once, so a
        //     cell that passes n heights waits for ceil(n / 4) loads, not n
        if (!quiet && !given) {
        for (int t = tid; t < n_pass; t += kNT) {
            const int e = sList[t];
            const int r = e / G::EW, s = e - r * G::EW;
            const int64_t cell = (int64_t)(ty0 - G::HE + r) * a.W + (tx0 - G::HE + s);
            const int32_t b = a.start[cell], end = a.start[cell + 1];
            const float zg0 = sEG[e];
            const uint32_t off = sOff[e];
            int32_t p = off < kSat ? b + (int32_t)off : upper_bound(a.zs, b, end, zg0);
            float zg = sZC[e], zc;     // zs[p] <= h: the ground is at least that
            for (;;) {
                const float z1 = p + 1 < end ? a.zs[p + 1] : INFINITY;
                const float z2 = p + 2 < end ? a.zs[p + 2] : INFINITY;
                const float z3 = p + 3 < end ? a.zs[p + 3] : INFINITY;
                const float z4 = p + 4 < end ? a.zs[p + 4] : INFINITY;
                if (z1 > h) { zc = z1; p += 1; break; }
                if (z2 > h) { zg = z1; zc = z2; p += 2; break; }
                if (z3 > h) { zg = z2; zc = z3; p += 3; break; }
                if (z4 > h) { zg = z3; zc = z4; p += 4; break; }
                zg = z4;
                p += 4;
            }
            sEG[e] = zg;
            sZC[e] = zc;
            sOff[e] = (uint16_t)min((uint32_t)(p - b), kSat);
            const uint32_t bit = 1u << (s & 31);
            if (zg != zg0) atomicOr(&sChgG[r * G::EWW + (s >> 5)], bit);
            atomicOr(&sChgC[r * G::EWW + (s >> 5)], bit);
        }
        __syncthreads();
        }

        // the next slice's change words are cleared here, a barrier ahead of their use
        {
            uint32_t *nG = sChgG0 + ((k + 1) & 1) * G::EH * G::EWW;
            uint32_t *nC = sChgC0 + ((k + 1) & 1) * G::EH * G::EWW;
            for (int i = tid; i < G::EH * G::EWW; i += kNT) { nG[i] = 0; nC[i] = 0; }
        }

        if (!quiet) {

        // ---- 2. gentle flags (Eq. 2: m^grad < theta_s) ----
        // 2a. one lane per 32-column row block: the block is dirty when a
        //     ground of its stencil rows (gr..gr+2, columns 32w..32w+33 of
        //     the elevation region) changed; dirty blocks are listed, clean
        //     ones get a zero change word
        for (int base = 32 * warp; base < G::GH * G::GPASS; base += 32 * kNW) {
            const int blk = base + lane;
            bool dirty = false;
            if (blk < G::GH * G::GPASS) {
                const int gr = blk / G::GPASS, w = blk - gr * G::GPASS;
                uint32_t v = 0;
#pragma unroll
                for (int dr = 0; dr < 3; ++dr)
                    v |= sChgG[(gr + dr) * G::EWW + w] | (sChgG[(gr + dr) * G::EWW + w + 1] & 3u);
                dirty = first || v != 0;
                if (!dirty) sGChg[gr * G::GWW + w] = 0;
            }
            const uint32_t m = __ballot_sync(0xffffffffu, dirty);
            if (m) {
                int at = 0;
                if (lane == 0) at = atomicAdd(&counters.nwork[0], __popc(m));
                at = __shfl_sync(0xffffffffu, at, 0);
                if (dirty) sList[at + __popc(m & ((1u << lane) - 1u))] = (uint16_t)blk;
            }
        }
        __syncthreads();
        // 2b. the listed blocks, spread over all warps
        {
            const int n_blk = counters.nwork[0];
#pragma unroll 1
            for (int t = warp; t < n_blk; t += kNW) {
                const int blk = sList[t];
                const int gr = blk / G::GPASS, w = blk - gr * G::GPASS;
                const int gs = 32 * w + lane;
                const int gsc = gs < G::GW ? gs : G::GW - 1;
                const float *ep = sEG + (gr + 1) * G::EW + (gsc + 1);
                const float e0 = ep[0], eL = ep[-1], eR = ep[1], eD = ep[-G::EW], eU = ep[G::EW];
                const bool ok = e0 > -INFINITY && eL > -INFINITY && eR > -INFINITY &&
                                eD > -INFINITY && eU > -INFINITY;
                const float gx = (eR - eL) * c.inv2r;
                const float gy = (eU - eD) * c.inv2r;
                const bool gentle = ok && __fmaf_rn(gx, gx, __fmul_rn(gy, gy)) < ts2 && gs < G::GW;
                const uint32_t bits = __ballot_sync(0xffffffffu, gentle);
                if (lane == 0) {
                    const uint32_t old = sGB[gr * G::GWW + w];
                    sGB[gr * G::GWW + w] = bits;
                    sGChg[gr * G::GWW + w] = first ? 0xffffffffu : (bits ^ old);
                }
            }
        }
        __syncthreads();

        // ---- the strip's own ground changes ----
        uint32_t gchbits = 0;
#pragma unroll
        for (int q = 0; q < kStrip; ++q) {
            const int er = tr0 + q + G::HE, es = ts + G::HE;
            const float eg = sEG[er * G::EW + es];
            if (first || ((sChgG[er * G::EWW + (es >> 5)] >> (es & 31)) & 1u)) {
                gchbits |= 1u << q;
                if (eg > -INFINITY) validbits |= 1u << q;
                else validbits &= ~(1u << q);
            }
        }

        // ---- 3. interval (Eq. 1), terrain (Eq. 3-4), initial cost (Eq. 5) ----
        // 3a. one lane per 32-column row block of the c^init region: dirty when
        //     a ground of rows cr+RP..cr+RP+2, the ceiling of row cr+RP+1 or a
        //     gentle flag of rows cr..cr+2RP changed; listed as in step 2
        for (int base = 32 * warp; base < G::CH * G::CPASS; base += 32 * kNW) {
            const int blk = base + lane;
            bool dirty = false;
            if (blk < G::CH * G::CPASS) {
                const int cr = blk / G::CPASS, w = blk - cr * G::CPASS;
                // exact column ranges: ground columns 32w+RP .. 32w+RP+33, the
                // ceiling's 32w+RP+1 .. 32w+RP+32, gentle flags 32w .. 32w+31+2RP
                uint32_t v = (sChgC[(cr + RP + 1) * G::EWW + w] & kCeilLo) |
                             (sChgC[(cr + RP + 1) * G::EWW + w + 1] & kCeilHi);
#pragma unroll
                for (int dr = 0; dr < 3; ++dr)
                    v |= (sChgG[(cr + RP + dr) * G::EWW + w] & kGrndLo) |
                         (sChgG[(cr + RP + dr) * G::EWW + w + 1] & kGrndHi);
#pragma unroll
                for (int dr = 0; dr <= 2 * RP; ++dr)
                    v |= sGChg[(cr + dr) * G::GWW + w] | (sGChg[(cr + dr) * G::GWW + w + 1] & kGentHi);
                dirty = first || v != 0;
                if (!dirty) sCIChg[cr * G::CWW + w] = 0;
            }
            const uint32_t m = __ballot_sync(0xffffffffu, dirty);
            if (m) {
                int at = 0;
                if (lane == 0) at = atomicAdd(&counters.nwork[1], __popc(m));
                at = __shfl_sync(0xffffffffu, at, 0);
                if (dirty) sList[at + __popc(m & ((1u << lane) - 1u))] = (uint16_t)blk;
            }
        }
        __syncthreads();
        // 3b. the listed blocks, spread over all warps
        {
            const int n_blk = counters.nwork[1];
#pragma unroll 1
            for (int t = warp; t < n_blk; t += kNW) {
                const int blk = sList[t];
                const int cr = blk / G::CPASS, w = blk - cr * G::CPASS;
                // branch-free over the warp: every lane evaluates Eq. 1-5 with
                // selects; p_s (Eq. 4) is counted when some lane needs it
                const int cs = 32 * w + lane;
                const bool live = cs < G::CW;
                const int csc = live ? cs : G::CW - 1;
                const int i = ty0 - RK + cr, j = tx0 - RK + csc;
                const bool in_map = live && i >= 0 && i < a.H && j >= 0 && j < a.W;
                const int eidx = (cr + RP + 1) * G::EW + (csc + RP + 1);
                const float *ep = sEG + eidx;
                const float eg = ep[0], zc = sZC[eidx];
                const float eL = ep[-1], eR = ep[1], eD = ep[-G::EW], eU = ep[G::EW];
                const bool valid = eg > -INFINITY;
                const float dI = zc - eg;
                const float cI = dI < c.d_min ? c.c_b
                                              : (isinf(dI) ? 0.0f : fmaxf(0.0f, c.alpha_d * (c.d_ref - dI)));
                const bool ok = eL > -INFINITY && eR > -INFINITY && eD > -INFINITY && eU > -INFINITY;
                const float gx = (eR - eL) * c.inv2r;
                const float gy = (eU - eD) * c.inv2r;
                const float m2 = __fmaf_rn(gx, gx, __fmul_rn(gy, gy));
                const float mxy = fmaxf(fabsf(gx), fabsf(gy));
                const bool barrier = !ok || mxy > c.theta_b;
                const bool step = in_map && valid && !barrier && !(m2 < ts2);
                float cg = barrier ? c.c_b : c.alpha_s * (m2 * inv_ts2);
                if (__any_sync(0xffffffffu, step)) {
                    int count = 0;
                    const int w0 = csc >> 5, off = csc & 31;
#pragma unroll
                    for (int dr = 0; dr <= 2 * RP; ++dr) {
                        const uint32_t *rowb = sGB + (cr + dr) * G::GWW;
                        const uint32_t bb = __funnelshift_r(rowb[w0], rowb[w0 + 1], off);
                        count += __popc(bb & ((1u << (2 * RP + 1)) - 1u));
                    }
                    const int cc = csc + RP;
                    count -= (sGB[(cr + RP) * G::GWW + (cc >> 5)] >> (cc & 31)) & 1u;
                    const float t = mxy * c.inv_tb;
                    if (step) cg = count > c.count_thresh ? c.alpha_b * (t * t) : c.c_b;
                }
                float ci = valid ? fminf(c.c_b, cI + cg) : c.c_b;
                ci = in_map ? ci : 0.0f;              // off-grid taps add nothing
                bool changed = false;
                if (live) {
                    const int cidx = cr * G::CW + cs;
                    changed = first || __float_as_uint(ci) != __float_as_uint(sCI[cidx]);
                    sCI[cidx] = ci;
                }
                const uint32_t cbits = __ballot_sync(0xffffffffu, changed);
                if (lane == 0) sCIChg[cr * G::CWW + w] = cbits;
            }
        }
        __syncthreads();

        // ---- 4. inflation (Eq. 6) of the strip, uniqueness, outputs ----
        uint32_t v = 0;
        for (int x = lane; x < 2 * (kStrip + 2 * RK); x += 32)
            v |= sCIChg[(tr0 + (x >> 1)) * G::CWW + half + (x & 1)] & ((x & 1) ? kWinHi : ~0u);
        const bool need_infl = __any_sync(0xffffffffu, v != 0);
        if (lane == 0 && need_infl) atomicOr(&counters.infl, 1u << warp);
        __syncthreads();
        const uint32_t dmask = counters.infl;
        const int ndirty = __popc(dmask);
        float acc[kStrip];
#pragma unroll
        for (int q = 0; q < kStrip; ++q) acc[q] = cT[q];
        if (ndirty > 0 && 2 * ndirty <= kNW) {
            // few strips changed: their halves (kStrip / 2 rows each) are
            // spread over the warps, half j on warp j, and handed to the
            // owner through the block list (free until the next slice)
            // (at most NW / 2 strips' halves of kStrip / 2 rows: TW TH / 2 floats,
            // within the list's NE >= TW TH 16-bit entries)
            float *slots = reinterpret_cast<float *>(sList);
            if (warp < 2 * ndirty) {
                uint32_t m = dmask;
                for (int r = warp >> 1; r > 0; --r) m &= m - 1u;
                const int owner = __ffs(m) - 1;
                const int o_tr0 = kStrip * (owner / G::NHALF) + (warp & 1) * (kStrip / 2);
                const int o_ts = 32 * (owner % G::NHALF) + lane;
                float a2[kStrip / 2];
                inflate_column<RK, kStrip / 2, G::CW>(sCI + o_tr0 * G::CW + o_ts, c, a2);
#pragma unroll
                for (int u = 0; u < kStrip / 2; ++u) slots[(warp * (kStrip / 2) + u) * 32 + lane] = a2[u];
            }
            __syncthreads();
            if (need_infl) {
                const int rank = __popc(dmask & ((1u << warp) - 1u));
#pragma unroll
                for (int q = 0; q < kStrip; ++q) acc[q] = slots[(2 * rank * (kStrip / 2) + q) * 32 + lane];
            }
            // the next slice's listing (step 1a) writes this region before its
            // first barrier: every owner has read its slots before any warp
            // passes here (the branch is uniform over the CTA: dmask was read
            // after a barrier)
            __syncthreads();
        } else if (need_infl) {
            inflate_column<RK, kStrip, G::CW>(sCI + tr0 * G::CW + ts, c, acc);
        }
        const bool need_simp = need_infl || __any_sync(0xffffffffu, gchbits != 0);
        if (need_simp) {
            // Eq. 9 of slice k-1 against slice k, then the rows p it is unique against
            int pre = 0;
            if (uniq) {
                uint32_t walk = 0;
#pragma unroll
                for (int q = 0; q < kStrip; ++q) {
                    const bool gq = (gchbits >> q) & 1u;
                    if (!first && ((inmap >> q) & 1u) && cT[q] < c.c_b && (gq || cT[q] < acc[q])) {
                        if (!((runle >> q) & 1u)) walk |= 1u << q;
                        pre = max(pre, run_get(q) + 1);
                    }
                }
                if (!first) mark_run(walk, k - 1);
            }
#pragma unroll
            for (int q = 0; q < kStrip; ++q) {
                const uint32_t bit = 1u << q;
                // the run state the uniqueness walks use
                if (uniq && (gchbits & bit)) {
                    run_set(q, k);
                    runle |= bit;
                } else if (uniq && !first) {
                    // the run now covers slice k-1 (cost cT) and the current cost is acc
                    if (runle & bit) {
                        // no earlier cost of the run exceeded cT, so the run's
                        // maximum is cT: the flag stays while cT <= acc, and the
                        // bound (unused while the flag holds) starts at cT
                        if (!(cT[q] <= acc[q])) {
                            runle &= ~bit;
                            rmax_set(q, __half_as_ushort(__float2half_ru(cT[q])));
                        }
                    } else {
                        // max(run, cT) <= acc  <=  cT <= acc and bound <= acc
                        const float mup = rmax_get(q);
                        if (cT[q] <= acc[q] && mup <= acc[q]) runle |= bit;
                        const __half hc = __float2half_ru(cT[q]);
                        if (__half2float(hc) > mup) rmax_set(q, __half_as_ushort(hc));
                    }
                }
                cT[q] = acc[q];
            }
            const int wmax = __reduce_max_sync(0xffffffffu, pre);
            if (lane == 0 && wmax > 0) atomicMax(&s_upre[k - 1], wmax);   // 0 unless uniq
            travbits = 0;
#pragma unroll
            for (int q = 0; q < kStrip; ++q)
                if (cT[q] < c.c_b) travbits |= 1u << q;
            wvalid = (int)__reduce_add_sync(0xffffffffu, (uint32_t)__popc(validbits & inmap));
            wtrav = (int)__reduce_add_sync(0xffffffffu, (uint32_t)__popc(travbits & inmap));
        }
        }   // !quiet
        if (lane == 0) {
            if (wvalid) atomicAdd(&s_valid[k], wvalid);
            if (wtrav) atomicAdd(&s_trav[k], wtrav);
        }
        if (inmap) {
            // this slice's layers, addressed by 32-bit offsets within the
            // slice (W H <= 2^30); ground and ceiling are still this slice's:
            // the next slice advances them after its first barrier
            const int64_t sl = (int64_t)k * HW;
            float *gk = given ? nullptr : a.ground + sl, *zk = given ? nullptr : a.ceil + sl;
            float *tk = a.cost + sl;
            uint8_t *mk = a.mask + sl;
            uint32_t o = (uint32_t)(ty0 + tr0) * (uint32_t)a.W + (uint32_t)j_out;
#pragma unroll
            for (int q = 0; q < kStrip; ++q, o += (uint32_t)a.W) {
                if ((inmap >> q) & 1u) {
                    if (!given) {
                        const int e = (tr0 + q + G::HE) * G::EW + ts + G::HE;
                        __stcs(gk + o, sEG[e]);
                        __stcs(zk + o, sZC[e]);
                    }
                    __stcs(tk + o, cT[q]);
                    mk[o] = (travbits >> q) & 1u;
                }
            }
        }
    }

    // Eq. 9 holds vacuously for the last slice
    if (uniq) {
        int pre = 0;
        uint32_t walk = 0;
#pragma unroll
        for (int q = 0; q < kStrip; ++q) {
            if (((inmap >> q) & 1u) && cT[q] < c.c_b) {
                if (!((runle >> q) & 1u)) walk |= 1u << q;
                pre = max(pre, run_get(q) + 1);
            }
        }
        mark_run(walk, a.N - 1);
        const int wmax = __reduce_max_sync(0xffffffffu, pre);
        if (lane == 0 && wmax > 0) atomicMax(&s_upre[a.N - 1], wmax);
    }
    __syncthreads();
    for (int k = tid; k < a.N; k += kNT) {
        if (s_upre[k]) atomicMax(&a.upre[k], s_upre[k]);
        if (s_valid[k])
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats->valid_cells[k]),
                      (unsigned long long)s_valid[k]);
        if (s_trav[k])
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats->trav_cells[k]),
                      (unsigned long long)s_trav[k]);
    }
}

// Resident CTAs per SM that the tile's shared memory and 64 registers per
// thread allow.
template <int RK, int RP, int TW, int TH, int KS>
struct Occupancy {
    using G = Geo<RK, RP, TW, TH, KS>;
    // 228 KB of shared memory per SM, 1 KB of it reserved per resident CTA,
    // plus the CTA's static shared memory
    static constexpr int by_smem =
        (int)(233472 / (G::smem_bytes() + sizeof(SliceCounters) + 64 + 1024));
    static constexpr int by_regs = 65536 / (64 * G::NT);
    static constexpr int value = by_smem < 1 ? 1 : (by_smem < by_regs ? by_smem : by_regs);
};

// ---------------------------------------------------------------- batches
//
// One persistent launch over the tiles of many maps: each CTA takes the next
// (map, tile) item from a queue; maps come largest first so the long tiles
// start early.  The descriptors travel in the kernel parameters.

struct BatchArgs {
    EvalConsts c;
    int32_t n_maps;
    int32_t total;                       // items
    int32_t *queue;                      // next item (zero before the launch)
    int32_t *done;                       // finished CTAs (zero before the launch); when set,
                                         // the last CTA runs every map's chain
    int32_t split;                       // slice ranges per tile (1: the whole stack, with the
                                         // uniqueness rows; more: items of one range each)
    int32_t item_start[TCT_MAX_BATCH + 1];
    int32_t tiles_x[TCT_MAX_BATCH];
    IncMap maps[TCT_MAX_BATCH];
};

template <int RK, int RP, int TW, int TH, int KS>
__global__ void __launch_bounds__(Geo<RK, RP, TW, TH, KS>::NT, (Occupancy<RK, RP, TW, TH, KS>::value))
k_stack_batched(const __grid_constant__ BatchArgs b) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SliceCounters counters;
    __shared__ int32_t s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(b.queue, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= b.total) break;
        int m = 0;
        while (m + 1 < b.n_maps && b.item_start[m + 1] <= item) ++m;
        const int t = (item - b.item_start[m]) / b.split, rg = (item - b.item_start[m]) % b.split;
        const int tx = t % b.tiles_x[m], ty = t / b.tiles_x[m];
        const int N = b.maps[m].N;
        // only the small-map shape is ever cut into slice ranges; the others
        // keep the uniqueness rows as a compile-time constant
        constexpr bool kMaySplit = TW == 32 && TH == 32;
        stack_tile<RK, RP, TW, TH, KS>(b.maps[m], b.c, tx * TW, ty * TH, smem, counters,
                                       (N * rg) / b.split, (N * (rg + 1)) / b.split,
                                       !kMaySplit || b.split == 1);
        __syncthreads();
    }
    if (b.done) {
        // the chain of Sec. III-C, once every tile's uniqueness bits are in: the
        // CTA that finishes last (its writes and the others' ordered before its
        // count by the fences) reads the rows through L2 and walks them
        __shared__ int32_t s_last;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = atomicAdd(b.done, 1) == (int)gridDim.x - 1;
        __syncthreads();
        if (s_last) {
            __threadfence();
            int32_t *s_pre = reinterpret_cast<int32_t *>(smem);     // the tile state is free now
            uint32_t *s_bits = reinterpret_cast<uint32_t *>(s_pre + TCT_MAX_SLICES + 1);
            for (int m = 0; m < b.n_maps; ++m) {
                const IncMap &mp = b.maps[m];
                for (int k = threadIdx.x; k < mp.N; k += blockDim.x) {
                    s_pre[k] = __ldcg(mp.upre + k);
#pragma unroll
                    for (int w = 0; w < 4; ++w) s_bits[4 * k + w] = __ldcg(mp.ubits + 4 * k + w);
                }
                __syncthreads();
                if (threadIdx.x == 0)
                    mp.stats->n_kept = chain_walk(mp.N, s_pre, s_bits, b.c.flags, mp.keep);
                __syncthreads();
            }
        }
    }
}

template <int RK, int RP, int TW, int TH, int KS>
cudaError_t run_batched(const BatchArgs &b, int ctas_per_sm, cudaStream_t s) {
    using G = Geo<RK, RP, TW, TH, KS>;
    const size_t smem = G::smem_bytes();
    auto fn = k_stack_batched<RK, RP, TW, TH, KS>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148, fit = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, fn, G::NT, smem);
    if (e != cudaSuccess) return e;
    if (fit < 1) fit = 1;
    int per_sm = ctas_per_sm > 0 && ctas_per_sm < fit ? ctas_per_sm : fit;
    int grid = sms * per_sm;
    if (grid > b.total) grid = b.total > 0 ? b.total : 1;
    fn<<<grid, G::NT, smem, s>>>(b);
    count_launches(1);
    return cudaGetLastError();
}

// Strip height of the 32 x 32 tile, the shape of small maps: two rows a
// thread, 16 warps, so that the few CTAs of a small map finish each slice's
// steps in fewer rounds.
constexpr int kStripSmall = 2;

// Launch of one (R_K, R_p) instance; defined in the tct_stack_inc_r*.cu units.
template <int RK, int RP>
cudaError_t run_radius(const BatchArgs &b, int tile, int ctas_per_sm, cudaStream_t s) {
    if (tile == TCT_TILE_32) return run_batched<RK, RP, 32, 32, kStripSmall>(b, ctas_per_sm, s);
    if (tile == TCT_TILE_64x56) return run_batched<RK, RP, 64, 56, 8>(b, ctas_per_sm, s);
    if (tile == TCT_TILE_64x40) return run_batched<RK, RP, 64, 40, 8>(b, ctas_per_sm, s);
    if (tile == TCT_TILE_128x56) return run_batched<RK, RP, 128, 56, 8>(b, ctas_per_sm, s);
    return run_batched<RK, RP, 64, 64, 8>(b, ctas_per_sm, s);
}

cudaError_t run_r4(const BatchArgs &b, int tile, int ctas_per_sm, cudaStream_t s);
cudaError_t run_r5(const BatchArgs &b, int tile, int ctas_per_sm, cudaStream_t s);
cudaError_t run_r12(const BatchArgs &b, int tile, int ctas_per_sm, cudaStream_t s);

}  // namespace inc
}  // namespace tct
