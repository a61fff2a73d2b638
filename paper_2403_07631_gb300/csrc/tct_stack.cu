// tct_stack.cu -- per-tile scene evaluation over the whole slice stack
// (Sec. III-B, Eq. 1-6) with the simplification bits of Sec. III-C.
//
// One CTA owns a TW x TH tile of the grid and walks the slices k = 0..N-1.
// For each slice it builds, in shared memory, the layers the stencils need on
// the tile plus a halo:
//   ground    e^G on tile + (R_K + R_p + 1)   (from the sorted per-cell z
//             segments of the build, or loaded from given layers)
//   gentle    m^grad < theta_s on tile + (R_K + R_p)          (Eq. 2)
//   c^init    on tile + R_K                                     (Eq. 1, 3-5)
// and then inflates c^init over the tile (Eq. 6) and writes e^G, e^C, c^T and
// the mask.  Nothing but the outputs goes back to HBM.
//
// Simplification (Eq. 7-9) needs, per slice k, which earlier slices p a
// traversable cell of k would be unique against.  Let A_k = trav_k and Eq. 9
// (against slice k+1); while ground is non-decreasing in k, Eq. 8 against p
// holds for every p below the start r_k of the cell's run of equal ground,
// and inside the run it reduces to c_k < c_p.  Each CTA ORs, per slice, the
// set of such p into a (N+1) x N bit matrix U(p, k); the sequential chain of
// Sec. III-C is then an O(N) walk over U (k_chain).
#include <cuda_runtime.h>

#include <algorithm>
#include <math.h>

#include "tct_internal.cuh"

namespace tct {
namespace {



struct Geo {
    int RK, RP, HE, EW, EH, GW, GH, CW, CH;
};

__device__ __forceinline__ Geo geometry(const EvalConsts &c, int TW, int TH) {
    Geo g;
    g.RK = c.rk;
    g.RP = c.patch_radius;
    g.HE = g.RK + g.RP + 1;
    g.EW = TW + 2 * g.HE;
    g.EH = TH + 2 * g.HE;
    g.GW = g.EW - 2;
    g.GH = g.EH - 2;
    g.CW = TW + 2 * g.RK;
    g.CH = TH + 2 * g.RK;
    return g;
}

template <int TW, int TH, int NT, int CPT, bool kLists, bool kAux>
__global__ void __launch_bounds__(NT)
k_stack(const __grid_constant__ StackArgs a) {
    constexpr int TPT = TW * TH / NT;
    static_assert(TW * TH % NT == 0, "tile cells must split evenly over the threads");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int32_t s_upre[TCT_MAX_SLICES + 1];
    __shared__ uint32_t s_ubits[TCT_MAX_SLICES + 1][4];
    __shared__ int32_t s_valid[TCT_MAX_SLICES + 1], s_trav[TCT_MAX_SLICES + 1];

    const EvalConsts &c = a.c;
    const Geo g = geometry(c, TW, TH);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int tx0 = blockIdx.x * TW, ty0 = blockIdx.y * TH;
    const int64_t HW = (int64_t)a.W * a.H;

    float *sEG0 = reinterpret_cast<float *>(smem);
    float *sEG1 = sEG0 + g.EW * g.EH;
    float *sEC = sEG1 + g.EW * g.EH;
    float *sMXY = sEC + g.CW * g.CH;
    float *sMGR = sMXY + g.CW * g.CH;
    float *sCI = sMGR + g.CW * g.CH;
    uint8_t *sGen = reinterpret_cast<uint8_t *>(sCI + g.CW * g.CH);

    for (int i = tid; i <= TCT_MAX_SLICES; i += NT) {
        s_upre[i] = 0;
        s_ubits[i][0] = s_ubits[i][1] = s_ubits[i][2] = s_ubits[i][3] = 0;
        s_valid[i] = 0;
        s_trav[i] = 0;
    }

    float z_min = a.z_min;
    if (kLists && a.zmin_from_data) {
        z_min = key_float(a.zkeys[0]);
        if (!isfinite(z_min)) z_min = 0.0f;
    }

    // ---- per-thread state of the elevation region cells (build path) ----
    const int ecount = g.EW * g.EH;
    int32_t ptr[CPT], end[CPT];
    float zg[CPT], zc[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        ptr[q] = end[q] = 0;
        zg[q] = -INFINITY;
        zc[q] = INFINITY;
        if (kLists) {
            const int e = tid + q * NT;
            if (e < ecount) {
                const int i = ty0 - g.HE + e / g.EW, j = tx0 - g.HE + e % g.EW;
                if (i >= 0 && i < a.H && j >= 0 && j < a.W) {
                    const int64_t cell = (int64_t)i * a.W + j;
                    ptr[q] = a.start[cell];
                    end[q] = a.start[cell + 1];
                    if (ptr[q] < end[q]) zc[q] = a.zs[ptr[q]];
                }
            }
        }
    }

    // ---- per-thread state of the owned tile cells (simplification) ----
    float e_prev[TPT], c_prev[TPT];
    int32_t run_prev[TPT];
    bool mono[TPT];
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
        e_prev[q] = -INFINITY;
        c_prev[q] = INFINITY;
        run_prev[q] = 0;
        mono[q] = true;
    }
    __syncthreads();

    const int ksz = 2 * g.RK + 1;

    // Uniqueness of slice kk = k-1 (or N-1 after the loop) for one tile cell:
    // A = trav_kk and Eq. 9; returns the prefix length of the rows p+1 it sets
    // and ORs the rows inside the run into s_ubits.
    auto unique_rows = [&](int kk, int q, int64_t cell, bool in_map, bool eq9) -> int {
        if (!in_map || !(c_prev[q] < c.c_b) || !eq9) return 0;
        if (mono[q]) {
            // rows p < r are set by the run prefix; rows in [r, kk-1] where c_p > c_kk
            for (int p = run_prev[q]; p < kk; ++p) {
                const float cp = a.cost[(int64_t)p * HW + cell];
                if (c_prev[q] < cp) atomicOr(&s_ubits[kk][(p + 1) >> 5], 1u << ((p + 1) & 31));
            }
            return run_prev[q] + 1;
        }
        // ground not monotone in k (given layers): test every earlier slice
        const float *gsrc = kLists ? a.ground : a.gin;
        for (int p = 0; p < kk; ++p) {
            const float ep = gsrc[(int64_t)p * HW + cell];
            const float cp = a.cost[(int64_t)p * HW + cell];
            if (e_prev[q] - ep > 0.0f || c_prev[q] < cp)
                atomicOr(&s_ubits[kk][(p + 1) >> 5], 1u << ((p + 1) & 31));
        }
        return 1;
    };

    for (int k = 0; k < a.N; ++k) {
        float *sEG = (k & 1) ? sEG1 : sEG0;
        const float h = __fmaf_rn((float)(k + 1), a.d_s, z_min);

        // ---- step 1: ground and ceiling of the region (Sec. III-A) ----
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int e = tid + q * NT;
            if (e >= ecount) break;
            const int r = e / g.EW, s = e % g.EW;
            const int i = ty0 - g.HE + r, j = tx0 - g.HE + s;
            const bool in_map = i >= 0 && i < a.H && j >= 0 && j < a.W;
            const int64_t cell = (int64_t)i * a.W + j;
            float eg, ec;
            if (kLists) {
                while (zc[q] <= h) {
                    zg[q] = zc[q];
                    ++ptr[q];
                    zc[q] = ptr[q] < end[q] ? a.zs[ptr[q]] : INFINITY;
                }
                eg = zg[q];
                ec = zc[q];
            } else {
                eg = in_map ? a.gin[(int64_t)k * HW + cell] : -INFINITY;
                ec = in_map ? a.cin[(int64_t)k * HW + cell] : INFINITY;
            }
            sEG[e] = eg;
            const int cr = r - g.RP - 1, cs = s - g.RP - 1;
            if (cr >= 0 && cr < g.CH && cs >= 0 && cs < g.CW) sEC[cr * g.CW + cs] = ec;
            if (kLists && r >= g.HE && r < g.HE + TH && s >= g.HE && s < g.HE + TW && in_map) {
                __stcs(&a.ground[(int64_t)k * HW + cell], eg);
                __stcs(&a.ceil[(int64_t)k * HW + cell], ec);
            }
        }
        __syncthreads();

        // ---- step 2: gradient magnitudes and the gentle flag (Eq. 2) ----
        for (int e = tid; e < g.GW * g.GH; e += NT) {
            const int gr = e / g.GW, gs = e % g.GW;
            const float *row = sEG + (gr + 1) * g.EW + (gs + 1);
            const float e0 = row[0], eL = row[-1], eR = row[1], eD = row[-g.EW], eU = row[g.EW];
            float mxy = INFINITY, mgr = INFINITY;
            if (e0 > -INFINITY && eL > -INFINITY && eR > -INFINITY && eD > -INFINITY &&
                eU > -INFINITY) {
                const float gx = (eR - eL) * c.inv2r;
                const float gy = (eU - eD) * c.inv2r;
                mxy = fmaxf(fabsf(gx), fabsf(gy));
                mgr = sqrtf(gx * gx + gy * gy);
            }
            sGen[e] = mgr < c.theta_s ? 1 : 0;
            const int cr = gr - g.RP, cs = gs - g.RP;
            if (cr >= 0 && cr < g.CH && cs >= 0 && cs < g.CW) {
                sMXY[cr * g.CW + cs] = mxy;
                sMGR[cr * g.CW + cs] = mgr;
            }
        }
        __syncthreads();

        // ---- step 3: interval, terrain and initial cost (Eq. 1, 3, 4, 5) ----
        for (int e = tid; e < g.CW * g.CH; e += NT) {
            const int cr = e / g.CW, cs = e % g.CW;
            const int i = ty0 - g.RK + cr, j = tx0 - g.RK + cs;
            if (i < 0 || i >= a.H || j < 0 || j >= a.W) {
                sCI[e] = 0.0f;                     // off-grid taps add nothing
                continue;
            }
            const float eg = sEG[(cr + g.RP + 1) * g.EW + (cs + g.RP + 1)];
            int count = 0;
            for (int dr = -g.RP; dr <= g.RP; ++dr) {
                const uint8_t *gl = sGen + (cr + g.RP + dr) * g.GW + (cs + g.RP);
                for (int ds = -g.RP; ds <= g.RP; ++ds) count += gl[ds];
            }
            count -= sGen[(cr + g.RP) * g.GW + (cs + g.RP)];
            const float dI = sEC[e] - eg;
            float cI;
            if (dI < c.d_min) cI = c.c_b;
            else if (isinf(dI)) cI = 0.0f;
            else cI = fmaxf(0.0f, c.alpha_d * (c.d_ref - dI));
            const float mxy = sMXY[e], mgr = sMGR[e];
            float cG;
            if (mxy > c.theta_b) {
                cG = c.c_b;
            } else if (mgr < c.theta_s) {
                const float t = mgr * c.inv_ts;
                cG = c.alpha_s * (t * t);
            } else if (count > c.count_thresh) {
                const float t = mxy * c.inv_tb;
                cG = c.alpha_b * (t * t);
            } else {
                cG = c.c_b;
            }
            const float ci = eg > -INFINITY ? fminf(c.c_b, cI + cG) : c.c_b;
            sCI[e] = ci;
            if (kAux) {
                const int tr = cr - g.RK, ts = cs - g.RK;
                if (tr >= 0 && tr < TH && ts >= 0 && ts < TW) {
                    const int64_t o = (int64_t)k * HW + (int64_t)i * a.W + j;
                    const int64_t L = (int64_t)a.N * HW;
                    a.aux[o] = mxy;
                    a.aux[L + o] = mgr;
                    a.aux[2 * L + o] = cI;
                    a.aux[3 * L + o] = cG;
                    a.aux[4 * L + o] = ci;
                }
            }
        }
        __syncthreads();

        // ---- step 4: inflation (Eq. 6), outputs, simplification bits ----
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            const int t = tid + q * NT;
            const int tr = t / TW, ts = t % TW;
            const int i = ty0 + tr, j = tx0 + ts;
            const bool in_map = i < a.H && j < a.W;
            const int64_t cell = (int64_t)i * a.W + j;
            float acc = 0.0f;
            const float *base = sCI + tr * g.CW + ts;
            for (int n = 0; n < ksz; ++n) {
                const float *krow = c.K + n * ksz;
                const float *crow = base + n * g.CW;
                for (int m = 0; m < ksz; ++m) {
                    const float w = krow[m];
                    if (w > 0.0f) acc = fmaxf(acc, w * crow[m]);
                }
            }
            const float e_k = sEG[(tr + g.HE) * g.EW + (ts + g.HE)];
            const bool trav = acc < c.c_b;
            if (in_map) {
                __stcs(&a.cost[(int64_t)k * HW + cell], acc);
                a.mask[(int64_t)k * HW + cell] = trav ? 1 : 0;
            }
            const unsigned nv = __ballot_sync(0xffffffffu, in_map && e_k > -INFINITY);
            const unsigned nt = __ballot_sync(0xffffffffu, in_map && trav);
            if (lane == 0) {
                if (nv) atomicAdd(&s_valid[k], __popc(nv));
                if (nt) atomicAdd(&s_trav[k], __popc(nt));
            }
            if (k > 0) {
                // Eq. 9 of slice k-1 against slice k
                const bool eq9 = (e_k - e_prev[q] > 0.0f) || (c_prev[q] < acc);
                const int pre = unique_rows(k - 1, q, cell, in_map, eq9);
                const int wmax = __reduce_max_sync(0xffffffffu, pre);
                if (lane == 0 && wmax > 0) atomicMax(&s_upre[k - 1], wmax);
            }
            if (k > 0 && e_k < e_prev[q]) mono[q] = false;
            if (k == 0 || !(e_k == e_prev[q])) run_prev[q] = k;
            e_prev[q] = e_k;
            c_prev[q] = acc;
        }
    }

    // Eq. 9 holds vacuously for the last slice
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
        const int t = tid + q * NT;
        const int i = ty0 + t / TW, j = tx0 + t % TW;
        const bool in_map = i < a.H && j < a.W;
        const int pre = unique_rows(a.N - 1, q, (int64_t)i * a.W + j, in_map, true);
        const int wmax = __reduce_max_sync(0xffffffffu, pre);
        if (lane == 0 && wmax > 0) atomicMax(&s_upre[a.N - 1], wmax);
    }
    __syncthreads();
    for (int k = tid; k < a.N; k += NT) {
        if (s_upre[k]) atomicMax(&a.upre[k], s_upre[k]);
#pragma unroll
        for (int w = 0; w < 4; ++w)
            if (s_ubits[k][w]) atomicOr(&a.ubits[4 * k + w], s_ubits[k][w]);
        if (s_valid[k])
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats->valid_cells[k]),
                      (unsigned long long)s_valid[k]);
        if (s_trav[k])
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats->trav_cells[k]),
                      (unsigned long long)s_trav[k]);
    }
}

// The sequential chain of Sec. III-C over the uniqueness matrix.
__global__ void k_chain(int n_slices, const int32_t *upre, const uint32_t *ubits, uint32_t flags,
                        uint8_t *keep, tct_stats *stats) {
    __shared__ int32_t s_pre[TCT_MAX_SLICES + 1];
    __shared__ uint32_t s_bits[4 * (TCT_MAX_SLICES + 1)];
    for (int k = threadIdx.x; k < n_slices; k += blockDim.x) {
        s_pre[k] = upre[k];
        s_bits[4 * k] = ubits[4 * k];
        s_bits[4 * k + 1] = ubits[4 * k + 1];
        s_bits[4 * k + 2] = ubits[4 * k + 2];
        s_bits[4 * k + 3] = ubits[4 * k + 3];
    }
    __syncthreads();
    if (threadIdx.x == 0) stats->n_kept = chain_walk(n_slices, s_pre, s_bits, flags, keep);
}

// Given layers whose ground falls somewhere from one slice to the next (not
// a build's): the uniqueness rows of Sec. III-C taken as the equations state
// them, every earlier slice p tested (Eq. 8 against p, Eq. 9 against k+1)
// from the given grounds and the evaluated costs, after the rows the slice
// stack accumulated are cleared.  Both kernels return at once when no
// ground fell.
__global__ void k_uniq_clear(const int32_t *falls, int32_t *upre, uint32_t *ubits) {
    if (!*falls) return;
    const int i = threadIdx.x;
    if (i <= TCT_MAX_SLICES) {
        upre[i] = 0;
        ubits[4 * i] = ubits[4 * i + 1] = ubits[4 * i + 2] = ubits[4 * i + 3] = 0;
    }
}

__global__ void __launch_bounds__(256)
k_uniq_general(const int32_t *falls, int64_t HW, int N, const float *__restrict__ ground,
               const float *__restrict__ cost, float c_b, uint32_t *ubits) {
    if (!*falls) return;
    __shared__ uint32_t s_bits[4 * (TCT_MAX_SLICES + 1)];
    for (int i = threadIdx.x; i < 4 * (TCT_MAX_SLICES + 1); i += blockDim.x) s_bits[i] = 0;
    __syncthreads();
    for (int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; cell < HW;
         cell += (int64_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < N; ++k) {
            const float ck = cost[(int64_t)k * HW + cell];
            if (!(ck < c_b)) continue;                       // not traversable
            const float ek = ground[(int64_t)k * HW + cell];
            if (k + 1 < N && !(ground[(int64_t)(k + 1) * HW + cell] - ek > 0.0f) &&
                !(ck < cost[(int64_t)(k + 1) * HW + cell]))
                continue;                                    // Eq. 9 fails
            atomicOr(&s_bits[4 * k], 1u);                    // row 0: no slice kept yet
            for (int p = 0; p < k; ++p) {
                if (ek - ground[(int64_t)p * HW + cell] > 0.0f || ck < cost[(int64_t)p * HW + cell])
                    atomicOr(&s_bits[4 * k + ((p + 1) >> 5)], 1u << ((p + 1) & 31));
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * N; i += blockDim.x)
        if (s_bits[i]) atomicOr(&ubits[i], s_bits[i]);
}

// The uniqueness rows of Sec. III-C for maps of up to kColSlices slices,
// straight from the finished layers (the same tests as k_uniq_general: Eq. 9
// against slice k+1, Eq. 8 against every earlier slice p): a thread holds its
// cell's column of grounds and costs, loaded at once, and a warp's rows leave
// with one shared atomic per slice.  The rows fit the first word of each
// slice's bits (p + 1 < 32).
constexpr int kColSlices = 16;

__global__ void __launch_bounds__(256)
k_uniq_columns(int64_t HW, int N, const float *__restrict__ ground,
               const float *__restrict__ cost, float c_b, uint32_t *ubits) {
    __shared__ uint32_t s_bits[kColSlices];
    if (threadIdx.x < kColSlices) s_bits[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < HW;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cell = base + lane;
        const bool live = cell < HW;
        float g[kColSlices], ct[kColSlices];
#pragma unroll
        for (int k = 0; k < kColSlices; ++k) {
            g[k] = live && k < N ? ground[(int64_t)k * HW + cell] : 0.0f;
            ct[k] = live && k < N ? cost[(int64_t)k * HW + cell] : INFINITY;
        }
#pragma unroll
        for (int k = 0; k < kColSlices; ++k) {
            const int kn = k + 1 < kColSlices ? k + 1 : k;   // slice k + 1 (read when k + 1 < N)
            uint32_t row = 0;
            if (k < N && ct[k] < c_b && (k + 1 >= N || g[kn] - g[k] > 0.0f || ct[k] < ct[kn])) {
                row = 1u;                                // row 0: no slice kept yet
#pragma unroll
                for (int p = 0; p < k; ++p)
                    if (g[k] - g[p] > 0.0f || ct[k] < ct[p]) row |= 1u << (p + 1);
            }
            row = __reduce_or_sync(0xffffffffu, row);
            if (lane == 0 && row) atomicOr(&s_bits[k], row);
        }
    }
    __syncthreads();
    if (threadIdx.x < N && s_bits[threadIdx.x]) atomicOr(&ubits[4 * threadIdx.x], s_bits[threadIdx.x]);
}

__global__ void k_stack_init(int32_t *upre, uint32_t *ubits, int32_t *queue, int32_t *falls) {
    const int i = threadIdx.x;
    if (i == 0 && queue) *queue = 0;
    if (i == 0 && falls) *falls = 0;
    if (i <= TCT_MAX_SLICES) {
        upre[i] = 0;
        ubits[4 * i] = ubits[4 * i + 1] = ubits[4 * i + 2] = ubits[4 * i + 3] = 0;
    }
}

size_t stack_smem(const EvalConsts &c, int TW, int TH) {
    const int RK = c.rk, RP = c.patch_radius, HE = RK + RP + 1;
    const size_t EW = TW + 2 * HE, EH = TH + 2 * HE;
    const size_t CW = TW + 2 * RK, CH = TH + 2 * RK;
    const size_t GW = EW - 2, GH = EH - 2;
    return sizeof(float) * (2 * EW * EH + 4 * CW * CH) + ((GW * GH + 15) / 16) * 16;
}

template <int TW, int TH, int NT, int CPT, bool kLists, bool kAux>
cudaError_t run_stack(const StackArgs &a, cudaStream_t s) {
    const size_t smem = stack_smem(a.c, TW, TH);
    auto fn = k_stack<TW, TH, NT, CPT, kLists, kAux>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.W + TW - 1) / TW, (a.H + TH - 1) / TH);
    fn<<<grid, NT, smem, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <int TW, int TH, int NT, bool kLists, bool kAux>
cudaError_t pick_cpt(const StackArgs &a, cudaStream_t s) {
    const int HE = a.c.rk + a.c.patch_radius + 1;
    const int cells = (TW + 2 * HE) * (TH + 2 * HE);
    const int need = (cells + NT - 1) / NT;
    if (need <= 4) return run_stack<TW, TH, NT, 4, kLists, kAux>(a, s);
    if (need <= 6) return run_stack<TW, TH, NT, 6, kLists, kAux>(a, s);
    if (need <= 8) return run_stack<TW, TH, NT, 8, kLists, kAux>(a, s);
    if (need <= 12) return run_stack<TW, TH, NT, 12, kLists, kAux>(a, s);
    if (need <= 16) return run_stack<TW, TH, NT, 16, kLists, kAux>(a, s);
    return cudaErrorInvalidConfiguration;
}

template <bool kLists, bool kAux>
cudaError_t pick_tile(const StackArgs &a, cudaStream_t s) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t big = (int64_t)((a.W + 31) / 32) * ((a.H + 31) / 32);
    if (big >= 2 * sms) return pick_cpt<32, 32, 512, kLists, kAux>(a, s);
    return pick_cpt<16, 16, 256, kLists, kAux>(a, s);
}

}  // namespace

cudaError_t launch_stack(const tct_grid &g, const EvalConsts &c, const Workspace *lists,
                         const int32_t *zkeys, const float *gin, const float *cin, float *ground,
                         float *ceil, float *cost, uint8_t *mask, float *aux, int32_t *upre,
                         uint32_t *ubits, tct_stats *stats, cudaStream_t s, int tile,
                         int32_t *queue, int32_t *falls, uint8_t *keep, bool *chained) {
    StackArgs a;
    a.W = g.W;
    a.H = g.H;
    a.N = g.n_slices;
    a.d_s = g.d_s;
    a.z_min = g.z_min;
    a.zmin_from_data = (g.flags & TCT_GRID_ZMIN_FROM_DATA) ? 1 : 0;
    a.zkeys = zkeys;
    a.start = lists ? lists->start : nullptr;
    a.zs = lists ? lists->zs : nullptr;
    a.gin = gin;
    a.cin = cin;
    a.ground = ground;
    a.ceil = ceil;
    a.cost = cost;
    a.aux = aux;
    a.mask = mask;
    a.upre = upre;
    a.ubits = ubits;
    a.stats = stats;
    a.c = c;
    a.falls = falls;
    a.keep = nullptr;
    a.done = nullptr;
    a.split = 1;
    if (chained) *chained = false;
    if (lists) {
        // the partition of this workspace has cleared its uniqueness rows,
        // queue and count of finished CTAs
        if (keep) {
            a.keep = keep;
            a.done = lists->queue + 1;
        }
        if (tile == TCT_TILE_AUTO && inc_supported(c, a.N)) tile = choose_tile(c, 1, &a, 1);
        // A small map (32 x 32 tiles, fewer than the SMs) of a few slices is a
        // latency chain of its slices: each tile's slices are cut into ranges
        // of at least four, one CTA each, so that more SMs walk shorter chains;
        // the uniqueness rows then come from the finished layers.
        const int64_t HW = (int64_t)a.W * a.H;
        if (tile == TCT_TILE_32 && a.N >= 8 && a.N <= kColSlices) {
            int dev = 0, sms = 148;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const int64_t tiles = (int64_t)((a.W + 31) / 32) * ((a.H + 31) / 32);
            a.split = (int)std::min<int64_t>(a.N / 4, std::max<int64_t>(1, sms / tiles));
        }
        const cudaError_t e = launch_stack_inc(a, lists->queue, tile, s);
        if (e != cudaErrorNotSupported) {
            if (e != cudaSuccess || a.split <= 1) {
                if (chained) *chained = e == cudaSuccess && keep != nullptr;
                return e;
            }
            const int blocks = (int)std::min<int64_t>((HW + 255) / 256, 4096);
            k_uniq_columns<<<blocks, 256, 0, s>>>(HW, a.N, ground, cost, c.c_b, ubits);
            count_launches(1);
            return cudaGetLastError();      // the caller launches the chain
        }
        a.keep = nullptr;
        a.done = nullptr;
        return pick_tile<true, false>(a, s);
    }
    k_stack_init<<<1, 128, 0, s>>>(upre, ubits, queue, falls);
    count_launches(1);
    if (!aux && queue && falls && inc_supported(c, a.N)) {
        // given layers on the incremental kernel; the general uniqueness rows
        // replace its own when a ground fell
        if (tile == TCT_TILE_AUTO) tile = choose_tile(c, 1, &a, 1);
        cudaError_t e = launch_stack_inc(a, queue, tile, s);
        if (e != cudaErrorNotSupported) {
            if (e != cudaSuccess) return e;
            const int64_t HW = (int64_t)a.W * a.H;
            k_uniq_clear<<<1, 128, 0, s>>>(falls, upre, ubits);
            const int blocks = (int)std::min<int64_t>((HW + 255) / 256, 4096);
            k_uniq_general<<<blocks, 256, 0, s>>>(falls, HW, a.N, gin, cost, c.c_b, ubits);
            count_launches(2);
            return cudaGetLastError();
        }
    }
    if (aux) return pick_tile<false, true>(a, s);
    return pick_tile<false, false>(a, s);
}

cudaError_t launch_stack_generic(const StackArgs &a, cudaStream_t s) {
    return pick_tile<true, false>(a, s);
}

cudaError_t launch_chain(int n_slices, const int32_t *upre, const uint32_t *ubits, uint32_t flags,
                         uint8_t *keep, tct_stats *stats, cudaStream_t s) {
    k_chain<<<1, 128, 0, s>>>(n_slices, upre, ubits, flags, keep, stats);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace tct
