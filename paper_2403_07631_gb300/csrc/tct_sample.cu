// tct_sample.cu -- cost and elevation queries on an evaluated tomogram and
// their adjoint (the C(q), e^G(q) queries of Sec. III-E, Eq. 10), and a fused
// path-refinement kernel built on them.
//
// A query (x, y, k) interpolates slice k bilinearly on the lattice of cell
// centres: u = (x - x0)/r_g - 1/2, v = (y - y0)/r_g - 1/2, clamped to the
// grid; the 2x2 stencil starts at (min(floor v, H-2), min(floor u, W-2)).
// The coordinate transform stays in float32 without losing the cell
// fraction: x - x0 is formed exactly as an unevaluated sum hi + lo (Knuth's
// TwoSum), the cell is estimated from hi / r_g and the remainder
// x - x0 - (j + 1/2) r_g is taken from hi, lo and the exact error of the
// product (j + 1/2) r_g (one fma); a plain float32 u would carry an error of
// 6e-5 cells 100 m from the origin (3e-3 in a cost of 50), this one about
// 1e-7 cells.  Interpolation and gradients are float32.  Invalid ground
// (-inf) reads as h_k - d_s.  Along an axis where the query was clamped the
// gradient is zero.
#include <cuda_runtime.h>
#include <math.h>

#include "tct_internal.cuh"

namespace tct {
namespace {

constexpr int kThreads = 256;

struct SampleGeo {
    float x0, y0, res;
    float inv_res, d_s, z_min;
    int32_t W, H, N;
};

SampleGeo sample_geo(const tct_grid &g) {
    SampleGeo s;
    s.x0 = g.x0;
    s.y0 = g.y0;
    s.res = g.res;
    s.inv_res = (float)(1.0 / (double)g.res);
    s.d_s = g.d_s;
    s.z_min = g.z_min;
    s.W = g.W;
    s.H = g.H;
    s.N = g.n_slices;
    return s;
}

struct Stencil {
    int64_t base;        // slice offset + first cell
    int dj, di;          // neighbour steps (0 on a one-cell axis)
    float fu, fv;
    bool cu, cv;         // clamped along x / y
};

// One axis of the transform u = (x - x0) / r - 1/2 on n cells: the first
// stencil cell j0, the fraction f in [0, 1] and whether u was clamped to
// [0, n-1] (as the FP64 definition clamps it).
__device__ __forceinline__ void locate_axis(float x, float x0, float r, float inv_r, int n,
                                            int &j0, float &f, bool &clamped) {
    // TwoSum: hi + lo == x - x0 exactly
    const float nx0 = -x0;
    const float hi = __fadd_rn(x, nx0);
    const float xv = __fsub_rn(hi, nx0);
    const float nv = __fsub_rn(hi, xv);
    const float lo = __fadd_rn(__fsub_rn(x, xv), __fsub_rn(nx0, nv));
    // cell estimate, then the remainder d - (j + 1/2) r with the exact
    // rounding error of the product
    const float q = __fmul_rn(hi, inv_r);
    int j = (int)floorf(__fsub_rn(q, 0.5f));
    j = max(-2, min(j, n + 1));
    float rem = 0.0f;
#pragma unroll 1
    for (int it = 0; it < 4; ++it) {
        const float t = (float)j + 0.5f;
        const float p = __fmul_rn(t, r);
        const float pe = __fmaf_rn(t, r, -p);
        rem = __fadd_rn(__fsub_rn(hi, p), __fsub_rn(lo, pe));
        if (rem < 0.0f) --j;
        else if (rem >= r) ++j;
        else break;
    }
    clamped = false;
    if (j < 0) {                                   // u < 0
        j0 = 0; f = 0.0f; clamped = true;
    } else if (j > n - 1 || (j == n - 1 && rem > 0.0f)) {   // u > n - 1
        j0 = n - 2; f = 1.0f; clamped = true;
    } else {
        j0 = j; f = fminf(__fmul_rn(rem, inv_r), 1.0f);
        if (j0 > n - 2) { j0 = n - 2; f = 1.0f; }  // u == n - 1 exactly
    }
    if (n < 2) { j0 = 0; f = 0.0f; }
}

__device__ __forceinline__ Stencil locate(const SampleGeo &g, float x, float y, int k) {
    Stencil s;
    int j0, i0;
    locate_axis(x, g.x0, g.res, g.inv_res, g.W, j0, s.fu, s.cu);
    locate_axis(y, g.y0, g.res, g.inv_res, g.H, i0, s.fv, s.cv);
    s.dj = g.W > 1 ? 1 : 0;
    s.di = g.H > 1 ? g.W : 0;
    s.base = (int64_t)k * g.W * g.H + (int64_t)i0 * g.W + j0;
    return s;
}

__device__ __forceinline__ float read(const float *__restrict__ L, int64_t idx, float fill) {
    const float v = __ldg(L + idx);
    return v > -INFINITY ? v : fill;
}

// value and gradient of the interpolant of L at the stencil
__device__ __forceinline__ void interp(const float *__restrict__ L, const Stencil &s, float fill,
                                       float inv_res, float &val, float &gx, float &gy) {
    const float c00 = read(L, s.base, fill), c01 = read(L, s.base + s.dj, fill);
    const float c10 = read(L, s.base + s.di, fill), c11 = read(L, s.base + s.di + s.dj, fill);
    const float fu = s.fu, fv = s.fv;
    val = (1.0f - fu) * (1.0f - fv) * c00 + fu * (1.0f - fv) * c01 + (1.0f - fu) * fv * c10 +
          fu * fv * c11;
    gx = (s.cu || s.dj == 0) ? 0.0f : ((1.0f - fv) * (c01 - c00) + fv * (c11 - c10)) * inv_res;
    gy = (s.cv || s.di == 0) ? 0.0f : ((1.0f - fu) * (c10 - c00) + fu * (c11 - c01)) * inv_res;
}

__device__ __forceinline__ bool query_ok(const SampleGeo &g, float x, float y, int k) {
    return k >= 0 && k < g.N && isfinite(x) && isfinite(y);
}

__global__ void __launch_bounds__(kThreads)
k_sample(SampleGeo g, const float *__restrict__ cost, const float *__restrict__ ground,
         const float2 *__restrict__ xy, const int32_t *__restrict__ slice, int64_t q,
         float *__restrict__ cost_out, float *__restrict__ elev_out, tct_stats *stats) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= q) return;
    const float2 p = xy[t];
    const int k = slice[t];
    if (!query_ok(g, p.x, p.y, k)) {
        if (cost_out) cost_out[t] = NAN;
        if (elev_out) elev_out[t] = NAN;
        if (stats) atomicOr(&stats->status, TCT_DEV_BAD_QUERY);
        return;
    }
    const Stencil s = locate(g, p.x, p.y, k);
    float v, gx, gy;
    if (cost_out) {
        interp(cost, s, 0.0f, g.inv_res, v, gx, gy);
        cost_out[t] = v;
    }
    if (elev_out) {
        const float fill = __fmaf_rn((float)(k + 1), g.d_s, g.z_min) - g.d_s;
        interp(ground, s, fill, g.inv_res, v, gx, gy);
        elev_out[t] = v;
    }
}

__global__ void __launch_bounds__(kThreads)
k_sample_backward(SampleGeo g, const float *__restrict__ cost, const float *__restrict__ ground,
                  const float2 *__restrict__ xy, const int32_t *__restrict__ slice, int64_t q,
                  const float *__restrict__ gcost, const float *__restrict__ gelev,
                  float2 *__restrict__ gxy) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= q) return;
    const float2 p = xy[t];
    const int k = slice[t];
    if (!query_ok(g, p.x, p.y, k)) {
        gxy[t] = make_float2(NAN, NAN);
        return;
    }
    const Stencil s = locate(g, p.x, p.y, k);
    float2 out = make_float2(0.0f, 0.0f);
    float v, gx, gy;
    if (gcost) {
        interp(cost, s, 0.0f, g.inv_res, v, gx, gy);
        const float w = gcost[t];
        out.x = fmaf(w, gx, out.x);
        out.y = fmaf(w, gy, out.y);
    }
    if (gelev) {
        const float fill = __fmaf_rn((float)(k + 1), g.d_s, g.z_min) - g.d_s;
        interp(ground, s, fill, g.inv_res, v, gx, gy);
        const float w = gelev[t];
        out.x = fmaf(w, gx, out.x);
        out.y = fmaf(w, gy, out.y);
    }
    gxy[t] = out;
}

// One CTA per path: all `steps` descent steps on
//   J = sum_w c^T(x_w) + lambda sum_{w=1}^{len-2} |x_{w+1} - 2 x_w + x_{w-1}|^2
// with the end points fixed, the waypoints held in shared memory.
constexpr int kRefineThreads = 256;
constexpr int kRefinePer = TCT_MAX_PATH_LEN / kRefineThreads;

__global__ void __launch_bounds__(kRefineThreads)
k_refine(SampleGeo g, const float *__restrict__ cost, const int32_t *__restrict__ slice,
         int32_t len, int32_t steps, float eta, float lambda, float2 *__restrict__ xy) {
    __shared__ float2 X[TCT_MAX_PATH_LEN];
    __shared__ float2 D[TCT_MAX_PATH_LEN];
    const int64_t base = (int64_t)blockIdx.x * len;
    for (int w = threadIdx.x; w < len; w += kRefineThreads) X[w] = xy[base + w];
    __syncthreads();
    for (int it = 0; it < steps; ++it) {
        for (int w = threadIdx.x; w < len; w += kRefineThreads) {
            float2 d = make_float2(0.0f, 0.0f);
            if (w >= 1 && w <= len - 2) {
                d.x = X[w + 1].x - 2.0f * X[w].x + X[w - 1].x;
                d.y = X[w + 1].y - 2.0f * X[w].y + X[w - 1].y;
            }
            D[w] = d;
        }
        __syncthreads();
        float2 nx[kRefinePer];
#pragma unroll
        for (int r = 0; r < kRefinePer; ++r) {
            const int w = threadIdx.x + r * kRefineThreads;
            if (w >= len) break;
            float2 p = X[w];
            if (w >= 1 && w <= len - 2) {
                const int k = slice[base + w];
                float gx = 0.0f, gy = 0.0f;
                if (query_ok(g, p.x, p.y, k)) {
                    float v;
                    interp(cost, locate(g, p.x, p.y, k), 0.0f, g.inv_res, v, gx, gy);
                }
                float sx = -2.0f * D[w].x, sy = -2.0f * D[w].y;
                if (w - 1 >= 1) { sx += D[w - 1].x; sy += D[w - 1].y; }
                if (w + 1 <= len - 2) { sx += D[w + 1].x; sy += D[w + 1].y; }
                gx = fmaf(2.0f * lambda, sx, gx);
                gy = fmaf(2.0f * lambda, sy, gy);
                p.x = fmaf(-eta, gx, p.x);
                p.y = fmaf(-eta, gy, p.y);
            }
            nx[r] = p;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kRefinePer; ++r) {
            const int w = threadIdx.x + r * kRefineThreads;
            if (w >= len) break;
            X[w] = nx[r];
        }
        __syncthreads();
    }
    for (int w = threadIdx.x; w < len; w += kRefineThreads) xy[base + w] = X[w];
}

bool sample_grid_ok(const tct_grid *g) {
    return g && g->W >= 1 && g->H >= 1 && g->n_slices >= 1 && g->res > 0.0f && isfinite(g->res) &&
           isfinite(g->x0) && isfinite(g->y0) && isfinite(g->z_min) && isfinite(g->d_s);
}

unsigned blocks_for(int64_t q) { return (unsigned)((q + kThreads - 1) / kThreads); }

}  // namespace
}  // namespace tct

using namespace tct;

extern "C" int tct_sample_cost(const tct_grid *grid, const float *d_cost, const float *d_ground,
                               const float *d_xy, const int32_t *d_slice, int64_t q,
                               float *d_cost_out, float *d_elev_out, tct_stats *d_stats,
                               tct_stream stream) {
    if (!sample_grid_ok(grid) || q < 0 || q > TCT_MAX_POINTS) return TCT_ERR_INVALID_ARG;
    if (q > 0 && (!d_xy || !d_slice)) return TCT_ERR_INVALID_ARG;
    if ((d_cost_out && !d_cost) || (d_elev_out && !d_ground)) return TCT_ERR_INVALID_ARG;
    if (q == 0 || (!d_cost_out && !d_elev_out)) return TCT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_sample<<<blocks_for(q), kThreads, 0, s>>>(sample_geo(*grid), d_cost, d_ground,
                                                 reinterpret_cast<const float2 *>(d_xy), d_slice, q,
                                                 d_cost_out, d_elev_out, d_stats);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? TCT_OK : TCT_ERR_CUDA;
}

extern "C" int tct_sample_cost_backward(const tct_grid *grid, const float *d_cost,
                                        const float *d_ground, const float *d_xy,
                                        const int32_t *d_slice, int64_t q, const float *d_gcost,
                                        const float *d_gelev, float *d_gxy, tct_stream stream) {
    if (!sample_grid_ok(grid) || q < 0 || q > TCT_MAX_POINTS) return TCT_ERR_INVALID_ARG;
    if (q > 0 && (!d_xy || !d_slice || !d_gxy)) return TCT_ERR_INVALID_ARG;
    if ((d_gcost && !d_cost) || (d_gelev && !d_ground)) return TCT_ERR_INVALID_ARG;
    if (q == 0) return TCT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_sample_backward<<<blocks_for(q), kThreads, 0, s>>>(
        sample_geo(*grid), d_cost, d_ground, reinterpret_cast<const float2 *>(d_xy), d_slice, q,
        d_gcost, d_gelev, reinterpret_cast<float2 *>(d_gxy));
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? TCT_OK : TCT_ERR_CUDA;
}

extern "C" int tct_refine_paths(const tct_grid *grid, const float *d_cost, const int32_t *d_slice,
                                int32_t paths, int32_t len, int32_t steps, float eta, float lambda,
                                float *d_xy, tct_stream stream) {
    if (!sample_grid_ok(grid) || paths < 0 || len < 2 || steps < 0) return TCT_ERR_INVALID_ARG;
    if (len > TCT_MAX_PATH_LEN) return TCT_ERR_UNSUPPORTED;
    if (!isfinite(eta) || !isfinite(lambda)) return TCT_ERR_INVALID_ARG;
    if (paths == 0 || steps == 0) return TCT_OK;
    if (!d_cost || !d_slice || !d_xy) return TCT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    k_refine<<<paths, kRefineThreads, 0, s>>>(sample_geo(*grid), d_cost, d_slice, len, steps, eta,
                                              lambda, reinterpret_cast<float2 *>(d_xy));
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? TCT_OK : TCT_ERR_CUDA;
}
