/*
 * oracle.c -- plain, slow FP64 CPU oracle for point-cloud tomography
 * (Yang et al., "Efficient Global Navigational Planning in 3D Structures
 * based on Point Cloud Tomography", arXiv 2403.07631).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py
 * load it.  It shares no code, header, table or constant generator with the
 * CUDA library; it follows the paper's definitions directly, in the paper's
 * order, by brute force.
 *
 * Readings of the paper that this file implements (each also listed in the
 * design notes):
 *   - planes (Sec. III-A): h_k = z_min + (k+1) d_s for k = 0..N-1, rounded
 *     once to float32 (fmaf); the first plane sits d_s above the lowest point.
 *   - groups (Sec. III-A, Alg. 1): the lower group of plane k is z <= h_k,
 *     the upper group is z > h_k; e^G = max z of the lower group in the cell,
 *     e^C = min z of the upper group; empty -> invalid (-inf / +inf).
 *     The stored elevation is the point's own float z (-0 folded to +0).
 *   - rasterize: j = floor(fl32(fl32(x - x0) / r_g)), i likewise from y;
 *     row i runs along +y, column j along +x.  Evaluated here in double and
 *     rounded to float, which equals the float32 operation exactly because
 *     double has more than 2*24+2 bits (double rounding is innocuous for a
 *     single +,-,*,/).
 *   - gradient (Eq. 2): central differences over 2 r_g; a border cell or a
 *     cell whose centre or any of its four neighbours is invalid gets
 *     m^xy = m^grad = +inf.
 *   - p_s (Eq. 4): square patch of radius R_p without the centre; off-map
 *     neighbours count as not gentle but stay in the denominator.
 *   - inflation (Eq. 6): K in cell units, D_inf = d_inf / r_g and
 *     D_sm = (d_sm - r_g) / r_g, each rounded to 6 decimals; off-map taps
 *     contribute nothing.
 *   - invalid ground -> c^init = c^B; invalid ceiling -> d^I = +inf, c^I = 0.
 *   - simplification (Sec. III-C, Eq. 7-9): the sequential chain; Eq. 8 is
 *     taken against the last kept slice p, Eq. 9 against the original k+1;
 *     Eq. 8 holds vacuously while no slice is kept, Eq. 9 for k = N-1.
 *   - fragile cells: a cell whose travel cost depends on a comparison that
 *     lies within 1e-6 * max(1, |threshold|) of its threshold and that float32
 *     arithmetic might decide the other way (a comparison whose operand float32
 *     holds exactly, or whose outcome another barrier branch overrides, is not
 *     fragile).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)
#define ORACLE_ENONFINITE (-3)

#define ORACLE_MAX_SLICES 127
#define ORACLE_FRAGILE_REL 1e-6

typedef struct oracle_grid {
    float x0, y0, res;  /* origin of cell (0,0) and resolution r_g (m)   */
    int32_t W, H;       /* columns (x) and rows (y)                      */
    float d_s;          /* slice interval d_s (m)                        */
    float z_min;        /* height the first plane is offset from         */
    int32_t N;          /* number of slices                              */
} oracle_grid;

typedef struct oracle_params {
    float d_min, d_ref;               /* Eq. 1 heights (m)                */
    float theta_b, theta_s, theta_p;  /* Eq. 3-4 thresholds               */
    float c_b, alpha_d, alpha_b, alpha_s; /* Eq. 1, 3, 4 costs/scales     */
    float d_inf, d_sm;                /* Eq. 6 inflation distances (m)    */
    int32_t patch_radius;             /* R_p of the p_s patch (cells)     */
} oracle_params;

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int finite3(float x, float y, float z)
{
    return isfinite(x) && isfinite(y) && isfinite(z);
}

static float fold_zero(float z) { return z == 0.0f ? 0.0f : z; }

/* Section III-A: h_k = z_min + (k+1) d_s, one rounding to float32. */
static float plane_height(const oracle_grid *g, int k)
{
    return fmaf((float)(k + 1), g->d_s, g->z_min);
}

int oracle_plane_heights(const oracle_grid *g, float *h)
{
    if (!g || !h || g->N < 1 || g->N > ORACLE_MAX_SLICES) return ORACLE_EINVAL;
    for (int k = 0; k < g->N; ++k) h[k] = plane_height(g, k);
    return ORACLE_OK;
}

/* fl32(fl32(x - x0) / r_g), computed in double and rounded once per op. */
static float grid_coord(float x, float x0, float res)
{
    float d = (float)((double)x - (double)x0);
    return (float)((double)d / (double)res);
}

/* Alg. 1 "rasterize": returns 1 and the cell when the point lies on the grid. */
static int rasterize(const oracle_grid *g, float x, float y, int *i, int *j)
{
    float u = grid_coord(x, g->x0, g->res);
    float v = grid_coord(y, g->y0, g->res);
    if (!(u >= 0.0f) || !(u < (float)g->W)) return 0;
    if (!(v >= 0.0f) || !(v < (float)g->H)) return 0;
    *j = (int)floorf(u);
    *i = (int)floorf(v);
    return 1;
}

/* min/max of x, y, z over the finite points; out = {xmin,ymin,zmin,xmax,ymax,zmax}. */
int oracle_bounds(const float *xyz, int64_t n, int32_t stride, double *out,
                  int64_t *n_nonfinite)
{
    if (!xyz || !out || (stride != 3 && stride != 4) || n < 0) return ORACLE_EINVAL;
    double lo[3] = {INFINITY, INFINITY, INFINITY};
    double hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int64_t bad = 0;
    for (int64_t u = 0; u < n; ++u) {
        const float *p = xyz + u * stride;
        if (!finite3(p[0], p[1], p[2])) { ++bad; continue; }
        for (int a = 0; a < 3; ++a) {
            double v = (double)fold_zero(p[a]);
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    }
    for (int a = 0; a < 3; ++a) { out[a] = lo[a]; out[3 + a] = hi[a]; }
    if (n_nonfinite) *n_nonfinite = bad;
    return ORACLE_OK;
}

/*
 * Section III-A: the grid covers the cloud (origin at its minimum x, y) and
 * N is the smallest number of planes whose last one lies at or above the
 * highest point.
 */
int oracle_derive_grid(const float *xyz, int64_t n, int32_t stride, float res,
                       float d_s, oracle_grid *g)
{
    if (!g || !(res > 0.0f) || !(d_s > 0.0f)) return ORACLE_EINVAL;
    double b[6];
    int64_t bad = 0;
    int rc = oracle_bounds(xyz, n, stride, b, &bad);
    if (rc) return rc;
    if (!(b[0] <= b[3])) return ORACLE_EINVAL; /* no finite point */
    g->x0 = (float)b[0];
    g->y0 = (float)b[1];
    g->res = res;
    g->W = (int32_t)floorf(grid_coord((float)b[3], g->x0, res)) + 1;
    g->H = (int32_t)floorf(grid_coord((float)b[4], g->y0, res)) + 1;
    g->d_s = d_s;
    g->z_min = (float)b[2];
    float zmax = (float)b[5];
    for (int N = 1; N <= ORACLE_MAX_SLICES; ++N) {
        g->N = N;
        if (plane_height(g, N - 1) >= zmax) return ORACLE_OK;
    }
    return ORACLE_EINVAL;
}

/*
 * The construction part of Algorithm 1, brute force: every slice scans every point.
 * eG, eC: [N][H][W] float32.  When zmin_from_data is set, g->z_min is
 * replaced by the lowest finite z of the whole cloud (the first step of Alg. 1).
 */
int oracle_build(const float *xyz, int64_t n, int32_t stride, oracle_grid *g,
                 int32_t zmin_from_data, float *eG, float *eC, int64_t *n_dropped,
                 int64_t *n_nonfinite)
{
    if (!xyz || !g || !eG || !eC || (stride != 3 && stride != 4) || n < 0) return ORACLE_EINVAL;
    if (g->N < 1 || g->N > ORACLE_MAX_SLICES || g->W < 1 || g->H < 1) return ORACLE_EINVAL;
    if (!(g->res > 0.0f) || !(g->d_s > 0.0f)) return ORACLE_EINVAL;
    int64_t bad = 0, dropped = 0;
    if (zmin_from_data) {
        double b[6];
        oracle_bounds(xyz, n, stride, b, &bad);
        g->z_min = isfinite(b[2]) ? (float)b[2] : 0.0f;
    }
    for (int64_t u = 0; u < n; ++u) {
        const float *p = xyz + u * stride;
        int i, j;
        if (!finite3(p[0], p[1], p[2])) continue;
        if (!rasterize(g, p[0], p[1], &i, &j)) ++dropped;
    }
    if (!zmin_from_data) {
        for (int64_t u = 0; u < n; ++u) {
            const float *p = xyz + u * stride;
            if (!finite3(p[0], p[1], p[2])) ++bad;
        }
    }
    const int64_t HW = (int64_t)g->H * g->W;
    const int N = g->N;
    int k;
#pragma omp parallel for schedule(dynamic, 1)
    for (k = 0; k < N; ++k) {
        const float h = plane_height(g, k);
        float *G = eG + (int64_t)k * HW;
        float *C = eC + (int64_t)k * HW;
        for (int64_t c = 0; c < HW; ++c) { G[c] = -INFINITY; C[c] = INFINITY; }
        for (int64_t u = 0; u < n; ++u) {
            const float *p = xyz + u * stride;
            int i, j;
            if (!finite3(p[0], p[1], p[2])) continue;
            if (!rasterize(g, p[0], p[1], &i, &j)) continue;
            const float z = fold_zero(p[2]);
            const int64_t c = (int64_t)i * g->W + j;
            if (z <= h) {            /* lower group: projected up, ground */
                if (z > G[c]) G[c] = z;
            } else {                 /* upper group: projected down, ceiling */
                if (z < C[c]) C[c] = z;
            }
        }
    }
    if (n_dropped) *n_dropped = dropped;
    if (n_nonfinite) *n_nonfinite = bad;
    return bad ? ORACLE_ENONFINITE : ORACLE_OK;
}

static double round6(double x) { return nearbyint(x * 1e6) / 1e6; }

/* Eq. 6 in cell units: D_inf = d_inf / r_g, D_sm = (d_sm - r_g) / r_g. */
static double kernel_weight(double d, double Dinf, double Dsm)
{
    if (Dsm <= 0.0) return d <= Dinf ? 1.0 : 0.0;
    double v = 1.0 - (d - Dinf) / Dsm;
    if (v > 1.0) v = 1.0;
    if (v < 0.0) v = 0.0;
    return v;
}

/*
 * The inflation kernel K(m, n) of Eq. 6 on a (2R+1) x (2R+1) window; R is the
 * largest offset with a positive weight.  K is written row-major (n, m).
 */
int oracle_kernel(const oracle_params *p, float res, int32_t *radius, double *K,
                  int32_t capacity)
{
    if (!p || !radius || !(res > 0.0f)) return ORACLE_EINVAL;
    const double Dinf = round6((double)p->d_inf / (double)res);
    const double Dsm = round6(((double)p->d_sm - (double)res) / (double)res);
    int R = 0;
    while (R < 64 && kernel_weight((double)(R + 1), Dinf, Dsm) > 0.0) ++R;
    *radius = R;
    const int side = 2 * R + 1;
    if (!K) return ORACLE_OK;
    if (side * side > capacity) return ORACLE_EINVAL;
    for (int n = -R; n <= R; ++n)
        for (int m = -R; m <= R; ++m)
            K[(n + R) * side + (m + R)] =
                kernel_weight(sqrt((double)(m * m + n * n)), Dinf, Dsm);
    return ORACLE_OK;
}

static int near_threshold(double v, double theta)
{
    if (!isfinite(v)) return 0;
    double tol = ORACLE_FRAGILE_REL * (fabs(theta) > 1.0 ? fabs(theta) : 1.0);
    return fabs(v - theta) <= tol;
}

/*
 * Section III-B, Eq. 1-6, on every slice.  Inputs eG, eC: [N][H][W] float32
 * (-inf / +inf mark invalid cells).  Outputs: cT [N][H][W] double, mask
 * (c^T < c^B) and fragile flags [N][H][W] uint8 (bit 0: the cost is not
 * pinned by FP64, bit 1: the mask is not).  aux, when not NULL,
 * receives five [N][H][W] double layers: m^xy, m^grad, c^I, c^G, c^init.
 */
int oracle_evaluate(const oracle_grid *g, const oracle_params *p, const float *eG,
                    const float *eC, double *cT, uint8_t *mask, uint8_t *fragile,
                    double *aux)
{
    if (!g || !p || !eG || !eC || !cT || !mask || !fragile) return ORACLE_EINVAL;
    if (g->N < 1 || g->W < 1 || g->H < 1 || !(g->res > 0.0f)) return ORACLE_EINVAL;
    if (p->patch_radius < 0 || p->patch_radius > 16) return ORACLE_EINVAL;
    int32_t R;
    if (oracle_kernel(p, g->res, &R, NULL, 0)) return ORACLE_EINVAL;
    const int side = 2 * R + 1;
    double *K = (double *)malloc(sizeof(double) * side * side);
    if (!K) return ORACLE_ENOMEM;
    oracle_kernel(p, g->res, &R, K, side * side);

    const int W = g->W, H = g->H, N = g->N, Rp = p->patch_radius;
    const int64_t HW = (int64_t)H * W;
    const double res = (double)g->res;
    const double c_b = p->c_b, d_min = p->d_min, d_ref = p->d_ref;
    const double th_b = p->theta_b, th_s = p->theta_s, th_p = p->theta_p;
    const double a_d = p->alpha_d, a_b = p->alpha_b, a_s = p->alpha_s;
    const int n_patch = (2 * Rp + 1) * (2 * Rp + 1) - 1;
    int failed = 0;
    int k;

#pragma omp parallel for schedule(dynamic, 1)
    for (k = 0; k < N; ++k) {
        const float *G = eG + (int64_t)k * HW;
        const float *C = eC + (int64_t)k * HW;
        double *mxy = (double *)malloc(sizeof(double) * HW);
        double *mgr = (double *)malloc(sizeof(double) * HW);
        double *cI = (double *)malloc(sizeof(double) * HW);
        double *cG = (double *)malloc(sizeof(double) * HW);
        double *ci = (double *)malloc(sizeof(double) * HW);
        uint8_t *fi = (uint8_t *)malloc(HW);
        if (!mxy || !mgr || !cI || !cG || !ci || !fi) {
#pragma omp atomic write
            failed = 1;
            free(mxy); free(mgr); free(cI); free(cG); free(ci); free(fi);
            continue;
        }
        /* Eq. 2: finite-difference gradient of the ground layer. */
        for (int i = 0; i < H; ++i) {
            for (int j = 0; j < W; ++j) {
                const int64_t c = (int64_t)i * W + j;
                double ax = INFINITY, ag = INFINITY;
                if (i > 0 && i < H - 1 && j > 0 && j < W - 1 &&
                    G[c] > -INFINITY && G[c - 1] > -INFINITY && G[c + 1] > -INFINITY &&
                    G[c - W] > -INFINITY && G[c + W] > -INFINITY) {
                    const double gx = ((double)G[c + 1] - (double)G[c - 1]) / (2.0 * res);
                    const double gy = ((double)G[c + W] - (double)G[c - W]) / (2.0 * res);
                    ax = fmax(fabs(gx), fabs(gy));
                    ag = sqrt(gx * gx + gy * gy);
                }
                mxy[c] = ax;
                mgr[c] = ag;
            }
        }
        /* Eq. 1, 3, 4, 5: interval cost, terrain cost, initial cost. */
        for (int i = 0; i < H; ++i) {
            for (int j = 0; j < W; ++j) {
                const int64_t c = (int64_t)i * W + j;
                /* p_s: share of the patch neighbours that are gentle surfaces */
                int count = 0, frag_patch = 0;
                for (int di = -Rp; di <= Rp; ++di) {
                    for (int dj = -Rp; dj <= Rp; ++dj) {
                        if (di == 0 && dj == 0) continue;
                        const int ii = i + di, jj = j + dj;
                        if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
                        const double m = mgr[(int64_t)ii * W + jj];
                        if (m < th_s) ++count;
                        if (near_threshold(m, th_s)) frag_patch = 1;
                    }
                }
                const double ps = n_patch > 0 ? (double)count / (double)n_patch : 0.0;
                /* Eq. 1 */
                double dI = INFINITY, vI;
                int bar_I = 0, frag_I = 0;
                if (C[c] < INFINITY && G[c] > -INFINITY) dI = (double)C[c] - (double)G[c];
                if (dI < d_min) { vI = c_b; bar_I = 1; }
                else if (isinf(dI)) vI = 0.0;
                else vI = fmax(0.0, a_d * (d_ref - dI));
                /* a difference of two floats that float32 holds exactly is
                 * compared identically in either precision */
                if (isfinite(dI) && near_threshold(dI, d_min) && (double)(float)dI != dI) frag_I = 1;
                /* Eq. 3 and Eq. 4 */
                double vG;
                int bar_G = 0, frag_G = 0;
                if (mxy[c] > th_b) { vG = c_b; bar_G = 1; }
                else if (mgr[c] < th_s) vG = a_s * (mgr[c] / th_s) * (mgr[c] / th_s);
                else if (ps > th_p) vG = a_b * (mxy[c] / th_b) * (mxy[c] / th_b);
                else { vG = c_b; bar_G = 1; }
                if (near_threshold(mxy[c], th_b)) frag_G = 1;
                else if (mxy[c] > th_b) frag_G = 0;
                else if (near_threshold(mgr[c], th_s)) frag_G = 1;
                else if (mgr[c] < th_s) frag_G = 0;
                else frag_G = frag_patch;           /* Eq. 4 branch: p_s decides */
                /* Eq. 5; a cell without ground is a barrier */
                const int valid = G[c] > -INFINITY;
                double v = valid ? fmin(c_b, vI + vG) : c_b;
                int frag = 0;
                if (valid) {
                    if (frag_I && !(bar_G && !frag_G)) frag = 1;
                    if (frag_G && !(bar_I && !frag_I)) frag = 1;
                    /* a continuous sum that meets the clip at c^B */
                    if (!bar_I && !bar_G && near_threshold(vI + vG, c_b)) frag = 1;
                }
                cI[c] = vI;
                cG[c] = vG;
                ci[c] = v;
                fi[c] = (uint8_t)frag;
            }
        }
        /*
         * Eq. 6 and the sliding window: max of K (Hadamard) c^init.  A fragile
         * c^init may take any value in [0, c^B] in float32 arithmetic, so the
         * window also yields bounds lo <= c^T <= hi; fragile bit 0 marks a
         * cost that is not pinned (lo != hi, or within the tolerance of c^B),
         * bit 1 a mask decision that is not.
         */
        double *T = cT + (int64_t)k * HW;
        uint8_t *M = mask + (int64_t)k * HW;
        uint8_t *F = fragile + (int64_t)k * HW;
        for (int i = 0; i < H; ++i) {
            for (int j = 0; j < W; ++j) {
                double best = 0.0, lo = 0.0, hi = 0.0;
                for (int n = -R; n <= R; ++n) {
                    for (int m = -R; m <= R; ++m) {
                        const double w = K[(n + R) * side + (m + R)];
                        const int ii = i + n, jj = j + m;
                        if (w <= 0.0) continue;
                        if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
                        const int64_t t = (int64_t)ii * W + jj;
                        const double v = w * ci[t];
                        if (v > best) best = v;
                        if (fi[t]) {
                            if (w * c_b > hi) hi = w * c_b;
                        } else {
                            if (v > lo) lo = v;
                            if (v > hi) hi = v;
                        }
                    }
                }
                const int64_t c = (int64_t)i * W + j;
                T[c] = best;
                M[c] = best < c_b ? 1 : 0;
                /* exactly c^B comes from a branch or the clip (exact in any
                 * precision); a value merely close to it is fragile */
                const int edge = best != c_b && near_threshold(best, c_b);
                const int fcost = edge || lo != hi;
                const int fmask = edge || ((lo < c_b) != (hi < c_b));
                F[c] = (uint8_t)(fcost | (fmask << 1));
            }
        }
        if (aux) {
            memcpy(aux + 0 * N * HW + (int64_t)k * HW, mxy, sizeof(double) * HW);
            memcpy(aux + 1 * N * HW + (int64_t)k * HW, mgr, sizeof(double) * HW);
            memcpy(aux + 2 * N * HW + (int64_t)k * HW, cI, sizeof(double) * HW);
            memcpy(aux + 3 * N * HW + (int64_t)k * HW, cG, sizeof(double) * HW);
            memcpy(aux + 4 * N * HW + (int64_t)k * HW, ci, sizeof(double) * HW);
        }
        free(mxy); free(mgr); free(cI); free(cG); free(ci); free(fi);
    }
    free(K);
    return failed ? ORACLE_ENOMEM : ORACLE_OK;
}

/* Is the FP64 comparison a < b too close to call for float32 arithmetic? */
static int close_pair(double a, double b)
{
    if (a == b) return 0;
    double s = fabs(b) > 1.0 ? fabs(b) : 1.0;
    return fabs(a - b) <= ORACLE_FRAGILE_REL * s;
}

/*
 * Section III-C, Eq. 7-9: the sequential simplification chain.  Starting
 * with no kept slice, slice k is kept when it has at least one unique
 * traversable cell; a cell is unique when Eq. 8 holds against the last kept
 * slice p (vacuous while none is kept) and Eq. 9 holds against the original
 * slice k+1 (vacuous for k = N-1).  keep_ends keeps slices 0 and N-1 in any
 * case.  robust[0] is cleared when some decision depends on a fragile cell
 * or on a cost comparison closer than the fragile tolerance.  counts, when
 * not NULL, receives per slice the unique cells, the unique cells that no
 * fragile comparison touches, and the cells that could be unique if every
 * fragile comparison went the other way ([N][3]).
 */
int oracle_simplify(int32_t N, int32_t H, int32_t W, const float *eG, const double *cT,
                    const uint8_t *fragile, double c_b, int32_t keep_ends, uint8_t *keep,
                    uint8_t *robust, int64_t *counts)
{
    if (!eG || !cT || !keep || N < 1 || H < 1 || W < 1) return ORACLE_EINVAL;
    const int64_t HW = (int64_t)H * W;
    int p = -1;
    int ok = 1;
    for (int k = 0; k < N; ++k) {
        int64_t unique = 0, sure = 0, maybe = 0;
        const float *Gk = eG + (int64_t)k * HW;
        const double *Tk = cT + (int64_t)k * HW;
        for (int64_t c = 0; c < HW; ++c) {
            const int fk = fragile ? (fragile[(int64_t)k * HW + c] & 1) : 0;
            const int fkm = fragile ? ((fragile[(int64_t)k * HW + c] >> 1) & 1) : 0;
            const int trav = Tk[c] < c_b;
            if (!trav && !fkm) continue;
            /* Eq. 8 against the last kept slice */
            int e8 = 1, f8 = 0;
            if (p >= 0) {
                const double dg = (double)Gk[c] - (double)eG[(int64_t)p * HW + c];
                const double cp = cT[(int64_t)p * HW + c];
                e8 = (dg > 0.0) || (Tk[c] < cp);
                if (!(dg > 0.0)) {
                    const int fp = fragile ? (fragile[(int64_t)p * HW + c] & 1) : 0;
                    f8 = fk || fp || close_pair(Tk[c], cp);
                }
            }
            /* Eq. 9 against the next original slice */
            int e9 = 1, f9 = 0;
            if (k < N - 1) {
                const double dg = (double)eG[(int64_t)(k + 1) * HW + c] - (double)Gk[c];
                const double cn = cT[(int64_t)(k + 1) * HW + c];
                e9 = (dg > 0.0) || (Tk[c] < cn);
                if (!(dg > 0.0)) {
                    const int fn = fragile ? (fragile[(int64_t)(k + 1) * HW + c] & 1) : 0;
                    f9 = fk || fn || close_pair(Tk[c], cn);
                }
            }
            if (trav && e8 && e9) ++unique;
            if (trav && !fkm && e8 && !f8 && e9 && !f9) ++sure;
            if ((trav || fkm) && (e8 || f8) && (e9 || f9)) ++maybe;
        }
        int kept = unique > 0;
        if ((sure > 0) != (maybe > 0)) ok = 0;
        if (counts) {
            counts[3 * k + 0] = unique;
            counts[3 * k + 1] = sure;
            counts[3 * k + 2] = maybe;
        }
        if (keep_ends && (k == 0 || k == N - 1)) kept = 1;
        keep[k] = (uint8_t)kept;
        if (kept) p = k;
    }
    if (robust) robust[0] = (uint8_t)ok;
    return ORACLE_OK;
}

/*
 * Cost and elevation queries of the trajectory program (Sec. III-E, Eq. 10
 * uses C(q) and e^G(q)): bilinear interpolation of slice k on the lattice of
 * cell centres.  u = (x - x0)/r_g - 1/2, v = (y - y0)/r_g - 1/2, clamped to
 * [0, W-1] x [0, H-1]; the 2x2 stencil starts at (min(floor(v), H-2),
 * min(floor(u), W-2)).  Invalid ground (-inf) reads as h_k - d_s.  The
 * gradient is that of the interpolant; along an axis where the query was
 * clamped it is zero.  out: value [q]; grad: [q][2] (d/dx, d/dy), may be NULL.
 * Slices outside [0, N) and non-finite queries give NaN.
 */
static double oracle_layer_at(const float *L, int W, int i, int j, double fill)
{
    const double v = (double)L[(int64_t)i * W + j];
    return v > -INFINITY ? v : fill;
}

/* One query at (x, y) on slice k; grad may be NULL. */
static void sample_one(const oracle_grid *g, const float *layer, int32_t is_ground, double x,
                       double y, int k, double *out, double *grad)
{
    const int W = g->W, H = g->H;
    const int64_t HW = (int64_t)W * H;
    const double r = (double)g->res;
    if (k < 0 || k >= g->N || !isfinite(x) || !isfinite(y)) {
        *out = NAN;
        if (grad) grad[0] = grad[1] = NAN;
        return;
    }
    const double fill = is_ground ? (double)plane_height(g, k) - (double)g->d_s : 0.0;
    const float *L = layer + (int64_t)k * HW;
    double u = (x - (double)g->x0) / r - 0.5, v = (y - (double)g->y0) / r - 0.5;
    int cu = 0, cv = 0;                     /* clamped along x / y */
    if (u < 0.0) { u = 0.0; cu = 1; }
    if (u > W - 1) { u = W - 1; cu = 1; }
    if (v < 0.0) { v = 0.0; cv = 1; }
    if (v > H - 1) { v = H - 1; cv = 1; }
    int j0 = (int)floor(u), i0 = (int)floor(v);
    if (j0 > W - 2) j0 = W - 2;
    if (i0 > H - 2) i0 = H - 2;
    if (j0 < 0) j0 = 0;
    if (i0 < 0) i0 = 0;
    const int j1 = W > 1 ? j0 + 1 : j0, i1 = H > 1 ? i0 + 1 : i0;
    const double fu = W > 1 ? u - j0 : 0.0, fv = H > 1 ? v - i0 : 0.0;
    const double c00 = oracle_layer_at(L, W, i0, j0, fill), c01 = oracle_layer_at(L, W, i0, j1, fill);
    const double c10 = oracle_layer_at(L, W, i1, j0, fill), c11 = oracle_layer_at(L, W, i1, j1, fill);
    *out = (1 - fu) * (1 - fv) * c00 + fu * (1 - fv) * c01 + (1 - fu) * fv * c10 + fu * fv * c11;
    if (grad) {
        grad[0] = (cu || W < 2) ? 0.0 : ((1 - fv) * (c01 - c00) + fv * (c11 - c10)) / r;
        grad[1] = (cv || H < 2) ? 0.0 : ((1 - fu) * (c10 - c00) + fu * (c11 - c01)) / r;
    }
}

/* Queries at float32 coordinates (the precision the library takes them in). */
int oracle_sample(const oracle_grid *g, const float *layer, int32_t is_ground, const float *xy,
                  const int32_t *slice, int64_t q, double *out, double *grad)
{
    if (!g || !layer || !xy || !slice || !out || q < 0) return ORACLE_EINVAL;
    for (int64_t t = 0; t < q; ++t)
        sample_one(g, layer, is_ground, (double)xy[2 * t], (double)xy[2 * t + 1], slice[t],
                   out + t, grad ? grad + 2 * t : NULL);
    return ORACLE_OK;
}

/* The same queries at FP64 coordinates (finite differences with steps far
 * below a float32 ulp of the coordinate). */
int oracle_sample_f64(const oracle_grid *g, const float *layer, int32_t is_ground,
                      const double *xy, const int32_t *slice, int64_t q, double *out,
                      double *grad)
{
    if (!g || !layer || !xy || !slice || !out || q < 0) return ORACLE_EINVAL;
    for (int64_t t = 0; t < q; ++t)
        sample_one(g, layer, is_ground, xy[2 * t], xy[2 * t + 1], slice[t], out + t,
                   grad ? grad + 2 * t : NULL);
    return ORACLE_OK;
}

/*
 * Gradient-based refinement of waypoint paths on one tomogram (an objective
 * of ours that uses the cost query C(q) of Eq. 10): for each path of `len`
 * waypoints (fixed end points), `steps` descent steps of size eta on
 *   J = sum_w c^T(x_w) + lambda sum_{w=1}^{len-2} |x_{w+1} - 2 x_w + x_{w-1}|^2,
 * every waypoint keeping the slice it starts on.  xy: [paths][len][2], updated
 * in place (double).
 */
int oracle_refine(const oracle_grid *g, const float *cost, const int32_t *slice, int32_t paths,
                  int32_t len, int32_t steps, double eta, double lambda, double *xy)
{
    if (!g || !cost || !slice || !xy || paths < 0 || len < 2 || steps < 0) return ORACLE_EINVAL;
    double *gr = (double *)malloc(sizeof(double) * 2 * len);
    double *d2 = (double *)malloc(sizeof(double) * 2 * len);
    float *pf = (float *)malloc(sizeof(float) * 2 * len);
    double *val = (double *)malloc(sizeof(double) * len);
    if (!gr || !d2 || !pf || !val) { free(gr); free(d2); free(pf); free(val); return ORACLE_ENOMEM; }
    for (int32_t p = 0; p < paths; ++p) {
        double *X = xy + (int64_t)p * len * 2;
        const int32_t *S = slice + (int64_t)p * len;
        for (int32_t s = 0; s < steps; ++s) {
            /* the sampler reads float coordinates, as the GPU does */
            for (int32_t w = 0; w < 2 * len; ++w) pf[w] = (float)X[w];
            int64_t nq = len;
            oracle_sample(g, cost, 0, pf, S, nq, val, gr);
            for (int32_t w = 0; w < 2 * len; ++w) d2[w] = 0.0;
            for (int32_t w = 1; w < len - 1; ++w)
                for (int a = 0; a < 2; ++a)
                    d2[2 * w + a] = X[2 * (w + 1) + a] - 2 * X[2 * w + a] + X[2 * (w - 1) + a];
            for (int32_t w = 1; w < len - 1; ++w) {
                for (int a = 0; a < 2; ++a) {
                    double sm = -2.0 * d2[2 * w + a];
                    if (w - 1 >= 1) sm += d2[2 * (w - 1) + a];
                    if (w + 1 <= len - 2) sm += d2[2 * (w + 1) + a];
                    gr[2 * w + a] += 2.0 * lambda * sm;
                }
            }
            for (int32_t w = 1; w < len - 1; ++w)
                for (int a = 0; a < 2; ++a) X[2 * w + a] -= eta * gr[2 * w + a];
        }
    }
    free(gr); free(d2); free(pf); free(val);
    return ORACLE_OK;
}
