// tct_stack_inc.cu -- dispatch of the incremental slice stack (tct_stack_inc.cuh)
// to its compiled window radii; one map is a batch of one.
#include "tct_stack_inc.cuh"

#include <algorithm>

namespace tct {
namespace {

using inc::BatchArgs;
using inc::IncMap;

IncMap inc_map(const StackArgs &a) {
    IncMap m;
    m.W = a.W; m.H = a.H; m.N = a.N;
    m.d_s = a.d_s; m.z_min = a.z_min; m.zmin_from_data = a.zmin_from_data && a.zkeys;
    m.zkeys = a.zkeys; m.start = a.start; m.zs = a.zs;
    m.gin = a.start ? nullptr : a.gin;
    m.cin = a.start ? nullptr : a.cin;
    m.falls = a.falls;
    m.ground = a.ground; m.ceil = a.ceil; m.cost = a.cost; m.mask = a.mask;
    m.upre = a.upre; m.ubits = a.ubits; m.stats = a.stats; m.keep = a.keep;
    return m;
}

cudaError_t dispatch(const BatchArgs &b, int tile, int ctas_per_sm, cudaStream_t s) {
    const int RK = b.c.rk, RP = b.c.patch_radius;
    if (RP == 2 && RK == 5) return inc::run_r5(b, tile, ctas_per_sm, s);
    if (RP == 2 && RK == 4) return inc::run_r4(b, tile, ctas_per_sm, s);
    if (RP == 2 && RK == 12) return inc::run_r12(b, tile, ctas_per_sm, s);
    return cudaErrorNotSupported;
}

// Tile edge lengths of a TCT_TILE_* shape.
void tile_dims(int tile, int *TW, int *TH) {
    *TW = tile == TCT_TILE_32 ? 32 : tile == TCT_TILE_128x56 ? 128 : 64;
    *TH = tile == TCT_TILE_32 ? 32
        : tile == TCT_TILE_64x56 || tile == TCT_TILE_128x56 ? 56
        : tile == TCT_TILE_64x40 ? 40 : 64;
}

// Resident CTAs per SM of an instance (the estimate its launch bounds use).
template <int RK, int RP>
int resident(int tile) {
    if (tile == TCT_TILE_32) return inc::Occupancy<RK, RP, 32, 32, inc::kStripSmall>::value;
    if (tile == TCT_TILE_64x56) return inc::Occupancy<RK, RP, 64, 56, 8>::value;
    if (tile == TCT_TILE_64x40) return inc::Occupancy<RK, RP, 64, 40, 8>::value;
    if (tile == TCT_TILE_128x56) return inc::Occupancy<RK, RP, 128, 56, 8>::value;
    return inc::Occupancy<RK, RP, 64, 64, 8>::value;
}

int resident_for(const EvalConsts &c, int tile) {
    if (c.rk == 5) return resident<5, 2>(tile);
    if (c.rk == 4) return resident<4, 2>(tile);
    return resident<12, 2>(tile);
}

}  // namespace

int choose_tile(const EvalConsts &c, int n_maps, const StackArgs *maps, int64_t small_tiles64) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t tiles64 = 0;
    for (int i = 0; i < n_maps; ++i)
        tiles64 += (int64_t)((maps[i].W + 63) / 64) * ((maps[i].H + 63) / 64);
    if (tiles64 < small_tiles64 * sms) return TCT_TILE_32;   // small maps: more, smaller CTAs
    // an SM's work over whole waves: waves x resident CTAs x the cells (with
    // halo) a CTA handles, divided by what co-resident CTAs gain by hiding
    // each other's barrier and memory waits (measured on the 1000 x 1000
    // parking structure: a second CTA per SM makes the slice stack 1.25x
    // faster, a third 1.05x more)
    static const double kResidentGain[] = {1.0, 1.0, 1.25, 1.31, 1.35};
    // One CTA of 28 warps (128 x 56) hides about as much as two of 14 (1.18x
    // against 1.25x, measured on the same map) and carries less halo per
    // cell.  Its 896 threads leave 72 registers a thread, fewer than the
    // window-radius-12 code takes in its other shapes (96 in the 64 x 40
    // tile), and there it measured slower (4000 x 4000 cave terrain: 12.70
    // against 12.28 ms for 64 x 40), so it is weighed for the smaller windows only.
    constexpr double kWideGain = 1.18;
    const bool wide_ok = c.rk <= 5;
    const int he = c.rk + c.patch_radius + 1;
    int best = TCT_TILE_64;
    double best_cost = INFINITY;
    for (int tile : {TCT_TILE_64, TCT_TILE_64x56, TCT_TILE_64x40, TCT_TILE_128x56}) {
        if (tile == TCT_TILE_128x56 && !wide_ok) continue;
        int TW, TH;
        tile_dims(tile, &TW, &TH);
        int64_t tiles = 0;
        for (int i = 0; i < n_maps; ++i)
            tiles += (int64_t)((maps[i].W + TW - 1) / TW) * ((maps[i].H + TH - 1) / TH);
        const int res = std::max(1, std::min(4, resident_for(c, tile)));
        const int64_t slots = (int64_t)sms * res;
        const int64_t waves = (tiles + slots - 1) / slots;
        // CTAs an SM runs at once in the last (or only) wave
        const int64_t per_sm = std::min<int64_t>(res, (tiles + sms - 1) / sms);
        const double gain = tile == TCT_TILE_128x56 ? kWideGain : kResidentGain[per_sm];
        const double cost = (double)waves * per_sm * (TW + 2 * he) * (TH + 2 * he) / gain;
        if (cost < best_cost) {
            best_cost = cost;
            best = tile;
        }
    }
    return best;
}

bool inc_supported(const EvalConsts &c, int n_slices) {
    if (n_slices > 255) return false;                // run starts are kept in bytes
    const int RK = c.rk, RP = c.patch_radius;
    return RP == 2 && (RK == 5 || RK == 4 || RK == 12);
}

cudaError_t launch_stack_inc(const StackArgs &a, int32_t *queue, int tile, cudaStream_t s) {
    return launch_stack_batched(a.c, 1, &a, queue, tile, 0, s);
}

cudaError_t launch_stack_batched(const EvalConsts &c, int n_maps, const StackArgs *maps,
                                 int32_t *queue, int tile, int ctas_per_sm, cudaStream_t s) {
    if (n_maps < 1 || n_maps > TCT_MAX_BATCH) return cudaErrorInvalidValue;
    for (int i = 0; i < n_maps; ++i)
        if (!inc_supported(c, maps[i].N)) return cudaErrorNotSupported;
    BatchArgs b;                 // kernel parameters, copied at launch
    b.c = c;
    b.n_maps = n_maps;
    b.queue = queue;
    // the chain runs in the last CTA when every map has its keep flags and
    // the first map brings the counter of finished CTAs
    b.done = maps[0].done;
    for (int i = 0; i < n_maps; ++i)
        if (!maps[i].keep) b.done = nullptr;
    // a single map's tiles may be cut into slice ranges (the uniqueness rows
    // then come from a pass over the finished layers, and the chain after it)
    b.split = n_maps == 1 && maps[0].split > 1 ? maps[0].split : 1;
    if (b.split > 1) b.done = nullptr;
    int TW, TH;
    tile_dims(tile, &TW, &TH);
    int total = 0;
    for (int i = 0; i < n_maps; ++i) {
        b.maps[i] = inc_map(maps[i]);
        b.item_start[i] = total;
        b.tiles_x[i] = (maps[i].W + TW - 1) / TW;
        total += b.tiles_x[i] * ((maps[i].H + TH - 1) / TH) * b.split;
    }
    b.item_start[n_maps] = total;
    b.total = total;
    return dispatch(b, tile, ctas_per_sm, s);
}

}  // namespace tct
