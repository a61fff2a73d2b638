// Path search across the kept slices of a tomogram (Sec. III-D): a host
// stage that reads the ground elevations and travel costs the GPU path
// produced (copied to host memory by the caller).
//
// Graph (Sec. III-D):
//  - a search state is a cell (i, j) on one kept slice m;
//  - cells (i, j) of adjacent kept slices whose ground elevations are equal
//    are one node in space; its node cost c^N is the minimum of their c^T
//    (equal elevations form one contiguous run, e^G being non-decreasing in
//    the slice index);
//  - on its slice a state connects to its eight neighbours; moving onto a
//    node costs its c^N plus the Euclidean distance between the two nodes
//    (in cell units, the elevation change divided by r_g), and a node with
//    c^N = c^B cannot be entered;
//  - a gateway joins (i, j, m) to (i, j, m+1) when their ground elevations
//    are equal and c^T is lower on m+1, and to (i, j, m-1) likewise going
//    down; being the same node, the move costs nothing;
//  - A* with the octile ("diagonal") distance to the goal cell as
//    heuristic, which never exceeds the remaining cost because every planar
//    step costs at least its length.
// The goal is reached on any slice whose cell is the goal node (the same
// cell, the same ground elevation as the goal's slice).

#include "tct.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <memory>
#include <mutex>
#include <queue>
#include <thread>
#include <vector>

namespace {

constexpr uint8_t kFromStart = 255;
constexpr uint8_t kFromBelow = 8;   // reached through a gateway from slice m-1
constexpr uint8_t kFromAbove = 9;   // reached through a gateway from slice m+1
constexpr int kDi[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
constexpr int kDj[8] = {-1, 0, 1, -1, 1, -1, 0, 1};

// Per-state search record, one cache-friendly 16 bytes: the best cost so
// far, the query it belongs to (records of earlier queries read as unseen)
// and the move that reached it.
struct Record {
    double g;
    uint32_t epoch;
    uint8_t from;
};

struct Search {
    std::vector<Record> rec;
    uint32_t current = 0;

    void prepare(size_t states)
    {
        if (rec.size() != states) {
            rec.assign(states, Record{0.0, 0u, kFromStart});
            current = 0;
        }
        if (++current == 0) {   // wrapped: forget every earlier query
            for (auto &r : rec) r.epoch = 0u;
            current = 1;
        }
    }
    bool seen(size_t s) const { return rec[s].epoch == current; }
};

struct Entry {
    double f, g;
    int64_t s;
    bool operator<(const Entry &o) const   // max-heap order: smallest f on top
    {
        if (f != o.f) return f > o.f;
        if (g != o.g) return g < o.g;     // ties: the deeper state first
        return s > o.s;
    }
};

}  // namespace

// What the search reads of one (kept slice, cell) state, packed together:
// its ground elevation, its c^T and the c^N of its node (c^B where the
// ground is invalid).
struct StateInfo {
    float e, t, cn;
};

struct tct_planner {
    int32_t H = 0, W = 0;
    float res = 0.f;
    float c_b = 0.f;
    std::vector<int32_t> kept;       // original index of kept slice m
    std::vector<StateInfo> info;     // [M][H][W]
    std::mutex mu;
    std::vector<std::unique_ptr<Search>> idle;

    int64_t HW() const { return (int64_t)H * W; }
    int32_t M() const { return (int32_t)kept.size(); }
    const StateInfo &at(int32_t m, int64_t cell) const { return info[(size_t)(m * HW() + cell)]; }

    // the table, from the caller's [N][H][W] layers: c^N of (m, cell) is the
    // minimum c^T over the run of kept slices around m with the same ground
    void fill(const float *ground, const float *cost)
    {
        const int64_t hw = HW();
        const int32_t nm = M();
        info.resize((size_t)nm * hw);
        for (int64_t c = 0; c < hw; ++c) {
            for (int32_t m = 0; m < nm;) {
                const float e = ground[(int64_t)kept[m] * hw + c];
                int32_t b = m + 1;
                float lo = cost[(int64_t)kept[m] * hw + c];
                if (std::isfinite(e))
                    for (; b < nm && ground[(int64_t)kept[b] * hw + c] == e; ++b)
                        lo = std::min(lo, cost[(int64_t)kept[b] * hw + c]);
                for (int32_t a = m; a < b; ++a) {
                    StateInfo &si = info[(size_t)(a * hw + c)];
                    si.e = e;
                    si.t = cost[(int64_t)kept[a] * hw + c];
                    si.cn = std::isfinite(e) ? lo : c_b;
                }
                m = b;
            }
        }
    }

    std::unique_ptr<Search> take()
    {
        std::lock_guard<std::mutex> lock(mu);
        if (idle.empty()) return std::make_unique<Search>();
        auto s = std::move(idle.back());
        idle.pop_back();
        return s;
    }
    void give(std::unique_ptr<Search> s)
    {
        std::lock_guard<std::mutex> lock(mu);
        idle.push_back(std::move(s));
    }
};

namespace {

struct Query {
    int32_t start[3], goal[3];   // i, j, original slice index
};

struct Result {
    std::vector<int32_t> path;   // (i, j, original slice) triples, start first
    double cost = INFINITY;
    int64_t expanded = 0;
};

int kept_index(const tct_planner &p, int32_t slice)
{
    auto it = std::lower_bound(p.kept.begin(), p.kept.end(), slice);
    return (it != p.kept.end() && *it == slice) ? (int)(it - p.kept.begin()) : -1;
}

bool valid_endpoint(const tct_planner &p, const int32_t *q)
{
    return q[0] >= 0 && q[0] < p.H && q[1] >= 0 && q[1] < p.W && kept_index(p, q[2]) >= 0;
}

void run_query(const tct_planner &p, Search &S, const Query &q, Result &r)
{
    const int64_t HW = p.HW();
    const int32_t M = p.M();
    S.prepare((size_t)M * HW);
    r.path.clear();
    r.cost = INFINITY;
    r.expanded = 0;

    const int32_t ms = kept_index(p, q.start[2]), mg = kept_index(p, q.goal[2]);
    const int64_t cs = (int64_t)q.start[0] * p.W + q.start[1];
    const int64_t cg = (int64_t)q.goal[0] * p.W + q.goal[1];
    const float eg = p.at(mg, cg).e;
    if (!(p.at(ms, cs).cn < p.c_b) || !(p.at(mg, cg).cn < p.c_b)) return;

    const int gi = q.goal[0], gj = q.goal[1];
    auto h = [&](int i, int j) {
        const double di = std::abs(i - gi), dj = std::abs(j - gj);
        return std::max(di, dj) + (std::sqrt(2.0) - 1.0) * std::min(di, dj);
    };
    std::priority_queue<Entry> open;
    const int64_t s0 = (int64_t)ms * HW + cs;
    S.rec[s0] = Record{0.0, S.current, kFromStart};
    open.push({h(q.start[0], q.start[1]), 0.0, s0});
    const double res = (double)p.res;
    int64_t reached = -1;

    auto relax = [&](int64_t t, double g, uint8_t code, int ti, int tj) {
        Record &rt = S.rec[t];
        if (rt.epoch != S.current || g < rt.g) {
            rt = Record{g, S.current, code};
            open.push({g + h(ti, tj), g, t});
        }
    };

    while (!open.empty()) {
        const Entry top = open.top();
        open.pop();
        if (top.g > S.rec[top.s].g) continue;   // stale entry
        ++r.expanded;
        const int32_t m = (int32_t)(top.s / HW);
        const int64_t c = top.s % HW;
        const int i = (int)(c / p.W), j = (int)(c % p.W);
        const StateInfo &here = p.at(m, c);
        const float e = here.e;
        if (c == cg && e == eg) {
            reached = top.s;
            break;
        }
        for (int d = 0; d < 8; ++d) {
            const int ni = i + kDi[d], nj = j + kDj[d];
            if (ni < 0 || ni >= p.H || nj < 0 || nj >= p.W) continue;
            const int64_t nc = (int64_t)ni * p.W + nj;
            const StateInfo &there = p.at(m, nc);
            const double cn = there.cn;   // c^B where the ground is invalid
            if (!(cn < p.c_b)) continue;
            const float ne = there.e;
            const double dz = ((double)ne - (double)e) / res;
            const double planar = (kDi[d] != 0 && kDj[d] != 0) ? 2.0 : 1.0;
            relax((int64_t)m * HW + nc, top.g + (cn + std::sqrt(planar + dz * dz)), (uint8_t)d,
                  ni, nj);
        }
        // gateways: the same node on the adjacent kept slice, cheaper there
        if (m + 1 < M && p.at(m + 1, c).e == e && p.at(m + 1, c).t < here.t)
            relax((int64_t)(m + 1) * HW + c, top.g, kFromBelow, i, j);
        if (m > 0 && p.at(m - 1, c).e == e && p.at(m - 1, c).t < here.t)
            relax((int64_t)(m - 1) * HW + c, top.g, kFromAbove, i, j);
    }
    if (reached < 0) return;
    r.cost = S.rec[reached].g;
    for (int64_t s = reached;;) {
        const int32_t m = (int32_t)(s / HW);
        const int64_t c = s % HW;
        r.path.push_back((int32_t)(c / p.W));
        r.path.push_back((int32_t)(c % p.W));
        r.path.push_back(p.kept[m]);
        const uint8_t f = S.rec[s].from;
        if (f == kFromStart) break;
        if (f == kFromBelow) s -= HW;
        else if (f == kFromAbove) s += HW;
        else s = (int64_t)m * HW + (c - (int64_t)kDi[f] * p.W - kDj[f]);
    }
    // reverse the triples: start first
    const size_t n = r.path.size() / 3;
    for (size_t a = 0, b = n - 1; a < b; ++a, --b)
        for (int t = 0; t < 3; ++t) std::swap(r.path[3 * a + t], r.path[3 * b + t]);
}

}  // namespace

extern "C" {

int tct_planner_create(const tct_grid *grid, const float *h_ground, const float *h_cost,
                       const uint8_t *h_keep, float c_b, tct_planner **out)
{
    if (!out) return TCT_ERR_INVALID_ARG;
    *out = nullptr;
    if (!grid || !h_ground || !h_cost || grid->W < 1 || grid->H < 1 || grid->n_slices < 1 ||
        grid->n_slices > TCT_MAX_SLICES || !(grid->res > 0.f) || !std::isfinite(grid->res) ||
        !(c_b > 0.f) || !std::isfinite(c_b))
        return TCT_ERR_INVALID_ARG;
    std::unique_ptr<tct_planner> p;
    try {
        p = std::make_unique<tct_planner>();
        p->H = grid->H;
        p->W = grid->W;
        p->res = grid->res;
        p->c_b = c_b;
        for (int32_t k = 0; k < grid->n_slices; ++k)
            if (!h_keep || h_keep[k]) p->kept.push_back(k);
        if (p->kept.empty()) return TCT_ERR_INVALID_ARG;
        p->fill(h_ground, h_cost);
    } catch (...) {   // the state table could not be allocated
        return TCT_ERR_UNSUPPORTED;
    }
    *out = p.release();
    return TCT_OK;
}

void tct_planner_destroy(tct_planner *planner) { delete planner; }

int tct_plan_paths(tct_planner *planner, int32_t n_queries, const int32_t *h_starts,
                   const int32_t *h_goals, int32_t max_len, int32_t *h_paths, int32_t *h_lens,
                   double *h_costs, int64_t *h_expanded, int32_t n_threads)
{
    if (!planner || n_queries < 0 || max_len < 0 || (n_queries > 0 && (!h_starts || !h_goals ||
        !h_lens || !h_costs || (max_len > 0 && !h_paths))))
        return TCT_ERR_INVALID_ARG;
    for (int32_t q = 0; q < n_queries; ++q)
        if (!valid_endpoint(*planner, h_starts + 3 * q) || !valid_endpoint(*planner, h_goals + 3 * q))
            return TCT_ERR_INVALID_ARG;
    if (n_queries == 0) return TCT_OK;
    const int32_t hw = (int32_t)std::max(1u, std::thread::hardware_concurrency());
    const int32_t workers = std::max(1, std::min(n_threads > 0 ? n_threads : hw, n_queries));
    std::atomic<int32_t> next{0};
    std::atomic<int> status{TCT_OK};

    auto work = [&]() {
        std::unique_ptr<Search> S;
        Result r;
        try {
            S = planner->take();
            for (int32_t q; (q = next.fetch_add(1)) < n_queries;) {
                Query qu;
                std::copy(h_starts + 3 * q, h_starts + 3 * q + 3, qu.start);
                std::copy(h_goals + 3 * q, h_goals + 3 * q + 3, qu.goal);
                run_query(*planner, *S, qu, r);
                const int32_t len = (int32_t)(r.path.size() / 3);
                h_lens[q] = len;
                h_costs[q] = r.cost;
                if (h_expanded) h_expanded[q] = r.expanded;
                const int32_t n = std::min(len, max_len);
                if (n > 0) std::copy(r.path.begin(), r.path.begin() + 3 * n,
                                     h_paths + (int64_t)3 * max_len * q);
                if (len > max_len) status.store(TCT_ERR_WORKSPACE_TOO_SMALL);
            }
        } catch (...) {   // allocation failure of the search state
            status.store(TCT_ERR_UNSUPPORTED);
        }
        if (S) planner->give(std::move(S));
    };
    if (workers == 1) {
        work();
    } else {
        std::vector<std::thread> pool;
        pool.reserve(workers);
        for (int32_t t = 0; t < workers; ++t) pool.emplace_back(work);
        for (auto &t : pool) t.join();
    }
    return status.load();
}

}  // extern "C"
