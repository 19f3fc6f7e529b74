// Host-side work partition of the persistent 1D kernel: the lane layout of one wall inside its warp,
// and the dealing of rounds of walls to the persistent blocks. Plain C++ without CUDA: the library
// (hygro_api.cu) includes it, and the CPU tests compile it on its own to check its invariants.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <vector>

namespace hygro {

constexpr int kLayoutMaxK = 16;   // most nodes per lane (the kernel's register arrays)

// Lane layout of a wall of N nodes: K nodes per lane, Wl lanes in use, lanes of K or K-1 nodes (bit i of
// short_mask: lane i holds K-1), the last lane full, so node 0 is lane 0's slot 0 and node N-1 lane
// Wl-1's slot K-1.
struct LaneLayout {
    int32_t K;
    int32_t Wl;
    uint32_t short_mask;
    int16_t aligned;   // 1 when every layer interface falls on a lane boundary
};

// Preferred: every layer interface on a lane boundary (each layer split into lanes of K or K-1 nodes,
// its short lanes first), trying K from ceil(N/32) up while the lanes fit in a warp. Otherwise the plain
// split (short lanes first), which may still be aligned by chance. first[l]: first node of layer l
// (first[0] = 0, increasing, below N); nl layers. Needs 1 <= N <= 32 * kLayoutMaxK.
inline LaneLayout wall_layout(int N, const int32_t *first, int nl)
{
    LaneLayout o;
    const int K0 = (N + 31) / 32;
    for (int K = K0; K <= kLayoutMaxK; ++K) {
        int lanes = 0;
        uint32_t mask = 0;
        bool ok = true;
        for (int l = 0; l < nl && ok; ++l) {
            const int Nl = (l + 1 < nl ? first[l + 1] : N) - first[l];
            const int c = (Nl + K - 1) / K;
            const int sh = c * K - Nl;
            const bool last = l + 1 == nl;
            if (sh > c - (last ? 1 : 0) || lanes + c > 32) {
                ok = false;
                break;
            }
            for (int i = 0; i < sh; ++i) mask |= 1u << (lanes + i);
            lanes += c;
        }
        if (ok) {
            o.K = K;
            o.Wl = lanes;
            o.short_mask = mask;
            o.aligned = 1;
            return o;
        }
    }
    o.K = K0;
    o.Wl = (N + K0 - 1) / K0;
    const int m = o.Wl * K0 - N;
    o.short_mask = m > 0 ? ((1u << m) - 1u) : 0u;
    // aligned by chance when every interface is a lane start
    int aligned = 1;
    for (int l = 1; l < nl; ++l) {
        int start = 0, lane = 0;
        bool hit = false;
        while (lane < o.Wl && start <= first[l]) {
            if (start == first[l]) hit = true;
            start += ((o.short_mask >> lane) & 1u) ? K0 - 1 : K0;
            ++lane;
        }
        if (!hit) aligned = 0;
    }
    o.aligned = (int16_t)aligned;
    return o;
}

// A wall of the persistent kernel as the scheduler sees it. kind: the kernel's code variant, 0 simple-heat
// with one layer per lane, 1 general with one layer per lane, 2 general with interfaces inside lanes,
// 3 simple-heat with interfaces inside lanes.
struct SchedWall {
    int32_t wall;
    int32_t K;
    int32_t kind;
    int32_t N;
};

// Time per step of a wall when an SM is shared by its full warp count, a[kind] + b[kind] K nanoseconds.
struct CostModel {
    double a[4], b[4];
};

// The built-in model: measured on GB300 with a per-wall trace at 16 warps per SM for variants 0 and 3;
// variants 1 and 2 scaled from an earlier 12-warp trace.
inline CostModel default_cost_model()
{
    return CostModel{{107.0, 234.0, 156.0, 191.0}, {64.2, 76.0, 125.0, 77.2}};
}

inline double sched_cost(const SchedWall &x, const CostModel &m) { return m.a[x.kind] + m.b[x.kind] * x.K; }
inline double sched_cost(const SchedWall &x) { return sched_cost(x, default_cost_model()); }

// Least-squares fit of a + b K per variant to measured step times ns[i] of walls[i] (ns[i] <= 0: not
// measured). A variant whose measured walls span two or more K values gets both coefficients (b kept
// >= 0); one with a single K keeps base's b and fits a; one with no measured wall keeps base. Returns the
// number of variants fitted.
inline int fit_cost_model(const std::vector<SchedWall> &walls, const std::vector<double> &ns, const CostModel &base,
                          CostModel &out)
{
    out = base;
    int fitted = 0;
    for (int v = 0; v < 4; ++v) {
        double n = 0, sk = 0, st = 0, skk = 0, skt = 0;
        int kmin = 1 << 30, kmax = -1;
        for (size_t i = 0; i < walls.size() && i < ns.size(); ++i) {
            if (walls[i].kind != v || !(ns[i] > 0.0)) continue;
            const double k = walls[i].K, t = ns[i];
            n += 1;
            sk += k;
            st += t;
            skk += k * k;
            skt += k * t;
            kmin = std::min(kmin, walls[i].K);
            kmax = std::max(kmax, walls[i].K);
        }
        if (n == 0) continue;
        const double var = skk - sk * sk / n;
        double b = base.b[v];
        if (kmax > kmin && var > 0) b = std::max(0.0, (skt - sk * st / n) / var);
        out.b[v] = b;
        out.a[v] = (st - b * sk) / n;
        ++fitted;
    }
    return fitted;
}

// Walls sorted by nodes per lane (descending), then variant, then N (descending), cut into rounds of R
// walls (warp i of a block takes entry i of each of its rounds); rounds dealt to the G blocks largest
// estimated cost first, each to the least loaded block (LPT); a block runs its rounds largest first.
// order: the rounds of block 0, then block 1, ..., R entries each (-1 for the empty entries of the last
// round); boff[g] .. boff[g + 1]: block g's entries. load (optional): each block's estimated cost.
inline void lpt_rounds(std::vector<SchedWall> walls, int G, int R, std::vector<int32_t> &order,
                       std::vector<int32_t> &boff, std::vector<double> *load_out = nullptr,
                       const CostModel &model = default_cost_model())
{
    std::stable_sort(walls.begin(), walls.end(), [](const SchedWall &x, const SchedWall &y) {
        if (x.K != y.K) return x.K > y.K;
        if (x.kind != y.kind) return x.kind < y.kind;
        return x.N > y.N;
    });
    const int Wf = (int)walls.size();
    const int n_rounds = (Wf + R - 1) / R;
    std::vector<double> rcost(n_rounds, 0.0);
    for (int i = 0; i < Wf; ++i) rcost[i / R] = std::max(rcost[i / R], sched_cost(walls[i], model));
    std::vector<int32_t> ridx(n_rounds);
    for (int r = 0; r < n_rounds; ++r) ridx[r] = r;
    std::stable_sort(ridx.begin(), ridx.end(), [&](int a, int b) { return rcost[a] > rcost[b]; });
    std::vector<double> load(G, 0.0);
    std::vector<std::vector<int32_t>> lists(G);
    for (int r : ridx) {
        int best = 0;
        for (int g = 1; g < G; ++g)
            if (load[g] < load[best]) best = g;
        load[best] += rcost[r];
        lists[best].push_back(r);
    }
    order.clear();
    boff.assign(G + 1, 0);
    order.reserve((size_t)n_rounds * R);
    for (int g = 0; g < G; ++g) {
        boff[g] = (int32_t)order.size();
        for (int r : lists[g])
            for (int i = 0; i < R; ++i) order.push_back(r * R + i < Wf ? walls[r * R + i].wall : -1);
    }
    boff[G] = (int32_t)order.size();
    if (load_out) *load_out = load;
}

}  // namespace hygro
