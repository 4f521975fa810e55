// Planner of the y-march runs (see plan.h).
//
// A run of h rows costs h + 2 * LAG + 1 row-times: its own rows, LAG halo rows pulled at either
// end (LAG = 2 where the run's box plus a 3-cell halo holds a solid node, else 1) and a fixed
// start-up.  For each candidate height the runs are assigned largest first to the least-loaded CTA
// (LPT); the height with the smallest makespan wins, ties going to the taller runs.
#include "plan.h"

#include <algorithm>
#include <functional>
#include <queue>
#include <utility>

namespace lbmwet {

namespace {

struct Block {
    int grid, x0;
    std::vector<int> solid_prefix;   // solid_prefix[y] = rows < y holding a solid in the block's x range
};

// any solid in rows y0 - 3 .. y1 + 2 (periodic) of the block
bool run_solid(const Block& b, int ny, int y0, int y1) {
    const int lo = y0 - 3, hi = y1 + 3;   // [lo, hi)
    if (hi - lo >= ny) return b.solid_prefix[ny] > 0;
    auto count = [&](int a, int c) { return b.solid_prefix[c] - b.solid_prefix[a]; };   // [a, c) within [0, ny]
    const int a = ((lo % ny) + ny) % ny;
    const int c = a + (hi - lo);
    if (c <= ny) return count(a, c) > 0;
    return count(a, ny) + count(0, c - ny) > 0;
}

}  // namespace

YPlan plan_ymarch(const std::vector<YGrid>& grids, int tw, int ctas_available) {
    const int ox = tw - 4;
    std::vector<Block> blocks;
    int max_ny = 1;
    for (size_t gi = 0; gi < grids.size(); ++gi) {
        const YGrid& g = grids[gi];
        max_ny = std::max(max_ny, g.ny);
        for (int x0 = 0; x0 < g.nx; x0 += ox) {
            Block b;
            b.grid = int(gi);
            b.x0 = x0;
            b.solid_prefix.assign(g.ny + 1, 0);
            // cells x0 - 3 .. x0 + tw - 2 (the types a run reads), periodic
            const int w = std::min(tw + 2, g.nx);
            for (int y = 0; y < g.ny; ++y) {
                const uint8_t* row = g.mask + (size_t)y * g.nx;
                bool any = false;
                for (int i = 0; i < w && !any; ++i) any = row[(((x0 - 3 + i) % g.nx) + g.nx) % g.nx] != 0;
                b.solid_prefix[y + 1] = b.solid_prefix[y] + (any ? 1 : 0);
            }
            blocks.push_back(std::move(b));
        }
    }

    const int cap = std::max(1, ctas_available);
    std::vector<int> heights;
    for (int h : {4, 6, 8, 10, 12, 14, 16, 20, 24, 28, 32, 40, 48, 56, 64, 80, 96, 112, 128, 160, 192, 256, 384, 512,
                  768, 1024, 2048, 4096})
        if (h < max_ny) heights.push_back(h);
    heights.push_back(max_ny);

    struct Run {
        int block, y0, y1, solid, cost;
    };
    YPlan best;
    std::vector<Run> best_runs;
    std::vector<int> best_owner;
    bool have = false;
    for (int h : heights) {
        std::vector<Run> runs;
        long long total = 0;
        for (size_t bi = 0; bi < blocks.size(); ++bi) {
            const int ny = grids[blocks[bi].grid].ny;
            for (int y0 = 0; y0 < ny; y0 += h) {
                const int y1 = std::min(ny, y0 + h);
                const int solid = run_solid(blocks[bi], ny, y0, y1) ? 1 : 0;
                const int cost = (y1 - y0) + (solid ? 4 : 2) + 1;
                runs.push_back({int(bi), y0, y1, solid, cost});
                total += cost;
            }
        }
        const int ctas = int(std::min<size_t>(runs.size(), size_t(cap)));
        std::vector<int> order(runs.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = int(i);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return runs[a].cost > runs[b].cost; });
        using Slot = std::pair<long long, int>;   // (load, cta)
        std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> pq;
        for (int c = 0; c < ctas; ++c) pq.push({0, c});
        std::vector<int> owner(runs.size());
        long long makespan = 0;
        for (int i : order) {
            Slot s = pq.top();
            pq.pop();
            owner[i] = s.second;
            s.first += runs[i].cost;
            makespan = std::max(makespan, s.first);
            pq.push(s);
        }
        if (!have || makespan < best.makespan || (makespan == best.makespan && h > best.run_rows)) {
            have = true;
            best.ctas = ctas;
            best.run_rows = h;
            best.makespan = double(makespan);
            best.efficiency = double(total) / (double(cap) * double(makespan));
            best_runs = std::move(runs);
            best_owner = std::move(owner);
        }
    }

    // group by CTA; within a CTA keep the runs in grid/block/row order
    std::vector<int> count(best.ctas + 1, 0);
    for (int o : best_owner) count[o + 1]++;
    best.begin.assign(best.ctas + 1, 0);
    for (int c = 0; c < best.ctas; ++c) best.begin[c + 1] = best.begin[c] + count[c + 1];
    best.items.assign(best_runs.size(), BatchItem{});
    std::vector<int> fill(best.begin.begin(), best.begin.end() - 1);
    for (size_t i = 0; i < best_runs.size(); ++i) {
        const Run& r = best_runs[i];
        const Block& b = blocks[r.block];
        BatchItem it = grids[b.grid].proto;
        it.nx = grids[b.grid].nx;
        it.ny = grids[b.grid].ny;
        it.N = it.nx * it.ny;
        it.x0 = b.x0;
        it.y0 = r.y0;
        it.y1 = r.y1;
        it.solid = r.solid;
        best.items[fill[best_owner[i]]++] = it;
    }
    return best;
}

}  // namespace lbmwet
