// Work plan of the D2Q9 y-march step kernel: every grid is cut into column blocks of tw - 4 own
// columns and each block into runs of consecutive rows; the runs are assigned to a fixed number of
// persistent CTAs so that the largest per-CTA row count (pulled rows, halo rows included) is as
// small as the run height allows.
#pragma once

#include <cstdint>
#include <vector>

#include "kernels.h"

namespace lbmwet {

struct YGrid {
    int nx, ny;
    const uint8_t* mask;   // host solid mask, nx * ny bytes (nonzero = solid)
    BatchItem proto;       // buffers, node types, wall ids, kappa and instance index of the grid
};

struct YPlan {
    std::vector<BatchItem> items;   // grouped by CTA
    std::vector<int> begin;         // CTA c walks items[begin[c] .. begin[c + 1])
    int ctas = 0;
    int run_rows = 0;               // rows per run (the last run of a block may be shorter)
    double makespan = 0;            // largest per-CTA cost, in pulled rows
    double efficiency = 0;          // total cost / (ctas_available * makespan)
};

// tw: threads (cells per row) of the kernel; ctas_available: resident CTAs of the whole GPU.
YPlan plan_ymarch(const std::vector<YGrid>& grids, int tw, int ctas_available);

}  // namespace lbmwet
