// Host pass over a solid mask at initialisation: the wall nodes (solid nodes with a fluid lattice
// neighbour, the nodes that carry virtual densities, Eqs. 16-17; the per-node index map is built from
// them on the device) and the solid flags per tile of the step kernels.  Row-based (no per-node index arithmetic), optionally split over threads by rows.
#pragma once
#include <cstdint>
#include <thread>
#include <vector>

namespace lbmwet {

struct MaskScan {
    long long nfluid = 0;
    std::vector<int64_t> wall_nodes;   // ascending linear indices
    std::vector<uint8_t> tile_solid;   // per tile of the step kernels
    std::vector<uint8_t> pair_solid;   // per tile of the D2Q9 FP32 pair kernel (empty unless asked for)
};

// Per tile of a t[0] x t[1] x t[2] tiling: does a solid node lie within the box of cells the tile
// touches (the full tile, including cells of a ragged tile that wrap past the grid edge, plus a
// 3-node halo; no z halo in 2D)?  Tiles without one skip the node-type staging.
std::vector<uint8_t> tile_solid_flags(const uint8_t* mask, int nx, int ny, int nz, const int t[3], int D,
                                      int threads = 1);

// The full scan: fluid count, wall list (neighbourhood of the D2Q9 or D3Q19 velocity set,
// periodic wrap), the step-kernel tile flags for tile shape t and, when pair_t is given, the pair
// kernel's.  `threads` > 1 splits the rows over that many threads.
void scan_mask(const uint8_t* mask, int nx, int ny, int nz, int D, const int t[3], const int* pair_t, int threads,
               MaskScan* out);

// Threads for scanning a grid of N nodes alone: one per 2^20 nodes, at most the host's cores and 16.
int scan_threads(long long N);

// f(i) for i in [0, n), spread over up to `threads` threads (the caller's among them).
template <class F>
void parallel_for(int n, int threads, F f) {
    if (threads > n) threads = n;
    if (threads <= 1) {
        for (int i = 0; i < n; ++i) f(i);
        return;
    }
    std::vector<std::thread> pool;
    pool.reserve(threads - 1);
    for (int k = 1; k < threads; ++k)
        pool.emplace_back([&, k] {
            for (int i = k; i < n; i += threads) f(i);
        });
    for (int i = 0; i < n; i += threads) f(i);
    for (auto& th : pool) th.join();
}

}  // namespace lbmwet
