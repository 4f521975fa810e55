// Test-only C entry points over the library's host mask scan (compiled by
// tests/test_maskscan_host.py with the host compiler; not part of the library).
#include <cstdint>
#include <cstring>

#include "../../paper_1908_04443_gb300/csrc/maskscan.h"

extern "C" {

// Returns the wall count; fills nfluid, wall_nodes (capacity N) and the tile flags (capacity
// max_tiles, count in *n_tiles) for tile shape t.
long long maskscan_run(const uint8_t* mask, int nx, int ny, int nz, int D, const int* t, int threads,
                       long long* nfluid, long long* wall_nodes, uint8_t* tiles, long long max_tiles,
                       long long* n_tiles) {
    lbmwet::MaskScan s;
    lbmwet::scan_mask(mask, nx, ny, nz, D, t, nullptr, threads, &s);
    *nfluid = s.nfluid;
    for (size_t i = 0; i < s.wall_nodes.size(); ++i) wall_nodes[i] = s.wall_nodes[i];
    *n_tiles = (long long)s.tile_solid.size();
    if (*n_tiles <= max_tiles) std::memcpy(tiles, s.tile_solid.data(), s.tile_solid.size());
    return (long long)s.wall_nodes.size();
}

}  // extern "C"
