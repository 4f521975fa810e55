// Host scan of the solid mask (see maskscan.h).
#include "maskscan.h"

#include <algorithm>
#include <cstring>

namespace lbmwet {
namespace {

// Per axis and coordinate: the tiles whose box (tile + halo, wrapped) covers it.
std::vector<std::vector<int>> cover_axis(int n, int t, int halo) {
    std::vector<std::vector<int>> cover(n);
    const int tiles = (n + t - 1) / t;
    for (int k = 0; k < tiles; ++k)
        for (int o = -halo; o < t + halo; ++o) {
            std::vector<int>& c = cover[((k * t + o) % n + n) % n];
            if (c.empty() || c.back() != k) c.push_back(k);
        }
    return cover;
}

inline bool zero_word(const uint8_t* p) {
    uint64_t w;
    std::memcpy(&w, p, sizeof w);
    return w == 0;
}

inline const uint8_t* row_at(const uint8_t* mask, int nx, int ny, int nz, int z, int y) {
    z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
    y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
    return mask + ((long long)z * ny + y) * nx;
}

// Rows [r0, r1) (row r = z * ny + y): solid count and wall nodes in ascending order.  A solid node is
// a wall node when one of its lattice neighbours is fluid: in D2Q9 the 8 nodes around it in the
// plane; in D3Q19 those 8 plus, in each neighbouring plane, the node above or below it and that
// node's 4 axis neighbours.
void scan_rows(const uint8_t* mask, int nx, int ny, int nz, int D, long long r0, long long r1,
               std::vector<int64_t>& walls, long long& nsolid) {
    long long ns = 0;
    for (long long r = r0; r < r1; ++r) {
        const int y = int(r % ny), z = int(r / ny);
        const uint8_t* row = mask + r * nx;
        const uint8_t* ym = row_at(mask, nx, ny, nz, z, y - 1);
        const uint8_t* yp = row_at(mask, nx, ny, nz, z, y + 1);
        const uint8_t *zm = row, *zmym = row, *zmyp = row, *zp = row, *zpym = row, *zpyp = row;
        if (D == 3) {
            zm = row_at(mask, nx, ny, nz, z - 1, y);
            zmym = row_at(mask, nx, ny, nz, z - 1, y - 1);
            zmyp = row_at(mask, nx, ny, nz, z - 1, y + 1);
            zp = row_at(mask, nx, ny, nz, z + 1, y);
            zpym = row_at(mask, nx, ny, nz, z + 1, y - 1);
            zpyp = row_at(mask, nx, ny, nz, z + 1, y + 1);
        }
        for (int x = 0; x < nx;) {
            if (x + 8 <= nx && zero_word(row + x)) {
                x += 8;
                continue;
            }
            if (row[x]) {
                ++ns;
                const int xl = x ? x - 1 : nx - 1, xr = x + 1 < nx ? x + 1 : 0;
                bool wall = !row[xl] || !row[xr] || !ym[xl] || !ym[x] || !ym[xr] || !yp[xl] || !yp[x] || !yp[xr];
                if (!wall && D == 3)
                    wall = !zm[xl] || !zm[x] || !zm[xr] || !zmym[x] || !zmyp[x] || !zp[xl] || !zp[x] || !zp[xr] ||
                           !zpym[x] || !zpyp[x];
                if (wall) walls.push_back(r * nx + x);
            }
            ++x;
        }
    }
    nsolid = ns;
}

}  // namespace

int scan_threads(long long N) {
    const long long hw = std::max(1u, std::thread::hardware_concurrency());
    return int(std::max(1LL, std::min(std::min(hw, 16LL), N >> 20)));
}

std::vector<uint8_t> tile_solid_flags(const uint8_t* mask, int nx, int ny, int nz, const int t[3], int D,
                                      int threads) {
    const int tiles[3] = {(nx + t[0] - 1) / t[0], (ny + t[1] - 1) / t[1], (nz + t[2] - 1) / t[2]};
    const auto cx = cover_axis(nx, t[0], 3);
    const auto cy = cover_axis(ny, t[1], 3);
    const auto cz = cover_axis(nz, t[2], D == 3 ? 3 : 0);
    // per row: the x tiles its solid nodes fall in (with the x halo)
    const long long rows = (long long)ny * nz;
    std::vector<uint8_t> rowt((size_t)rows * tiles[0], 0), rowany((size_t)rows, 0);
    const int nt = int(std::max(1LL, std::min<long long>(threads, rows)));
    parallel_for(nt, nt, [&](int k) {
        const long long r0 = rows * k / nt, r1 = rows * (k + 1) / nt;
        for (long long r = r0; r < r1; ++r) {
            const uint8_t* row = mask + r * nx;
            uint8_t* rt = rowt.data() + (size_t)r * tiles[0];
            for (int x = 0; x < nx;) {
                if (x + 8 <= nx && zero_word(row + x)) {
                    x += 8;
                    continue;
                }
                if (row[x]) {
                    rowany[r] = 1;
                    for (int kx : cx[x]) rt[kx] = 1;
                }
                ++x;
            }
        }
    });
    // per tile: any row of its box
    std::vector<uint8_t> out((size_t)tiles[0] * tiles[1] * tiles[2], 0);
    for (long long r = 0; r < rows; ++r) {
        if (!rowany[r]) continue;
        const int y = int(r % ny), z = int(r / ny);
        const uint8_t* rt = rowt.data() + (size_t)r * tiles[0];
        for (int kz : cz[z])
            for (int ky : cy[y]) {
                uint8_t* o = out.data() + ((size_t)kz * tiles[1] + ky) * tiles[0];
                for (int kx = 0; kx < tiles[0]; ++kx) o[kx] |= rt[kx];
            }
    }
    return out;
}

void scan_mask(const uint8_t* mask, int nx, int ny, int nz, int D, const int t[3], const int* pair_t, int threads,
               MaskScan* out) {
    const long long rows = (long long)ny * nz, N = rows * nx;
    const int nt = int(std::max(1LL, std::min<long long>(threads, rows)));
    std::vector<std::vector<int64_t>> part(nt);
    std::vector<long long> solid(nt, 0);
    parallel_for(nt, nt, [&](int k) {
        scan_rows(mask, nx, ny, nz, D, rows * k / nt, rows * (k + 1) / nt, part[k], solid[k]);
    });
    long long ns = 0;
    size_t nw = 0;
    std::vector<size_t> off(nt + 1, 0);
    for (int k = 0; k < nt; ++k) {
        ns += solid[k];
        off[k + 1] = off[k] + part[k].size();
    }
    nw = off[nt];
    out->nfluid = N - ns;
    out->wall_nodes.resize(nw);
    parallel_for(nt, nt, [&](int k) { std::copy(part[k].begin(), part[k].end(), out->wall_nodes.begin() + off[k]); });
    out->tile_solid = tile_solid_flags(mask, nx, ny, nz, t, D, nt);
    if (pair_t) {
        const int tp[3] = {pair_t[0], pair_t[1], 1};
        out->pair_solid = tile_solid_flags(mask, nx, ny, nz, tp, 2, nt);
    } else {
        out->pair_solid.clear();
    }
}

}  // namespace lbmwet
