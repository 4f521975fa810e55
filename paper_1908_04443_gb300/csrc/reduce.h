// Observables reductions of several grids in one pair of launches, each grid's results and error
// word into a caller-given slot, for callers that gather them in one device array and copy it to the
// host at once (the batch).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace lbmwet {

// One grid of a several-grid reduction: its fields and node types, its partials array (room for
// reduce_blocks(N) * NRED doubles) and result slot (NRED + 1 doubles), the
// first block of the launch that is its and its block count (= reduce_blocks(N)).  The slot gets the
// NRED results in out[0 .. NRED) and, when err is not null, the grid's 4-byte device error word in
// the first 4 bytes of out[NRED] (out holds NRED + 1 doubles).
struct RedGrid {
    const double* rho;
    const double* u;
    const uint8_t* type;
    const unsigned* err;
    double* partials;
    double* out;
    double rho_mid;
    double hint[3];
    int nx, ny, nz, block0, nblk;
};

// Blocks of the partial reduction of a grid of N nodes.
int reduce_blocks(long long N);

// The reductions of several grids of one lattice (dim 2 or 3) in two launches: `grids` (device
// array, ngrids entries, block0 ascending from 0, total_blocks = the sum of nblk) is read by the
// kernels; each grid's results equal those of launch_reduce on it alone, bit for bit.
cudaError_t launch_reduce_grids(int dim, const RedGrid* grids, int ngrids, int total_blocks, cudaStream_t s);

}  // namespace lbmwet
