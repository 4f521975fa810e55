// Observables reduction of one grid into a caller-given slot, for callers that gather several
// grids' results in one device array and copy them to the host at once (the batch).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace lbmwet {

// As launch_reduce (per-block partials, then one block combining them), with the NRED results
// written to out[0 .. NRED) and, when err is not null, the grid's 4-byte device error word copied by
// the combining block into the first 4 bytes of out[NRED] (out then holds NRED + 1 doubles).  Stream
// order on s makes the word the one left by the kernels enqueued before.
cudaError_t launch_reduce_slot(int dim, const double* rho, const double* u, const uint8_t* type, int nx, int ny,
                               int nz, double rho_mid, const double* hint, double* partials, const unsigned* err,
                               double* out, cudaStream_t s);

}  // namespace lbmwet
