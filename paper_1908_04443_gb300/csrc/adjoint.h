// Internal interface of the D2Q9 discrete adjoint kernels (not part of the ABI).
#pragma once

#include "kernels.h"

namespace lbmwet {

// Work buffer of the adjoint step: adjoint_scratch_elems(N) values of the storage precision.
struct AdjointScratch {
    void* buf;
};
size_t adjoint_scratch_elems(long long N);

// One adjoint step: given the stored forward state f*_k (whose pull is the post-streaming state
// that step k collides) and mu_next = dL/df*_{k+1}, write mu_prev = dL/df*_k and add the step's
// dL/dkappa to dkappa (one double per wall node).
cudaError_t launch_adjoint_step(int prec, const void* fstar_k, const void* mu_next, void* mu_prev, const DevParams& p,
                                const AdjointScratch& w, double* dkappa, cudaStream_t s);

// mu_n = dL/df*_n for a loss of the final density rho_T = sum_a pull(f*_n)_a: the transpose of the
// pull applied to dL/drho_T (N doubles, device).
cudaError_t launch_adjoint_final(int prec, const double* drho_final, void* mu, const DevParams& p, cudaStream_t s);

}  // namespace lbmwet
