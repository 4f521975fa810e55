// Internal interface of the D2Q9 discrete adjoint kernels (not part of the ABI).
#pragma once

#include "kernels.h"

namespace lbmwet {

// Work buffer of the adjoint step: adjoint_scratch_elems(N) values of the storage precision.
struct AdjointScratch {
    void* buf;
};
size_t adjoint_scratch_elems(long long N);

// Node fields of the adjoint step (storage precision; [a][node] for mu and lam, one per node else).
struct AdjointFields {
    const void* mu;
    void *lam, *fmb_x, *fmb_y, *psib, *psi, *dpsi, *drw_k, *drw_a;
};

// Local part of an adjoint step (tile kernel sharing the forward's halo machinery): recomputes the
// state pulled from f*_k and writes, per node, the reverse of the collision and psi data.
cudaError_t launch_adjoint_local(int prec, const void* fstar, const DevParams& p, const AdjointFields& w,
                                 cudaStream_t s);

// One adjoint step: given the stored forward state f*_k (whose pull is the post-streaming state
// that step k collides) and mu_next = dL/df*_{k+1}, write mu_prev = dL/df*_k and add the step's
// dL/dkappa to dkappa (one double per wall node).
cudaError_t launch_adjoint_step(int prec, const void* fstar_k, const void* mu_next, void* mu_prev, const DevParams& p,
                                const AdjointScratch& w, double* dkappa, cudaStream_t s);

// mu_n = dL/df*_n for a loss of the final density rho_T = sum_a pull(f*_n)_a: the transpose of the
// pull applied to dL/drho_T (N doubles, device).
cudaError_t launch_adjoint_final(int prec, const double* drho_final, void* mu, const DevParams& p, cudaStream_t s);

}  // namespace lbmwet
