// Discrete adjoint of the D2Q9 time step with respect to the per-wall-node wettability parameter.
//
// Forward step k (GPU storage): stored post-collision f*_k --pull (Eq. 3, Fig. 3)--> f (post-
// streaming) --rho, psi, rho_w (Eqs. 4, 6, 16-17), F_m (Eq. 5), collision (Eqs. 2, 7)--> f*_{k+1}.
// Its adjoint maps mu_{k+1} = dL/df*_{k+1} to mu_k = dL/df*_k and adds dL/dkappa_j, in two kernels:
//   A (the forward tile body in its adjoint mode, step.cu): recompute rho, psi and rho_w of the
//     state pulled from f*_k; per fluid node the reverse of the collision, lambda_loc = dL/df,
//     Fmbar = dL/dF_m and the node's own psi-bar; psi'(rho), and at wall nodes d rho_w/d kappa and
//     d rho_w/d rho_ave / den (zero where the limiter clamps);
//   B (adj_gather_push): psi-bar gathered through Eq. 5 from the neighbours' Fmbar; fluid nodes
//     turn it into rho-bar, wall nodes into kappa-bar and an Eq. 17 weight; then per fluid node
//     lambda = lambda_loc + rho-bar (own psi and wall neighbours' averages) and the transpose of the
//     pull (a push) into mu_k.
#include <cmath>
#include <type_traits>

#include "adjoint.h"
#include "lattice.cuh"

namespace lbmwet {

namespace {

__device__ __forceinline__ int wrap_any(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// psi-bar gathered through Eq. 5, rho-bar / kappa-bar, and the push (transpose of the pull), for a
// TX x TY tile.  psi-bar(y) = psib(y) + sum_a [x = y - e_a fluid] (-G psi(x) w_a e_a . Fmbar(x)).
template <class C, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) adj_gather_push(DevParams p, const C* __restrict__ psi,
                                                          const C* __restrict__ dpsi, const C* __restrict__ drw_k,
                                                          const C* __restrict__ drw_a, const C* __restrict__ fmb_x,
                                                          const C* __restrict__ fmb_y, const C* __restrict__ psib,
                                                          const C* __restrict__ lam, double* __restrict__ dkappa,
                                                          C* __restrict__ mu_out) {
    constexpr int RX = TX + 4, RY = TY + 4, PX = TX + 2, PY = TY + 2, NT = TX * TY;
    __shared__ uint8_t s_t[RY * RX];
    __shared__ C s_psi[RY * RX], s_fx[RY * RX], s_fy[RY * RX];
    __shared__ C s_rb[PY * PX], s_wb[PY * PX];
    const int nx = p.nx, ny = p.ny, N = int(p.N);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const C G = C(p.G);
    // 0. types, psi and Fmbar on the tile + 2-node halo
    for (int i = tid; i < RX * RY; i += NT) {
        const int gx = wrap_any(x0 + i % RX - 2, nx), gy = wrap_any(y0 + i / RX - 2, ny);
        const int g = gy * nx + gx;
        s_t[i] = p.type[g];
        s_psi[i] = psi[g];
        s_fx[i] = fmb_x[g];
        s_fy[i] = fmb_y[g];
    }
    __syncthreads();
    // 1. psi-bar on the tile + 1-node halo; fluid -> rho-bar, wall -> kappa-bar and the Eq. 17 weight
    for (int i = tid; i < PX * PY; i += NT) {
        const int px = i % PX, py = i / PX;
        const int r = (py + 1) * RX + px + 1;
        const uint8_t t = s_t[r];
        const bool fluid = !(t & T_SOLID);
        if (!fluid && !(t & T_WALL)) {
            s_rb[i] = C(0);
            s_wb[i] = C(0);
            continue;
        }
        const int gx = wrap_any(x0 + px - 1, nx), gy = wrap_any(y0 + py - 1, ny);
        const int g = gy * nx + gx;
        C pb = fluid ? psib[g] : C(0);
#pragma unroll
        for (int a = 1; a < 9; ++a) {
            const int rs = r - D2Q9::ex(a) - D2Q9::ey(a) * RX;
            if (s_t[rs] & T_SOLID) continue;
            pb += -G * s_psi[rs] * C(D2Q9::wf(a)) * (s_fx[rs] * C(D2Q9::ex(a)) + s_fy[rs] * C(D2Q9::ey(a)));
        }
        const C rb = pb * dpsi[g];
        if (fluid) {
            s_rb[i] = rb;
            s_wb[i] = C(0);
        } else {
            s_rb[i] = C(0);
            s_wb[i] = rb * drw_a[g];
            const bool own = px >= 1 && px <= TX && py >= 1 && py <= TY && x0 + px - 1 < nx && y0 + py - 1 < ny;
            if (own && p.kappa_w) dkappa[p.wall_id[g]] += double(rb * drw_k[g]);
        }
    }
    __syncthreads();
    // 2. lambda = lam + rho-bar at the tile's fluid nodes, pushed to mu (the transpose of the pull)
    const int lx = threadIdx.x, ly = threadIdx.y;
    if (x0 + lx >= nx || y0 + ly >= ny) return;
    const int r = (ly + 2) * RX + lx + 2;
    if (s_t[r] & T_SOLID) return;
    const int pi = (ly + 1) * PX + lx + 1;
    C rb = s_rb[pi];
#pragma unroll
    for (int a = 1; a < 9; ++a) {
        if (s_t[r + D2Q9::ex(a) + D2Q9::ey(a) * RX] & T_WALL)
            rb += C(D2Q9::wf(a)) * s_wb[pi + D2Q9::ex(a) + D2Q9::ey(a) * PX];
    }
    const int gx = x0 + lx, gy = y0 + ly, g = gy * nx + gx;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const C l = lam[a * N + g] + rb;
        const int rs = r - D2Q9::ex(a) - D2Q9::ey(a) * RX;
        if (s_t[rs] & T_SOLID) {
            mu_out[D2Q9::opp(a) * N + g] = l;
        } else {
            const int sx = wrap_any(gx - D2Q9::ex(a), nx), sy = wrap_any(gy - D2Q9::ey(a), ny);
            mu_out[a * N + sy * nx + sx] = l;
        }
    }
}

// mu_n from dL/drho_T: every direction of a fluid node carries dL/drho_T, pushed like step 2 above
template <class C>
__global__ void __launch_bounds__(256) adj_final_push(DevParams p, const double* __restrict__ drho,
                                                      C* __restrict__ mu_out) {
    const int N = int(p.N), nx = p.nx, ny = p.ny;
    for (int g = blockIdx.x * 256 + threadIdx.x; g < N; g += gridDim.x * 256) {
        if (p.type[g] & T_SOLID) continue;
        const int x = g % nx, y = g / nx;
        const C l = C(drho[g]);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const int s = wrap_any(y - D2Q9::ey(a), ny) * nx + wrap_any(x - D2Q9::ex(a), nx);
            if (p.type[s] & T_SOLID) mu_out[D2Q9::opp(a) * N + g] = l;
            else mu_out[a * N + s] = l;
        }
    }
}

constexpr int GX = 32, GY = 8;

template <class S>
cudaError_t adjoint_step_t(const void* fstar_k, const void* mu_next, void* mu_prev, const DevParams& p,
                           const AdjointScratch& w, double* dkappa, cudaStream_t s) {
    const size_t N = size_t(p.N);
    S* b = static_cast<S*>(w.buf);
    AdjointFields f;
    f.mu = mu_next;
    f.lam = b;
    f.fmb_x = b + 9 * N;
    f.fmb_y = b + 10 * N;
    f.psib = b + 11 * N;
    f.psi = b + 12 * N;
    f.dpsi = b + 13 * N;
    f.drw_k = b + 14 * N;
    f.drw_a = b + 15 * N;
    cudaError_t e = launch_adjoint_local(std::is_same<S, double>::value ? PREC_FP64 : PREC_FP32, fstar_k, p, f, s);
    if (e != cudaSuccess) return e;
    dim3 grid((p.nx + GX - 1) / GX, (p.ny + GY - 1) / GY, 1);
    adj_gather_push<S, GX, GY><<<grid, dim3(GX, GY, 1), 0, s>>>(
        p, static_cast<const S*>(f.psi), static_cast<const S*>(f.dpsi), static_cast<const S*>(f.drw_k),
        static_cast<const S*>(f.drw_a), static_cast<const S*>(f.fmb_x), static_cast<const S*>(f.fmb_y),
        static_cast<const S*>(f.psib), static_cast<const S*>(f.lam), dkappa, static_cast<S*>(mu_prev));
    return cudaGetLastError();
}

unsigned grid_of(long long n) {
    long long b = (n + 255) / 256;
    if (b > 152LL * 16) b = 152LL * 16;
    return unsigned(b < 1 ? 1 : b);
}

}  // namespace

size_t adjoint_scratch_elems(long long N) { return size_t(N) * 16; }

cudaError_t launch_adjoint_step(int prec, const void* fstar_k, const void* mu_next, void* mu_prev, const DevParams& p,
                                const AdjointScratch& w, double* dkappa, cudaStream_t s) {
    if (prec == PREC_FP64) return adjoint_step_t<double>(fstar_k, mu_next, mu_prev, p, w, dkappa, s);
    return adjoint_step_t<float>(fstar_k, mu_next, mu_prev, p, w, dkappa, s);
}

cudaError_t launch_adjoint_final(int prec, const double* drho_final, void* mu, const DevParams& p, cudaStream_t s) {
    const unsigned g = grid_of(p.N);
    if (prec == PREC_FP64) adj_final_push<double><<<g, 256, 0, s>>>(p, drho_final, static_cast<double*>(mu));
    else adj_final_push<float><<<g, 256, 0, s>>>(p, drho_final, static_cast<float*>(mu));
    return cudaGetLastError();
}

}  // namespace lbmwet
