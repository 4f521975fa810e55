// Discrete adjoint of the D2Q9 time step with respect to the per-wall-node wettability parameter.
//
// Forward step k (GPU storage): stored post-collision f*_k --pull (Eq. 3, Fig. 3)--> f (post-
// streaming) --rho, psi, rho_w (Eqs. 4, 6, 16-17), F_m (Eq. 5), collision (Eqs. 2, 7)--> f*_{k+1}.
// Its adjoint maps mu_{k+1} = dL/df*_{k+1} to mu_k = dL/df*_k and adds dL/dkappa_j:
//   1. rho of the recomputed state                                    (adj_density)
//   2. psi, psi'(rho), and at wall nodes rho_w with d rho_w/d kappa and d rho_w/d rho_ave / den
//      (zero where the limiter clamps)                                  (adj_psi)
//   3. per fluid node, the reverse of the collision: lambda_loc = dL/df, Fmbar = dL/dF_m and the
//      node's own psi-bar                                               (adj_local)
//   4. per node, psi-bar gathered through Eq. 5 from the neighbours' Fmbar; fluid nodes turn it
//      into rho-bar, wall nodes into kappa-bar (accumulated) and a rho_ave-bar weight  (adj_psibar)
//   5. per fluid node, rho-bar from its own psi and from its wall neighbours' Eq. 17 averages,
//      lambda = lambda_loc + rho-bar, and the transpose of the pull (a push) into mu_k  (adj_push)
#include <cmath>

#include "adjoint.h"
#include "lattice.cuh"

namespace lbmwet {

namespace {

constexpr int AB = 256;

__device__ __forceinline__ int wrapn(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

template <class C>
struct EosA {
    int kind;
    C RT, a, b, b4, aphi, two_over_G, G;
};

template <class C>
__host__ __device__ EosA<C> eos_of(const DevParams& p) {
    EosA<C> e;
    e.kind = p.eos_kind;
    e.RT = C(p.RT);
    e.a = C(p.a);
    e.b = C(p.b);
    e.b4 = C(0.25 * p.b);
    e.aphi = C(p.aphi);
    e.two_over_G = C(p.two_over_G);
    e.G = C(p.G);
    return e;
}

// p(rho) and dp/drho
template <class C>
__device__ __forceinline__ void pressure_and_slope(C rho, const EosA<C>& e, C& p, C& dp) {
    if (e.kind == 1) {
        const C eta = e.b4 * rho, om = C(1) - eta;
        const C om3 = om * om * om;
        const C Z = (C(1) + eta + eta * eta - eta * eta * eta) / om3;
        const C dZ = (C(4) + C(4) * eta - C(2) * eta * eta) / (om3 * om);
        p = rho * e.RT * Z - e.a * rho * rho;
        dp = e.RT * (Z + eta * dZ) - C(2) * e.a * rho;
    } else {
        const C den = C(1) + C(2) * e.b * rho - e.b * e.b * rho * rho;
        const C dden = C(2) * e.b - C(2) * e.b * e.b * rho;
        const C om = C(1) - e.b * rho;
        p = rho * e.RT / om - e.aphi * rho * rho / den;
        dp = e.RT / (om * om) - e.aphi * (C(2) * rho * den - rho * rho * dden) / (den * den);
    }
}

// psi (Eq. 6) and d psi / d rho = (p'(rho) - 1/3) / (G psi)
template <class C>
__device__ __forceinline__ void psi_and_slope(C rho, const EosA<C>& e, C& psi, C& dpsi) {
    C p, dp;
    pressure_and_slope(rho, e, p, dp);
    const C arg = e.two_over_G * (p - rho * C(1.0 / 3.0));
    psi = arg > C(0) ? sqrt(arg) : C(0);
    dpsi = psi > C(0) ? (dp - C(1.0 / 3.0)) / (e.G * psi) : C(0);
}

template <class S, class C>
__device__ __forceinline__ void pull9(const S* __restrict__ fin, const uint8_t* __restrict__ type, int x, int y,
                                      int nx, int ny, int N, C (&f)[9]) {
    const int g = y * nx + x;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const int sx = wrapn(x - D2Q9::ex(a), nx), sy = wrapn(y - D2Q9::ey(a), ny);
        const int s = sy * nx + sx;
        f[a] = (type[s] & T_SOLID) ? C(fin[D2Q9::opp(a) * N + g]) : C(fin[a * N + s]);
    }
}

template <class S, class C>
__global__ void __launch_bounds__(AB) adj_density(const S* __restrict__ fin, DevParams p, C* __restrict__ rho_out) {
    const int N = int(p.N), nx = p.nx, ny = p.ny;
    const C rho_ref = C(p.rho_ref);
    for (int g = blockIdx.x * AB + threadIdx.x; g < N; g += gridDim.x * AB) {
        if (p.type[g] & T_SOLID) {
            rho_out[g] = C(0);
            continue;
        }
        C f[9];
        pull9<S, C>(fin, p.type, g % nx, g / nx, nx, ny, N, f);
        C d = C(0);
#pragma unroll
        for (int a = 0; a < 9; ++a) d += f[a];
        rho_out[g] = rho_ref + d;
    }
}

template <class C>
__global__ void __launch_bounds__(AB) adj_psi(DevParams p, const C* __restrict__ rho, C* __restrict__ psi,
                                              C* __restrict__ dpsi, C* __restrict__ drw_k, C* __restrict__ drw_a) {
    const int N = int(p.N), nx = p.nx, ny = p.ny;
    const EosA<C> e = eos_of<C>(p);
    const C rho_l = C(p.rho_l), rho_g = C(p.rho_g);
    for (int g = blockIdx.x * AB + threadIdx.x; g < N; g += gridDim.x * AB) {
        const uint8_t t = p.type[g];
        C ps = C(0), dps = C(0), dk = C(0), da = C(0);
        if (!(t & T_SOLID)) {
            psi_and_slope(rho[g], e, ps, dps);
        } else if (t & T_WALL) {
            C rw;
            if (p.wall_kind == 1) {
                rw = C(p.rho_w_const);
            } else {
                const int x = g % nx, y = g / nx;
                C num = C(0), den = C(0);
#pragma unroll
                for (int a = 1; a < 9; ++a) {
                    const int s = wrapn(y + D2Q9::ey(a), ny) * nx + wrapn(x + D2Q9::ex(a), nx);
                    if (!(p.type[s] & T_SOLID)) {
                        num += C(D2Q9::wf(a)) * rho[s];
                        den += C(D2Q9::wf(a));
                    }
                }
                const C ra = num / den;
                const C kap = p.kappa_w ? C(p.kappa_w[p.wall_id[g]]) : C(p.kappa);
                const C raw = kap >= C(0) ? (C(1) + kap) * ra : ra + kap;
                rw = raw > rho_l ? rho_l : (raw < rho_g ? rho_g : raw);
                if (raw < rho_l && raw > rho_g) {   // the limiter is inactive
                    dk = kap >= C(0) ? ra : C(1);
                    da = (kap >= C(0) ? C(1) + kap : C(1)) / den;
                }
            }
            psi_and_slope(rw, e, ps, dps);
        }
        psi[g] = ps;
        dpsi[g] = dps;
        drw_k[g] = dk;
        drw_a[g] = da;
    }
}

template <class S, class C>
__global__ void __launch_bounds__(AB) adj_local(const S* __restrict__ fin, const C* __restrict__ mu, DevParams p,
                                                const C* __restrict__ psi, C* __restrict__ lam, C* __restrict__ fmb_x,
                                                C* __restrict__ fmb_y, C* __restrict__ psib) {
    const int N = int(p.N), nx = p.nx, ny = p.ny;
    Rates<C> r;
    r.s_e = C(p.s_e);
    r.s_eps = C(p.s_eps);
    r.s_q = C(p.s_q);
    r.s_nu = C(p.s_nu);
    r.s_pi = C(p.s_pi);
    r.s_m = C(p.s_m);
    r.c_e = C(p.c_e);
    r.c_eps = C(p.c_eps);
    const C G = C(p.G), rho_ref = C(p.rho_ref);
    for (int g = blockIdx.x * AB + threadIdx.x; g < N; g += gridDim.x * AB) {
        if (p.type[g] & T_SOLID) {
            fmb_x[g] = C(0);
            fmb_y[g] = C(0);
            psib[g] = C(0);
            continue;
        }
        const int x = g % nx, y = g / nx;
        C f[9];
        pull9<S, C>(fin, p.type, x, y, nx, ny, N, f);
        const C psi_c = psi[g];
        C sx = C(0), sy = C(0);
#pragma unroll
        for (int a = 1; a < 9; ++a) {
            const C v = C(D2Q9::wf(a)) * psi[wrapn(y + D2Q9::ey(a), ny) * nx + wrapn(x + D2Q9::ex(a), nx)];
            sx += C(D2Q9::ex(a)) * v;
            sy += C(D2Q9::ey(a)) * v;
        }
        const C Fmx = -G * psi_c * sx, Fmy = -G * psi_c * sy;
        const C Fx = Fmx + C(p.fx), Fy = Fmy + C(p.fy);
        C drho = C(0), jx = C(0), jy = C(0);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            drho += f[a];
            jx += C(D2Q9::ex(a)) * f[a];
            jy += C(D2Q9::ey(a)) * f[a];
        }
        const C rho = rho_ref + drho;
        const C ux = (jx + C(0.5) * Fx) / rho, uy = (jy + C(0.5) * Fy) / rho;
        C m[9], fb[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) m[a] = mu[a * N + g];
        C bx, by, pb;
        collide_d2q9_adjoint<C>(f, m, rho, ux, uy, Fx, Fy, Fmx, Fmy, psi_c, r, fb, bx, by, pb);
#pragma unroll
        for (int a = 0; a < 9; ++a) lam[a * N + g] = fb[a];
        fmb_x[g] = bx;
        fmb_y[g] = by;
        // F_m = -G psi(x) sum w psi(x+e) e: its dependence on psi(x) is F_m / psi(x)
        psib[g] = pb + (bx * Fmx + by * Fmy) / psi_c;
    }
}

template <class C>
__global__ void __launch_bounds__(AB) adj_psibar(DevParams p, const C* __restrict__ psi, const C* __restrict__ dpsi,
                                                 const C* __restrict__ drw_k, const C* __restrict__ drw_a,
                                                 const C* __restrict__ fmb_x, const C* __restrict__ fmb_y,
                                                 const C* __restrict__ psib, C* __restrict__ rhob, C* __restrict__ wb,
                                                 double* __restrict__ dkappa) {
    const int N = int(p.N), nx = p.nx, ny = p.ny;
    const C G = C(p.G);
    for (int g = blockIdx.x * AB + threadIdx.x; g < N; g += gridDim.x * AB) {
        const uint8_t t = p.type[g];
        const bool fluid = !(t & T_SOLID);
        if (!fluid && !(t & T_WALL)) {
            rhob[g] = C(0);
            wb[g] = C(0);
            continue;
        }
        const int x = g % nx, y = g / nx;
        // psi(y) enters F_m(x) of every fluid x = y - e_a with weight -G psi(x) w_a e_a
        C pb = fluid ? psib[g] : C(0);
#pragma unroll
        for (int a = 1; a < 9; ++a) {
            const int s = wrapn(y - D2Q9::ey(a), ny) * nx + wrapn(x - D2Q9::ex(a), nx);
            if (p.type[s] & T_SOLID) continue;
            const C proj = fmb_x[s] * C(D2Q9::ex(a)) + fmb_y[s] * C(D2Q9::ey(a));
            pb += -G * psi[s] * C(D2Q9::wf(a)) * proj;
        }
        const C rb = pb * dpsi[g];
        if (fluid) {
            rhob[g] = rb;
            wb[g] = C(0);
        } else {
            rhob[g] = C(0);
            wb[g] = rb * drw_a[g];
            if (p.kappa_w) dkappa[p.wall_id[g]] += double(rb * drw_k[g]);
        }
    }
}

// lambda = lam + rho-bar (own psi and wall neighbours' averages); push: lambda_a(z) -> mu_a(z - e_a)
// if z - e_a is fluid, else mu_abar(z)
template <class C, bool FINAL>
__global__ void __launch_bounds__(AB) adj_push(DevParams p, const C* __restrict__ lam, const C* __restrict__ rhob,
                                               const C* __restrict__ wb, const double* __restrict__ drho_final,
                                               C* __restrict__ mu_out) {
    const int N = int(p.N), nx = p.nx, ny = p.ny;
    for (int g = blockIdx.x * AB + threadIdx.x; g < N; g += gridDim.x * AB) {
        if (p.type[g] & T_SOLID) continue;
        const int x = g % nx, y = g / nx;
        C rb;
        if (FINAL) {
            rb = C(drho_final[g]);
        } else {
            rb = rhob[g];
#pragma unroll
            for (int a = 1; a < 9; ++a) {
                const int s = wrapn(y + D2Q9::ey(a), ny) * nx + wrapn(x + D2Q9::ex(a), nx);
                if (p.type[s] & T_WALL) rb += C(D2Q9::wf(a)) * wb[s];
            }
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const C l = FINAL ? rb : lam[a * N + g] + rb;
            const int s = wrapn(y - D2Q9::ey(a), ny) * nx + wrapn(x - D2Q9::ex(a), nx);
            if (p.type[s] & T_SOLID) mu_out[D2Q9::opp(a) * N + g] = l;
            else mu_out[a * N + s] = l;
        }
    }
}

unsigned grid_of(long long n) {
    long long b = (n + AB - 1) / AB;
    if (b > 152LL * 16) b = 152LL * 16;
    return unsigned(b < 1 ? 1 : b);
}

template <class S>
cudaError_t adjoint_step_t(const void* fstar_k, const void* mu_next, void* mu_prev, const DevParams& p,
                           const AdjointScratch& w, double* dkappa, cudaStream_t s) {
    using C = S;
    const unsigned g = grid_of(p.N);
    const int N = int(p.N);
    C* rho = static_cast<C*>(w.buf) + 0 * (size_t)N;
    C* psi = static_cast<C*>(w.buf) + 1 * (size_t)N;
    C* dpsi = static_cast<C*>(w.buf) + 2 * (size_t)N;
    C* drw_k = static_cast<C*>(w.buf) + 3 * (size_t)N;
    C* drw_a = static_cast<C*>(w.buf) + 4 * (size_t)N;
    C* fmb_x = static_cast<C*>(w.buf) + 5 * (size_t)N;
    C* fmb_y = static_cast<C*>(w.buf) + 6 * (size_t)N;
    C* psib = static_cast<C*>(w.buf) + 7 * (size_t)N;
    C* rhob = static_cast<C*>(w.buf) + 8 * (size_t)N;
    C* wb = static_cast<C*>(w.buf) + 9 * (size_t)N;
    C* lam = static_cast<C*>(w.buf) + 10 * (size_t)N;   // 9 N values
    const S* fin = static_cast<const S*>(fstar_k);
    adj_density<S, C><<<g, AB, 0, s>>>(fin, p, rho);
    adj_psi<C><<<g, AB, 0, s>>>(p, rho, psi, dpsi, drw_k, drw_a);
    adj_local<S, C><<<g, AB, 0, s>>>(fin, static_cast<const C*>(mu_next), p, psi, lam, fmb_x, fmb_y, psib);
    adj_psibar<C><<<g, AB, 0, s>>>(p, psi, dpsi, drw_k, drw_a, fmb_x, fmb_y, psib, rhob, wb, dkappa);
    adj_push<C, false><<<g, AB, 0, s>>>(p, lam, rhob, wb, nullptr, static_cast<C*>(mu_prev));
    return cudaGetLastError();
}

}  // namespace

size_t adjoint_scratch_elems(long long N) { return size_t(N) * 19; }

cudaError_t launch_adjoint_step(int prec, const void* fstar_k, const void* mu_next, void* mu_prev, const DevParams& p,
                                const AdjointScratch& w, double* dkappa, cudaStream_t s) {
    if (prec == PREC_FP64) return adjoint_step_t<double>(fstar_k, mu_next, mu_prev, p, w, dkappa, s);
    return adjoint_step_t<float>(fstar_k, mu_next, mu_prev, p, w, dkappa, s);
}

cudaError_t launch_adjoint_final(int prec, const double* drho_final, void* mu, const DevParams& p, cudaStream_t s) {
    const unsigned g = grid_of(p.N);
    if (prec == PREC_FP64)
        adj_push<double, true><<<g, AB, 0, s>>>(p, nullptr, nullptr, nullptr, drho_final, static_cast<double*>(mu));
    else
        adj_push<float, true><<<g, AB, 0, s>>>(p, nullptr, nullptr, nullptr, drho_final, static_cast<float*>(mu));
    return cudaGetLastError();
}

}  // namespace lbmwet
