// Fused time-step kernels of the pseudopotential MRT-LB method with improved virtual-density walls.
//
// One CTA owns a TX x TY (x TZ) tile of nodes.  The state in global memory is the post-collision
// f* of the previous step (structure of arrays, [a][node]); a step is
//   0. node-type flags of the tile + 3-node halo into shared memory;
//   1. pull-streaming (Eq. 3) with halfway bounce-back (Fig. 3) of every node of the tile + 2-node
//      halo, and its density (Eq. 4) into shared memory (the tile's own pulled f stay in registers);
//   2. psi (Eq. 6) on the tile + 1-node halo: from rho at fluid nodes, and at wall nodes from the
//      virtual density of Eqs. 16-17 (improved scheme with limiter, Sec. III.B) or the constant one
//      (Sec. II.B), itself averaged from the shared-memory densities of its fluid neighbours;
//   3. at the tile's fluid nodes: F_m (Eq. 5) from shared psi, F = F_m + body force, u (Eq. 4), the
//      MRT collision with the consistency source (Eqs. 2, 7), and a coalesced store of f*.
// Steps 1-2 need neighbour values of the same time level, hence the halo recomputation: nothing
// but f* is written to global memory per step.
#include <cmath>

#include "kernels.h"
#include "lattice.cuh"

namespace lbmwet {

template <class C>
struct EosC {
    int kind;
    C RT, a, b, b4, aphi, two_over_G;
};

template <class C>
__device__ __forceinline__ C psi_arg(C rho, const EosC<C>& e) {
    C p;
    if (e.kind == 1) {  // Carnahan-Starling
        const C eta = e.b4 * rho;
        const C om = C(1) - eta;
        p = rho * e.RT * (C(1) + eta + eta * eta - eta * eta * eta) / (om * om * om) - e.a * rho * rho;
    } else {            // Peng-Robinson, Eq. 18
        p = rho * e.RT / (C(1) - e.b * rho) - e.aphi * rho * rho / (C(1) + C(2) * e.b * rho - e.b * e.b * rho * rho);
    }
    return e.two_over_G * (p - rho * C(1.0 / 3.0));   // Eq. 6 argument: 2 (p - rho c_s^2) / (G c^2)
}

template <class C>
__device__ __forceinline__ C psi_checked(C rho, const EosC<C>& e, unsigned* err) {
    const C arg = psi_arg(rho, e);
    if (!(arg > C(0))) {
        atomicOr(err, ERR_PSI);
        return C(0);
    }
    return sqrt(arg);
}

__device__ __forceinline__ int wrap_full(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}
__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

template <class L, class S, class C, int TX, int TY, int TZ, int BY, int MODE>
__global__ void __launch_bounds__(TX* BY) fused_step(const S* __restrict__ fin, S* __restrict__ fout, DevParams p,
                                                     double* __restrict__ rho_out, double* __restrict__ u_out) {
    constexpr int D = L::D, Q = L::Q;
    constexpr int HZ = (D == 3) ? 2 : 0;        // rho halo along z
    constexpr int PZH = (D == 3) ? 1 : 0;       // psi halo along z
    constexpr int YZH = (D == 3) ? 3 : 0;       // type halo along z
    constexpr int RX = TX + 4, RY = TY + 4, RZ = TZ + 2 * HZ;
    constexpr int PX = TX + 2, PY = TY + 2, PZ = TZ + 2 * PZH;
    constexpr int YX = TX + 6, YY = TY + 6, YZ = TZ + 2 * YZH;
    constexpr int NT = TX * BY;
    constexpr int RPT = (TY * TZ) / BY;
    static_assert((TY * TZ) % BY == 0, "rows per thread");

    __shared__ uint8_t s_type[YZ * YY * YX];
    __shared__ C s_rho[RZ * RY * RX];
    __shared__ C s_psi[PZ * PY * PX];

    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const long long N = p.N;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const int tid = threadIdx.y * TX + threadIdx.x;

    EosC<C> eos;
    eos.kind = p.eos_kind;
    eos.RT = C(p.RT);
    eos.a = C(p.a);
    eos.b = C(p.b);
    eos.b4 = C(p.b * 0.25);
    eos.aphi = C(p.aphi);
    eos.two_over_G = C(p.two_over_G);
    const C rho_ref = C(p.rho_ref);

    auto tidx = [&](int lx, int ly, int lz) { return (lz * YY + ly) * YX + lx; };
    auto ridx = [&](int lx, int ly, int lz) { return (lz * RY + ly) * RX + lx; };
    auto pidx = [&](int lx, int ly, int lz) { return (lz * PY + ly) * PX + lx; };

    // 0. node types of the tile + 3-node halo
    for (int i = tid; i < YX * YY * YZ; i += NT) {
        const int lx = i % YX, t = i / YX, ly = t % YY, lz = t / YY;
        const int gx = wrap_full(x0 + lx - 3, nx), gy = wrap_full(y0 + ly - 3, ny);
        const int gz = (D == 3) ? wrap_full(z0 + lz - YZH, nz) : 0;
        s_type[i] = p.type[((long long)gz * ny + gy) * nx + gx];
    }
    __syncthreads();

    // pull of one node: f_a(x) = f*_a(x - e_a) if x - e_a is fluid, else f*_abar(x)
    auto pull = [&](C (&f)[Q], int gx, int gy, int gz, int tx, int ty, int tz) {
        const long long g = ((long long)gz * ny + gy) * nx + gx;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
            if (s_type[tidx(tx - ex, ty - ey, tz - ez)] & T_SOLID) {
                f[a] = C(fin[(long long)L::opp(a) * N + g]);
            } else {
                const int sx = ex ? wrap1(gx - ex, nx) : gx;
                const int sy = ey ? wrap1(gy - ey, ny) : gy;
                const int sz = ez ? wrap1(gz - ez, nz) : gz;
                f[a] = C(fin[(long long)a * N + ((long long)sz * ny + sy) * nx + sx]);
            }
        }
    };

    // 1a. the tile's own nodes: pull into registers, density into shared memory
    C f[RPT][Q];
    int gxs[RPT], gys[RPT], gzs[RPT];
    bool fluid[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int j = threadIdx.y + r * BY;
        const int lx = threadIdx.x, ly = j % TY, lz = j / TY;
        const int gx = wrap_full(x0 + lx, nx), gy = wrap_full(y0 + ly, ny);
        const int gz = (D == 3) ? wrap_full(z0 + lz, nz) : 0;
        gxs[r] = gx;
        gys[r] = gy;
        gzs[r] = gz;
        const int tx = lx + 3, ty = ly + 3, tz = lz + YZH;
        fluid[r] = !(s_type[tidx(tx, ty, tz)] & T_SOLID);
        C drho = C(0);
        if (fluid[r]) {
            pull(f[r], gx, gy, gz, tx, ty, tz);
#pragma unroll
            for (int a = 0; a < Q; ++a) drho += f[r][a];
        } else {
#pragma unroll
            for (int a = 0; a < Q; ++a) f[r][a] = C(0);
        }
        s_rho[ridx(lx + 2, ly + 2, lz + HZ)] = fluid[r] ? rho_ref + drho : C(0);
    }
    // 1b. the 2-node halo ring: density only
    for (int i = tid; i < RX * RY * RZ; i += NT) {
        const int lx = i % RX, t = i / RX, ly = t % RY, lz = t / RY;
        if (lx >= 2 && lx < TX + 2 && ly >= 2 && ly < TY + 2 && lz >= HZ && lz < TZ + HZ) continue;
        const int gx = wrap_full(x0 + lx - 2, nx), gy = wrap_full(y0 + ly - 2, ny);
        const int gz = (D == 3) ? wrap_full(z0 + lz - HZ, nz) : 0;
        const int tx = lx + 1, ty = ly + 1, tz = lz + (YZH - HZ);
        C rho = C(0);
        if (!(s_type[tidx(tx, ty, tz)] & T_SOLID)) {
            C g[Q];
            pull(g, gx, gy, gz, tx, ty, tz);
            C drho = C(0);
#pragma unroll
            for (int a = 0; a < Q; ++a) drho += g[a];
            rho = rho_ref + drho;
        }
        s_rho[i] = rho;
    }
    __syncthreads();

    // 2. psi on the tile + 1-node halo
    const C rho_g = C(p.rho_g), rho_l = C(p.rho_l);
    for (int i = tid; i < PX * PY * PZ; i += NT) {
        const int lx = i % PX, t = i / PX, ly = t % PY, lz = t / PY;
        const int rx = lx + 1, ry = ly + 1, rz = lz + (HZ - PZH);
        const int tx = lx + 2, ty = ly + 2, tz = lz + (YZH - PZH);
        const uint8_t ty_ = s_type[tidx(tx, ty, tz)];
        C psi = C(0);
        if (!(ty_ & T_SOLID)) {
            psi = psi_checked(s_rho[ridx(rx, ry, rz)], eos, p.err);
        } else if (ty_ & T_WALL) {
            C rw;
            if (p.wall_kind == 1) {
                rw = C(p.rho_w_const);
            } else {
                // Eq. 17: weighted mean of the fluid neighbours' densities
                C num = C(0), den = C(0);
#pragma unroll
                for (int a = 1; a < Q; ++a) {
                    const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
                    if (!(s_type[tidx(tx + ex, ty + ey, tz + ez)] & T_SOLID)) {
                        num += C(L::wf(a)) * s_rho[ridx(rx + ex, ry + ey, rz + ez)];
                        den += C(L::wf(a));
                    }
                }
                const C rho_ave = num / den;
                C kap;
                if (p.kappa_w) {
                    const int gx = wrap_full(x0 + lx - 1, nx), gy = wrap_full(y0 + ly - 1, ny);
                    const int gz = (D == 3) ? wrap_full(z0 + lz - PZH, nz) : 0;
                    kap = C(p.kappa_w[p.wall_id[((long long)gz * ny + gy) * nx + gx]]);
                } else {
                    kap = C(p.kappa);
                }
                // Eq. 16 (kappa >= 0: phi = 1 + kappa; kappa < 0: drho = -kappa) and the limiter
                rw = (kap >= C(0)) ? (C(1) + kap) * rho_ave : rho_ave + kap;
                rw = rw > rho_l ? rho_l : rw;
                rw = rw < rho_g ? rho_g : rw;
            }
            psi = psi_checked(rw, eos, p.err);
        }
        s_psi[i] = psi;
    }
    __syncthreads();

    // 3. force, velocity and collision of the tile's fluid nodes
    Rates<C> rates;
    rates.s_e = C(p.s_e);
    rates.s_eps = C(p.s_eps);
    rates.s_q = C(p.s_q);
    rates.s_nu = C(p.s_nu);
    rates.s_pi = C(p.s_pi);
    rates.s_m = C(p.s_m);
    rates.c_e = C(p.c_e);
    rates.c_eps = C(p.c_eps);
    const C G = C(p.G);
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int j = threadIdx.y + r * BY;
        const int lx = threadIdx.x, ly = j % TY, lz = j / TY;
        const bool valid = (x0 + lx < nx) && (y0 + ly < ny) && (D == 2 || z0 + lz < nz);
        if (!valid) continue;
        const long long g = ((long long)gzs[r] * ny + gys[r]) * nx + gxs[r];
        if (!fluid[r]) {
            if (MODE == 1) {
                if (rho_out) rho_out[g] = 0.0;
                if (u_out) {
                    for (int c = 0; c < D; ++c) u_out[(long long)c * N + g] = 0.0;
                }
            }
            continue;
        }
        const int px = lx + 1, py = ly + 1, pz = lz + PZH;
        const C psi_c = s_psi[pidx(px, py, pz)];
        // sum_a w_a psi(x + e_a) e_a, taken over opposite pairs: w_a e_a (psi(x + e_a) - psi(x - e_a))
        // (nearly equal values cancel exactly in the difference, which keeps FP32 accurate in bulk)
        C sx = C(0), sy = C(0), sz = C(0);
#pragma unroll
        for (int a = 1; a < Q; ++a) {
            if (L::opp(a) < a) continue;
            const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
            const C dpsi = s_psi[pidx(px + ex, py + ey, pz + ez)] - s_psi[pidx(px - ex, py - ey, pz - ez)];
            const C wd = C(L::wf(a)) * dpsi;
            if (ex) sx += C(ex) * wd;
            if (ey) sy += C(ey) * wd;
            if (D == 3 && ez) sz += C(ez) * wd;
        }
        // Eq. 5
        const C Fmx = -G * psi_c * sx, Fmy = -G * psi_c * sy, Fmz = -G * psi_c * sz;
        const C Fx = Fmx + C(p.fx), Fy = Fmy + C(p.fy), Fz = Fmz + C(p.fz);
        C drho = C(0), jx = C(0), jy = C(0), jz = C(0);
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            drho += f[r][a];
            if (L::ex(a)) jx += C(L::ex(a)) * f[r][a];
            if (L::ey(a)) jy += C(L::ey(a)) * f[r][a];
            if (D == 3 && L::ez(a)) jz += C(L::ez(a)) * f[r][a];
        }
        const C rho = rho_ref + drho;
        if (!(rho > C(0))) atomicOr(p.err, ERR_RHO);
        // Eq. 4: rho u = sum e f + F/2
        const C inv = C(1) / rho;
        const C ux = (jx + C(0.5) * Fx) * inv, uy = (jy + C(0.5) * Fy) * inv, uz = (jz + C(0.5) * Fz) * inv;
        if (MODE == 1) {
            if (rho_out) rho_out[g] = double(rho);
            if (u_out) {
                u_out[g] = double(ux);
                u_out[N + g] = double(uy);
                if (D == 3) u_out[2 * N + g] = double(uz);
            }
            continue;
        }
        const C X = (Fmx * Fmx + Fmy * Fmy + Fmz * Fmz) / (psi_c * psi_c);
        if constexpr (D == 2) {
            collide_d2q9<C>(f[r], drho, rho, ux, uy, Fx, Fy, X, rates);
        } else {
            collide_d3q19<C>(f[r], drho, rho, ux, uy, uz, Fx, Fy, Fz, X, rates);
        }
#pragma unroll
        for (int a = 0; a < Q; ++a) fout[(long long)a * N + g] = S(f[r][a]);
    }
}

// ---------------------------------------------------------------------------------------------
// Initial state, state transfer and node classification (simple one-node-per-thread kernels).
// ---------------------------------------------------------------------------------------------

template <class L>
__device__ __forceinline__ double feq_a(int a, double rho, double ux, double uy, double uz) {
    const double eu = L::ex(a) * ux + L::ey(a) * uy + L::ez(a) * uz;
    const double uu = ux * ux + uy * uy + uz * uz;
    return L::w(a) * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
}

__device__ __forceinline__ void coords(long long g, int nx, int ny, int& x, int& y, int& z) {
    x = int(g % nx);
    const long long t = g / nx;
    y = int(t % ny);
    z = int(t / ny);
}

// Stored f* whose pull gives f_post: f*_b(y) = f_post_b(y + e_b) if y + e_b is fluid, else
// f_post_bbar(y) (the inverse of the pull with bounce-back).  Source is either f^eq(rho0, u0) or
// explicit post-streaming values.
template <class L, class S, bool FROM_FEQ>
__global__ void unstream_kernel(S* __restrict__ fout, DevParams p, const double* __restrict__ src0,
                                const double* __restrict__ src1) {
    constexpr int Q = L::Q;
    const long long N = p.N;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
        if (p.type[g] & T_SOLID) {
            for (int b = 0; b < Q; ++b) fout[(long long)b * N + g] = S(0);
            continue;
        }
        int x, y, z;
        coords(g, p.nx, p.ny, x, y, z);
        for (int b = 0; b < Q; ++b) {
            const int tx = wrap1(x + L::ex(b), p.nx), ty = wrap1(y + L::ey(b), p.ny);
            const int tz = (L::D == 3) ? wrap1(z + L::ez(b), p.nz) : 0;
            const long long t = ((long long)tz * p.ny + ty) * p.nx + tx;
            long long src;
            int a;
            if (!(p.type[t] & T_SOLID)) {
                src = t;
                a = b;
            } else {
                src = g;
                a = L::opp(b);
            }
            double v;
            if (FROM_FEQ) {
                const double* rho0 = src0;
                const double* u0 = src1;
                const double ux = u0 ? u0[src] : 0.0, uy = u0 ? u0[N + src] : 0.0;
                const double uz = (u0 && L::D == 3) ? u0[2 * N + src] : 0.0;
                v = feq_a<L>(a, rho0[src], ux, uy, uz);
            } else {
                v = src0[(long long)a * N + src];
            }
            fout[(long long)b * N + g] = S(v - L::w(b) * p.rho_ref);
        }
    }
}

template <class L, class S>
__global__ void get_state_kernel(const S* __restrict__ fin, DevParams p, double* __restrict__ fpost) {
    constexpr int Q = L::Q;
    const long long N = p.N;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
        if (p.type[g] & T_SOLID) {
            for (int a = 0; a < Q; ++a) fpost[(long long)a * N + g] = 0.0;
            continue;
        }
        int x, y, z;
        coords(g, p.nx, p.ny, x, y, z);
        for (int a = 0; a < Q; ++a) {
            const int sx = wrap1(x - L::ex(a), p.nx), sy = wrap1(y - L::ey(a), p.ny);
            const int sz = (L::D == 3) ? wrap1(z - L::ez(a), p.nz) : 0;
            const long long s = ((long long)sz * p.ny + sy) * p.nx + sx;
            double v;
            if (p.type[s] & T_SOLID) v = double(fin[(long long)L::opp(a) * N + g]);
            else v = double(fin[(long long)a * N + s]);
            fpost[(long long)a * N + g] = v + L::w(a) * p.rho_ref;
        }
    }
}

template <class L>
__global__ void classify_kernel(const uint8_t* __restrict__ mask, uint8_t* __restrict__ type, int nx, int ny, int nz) {
    const long long N = (long long)nx * ny * nz;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords(g, nx, ny, x, y, z);
        uint8_t t = 0;
        const bool solid = mask[g] != 0;
        if (solid) {
            t |= T_SOLID;
            for (int a = 1; a < L::Q; ++a) {
                const int sx = wrap1(x + L::ex(a), nx), sy = wrap1(y + L::ey(a), ny);
                const int sz = (L::D == 3) ? wrap1(z + L::ez(a), nz) : 0;
                if (!mask[((long long)sz * ny + sy) * nx + sx]) {
                    t |= T_WALL;
                    break;
                }
            }
        }
        // within Euclidean distance 3 of a solid node
        bool near = false;
        const int rz = (L::D == 3) ? 3 : 0;
        for (int dz = -rz; dz <= rz && !near; ++dz)
            for (int dy = -3; dy <= 3 && !near; ++dy)
                for (int dx = -3; dx <= 3 && !near; ++dx) {
                    if (dx * dx + dy * dy + dz * dz > 9) continue;
                    const int sx = wrap_full(x + dx, nx), sy = wrap_full(y + dy, ny);
                    const int sz = (L::D == 3) ? wrap_full(z + dz, nz) : 0;
                    if (mask[((long long)sz * ny + sy) * nx + sx]) near = true;
                }
        if (near) t |= T_NEARWALL;
        type[g] = t;
    }
}

// ---------------------------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------------------------

template <class L, class S, class C, int TX, int TY, int TZ, int BY, int MODE>
static cudaError_t launch_tile(const void* fin, void* fout, const DevParams& p, double* rho, double* u, cudaStream_t s) {
    dim3 grid((p.nx + TX - 1) / TX, (p.ny + TY - 1) / TY, (p.nz + TZ - 1) / TZ);
    dim3 block(TX, BY, 1);
    fused_step<L, S, C, TX, TY, TZ, BY, MODE>
        <<<grid, block, 0, s>>>(static_cast<const S*>(fin), static_cast<S*>(fout), p, rho, u);
    return cudaGetLastError();
}

// Tile shapes: 2D 32x16 tiles with 256 threads (2 nodes per thread); 3D 32x4x4 tiles, 256 threads.
template <int MODE>
static cudaError_t dispatch(int lat, int prec, const void* fin, void* fout, const DevParams& p, double* rho, double* u,
                            cudaStream_t s) {
    if (lat == LAT_D2Q9) {
        if (prec == PREC_FP64) return launch_tile<D2Q9, double, double, 32, 16, 1, 8, MODE>(fin, fout, p, rho, u, s);
        return launch_tile<D2Q9, float, float, 32, 16, 1, 8, MODE>(fin, fout, p, rho, u, s);
    }
    if (prec == PREC_FP64) return launch_tile<D3Q19, double, double, 32, 4, 4, 16, MODE>(fin, fout, p, rho, u, s);
    return launch_tile<D3Q19, float, float, 32, 4, 4, 8, MODE>(fin, fout, p, rho, u, s);
}

cudaError_t launch_step(int lat, int prec, const void* fin, void* fout, const DevParams& p, cudaStream_t s) {
    return dispatch<0>(lat, prec, fin, fout, p, nullptr, nullptr, s);
}

cudaError_t launch_fields(int lat, int prec, const void* fin, const DevParams& p, double* rho, double* u,
                          cudaStream_t s) {
    return dispatch<1>(lat, prec, fin, nullptr, p, rho, u, s);
}

static unsigned grid_for(long long n) {
    long long b = (n + 255) / 256;
    if (b > 152LL * 32) b = 152LL * 32;
    return unsigned(b < 1 ? 1 : b);
}

template <class L, bool FEQ>
static cudaError_t unstream_l(int prec, void* fout, const DevParams& p, const double* a, const double* b, cudaStream_t s) {
    if (prec == PREC_FP64)
        unstream_kernel<L, double, FEQ><<<grid_for(p.N), 256, 0, s>>>(static_cast<double*>(fout), p, a, b);
    else
        unstream_kernel<L, float, FEQ><<<grid_for(p.N), 256, 0, s>>>(static_cast<float*>(fout), p, a, b);
    return cudaGetLastError();
}

cudaError_t launch_init(int lat, int prec, void* fout, const DevParams& p, const double* rho0, const double* u0,
                        cudaStream_t s) {
    return lat == LAT_D2Q9 ? unstream_l<D2Q9, true>(prec, fout, p, rho0, u0, s)
                           : unstream_l<D3Q19, true>(prec, fout, p, rho0, u0, s);
}

cudaError_t launch_set_state(int lat, int prec, void* fout, const DevParams& p, const double* fpost, cudaStream_t s) {
    return lat == LAT_D2Q9 ? unstream_l<D2Q9, false>(prec, fout, p, fpost, nullptr, s)
                           : unstream_l<D3Q19, false>(prec, fout, p, fpost, nullptr, s);
}

cudaError_t launch_get_state(int lat, int prec, const void* fin, const DevParams& p, double* fpost, cudaStream_t s) {
    const unsigned g = grid_for(p.N);
    if (lat == LAT_D2Q9) {
        if (prec == PREC_FP64) get_state_kernel<D2Q9, double><<<g, 256, 0, s>>>(static_cast<const double*>(fin), p, fpost);
        else get_state_kernel<D2Q9, float><<<g, 256, 0, s>>>(static_cast<const float*>(fin), p, fpost);
    } else {
        if (prec == PREC_FP64) get_state_kernel<D3Q19, double><<<g, 256, 0, s>>>(static_cast<const double*>(fin), p, fpost);
        else get_state_kernel<D3Q19, float><<<g, 256, 0, s>>>(static_cast<const float*>(fin), p, fpost);
    }
    return cudaGetLastError();
}

cudaError_t launch_classify(int lat, const uint8_t* mask, uint8_t* type, int nx, int ny, int nz, cudaStream_t s) {
    const unsigned g = grid_for((long long)nx * ny * nz);
    if (lat == LAT_D2Q9) classify_kernel<D2Q9><<<g, 256, 0, s>>>(mask, type, nx, ny, nz);
    else classify_kernel<D3Q19><<<g, 256, 0, s>>>(mask, type, nx, ny, nz);
    return cudaGetLastError();
}

}  // namespace lbmwet
