// D3Q19 time step as a z-march: one CTA owns a TX x TY column of the grid and walks a chunk of
// z-planes, keeping rolling shared-memory rings of
//   node types   5 planes of the column + 3-node xy halo,
//   densities    3 planes (+2-node xy halo),
//   psi          4 planes (+1-node xy halo),
//   distributions 3 planes of the column's own nodes (pulled once, collided two planes later).
// For lead plane zl the CTA
//   A. pulls (Eq. 3 with halfway bounce-back, Fig. 3) every node of plane zl in the 1-node xy halo
//      (the 2-node halo too where the column holds solid nodes), stores rho (Eq. 4) and, at fluid
//      nodes, psi (Eq. 6); wall nodes are queued;
//   B. gives the queued wall nodes of plane zl - 1 their virtual density (Eqs. 16-17 with the
//      limiter, or the constant one) from the densities of planes zl - 2 .. zl, and its psi;
//   C. collides plane zl - 2: F_m (Eq. 5) from psi of planes zl - 3 .. zl - 1, u (Eq. 4), the MRT
//      collision with the consistency source (Eqs. 2, 7), and a coalesced store of f*.
// Each node is pulled once plus the thin xy halo, instead of the full 3D halo shell of a cubic tile.
#include <cmath>

#include "kernels.h"
#include "lattice.cuh"
#include "tile_common.cuh"

namespace lbmwet {

namespace {

template <class C, int TX, int TY>
struct ZSmem {
    static constexpr int YX = TX + 6, YY = TY + 6;   // type planes (3-node xy halo)
    static constexpr int RX = TX + 4, RY = TY + 4;   // density planes (2-node xy halo)
    static constexpr int PX = TX + 2, PY = TY + 2;   // psi planes (1-node xy halo)
    uint8_t type[5][YY * YX];
    C rho[3][RY * RX];
    C psi[4][PY * PX];
    C f[3][19][TY * TX];
    short wq[2][PY * PX];
    int nw[2];
};

__device__ __forceinline__ int ring(int z, int r) {
    const int m = z % r;
    return m < 0 ? m + r : m;
}

template <class S>
struct ZShape;
template <> struct ZShape<float> {
    static constexpr int X = LBMWET_Z3F_X, Y = LBMWET_Z3F_Y, Z = LBMWET_Z3F_Z, MINB = LBMWET_Z3F_MINB;
};
template <> struct ZShape<double> { static constexpr int X = 32, Y = 4, Z = 32, MINB = 1; };

template <class S, class C, int MODE>
__global__ void __launch_bounds__(ZShape<S>::X* ZShape<S>::Y, ZShape<S>::MINB)
    zmarch_step(const S* __restrict__ fin, S* __restrict__ fout, Geo g, Phys<C> ph, unsigned* err,
                double* __restrict__ rho_out, double* __restrict__ u_out) {
    using L = D3Q19;
    constexpr int Q = 19, TX = ZShape<S>::X, TY = ZShape<S>::Y, ZC = ZShape<S>::Z, NT = TX * TY;
    using Sm = ZSmem<C, TX, TY>;
    constexpr int YX = Sm::YX, YY = Sm::YY, RX = Sm::RX, RY = Sm::RY, PX = Sm::PX, PY = Sm::PY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Sm& sm = *reinterpret_cast<Sm*>(smem_raw);

    const int nx = g.nx, ny = g.ny, nz = g.nz, N = g.N;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, zb = blockIdx.z * ZC;
    const int ze = min(zb + ZC, nz);
    const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * TX + lx;
    const bool small = nx < TX + 8 || ny < TY + 8 || nz < 8;
    auto wx = [&](int v) { return small ? wrap_full(v, nx) : wrap1(v, nx); };
    auto wy = [&](int v) { return small ? wrap_full(v, ny) : wrap1(v, ny); };
    auto wz = [&](int v) { return small ? wrap_full(v, nz) : wrap1(v, nz); };
    const int tile = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const bool solid = g.tile_solid ? g.tile_solid[tile] != 0 : true;
    const int nxy = nx * ny;

    auto load_types = [&](int z) {
        if (!solid) return;
        uint8_t* dst = sm.type[ring(z, 5)];
        const int gz = wz(z);
        for (int i = tid; i < YX * YY; i += NT) {
            const int gx = wx(x0 + i % YX - 3), gy = wy(y0 + i / YX - 3);
            dst[i] = g.type[gz * nxy + gy * nx + gx];
        }
    };
    auto type_at = [&](int z, int ti) -> uint8_t { return solid ? sm.type[ring(z, 5)][ti] : uint8_t(T_BULK); };

    // pull of node (gx, gy, gz) of plane z whose type-plane cell is ti
    auto pull = [&](C (&f)[Q], int gx, int gy, int gz, int z, int ti, uint8_t self) {
        const int cx[3] = {wrap1(gx - 1, nx), gx, wrap1(gx + 1, nx)};
        const int ry[3] = {wrap1(gy - 1, ny) * nx, gy * nx, wrap1(gy + 1, ny) * nx};
        const int pz[3] = {wrap1(gz - 1, nz) * nxy, gz * nxy, wrap1(gz + 1, nz) * nxy};
        const int gi = pz[1] + ry[1] + cx[1];
        if (self & T_BULK) {
#pragma unroll
            for (int a = 0; a < Q; ++a)
                f[a] = C(fin[a * N + pz[1 - L::ez(a)] + ry[1 - L::ey(a)] + cx[1 - L::ex(a)]]);
        } else {
            const uint8_t* tm = sm.type[ring(z - 1, 5)];
            const uint8_t* t0 = sm.type[ring(z, 5)];
            const uint8_t* tp = sm.type[ring(z + 1, 5)];
            // next to a solid: one load per direction, the bounce-back source chosen by address
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
                const uint8_t* tz = ez > 0 ? tm : (ez < 0 ? tp : t0);   // upstream plane is z - ez
                const bool bb = (tz[ti - ex - ey * YX] & T_SOLID) != 0;
                f[a] = C(fin[bb ? L::opp(a) * N + gi : a * N + pz[1 - ez] + ry[1 - ey] + cx[1 - ex]]);
            }
        }
    };
    // pull, density and (fluid) psi of a cell of plane z at xy halo coordinates (hx, hy) relative to
    // the 2-node density plane; returns the cell's type
    auto do_cell = [&](int z, int hx, int hy, bool keep_f, bool want_psi) -> uint8_t {
        const int gx = wx(x0 + hx - 2), gy = wy(y0 + hy - 2), gz = wz(z);
        const int ti = (hy + 1) * YX + hx + 1;
        const uint8_t t = type_at(z, ti);
        C rho = C(0), psi = C(0);
        if (!(t & T_SOLID)) {
            C h[Q];
            pull(h, gx, gy, gz, z, ti, t);
            C d = C(0);
#pragma unroll
            for (int a = 0; a < Q; ++a) d += h[a];
            rho = ph.rho_ref + d;
            if (want_psi) psi = psi_checked(rho, ph, err);
            if (keep_f) {
#pragma unroll
                for (int a = 0; a < Q; ++a) sm.f[ring(z, 3)][a][(hy - 2) * TX + hx - 2] = h[a];
            }
        } else if (want_psi && (t & T_WALL)) {
            sm.wq[ring(z, 2)][atomicAdd(&sm.nw[ring(z, 2)], 1)] = short((hy - 1) * PX + hx - 1);
        }
        sm.rho[ring(z, 3)][hy * RX + hx] = rho;
        if (want_psi) sm.psi[ring(z, 4)][(hy - 1) * PX + hx - 1] = psi;
        return t;
    };

    // prologue: type planes zb - 4 .. zb - 1, empty wall queue of the first lead plane
    for (int z = zb - 4; z <= zb - 1; ++z) load_types(z);
    if (tid == 0) sm.nw[ring(zb - 2, 2)] = 0;
    __syncthreads();

    for (int zl = zb - 2; zl <= ze + 1; ++zl) {
        // A. the lead plane: own node, 1-node xy halo shell, and the 2-node shell near solids
        const bool keep = zl >= zb && zl < ze;
        do_cell(zl, lx + 2, ly + 2, keep, true);
        using Shell1 = Shell<PX, PY, 1, 2>;
        for (int k = tid; k < Shell1::COUNT; k += NT) {
            int px, py, pz;
            Shell1::cell(k, px, py, pz);
            do_cell(zl, px + 1, py + 1, false, true);
        }
        if (solid) {
            using Shell2 = Shell<RX, RY, 1, 2>;
            for (int k = tid; k < Shell2::COUNT; k += NT) {
                int rx, ry, rz;
                Shell2::cell(k, rx, ry, rz);
                do_cell(zl, rx, ry, false, false);
            }
        }
        __syncthreads();

        // B. wall nodes of plane zl - 1
        const int zw = zl - 1;
        const int nwb = sm.nw[ring(zw, 2)];
        // (the solid-fluid interaction scheme keeps psi = 0 on solids)
        if (zw >= zb - 1 && zw <= ze && nwb > 0 && ph.wall_kind != 2) {
            const short* q = sm.wq[ring(zw, 2)];
            for (int k = tid; k < nwb; k += NT) {
                const int i = q[k];
                const int px = i % PX, py = i / PX;
                const int rc = (py + 1) * RX + px + 1, tc = (py + 2) * YX + px + 2;
                C rw;
                if (ph.wall_kind == 1) {
                    rw = ph.wall_param;
                } else {
                    C num = C(0), den = C(0);
#pragma unroll
                    for (int a = 1; a < Q; ++a) {
                        const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
                        if (!(sm.type[ring(zw + ez, 5)][tc + ex + ey * YX] & T_SOLID)) {
                            num += C(L::wf(a)) * sm.rho[ring(zw + ez, 3)][rc + ex + ey * RX];
                            den += C(L::wf(a));
                        }
                    }
                    const C rho_ave = cdiv(num, den);
                    C kap;
                    if (g.kappa_w) {
                        const int gx = wx(x0 + px - 1), gy = wy(y0 + py - 1), gz = wz(zw);
                        kap = C(g.kappa_w[g.wall_id[gz * nxy + gy * nx + gx]]);
                    } else {
                        kap = C(g.kappa);
                    }
                    rw = (kap >= C(0)) ? (C(1) + kap) * rho_ave : rho_ave + kap;
                    rw = rw > ph.rho_l ? ph.rho_l : rw;
                    rw = rw < ph.rho_g ? ph.rho_g : rw;
                }
                sm.psi[ring(zw, 4)][i] = psi_checked(rw, ph, err);
            }
            __syncthreads();
        }

        // C. collide plane zl - 2
        const int zc = zl - 2;
        if (zc >= zb && zc < ze && x0 + lx < nx && y0 + ly < ny) {
            const int gi = zc * nxy + (y0 + ly) * nx + x0 + lx;
            const uint8_t t = type_at(zc, (ly + 3) * YX + lx + 3);
            if (t & T_SOLID) {
                if (MODE == 1) {
                    if (rho_out) rho_out[gi] = 0.0;
                    if (u_out)
                        for (int c = 0; c < 3; ++c) u_out[c * N + gi] = 0.0;
                }
            } else {
                C f[Q];
#pragma unroll
                for (int a = 0; a < Q; ++a) f[a] = sm.f[ring(zc, 3)][a][ly * TX + lx];
                const int pc = (ly + 1) * PX + lx + 1;
                const C* p0 = sm.psi[ring(zc, 4)];
                const C psi_c = p0[pc];
                C sx = C(0), sy = C(0), sz = C(0);
#pragma unroll
                for (int a = 1; a < Q; ++a) {
                    if (L::opp(a) < a) continue;
                    const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
                    const C* pp = sm.psi[ring(zc + ez, 4)];
                    const C* pm = sm.psi[ring(zc - ez, 4)];
                    const int off = ex + ey * PX;
                    const C wd = C(L::wf(a)) * (pp[pc + off] - pm[pc - off]);
                    if (ex) sx += C(ex) * wd;
                    if (ey) sy += C(ey) * wd;
                    if (ez) sz += C(ez) * wd;
                }
                const C Fmx = -ph.G * psi_c * sx, Fmy = -ph.G * psi_c * sy, Fmz = -ph.G * psi_c * sz;
                C drho = C(0), jx = C(0), jy = C(0), jz = C(0);
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    drho += f[a];
                    if (L::ex(a)) jx += C(L::ex(a)) * f[a];
                    if (L::ey(a)) jy += C(L::ey(a)) * f[a];
                    if (L::ez(a)) jz += C(L::ez(a)) * f[a];
                }
                const C rho = ph.rho_ref + drho;
                C Fx = Fmx + ph.fx, Fy = Fmy + ph.fy, Fz = Fmz + ph.fz;
                // Eq. 8 (solid-fluid interaction scheme): F_ads = -G_w rho sum_a w_a s(x + e_a) e_a
                if (solid && ph.wall_kind == 2 && !(t & T_BULK)) {
                    const int tc = (ly + 3) * YX + lx + 3;
                    C ax = C(0), ay = C(0), az = C(0);
#pragma unroll
                    for (int a = 1; a < Q; ++a) {
                        const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
                        if (sm.type[ring(zc + ez, 5)][tc + ex + ey * YX] & T_SOLID) {
                            if (ex) ax += C(L::wf(a) * ex);
                            if (ey) ay += C(L::wf(a) * ey);
                            if (ez) az += C(L::wf(a) * ez);
                        }
                    }
                    const C gr = -ph.wall_param * rho;
                    Fx = (Fmx + gr * ax) + ph.fx;
                    Fy = (Fmy + gr * ay) + ph.fy;
                    Fz = (Fmz + gr * az) + ph.fz;
                }
                if (!(rho > C(0))) atomicOr(err, ERR_RHO);
                const C inv = cdiv(C(1), rho);
                const C ux = (jx + C(0.5) * Fx) * inv, uy = (jy + C(0.5) * Fy) * inv, uz = (jz + C(0.5) * Fz) * inv;
                if (MODE == 1) {
                    if (rho_out) rho_out[gi] = double(rho);
                    if (u_out) {
                        u_out[gi] = double(ux);
                        u_out[N + gi] = double(uy);
                        u_out[2 * N + gi] = double(uz);
                    }
                } else {
                    const C X = cdiv(Fmx * Fmx + Fmy * Fmy + Fmz * Fmz, psi_c * psi_c);
                    collide_d3q19<C>(f, drho, rho, ux, uy, uz, Fx, Fy, Fz, X, ph.r);
#pragma unroll
                    for (int a = 0; a < Q; ++a) fout[a * N + gi] = S(f[a]);
                }
            }
        }
        // prefetch the type plane the next lead plane's pulls need; empty its wall queue
        load_types(zl + 2);
        if (tid == 0) sm.nw[ring(zl + 1, 2)] = 0;
        __syncthreads();
    }
}

template <class S, int MODE>
cudaError_t launch_z(const void* fin, void* fout, const Geo& g, const DevParams& p, double* rho, double* u,
                     cudaStream_t s) {
    using Z = ZShape<S>;
    constexpr size_t bytes = sizeof(ZSmem<S, Z::X, Z::Y>);
    // the shared-memory limit is raised once per device (before any capture of this launch)
    static bool attr[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr[dev]) {
        cudaError_t e = cudaFuncSetAttribute(zmarch_step<S, S, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(bytes));
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    dim3 grid((p.nx + Z::X - 1) / Z::X, (p.ny + Z::Y - 1) / Z::Y, (p.nz + Z::Z - 1) / Z::Z);
    zmarch_step<S, S, MODE><<<grid, dim3(Z::X, Z::Y, 1), bytes, s>>>(
        static_cast<const S*>(fin), static_cast<S*>(fout), g, make_phys<S>(p), p.err, rho, u);
    return cudaGetLastError();
}

}  // namespace

void zmarch_tile_shape(int prec, int* tx, int* ty, int* tz) {
    if (prec == PREC_FP64) {
        *tx = ZShape<double>::X;
        *ty = ZShape<double>::Y;
        *tz = ZShape<double>::Z;
    } else {
        *tx = ZShape<float>::X;
        *ty = ZShape<float>::Y;
        *tz = ZShape<float>::Z;
    }
}

cudaError_t launch_step3d(int prec, int mode, const void* fin, void* fout, const Geo& g, const DevParams& p,
                          double* rho, double* u, cudaStream_t s) {
    if (prec == PREC_FP32 && mode == 0 && p.step3 == 0 && p.ztmap)
        return launch_ztma_step(fin, fout, static_cast<const char*>(p.ztmap) + (fin == p.zf0 ? 0 : 128), g, p, s);
    if (prec == PREC_FP32 && mode == 0 && p.step3 != 2) return launch_zpair_step(fin, fout, g, p, s);
    if (prec == PREC_FP64)
        return mode == 0 ? launch_z<double, 0>(fin, fout, g, p, rho, u, s) : launch_z<double, 1>(fin, fout, g, p, rho, u, s);
    return mode == 0 ? launch_z<float, 0>(fin, fout, g, p, rho, u, s) : launch_z<float, 1>(fin, fout, g, p, rho, u, s);
}

}  // namespace lbmwet
