// Fused time-step kernels of the pseudopotential MRT-LB method with improved virtual-density walls.
//
// One CTA owns a TX x TY (x TZ) tile of nodes, one thread per node.  The state in global memory is
// the post-collision f* of the previous step (structure of arrays, [a][node]); a step is
//   0. node-type flags of the tile + 3-node halo into shared memory;
//   1. pull-streaming (Eq. 3) with halfway bounce-back (Fig. 3) and the density (Eq. 4) of every
//      node of the tile + 1-node halo (the tile's own pulled f stay in registers), and psi (Eq. 6)
//      of its fluid nodes; wall nodes are queued; tiles that contain a wall node also pull their
//      2-node halo ring, whose densities Eq. 17 needs;
//   2. at the queued wall nodes: the virtual density of Eqs. 16-17 (improved scheme with limiter,
//      Sec. III.B) or the constant one (Sec. II.B), averaged from the shared-memory densities of
//      their fluid neighbours, and its psi;
//   3. at the tile's fluid nodes: F_m (Eq. 5) from shared psi, F = F_m + body force, u (Eq. 4), the
//      MRT collision with the consistency source (Eqs. 2, 7), and a coalesced store of f*.
// Neighbour values of the same time level come from the halo recomputation: nothing but f* is
// written to global memory per step.  The same tile body serves a single grid (tiles from the
// CUDA grid) and a batch of grids (a persistent grid walking a work list of (instance, tile)).
#include <cmath>

#include "adjoint.h"
#include "kernels.h"
#include "lattice.cuh"
#include "tile_common.cuh"

namespace lbmwet {

template <class L, class C, int TX, int TY, int TZ, bool ADJ = false>
struct TileSmem {
    static constexpr int D = L::D;
    static constexpr int HZ = (D == 3) ? 2 : 0, PZH = (D == 3) ? 1 : 0, YZH = (D == 3) ? 3 : 0;
    static constexpr int RX = TX + 4, RY = TY + 4, RZ = TZ + 2 * HZ;    // density tile (2-node halo)
    static constexpr int PX = TX + 2, PY = TY + 2, PZ = TZ + 2 * PZH;   // psi tile (1-node halo)
    static constexpr int YX = TX + 6, YY = TY + 6, YZ = TZ + 2 * YZH;   // type tile (3-node halo)
    uint8_t type[YZ * YY * YX];
    C rho[RZ * RY * RX];
    C psi[PZ * PY * PX];
    short wall[PZ * PY * PX];    // queued wall cells (psi-tile indices)
    int nwall;
    // adjoint mode: at wall cells d rho_w/d kappa, d rho_w/d rho_ave / den and d psi/d rho at rho_w
    C wdk[ADJ ? PZ * PY * PX : 1], wda[ADJ ? PZ * PY * PX : 1], wdpsi[ADJ ? PZ * PY * PX : 1];
};

// Outputs of the adjoint mode of the tile body (one value per node unless noted).
template <class C>
struct AdjIO {
    const C* mu;      // dL/df* of the step's output, [a][node]
    C* lam;           // dL/df through the collision, [a][node]
    C* fmb_x;         // dL/dF_m
    C* fmb_y;
    C* psib;          // dL/dpsi(x) through the node's own collision (X term and F_m's psi(x) factor)
    C* psi;           // psi (fluid) or psi(rho_w) (wall)
    C* dpsi;          // d psi/d rho at rho or rho_w
    C* drw_k;         // walls: d rho_w / d kappa (0 when the limiter clamps)
    C* drw_a;         // walls: d rho_w / d rho_ave / den
};

// d psi / d rho = (p'(rho) - 1/3) / (G psi), with p' from the equation of state
template <class C>
__device__ __forceinline__ C psi_slope(C rho, C psi, const Phys<C>& e) {
    C dp;
    if (e.eos_kind == 1) {
        const C eta = e.b4 * rho, om = C(1) - eta;
        const C om3 = om * om * om;
        const C Z = (C(1) + eta + eta * eta - eta * eta * eta) / om3;
        const C dZ = (C(4) + C(4) * eta - C(2) * eta * eta) / (om3 * om);
        dp = e.RT * (Z + eta * dZ) - C(2) * e.a * rho;
    } else {
        const C den = C(1) + C(2) * e.b * rho - e.b * e.b * rho * rho;
        const C dden = C(2) * e.b - C(2) * e.b * e.b * rho;
        const C om = C(1) - e.b * rho;
        dp = e.RT / (om * om) - e.aphi * (C(2) * rho * den - rho * rho * dden) / (den * den);
    }
    return psi > C(0) ? (dp - C(1.0 / 3.0)) / (e.G * psi) : C(0);
}

// One tile: x0, y0, z0 is its first node.  All threads of the CTA call this together.
// MODE 0: time step (writes f*); 1: fields (writes rho, u); 2: adjoint local part (writes AdjIO).
// SOLID = false compiles the body of a tile with no solid node within its box (every cell a bulk
// fluid node: no node-type staging, no bounce-back, no wall nodes).  WRAP 0 compiles a tile whose
// pulls touch no cell beyond the grid (no periodic wrapping: neighbours at constant offsets),
// 1 a tile that wraps once, 2 a grid narrower than a tile plus its halo (full modulo).
template <class L, class S, class C, int TX, int TY, int TZ, int MODE, bool SOLID = true, int WRAP = 2>
__device__ __forceinline__ void tile_body(const S* __restrict__ fin, S* __restrict__ fout, const Geo& g,
                                          const Phys<C>& ph, int x0, int y0, int z0, bool tile_solid_arg,
                                          unsigned* err, double* __restrict__ rho_out, double* __restrict__ u_out,
                                          TileSmem<L, C, TX, TY, TZ, MODE == 2>& sm, const AdjIO<C>* adj = nullptr) {
    using T = TileSmem<L, C, TX, TY, TZ, MODE == 2>;
    constexpr int D = L::D, Q = L::Q;
    const bool tile_solid = SOLID && tile_solid_arg;
    constexpr int NT = TX * TY * TZ;
    constexpr int RX = T::RX, RY = T::RY, RZ = T::RZ, PX = T::PX, PY = T::PY, PZ = T::PZ;
    constexpr int YX = T::YX, YY = T::YY, YZ = T::YZ, HZ = T::HZ, PZH = T::PZH, YZH = T::YZH;
    const int nx = g.nx, ny = g.ny, nz = g.nz, N = g.N;
    const int fp = g.fp, fs = g.fs;   // distribution row pitch and direction stride
    const int tid = threadIdx.x + TX * (threadIdx.y + TY * threadIdx.z);
    auto wrapc = [](int v, int n) { return WRAP == 0 ? v : (WRAP == 1 ? wrap1(v, n) : wrap_full(v, n)); };
    auto wx = [&](int v) { return wrapc(v, nx); };
    auto wy = [&](int v) { return wrapc(v, ny); };
    auto wz = [&](int v) { return (D == 3) ? wrapc(v, nz) : 0; };
    auto tix = [](int lx, int ly, int lz) { return (lz * YY + ly) * YX + lx; };
    auto rix = [](int lx, int ly, int lz) { return (lz * RY + ly) * RX + lx; };
    auto pix = [](int lx, int ly, int lz) { return (lz * PY + ly) * PX + lx; };

    // 0. node types of the tile + 3-node halo (skipped when no solid node lies within it: then
    //    every cell is a bulk fluid node); does the 1-node halo region hold a wall node?
    if (tid == 0) sm.nwall = 0;
    bool tile_has_wall = false;
    if constexpr (SOLID) {
        int wall_seen = 0;
        for (int i = tid; tile_solid && i < YX * YY * YZ; i += NT) {
            const int lx = i % YX, t = i / YX, ly = t % YY, lz = t / YY;
            const int gx = wx(x0 + lx - 3), gy = wy(y0 + ly - 3), gz = wz(z0 + lz - YZH);
            const uint8_t ty = g.type[(gz * ny + gy) * nx + gx];
            sm.type[i] = ty;
            const bool in_p = lx >= 2 && lx < TX + 4 && ly >= 2 && ly < TY + 4 &&
                              (D == 2 || (lz >= YZH - PZH && lz < TZ + YZH + PZH));
            if (in_p && (ty & T_WALL)) wall_seen = 1;
        }
        tile_has_wall = __syncthreads_or(wall_seen);
    }
    auto type_at = [&](int ti) -> uint8_t {
        if constexpr (!SOLID) return uint8_t(T_BULK);
        return tile_solid ? sm.type[ti] : uint8_t(T_BULK);
    };

    // pull of one node at global (gx, gy, gz) whose type-tile cell is ti
    auto pull = [&](C (&f)[Q], int gx, int gy, int gz, int ti, uint8_t self) {
        if constexpr (WRAP == 0) {
            // every upstream node at a constant offset from the node itself
            const int fpy = fp * ny;
            const S* p = fin + ((gz * ny + gy) * fp + gx);
            if (!SOLID || (self & T_BULK)) {
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
                    f[a] = C(p[a * fs - ex - ey * fp - ez * fpy]);
                }
            } else {
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
                    const bool bb = (sm.type[ti - ex - ey * YX - ez * YX * YY] & T_SOLID) != 0;
                    f[a] = C(p[bb ? L::opp(a) * fs : a * fs - ex - ey * fp - ez * fpy]);
                }
            }
            return;
        }
        const int xm = wrap1(gx - 1, nx), xp = wrap1(gx + 1, nx);
        const int ym = wrap1(gy - 1, ny), yp = wrap1(gy + 1, ny);
        const int cx[3] = {xm, gx, xp};
        const int ry[3] = {ym * fp, gy * fp, yp * fp};
        int pz[3];
        if (D == 3) {
            const int fpy = fp * ny;
            pz[0] = wrap1(gz - 1, nz) * fpy;
            pz[1] = gz * fpy;
            pz[2] = wrap1(gz + 1, nz) * fpy;
        } else {
            pz[0] = pz[1] = pz[2] = 0;
        }
        const int gi = pz[1] + ry[1] + cx[1];
        if (!SOLID || (self & T_BULK)) {
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
                f[a] = C(fin[a * fs + pz[1 - ez] + ry[1 - ey] + cx[1 - ex]]);
            }
        } else {
            // next to a solid: one load per direction, the bounce-back source chosen by address
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
                const bool bb = (sm.type[ti - ex - ey * YX - ez * YX * YY] & T_SOLID) != 0;
                f[a] = C(fin[bb ? L::opp(a) * fs + gi : a * fs + pz[1 - ez] + ry[1 - ey] + cx[1 - ex]]);
            }
        }
    };

    // 1a. the tile's own node
    const int lx = threadIdx.x, ly = threadIdx.y, lz = threadIdx.z;
    const int gx = wx(x0 + lx), gy = wy(y0 + ly), gz = wz(z0 + lz);
    const int gi = (gz * ny + gy) * nx + gx;   // node index (per-node arrays)
    const int fi = (gz * ny + gy) * fp + gx;   // distribution index
    const int my_ti = tix(lx + 3, ly + 3, lz + YZH);
    const uint8_t my_type = type_at(my_ti);
    const bool my_fluid = !(my_type & T_SOLID);
    C f[Q];
    C my_drho = C(0);
    {
        C rho = C(0);
        if (my_fluid) {
            pull(f, gx, gy, gz, my_ti, my_type);
            C drho = C(0);
#pragma unroll
            for (int a = 0; a < Q; ++a) drho += f[a];
            my_drho = drho;
            rho = ph.rho_ref + drho;
            sm.psi[pix(lx + 1, ly + 1, lz + PZH)] = psi_checked(rho, ph, err);
        } else {
#pragma unroll
            for (int a = 0; a < Q; ++a) f[a] = C(0);
            const int pi = pix(lx + 1, ly + 1, lz + PZH);
            sm.psi[pi] = C(0);
            if (my_type & T_WALL) sm.wall[atomicAdd(&sm.nwall, 1)] = short(pi);
        }
        sm.rho[rix(lx + 2, ly + 2, lz + HZ)] = rho;
    }
    // 1b. the 1-node halo ring: density and psi (fluid) or queue (wall)
    using ShellP = Shell<PX, PY, PZ, D>;
    for (int k = tid; k < ShellP::COUNT; k += NT) {
        int px, py, pz;
        ShellP::cell(k, px, py, pz);
        const int i = pix(px, py, pz);
        const int cgx = wx(x0 + px - 1), cgy = wy(y0 + py - 1), cgz = wz(z0 + pz - PZH);
        const int ti = tix(px + 2, py + 2, pz + (YZH - PZH));
        const uint8_t ty = type_at(ti);
        C rho = C(0), psi = C(0);
        if (!(ty & T_SOLID)) {
            C h[Q];
            pull(h, cgx, cgy, cgz, ti, ty);
            C drho = C(0);
#pragma unroll
            for (int a = 0; a < Q; ++a) drho += h[a];
            rho = ph.rho_ref + drho;
            psi = psi_checked(rho, ph, err);
        } else if (ty & T_WALL) {
            sm.wall[atomicAdd(&sm.nwall, 1)] = short(i);
        }
        sm.rho[rix(px + 1, py + 1, pz + (HZ - PZH))] = rho;
        sm.psi[i] = psi;
    }
    // 1c. the 2-node halo ring, only where Eq. 17 will need it
    if (SOLID && tile_has_wall) {
        using ShellR = Shell<RX, RY, RZ, D>;
        for (int k = tid; k < ShellR::COUNT; k += NT) {
            int rx, ry, rz;
            ShellR::cell(k, rx, ry, rz);
            const int cgx = wx(x0 + rx - 2), cgy = wy(y0 + ry - 2), cgz = wz(z0 + rz - HZ);
            const int ti = tix(rx + 1, ry + 1, rz + (YZH - HZ));
            const uint8_t ty = sm.type[ti];
            C rho = C(0);
            if (!(ty & T_SOLID)) {
                C h[Q];
                pull(h, cgx, cgy, cgz, ti, ty);
                C drho = C(0);
#pragma unroll
                for (int a = 0; a < Q; ++a) drho += h[a];
                rho = ph.rho_ref + drho;
            }
            sm.rho[rix(rx, ry, rz)] = rho;
        }
    }
    __syncthreads();

    // 2. wall nodes of the tile + 1-node halo: virtual density and its psi (the solid-fluid
    //    interaction scheme keeps psi = 0 on solids)
    const int nwall = SOLID ? sm.nwall : 0;
    if (SOLID && nwall > 0 && ph.wall_kind != 2) {
        for (int k = tid; k < nwall; k += NT) {
            const int i = sm.wall[k];
            const int px = i % PX, t = i / PX, py = t % PY, pz = t / PY;
            const int rx = px + 1, ry = py + 1, rz = pz + (HZ - PZH);
            const int ti = tix(px + 2, py + 2, pz + (YZH - PZH));
            C rw;
            if (ph.wall_kind == 1) {
                rw = ph.wall_param;
            } else {
                // Eq. 17: weighted mean of the fluid neighbours' densities
                C num = C(0), den = C(0);
#pragma unroll
                for (int a = 1; a < Q; ++a) {
                    const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
                    if (!(sm.type[ti + ex + ey * YX + ez * YX * YY] & T_SOLID)) {
                        num += C(L::wf(a)) * sm.rho[rix(rx + ex, ry + ey, rz + ez)];
                        den += C(L::wf(a));
                    }
                }
                const C rho_ave = cdiv(num, den);
                if (D == 2 && ph.wall_kind == 3) {
                    // geometric formulation (Eqs. 10-15): crossings of the characteristic lines
                    const int cgx = wx(x0 + px - 1), cgy = wy(y0 + py - 1);
                    const double* t = g.kappa_w + GF_STRIDE * g.wall_id[cgy * nx + cgx];
                    rw = gf_wall_density(t, rho_ave, [&](int dx, int dy) { return sm.rho[rix(rx + dx, ry + dy, rz)]; });
                } else {
                    C kap;
                    if (g.kappa_w) {
                        const int cgx = wx(x0 + px - 1), cgy = wy(y0 + py - 1), cgz = wz(z0 + pz - PZH);
                        kap = C(g.kappa_w[g.wall_id[(cgz * ny + cgy) * nx + cgx]]);
                    } else {
                        kap = C(g.kappa);
                    }
                    // Eq. 16 (kappa >= 0: phi = 1 + kappa; kappa < 0: drho = -kappa) and the limiter
                    const C raw = (kap >= C(0)) ? (C(1) + kap) * rho_ave : rho_ave + kap;
                    rw = raw > ph.rho_l ? ph.rho_l : raw;
                    rw = rw < ph.rho_g ? ph.rho_g : rw;
                    if constexpr (MODE == 2) {
                        const bool free = raw < ph.rho_l && raw > ph.rho_g;   // limiter inactive
                        sm.wdk[i] = free ? (kap >= C(0) ? rho_ave : C(1)) : C(0);
                        sm.wda[i] = free ? (kap >= C(0) ? C(1) + kap : C(1)) / den : C(0);
                    }
                }
            }
            if constexpr (MODE == 2) {
                if (ph.wall_kind != 0) sm.wdk[i] = sm.wda[i] = C(0);   // the adjoint covers IVD only
            }
            sm.psi[i] = psi_checked(rw, ph, err);
            if constexpr (MODE == 2) sm.wdpsi[i] = psi_slope(rw, sm.psi[i], ph);
        }
        __syncthreads();
    }

    // 3. force, velocity and collision of the tile's fluid node
    const bool valid = (x0 + lx < nx) && (y0 + ly < ny) && (D == 2 || z0 + lz < nz);
    if (!valid) return;
    const int pc = pix(lx + 1, ly + 1, lz + PZH);
    if (!my_fluid) {
        if (MODE == 1) {
            if (rho_out) rho_out[gi] = 0.0;
            if (u_out)
                for (int c = 0; c < D; ++c) u_out[c * N + gi] = 0.0;
        }
        if constexpr (MODE == 2) {
            const bool wall = (my_type & T_WALL) != 0;
            adj->psi[gi] = wall ? sm.psi[pc] : C(0);
            adj->dpsi[gi] = wall ? sm.wdpsi[pc] : C(0);
            adj->drw_k[gi] = wall ? sm.wdk[pc] : C(0);
            adj->drw_a[gi] = wall ? sm.wda[pc] : C(0);
            adj->fmb_x[gi] = C(0);
            adj->fmb_y[gi] = C(0);
            adj->psib[gi] = C(0);
        }
        return;
    }
    const C psi_c = sm.psi[pc];
    // sum_a w_a psi(x + e_a) e_a, taken over opposite pairs: w_a e_a (psi(x + e_a) - psi(x - e_a))
    // (nearly equal values cancel exactly in the difference, which keeps FP32 accurate in bulk)
    C sx = C(0), sy = C(0), sz = C(0);
#pragma unroll
    for (int a = 1; a < Q; ++a) {
        if (L::opp(a) < a) continue;
        const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
        const int off = ex + ey * PX + ez * PX * PY;
        const C wd = C(L::wf(a)) * (sm.psi[pc + off] - sm.psi[pc - off]);
        if (ex) sx += C(ex) * wd;
        if (ey) sy += C(ey) * wd;
        if (D == 3 && ez) sz += C(ez) * wd;
    }
    // Eq. 5
    const C Fmx = -ph.G * psi_c * sx, Fmy = -ph.G * psi_c * sy, Fmz = -ph.G * psi_c * sz;
    C Fx = Fmx + ph.fx, Fy = Fmy + ph.fy, Fz = Fmz + ph.fz;
    // Eq. 8 (solid-fluid interaction scheme): F_ads = -G_w rho sum_a w_a s(x + e_a) e_a
    if constexpr (SOLID) {
        if (tile_solid && ph.wall_kind == 2 && !(my_type & T_BULK)) {
            C ax = C(0), ay = C(0), az = C(0);
#pragma unroll
            for (int a = 1; a < Q; ++a) {
                const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
                if (sm.type[my_ti + ex + ey * YX + ez * YX * YY] & T_SOLID) {
                    if (ex) ax += C(L::wf(a) * ex);
                    if (ey) ay += C(L::wf(a) * ey);
                    if (D == 3 && ez) az += C(L::wf(a) * ez);
                }
            }
            const C gr = -ph.wall_param * (ph.rho_ref + my_drho);
            Fx = (Fmx + gr * ax) + ph.fx;
            Fy = (Fmy + gr * ay) + ph.fy;
            Fz = (Fmz + gr * az) + ph.fz;
        }
    }
    const C drho = my_drho;   // sum of f in the order of the pull's density
    C jx = C(0), jy = C(0), jz = C(0);
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        if (L::ex(a)) jx += C(L::ex(a)) * f[a];
        if (L::ey(a)) jy += C(L::ey(a)) * f[a];
        if (D == 3 && L::ez(a)) jz += C(L::ez(a)) * f[a];
    }
    const C rho = ph.rho_ref + drho;
    if (!(rho > C(0))) atomicOr(err, ERR_RHO);
    // Eq. 4: rho u = sum e f + F/2
    const C inv = cdiv(C(1), rho);
    const C ux = (jx + C(0.5) * Fx) * inv, uy = (jy + C(0.5) * Fy) * inv, uz = (jz + C(0.5) * Fz) * inv;
    if (MODE == 1) {
        if (rho_out) rho_out[gi] = double(rho);
        if (u_out) {
            u_out[gi] = double(ux);
            u_out[N + gi] = double(uy);
            if (D == 3) u_out[2 * N + gi] = double(uz);
        }
        return;
    }
    if constexpr (MODE == 2) {
        if constexpr (D == 2) {
            C m[Q], fb[Q];
#pragma unroll
            for (int a = 0; a < Q; ++a) m[a] = adj->mu[a * N + gi];
            C bx, by, pb;
            collide_d2q9_adjoint<C>(f, m, rho, ux, uy, Fx, Fy, Fmx, Fmy, psi_c, ph.r, fb, bx, by, pb);
#pragma unroll
            for (int a = 0; a < Q; ++a) adj->lam[a * N + gi] = fb[a];
            adj->fmb_x[gi] = bx;
            adj->fmb_y[gi] = by;
            // F_m = -G psi(x) sum w psi(x+e) e: its dependence on psi(x) is F_m / psi(x)
            adj->psib[gi] = pb + (bx * Fmx + by * Fmy) / psi_c;
            adj->psi[gi] = psi_c;
            adj->dpsi[gi] = psi_slope(rho, psi_c, ph);
            adj->drw_k[gi] = C(0);
            adj->drw_a[gi] = C(0);
        }
        return;
    }
    const C X = cdiv(Fmx * Fmx + Fmy * Fmy + Fmz * Fmz, psi_c * psi_c);
    if constexpr (D == 2) {
        collide_d2q9<C>(f, drho, rho, ux, uy, Fx, Fy, X, ph.r);
    } else {
        collide_d3q19<C>(f, drho, rho, ux, uy, uz, Fx, Fy, Fz, X, ph.r);
    }
#pragma unroll
    for (int a = 0; a < Q; ++a) fout[a * fs + fi] = S(f[a]);
}

// Tile shapes per lattice and precision (one thread per node).
template <class L, class S>
struct TileShape;
#ifndef LBMWET_T2F_X   // tile of the FP32 D2Q9 kernels (compile-time; chosen by measurement)
#define LBMWET_T2F_X 32
#define LBMWET_T2F_Y 8
#define LBMWET_T2F_MINB 4
#endif
template <> struct TileShape<D2Q9, float> {
    static constexpr int X = LBMWET_T2F_X, Y = LBMWET_T2F_Y, Z = 1, MINB = LBMWET_T2F_MINB;
};
template <> struct TileShape<D2Q9, double> { static constexpr int X = 32, Y = 8, Z = 1, MINB = 2; };

// Wrap mode of a tile (the WRAP parameter of tile_body): 0 when every cell its pulls touch (the
// tile + 3 cells on each side) lies inside the grid, 2 for grids narrower than a tile plus its
// halo, else 1.
template <int D, int TX, int TY, int TZ>
__device__ __forceinline__ int tile_wrap(int x0, int y0, int z0, int nx, int ny, int nz) {
    if (nx < TX + 8 || ny < TY + 8 || (D == 3 && nz < TZ + 8)) return 2;
    const bool inside = x0 >= 3 && x0 + TX + 2 < nx && y0 >= 3 && y0 + TY + 2 < ny &&
                        (D == 2 || (z0 >= 3 && z0 + TZ + 2 < nz));
    return inside ? 0 : 1;
}

// tile_body with the wrap mode chosen at run time (uniform per CTA)
template <class L, class S, class C, int TX, int TY, int TZ, int MODE, bool SOLID>
__device__ __forceinline__ void tile_body_w(const S* __restrict__ fin, S* __restrict__ fout, const Geo& g,
                                            const Phys<C>& ph, int x0, int y0, int z0, bool tile_solid_arg,
                                            unsigned* err, double* __restrict__ rho_out, double* __restrict__ u_out,
                                            TileSmem<L, C, TX, TY, TZ, MODE == 2>& sm, const AdjIO<C>* adj = nullptr) {
    const int w = tile_wrap<L::D, TX, TY, TZ>(x0, y0, z0, g.nx, g.ny, g.nz);
    if (w == 0)
        tile_body<L, S, C, TX, TY, TZ, MODE, SOLID, 0>(fin, fout, g, ph, x0, y0, z0, tile_solid_arg, err, rho_out,
                                                       u_out, sm, adj);
    else if (w == 1)
        tile_body<L, S, C, TX, TY, TZ, MODE, SOLID, 1>(fin, fout, g, ph, x0, y0, z0, tile_solid_arg, err, rho_out,
                                                       u_out, sm, adj);
    else
        tile_body<L, S, C, TX, TY, TZ, MODE, SOLID, 2>(fin, fout, g, ph, x0, y0, z0, tile_solid_arg, err, rho_out,
                                                       u_out, sm, adj);
}


template <class L, class S, class C, int MODE>
__global__ void __launch_bounds__(TileShape<L, S>::X* TileShape<L, S>::Y* TileShape<L, S>::Z, TileShape<L, S>::MINB)
    fused_step(const S* __restrict__ fin, S* __restrict__ fout, Geo g, Phys<C> ph, unsigned* err,
               double* __restrict__ rho_out, double* __restrict__ u_out) {
    using TS = TileShape<L, S>;
    __shared__ TileSmem<L, C, TS::X, TS::Y, TS::Z> sm;
    const int tile = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const bool solid = g.tile_solid ? g.tile_solid[tile] != 0 : true;
    if (solid)
        tile_body_w<L, S, C, TS::X, TS::Y, TS::Z, MODE, true>(fin, fout, g, ph, blockIdx.x * TS::X, blockIdx.y * TS::Y,
                                                              blockIdx.z * TS::Z, true, err, rho_out, u_out, sm);
    else
        tile_body_w<L, S, C, TS::X, TS::Y, TS::Z, MODE, false>(fin, fout, g, ph, blockIdx.x * TS::X,
                                                               blockIdx.y * TS::Y, blockIdx.z * TS::Z, false, err,
                                                               rho_out, u_out, sm);
}

// Adjoint local part (D2Q9): the forward tile machinery recomputes rho, psi and rho_w of the state
// pulled from f*_k, then each node writes the reverse of its collision and its psi data.
template <class S>
__global__ void __launch_bounds__(TileShape<D2Q9, S>::X* TileShape<D2Q9, S>::Y, TileShape<D2Q9, S>::MINB)
    adjoint_local_tile(const S* __restrict__ fin, Geo g, Phys<S> ph, unsigned* err, AdjIO<S> io) {
    using TS = TileShape<D2Q9, S>;
    __shared__ TileSmem<D2Q9, S, TS::X, TS::Y, 1, true> sm;
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    const bool solid = g.tile_solid ? g.tile_solid[tile] != 0 : true;
    tile_body_w<D2Q9, S, S, TS::X, TS::Y, 1, 2, true>(fin, nullptr, g, ph, blockIdx.x * TS::X, blockIdx.y * TS::Y, 0,
                                                       solid, err, nullptr, nullptr, sm, &io);
}

// Batched step: CTAs walk the work list; each item is one tile of one instance.  The next item's
// record is fetched into registers by the first lanes while the current tile runs and handed over
// through shared memory at the end of the iteration.
template <class L, class S, class C>
__global__ void __launch_bounds__(TileShape<L, S>::X* TileShape<L, S>::Y* TileShape<L, S>::Z, TileShape<L, S>::MINB)
    fused_step_batched(int parity, const BatchInstance* __restrict__ insts, const BatchItem* __restrict__ items,
                       int n_items, Phys<C> ph, unsigned* err) {
    (void)insts;
    using TS = TileShape<L, S>;
    constexpr int WORDS = int(sizeof(BatchItem) / 4);
    __shared__ TileSmem<L, C, TS::X, TS::Y, TS::Z> sm;
    __shared__ BatchItem s_item[2];
    const int tid = threadIdx.x + TS::X * (threadIdx.y + TS::Y * threadIdx.z);
    if (tid < WORDS && blockIdx.x < n_items)
        reinterpret_cast<uint32_t*>(&s_item[0])[tid] = reinterpret_cast<const uint32_t*>(&items[blockIdx.x])[tid];
    __syncthreads();
    int slot = 0;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const BatchItem& item = s_item[slot];
        const int next = it + gridDim.x;
        uint32_t w = 0;
        const bool fetch = tid < WORDS && next < n_items;
        if (fetch) w = reinterpret_cast<const uint32_t*>(&items[next])[tid];
        Geo g;
        g.nx = item.nx;
        g.ny = item.ny;
        g.nz = 1;
        g.N = item.N;
        g.fp = item.fp;
        g.fs = item.fs;
        g.type = item.type;
        g.tile_solid = nullptr;
        g.wall_id = item.wall_id;
        g.kappa_w = item.kappa_w;
        g.kappa = item.kappa;
        const S* fin = static_cast<const S*>(item.f[parity]);
        S* fout = static_cast<S*>(const_cast<void*>(item.f[parity ^ 1]));
        if (item.solid)
            tile_body_w<L, S, C, TS::X, TS::Y, TS::Z, 0, true>(fin, fout, g, ph, item.x0, item.y0, 0, true, err,
                                                               nullptr, nullptr, sm);
        else
            tile_body_w<L, S, C, TS::X, TS::Y, TS::Z, 0, false>(fin, fout, g, ph, item.x0, item.y0, 0, false, err,
                                                                nullptr, nullptr, sm);
        if (fetch) reinterpret_cast<uint32_t*>(&s_item[slot ^ 1])[tid] = w;
        __syncthreads();   // the next record is visible, and this tile's threads are done with shared memory
        slot ^= 1;
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

// (32-bit division: a grid holds fewer than 2^31 / 19 nodes, checked at initialisation)
__device__ __forceinline__ void coords(long long g, int nx, int ny, int& x, int& y, int& z) {
    const unsigned u = unsigned(g), t = u / unsigned(nx);
    x = int(u - t * unsigned(nx));
    y = int(t % unsigned(ny));
    z = int(t / unsigned(ny));
}

// Stored f* whose pull gives f_post: f*_b(y) = f_post_b(y + e_b) if y + e_b is fluid, else
// f_post_bbar(y) (the inverse of the pull with bounce-back).  Source is either f^eq(rho0, u0) or
// explicit post-streaming values.
template <class L>
constexpr bool opposite_weights_equal() {
    for (int a = 0; a < L::Q; ++a)
        if (L::w(a) != L::w(L::opp(a))) return false;
    return true;
}
static_assert(opposite_weights_equal<D2Q9>() && opposite_weights_equal<D3Q19>(),
              "the initial state takes w_b for the weight of the opposite direction");

template <class L, class S, bool FROM_FEQ>
__global__ void unstream_kernel(S* __restrict__ fout, DevParams p, const double* __restrict__ src0,
                                const double* __restrict__ src1) {
    constexpr int Q = L::Q;
    const long long N = p.N, fs = p.fs;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords(g, p.nx, p.ny, x, y, z);
        const long long fg = ((long long)z * p.ny + y) * p.fp + x;   // distribution index of node g
        if (p.type[g] & T_SOLID) {
            for (int b = 0; b < Q; ++b) fout[b * fs + fg] = S(0);
            continue;
        }
        // (unrolled: every lattice constant is a compile-time value; a runtime-indexed weight table
        // would sit in local memory)
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            const int tx = wrap1(x + L::ex(b), p.nx), ty = wrap1(y + L::ey(b), p.ny);
            const int tz = (L::D == 3) ? wrap1(z + L::ez(b), p.nz) : 0;
            const long long t = ((long long)tz * p.ny + ty) * p.nx + tx;
            const bool bounce = (p.type[t] & T_SOLID) != 0;
            const long long src = bounce ? g : t;
            double v;
            if (FROM_FEQ && src1 == nullptr) {
                // u0 = 0: every velocity term of the bracket is an exact zero, so this is feq_a's
                // value bit for bit (w of the opposite direction equals w_b); the product is rounded
                // on its own, as feq_a's is, so that it is not fused with the subtraction below
                v = __dmul_rn(L::w(b), src0[src]);
            } else if (FROM_FEQ) {
                const double* rho0 = src0;
                const double* u0 = src1;
                const double ux = u0[src], uy = u0[N + src];
                const double uz = L::D == 3 ? u0[2 * N + src] : 0.0;
                v = bounce ? feq_a<L>(L::opp(b), rho0[src], ux, uy, uz) : feq_a<L>(b, rho0[src], ux, uy, uz);
            } else {
                v = src0[(long long)(bounce ? L::opp(b) : b) * N + src];
            }
            fout[b * fs + fg] = S(v - L::w(b) * p.rho_ref);
        }
    }
}

template <class L, class S>
__global__ void get_state_kernel(const S* __restrict__ fin, DevParams p, double* __restrict__ fpost) {
    constexpr int Q = L::Q;
    const long long N = p.N, fs = p.fs;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
        if (p.type[g] & T_SOLID) {
            for (int a = 0; a < Q; ++a) fpost[(long long)a * N + g] = 0.0;
            continue;
        }
        int x, y, z;
        coords(g, p.nx, p.ny, x, y, z);
        const long long fg = ((long long)z * p.ny + y) * p.fp + x;
        for (int a = 0; a < Q; ++a) {
            const int sx = wrap1(x - L::ex(a), p.nx), sy = wrap1(y - L::ey(a), p.ny);
            const int sz = (L::D == 3) ? wrap1(z - L::ez(a), p.nz) : 0;
            const long long s = ((long long)sz * p.ny + sy) * p.nx + sx;
            const long long fsrc = ((long long)sz * p.ny + sy) * p.fp + sx;
            double v;
            if (p.type[s] & T_SOLID) v = double(fin[L::opp(a) * fs + fg]);
            else v = double(fin[a * fs + fsrc]);
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
        // within Euclidean distance 3 of a solid node (wrapped offsets computed once per axis)
        bool near = false;
        const int rz = (L::D == 3) ? 3 : 0;
        int wx[7], wy[7], wz[7];
#pragma unroll
        for (int d = 0; d < 7; ++d) {
            wx[d] = wrap_full(x + d - 3, nx);
            wy[d] = wrap_full(y + d - 3, ny);
            wz[d] = (L::D == 3) ? wrap_full(z + d - 3, nz) : 0;
        }
        for (int dz = -rz; dz <= rz && !near; ++dz)
            for (int dy = -3; dy <= 3 && !near; ++dy) {
                const uint8_t* row = mask + ((long long)wz[dz + 3] * ny + wy[dy + 3]) * nx;
                for (int dx = -3; dx <= 3 && !near; ++dx) {
                    if (dx * dx + dy * dy + dz * dz > 9) continue;
                    if (row[wx[dx + 3]]) near = true;
                }
            }
        if (near) t |= T_NEARWALL;
        if (!solid) {
            bool bulk = true;
            for (int a = 1; a < L::Q; ++a) {
                const int sx = wrap1(x + L::ex(a), nx), sy = wrap1(y + L::ey(a), ny);
                const int sz = (L::D == 3) ? wrap1(z + L::ez(a), nz) : 0;
                if (mask[((long long)sz * ny + sy) * nx + sx]) bulk = false;
            }
            if (bulk) t |= T_BULK;
        }
        type[g] = t;
    }
}

// ---------------------------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------------------------

static Geo geo_of(const DevParams& p) {
    Geo g;
    g.nx = p.nx;
    g.ny = p.ny;
    g.nz = p.nz;
    g.N = int(p.N);
    g.fp = p.fp;
    g.fs = int(p.fs);
    g.type = p.type;
    g.tile_solid = p.tile_solid;
    g.wall_id = p.wall_id;
    g.kappa_w = p.kappa_w;
    g.kappa = p.kappa;
    return g;
}

template <class L, class S, int MODE>
static cudaError_t launch_tile(const void* fin, void* fout, const DevParams& p, double* rho, double* u, cudaStream_t s) {
    using TS = TileShape<L, S>;
    dim3 grid((p.nx + TS::X - 1) / TS::X, (p.ny + TS::Y - 1) / TS::Y, (p.nz + TS::Z - 1) / TS::Z);
    dim3 block(TS::X, TS::Y, TS::Z);
    fused_step<L, S, S, MODE><<<grid, block, 0, s>>>(static_cast<const S*>(fin), static_cast<S*>(fout), geo_of(p),
                                                     make_phys<S>(p), p.err, rho, u);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t dispatch(int lat, int prec, const void* fin, void* fout, const DevParams& p, double* rho, double* u,
                            cudaStream_t s) {
    if (lat == LAT_D2Q9) {
        if (prec == PREC_FP64) return launch_tile<D2Q9, double, MODE>(fin, fout, p, rho, u, s);
        return launch_tile<D2Q9, float, MODE>(fin, fout, p, rho, u, s);
    }
    return launch_step3d(prec, MODE, fin, fout, geo_of(p), p, rho, u, s);
}

cudaError_t launch_step(int lat, int prec, const void* fin, void* fout, const DevParams& p, cudaStream_t s) {
    if (lat == LAT_D2Q9 && prec == PREC_FP32 && p.pair_solid) return launch_pair_step(fin, fout, p, s);
    return dispatch<0>(lat, prec, fin, fout, p, nullptr, nullptr, s);
}

cudaError_t launch_fields(int lat, int prec, const void* fin, const DevParams& p, double* rho, double* u,
                          cudaStream_t s) {
    return dispatch<1>(lat, prec, fin, nullptr, p, rho, u, s);
}

template <class L, class S>
static cudaError_t batched_l(int parity, const DevParams& p, const BatchInstance* insts, const BatchItem* items,
                             int n_items, int ctas, cudaStream_t s) {
    using TS = TileShape<L, S>;
    dim3 block(TS::X, TS::Y, TS::Z);
    fused_step_batched<L, S, S><<<ctas, block, 0, s>>>(parity, insts, items, n_items, make_phys<S>(p), p.err);
    return cudaGetLastError();
}

cudaError_t launch_step_batched(int lat, int prec, int parity, const DevParams& p, const BatchInstance* insts,
                                const BatchItem* items, int n_items, int ctas, cudaStream_t s) {
    if (lat == LAT_D2Q9) {
        if (prec == PREC_FP64) return batched_l<D2Q9, double>(parity, p, insts, items, n_items, ctas, s);
        return batched_l<D2Q9, float>(parity, p, insts, items, n_items, ctas, s);
    }
    return cudaErrorInvalidValue;   // batches are D2Q9
}

template <class S>
static cudaError_t adj_local_t(const void* fstar, const DevParams& p, const AdjointFields& w, cudaStream_t s) {
    using TS = TileShape<D2Q9, S>;
    AdjIO<S> io;
    io.mu = static_cast<const S*>(w.mu);
    io.lam = static_cast<S*>(w.lam);
    io.fmb_x = static_cast<S*>(w.fmb_x);
    io.fmb_y = static_cast<S*>(w.fmb_y);
    io.psib = static_cast<S*>(w.psib);
    io.psi = static_cast<S*>(w.psi);
    io.dpsi = static_cast<S*>(w.dpsi);
    io.drw_k = static_cast<S*>(w.drw_k);
    io.drw_a = static_cast<S*>(w.drw_a);
    dim3 grid((p.nx + TS::X - 1) / TS::X, (p.ny + TS::Y - 1) / TS::Y, 1);
    adjoint_local_tile<S><<<grid, dim3(TS::X, TS::Y, 1), 0, s>>>(static_cast<const S*>(fstar), geo_of(p),
                                                                  make_phys<S>(p), p.err, io);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_local(int prec, const void* fstar, const DevParams& p, const AdjointFields& w,
                                 cudaStream_t s) {
    return prec == PREC_FP64 ? adj_local_t<double>(fstar, p, w, s) : adj_local_t<float>(fstar, p, w, s);
}

void step_tile_shape(int lat, int prec, int* tx, int* ty, int* tz) {
    if (lat == LAT_D2Q9) {
        if (prec == PREC_FP64) { *tx = TileShape<D2Q9, double>::X; *ty = TileShape<D2Q9, double>::Y; *tz = 1; }
        else { *tx = TileShape<D2Q9, float>::X; *ty = TileShape<D2Q9, float>::Y; *tz = 1; }
    } else {
        zmarch_tile_shape(prec, tx, ty, tz);
    }
}

template <class L, class S>
static int occ() {
    using TS = TileShape<L, S>;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_step_batched<L, S, S>, TS::X * TS::Y * TS::Z, 0) !=
        cudaSuccess)
        n = 1;
    return n < 1 ? 1 : n;
}

int batched_ctas_per_sm(int lat, int prec) {
    (void)lat;
    return prec == PREC_FP64 ? occ<D2Q9, double>() : occ<D2Q9, float>();
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

// wall_id[idx[i]] = i for the nw wall nodes (every other entry was set to -1 before)
__global__ void wall_id_scatter(const int* __restrict__ idx, int nw, int* __restrict__ wall_id) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += gridDim.x * blockDim.x) wall_id[idx[i]] = i;
}

cudaError_t launch_wall_ids(const int* idx, int nw, int* wall_id, long long N, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(wall_id, 0xFF, sizeof(int) * (size_t)N, s);   // -1 everywhere
    if (e != cudaSuccess || nw == 0) return e;
    wall_id_scatter<<<grid_for(nw), 256, 0, s>>>(idx, nw, wall_id);
    return cudaGetLastError();
}

cudaError_t launch_classify(int lat, const uint8_t* mask, uint8_t* type, int nx, int ny, int nz, cudaStream_t s) {
    const unsigned g = grid_for((long long)nx * ny * nz);
    if (lat == LAT_D2Q9) classify_kernel<D2Q9><<<g, 256, 0, s>>>(mask, type, nx, ny, nz);
    else classify_kernel<D3Q19><<<g, 256, 0, s>>>(mask, type, nx, ny, nz);
    return cudaGetLastError();
}

}  // namespace lbmwet
