// D2Q9 time step as a y-march.  A CTA of TW threads owns a block of TW - 4 columns and walks a run
// of rows [y0, y1) of one grid; lane hx holds the cell at x = x0 + hx - 2 of every row, so each
// row is TW cells: the block's own columns plus a 2-cell x halo on either side.  For lead row yl
// the CTA
//   A. finishes the pull (Eq. 3 with halfway bounce-back, Fig. 3) of row yl, whose distributions
//      were copied into the lane's private shared-memory slot one or two rows earlier
//      (cp.async), and stores rho (Eq. 4) and psi (Eq. 6) of its fluid cells;
//   B. gives the wall cells of row yl - 1 their virtual density (Eqs. 16-17 with the limiter, or
//      the constant one) from the densities of rows yl - 2 .. yl, and its psi;
//   C. collides row yl - LAG: F_m (Eq. 5) from psi of the rows around it, u (Eq. 4), the MRT
//      collision with the consistency source (Eqs. 2, 7), and a coalesced store of f*.
// A run whose box (plus a 3-cell halo) holds no solid node skips the node types, B and the second
// halo row (LAG = 1, pulls two rows ahead); otherwise LAG = 2 and pulls run one row ahead.
// Each node is pulled once, plus 4 halo cells per row of TW - 4 nodes and LAG halo rows at each
// end of a run.  Rings (power-of-two, indexed by the absolute row): f 4 rows, rho 4, psi 8,
// node types 8.  Persistent CTAs walk a host-planned list of runs (the planner balances the rows
// per CTA).
#include <cmath>

#include "kernels.h"
#include "lattice.cuh"
#include "tile_common.cuh"

namespace lbmwet {

namespace {

template <class S>
struct YShape;
#ifndef LBMWET_Y2F_TW   // threads (cells per row) and resident CTAs per SM of the FP32 y-march
#define LBMWET_Y2F_TW 128
#define LBMWET_Y2F_MINB 8
#endif
template <> struct YShape<float> { static constexpr int TW = LBMWET_Y2F_TW, MINB = LBMWET_Y2F_MINB; };
template <> struct YShape<double> { static constexpr int TW = 128, MINB = 4; };

template <class C, int TW>
struct YSmem {
    C f[4][9][TW];            // lane-private: pulled distributions of the lane's cell, by row
    C rho[4][TW];
    C psi[8][TW];
    uint8_t type[8][TW + 8];  // cell hx at index hx + 1 (x = x0 + index - 3)
};

// One run: columns x0 .. x0 + TW - 5 (those below nx), rows yb .. ye - 1.
template <class S, bool SOLID>
__device__ __forceinline__ void ymarch_run(const S* __restrict__ fin, S* __restrict__ fout, const Geo& g,
                                           const Phys<S>& ph, int x0, int yb, int ye, unsigned* err,
                                           YSmem<S, YShape<S>::TW>& sm) {
    using L = D2Q9;
    using C = S;
    constexpr int Q = 9, TW = YShape<S>::TW;
    constexpr int LAG = SOLID ? 2 : 1;      // rows between pull and collision
    constexpr int AHEAD = SOLID ? 1 : 2;    // rows of pulls in flight
    const int nx = g.nx, ny = g.ny;
    const int fp = g.fp, fs = g.fs;   // distribution row pitch and direction stride
    const int hx = threadIdx.x, ti = hx + 1;
    const bool small = nx < TW + 8 || ny < 8;
    auto wx = [&](int v) { return small ? wrap_full(v, nx) : wrap1(v, nx); };
    auto wy = [&](int v) { return small ? wrap_full(v, ny) : wrap1(v, ny); };
    const int gx = wx(x0 + hx - 2);
    const int col[3] = {wrap1(gx - 1, nx), gx, wrap1(gx + 1, nx)};   // columns x - 1, x, x + 1
    const bool own = hx >= 2 && hx < TW - 2 && x0 + hx - 2 < nx;
    const bool inner = hx >= 1 && hx < TW - 1;   // cells whose psi is used
    const bool active = SOLID || inner;           // cells pulled (the outer halo only feeds Eq. 17)

    auto load_types = [&](int y) {
        if constexpr (SOLID) {
            uint8_t* dst = sm.type[y & 7];
            const int row = wy(y) * nx;
            for (int i = hx; i < TW + 2; i += TW) dst[i] = g.type[row + wx(x0 + i - 3)];
        }
    };
    // copy the distributions that stream into the lane's cell of row y into its slot
    auto issue = [&](int y) {
        if (active) {
            const int gy = wy(y);
            const int r[3] = {wrap1(gy - 1, ny) * fp, gy * fp, wrap1(gy + 1, ny) * fp};
            S* dst = &sm.f[y & 3][0][hx];
            uint8_t self = uint8_t(T_BULK);
            if constexpr (SOLID) self = sm.type[y & 7][ti];
            if (!SOLID || (self & T_BULK)) {
#pragma unroll
                for (int a = 0; a < Q; ++a) cp_async(dst + a * TW, fin + a * fs + r[1 - L::ey(a)] + col[1 - L::ex(a)]);
            } else if (!(self & T_SOLID)) {
                // next to a solid: a link whose upstream node is solid brings back the cell's own
                // outgoing population (halfway bounce-back)
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    const int ex = L::ex(a), ey = L::ey(a);
                    const bool bb = (sm.type[(y - ey) & 7][ti - ex] & T_SOLID) != 0;
                    cp_async(dst + a * TW, fin + (bb ? L::opp(a) * fs + r[1] + gx : a * fs + r[1 - ey] + col[1 - ex]));
                }
            }
        }
        cp_commit();
    };

    const int ys = yb - LAG, ylast = ye + LAG - 1;   // lead rows
    load_types(yb - 3);
    load_types(yb - 2);
    load_types(yb - 1);
    load_types(yb);
    __syncthreads();
    issue(ys);
    if (AHEAD == 2) issue(ys + 1);
    int walls_prev = 0;   // row yl - 1 has wall cells in lanes 1 .. TW - 2
    for (int yl = ys; yl <= ylast; ++yl) {
        // A. density and psi of row yl
        cp_wait<AHEAD - 1>();
        uint8_t t = uint8_t(T_BULK);
        if constexpr (SOLID) t = sm.type[yl & 7][ti];
        if (active && !(t & T_SOLID)) {
            const S* fr = &sm.f[yl & 3][0][hx];
            C drho = C(0);
#pragma unroll
            for (int a = 0; a < Q; ++a) drho += C(fr[a * TW]);
            const C rho = ph.rho_ref + drho;
            if constexpr (SOLID) sm.rho[yl & 3][hx] = rho;
            sm.psi[yl & 7][hx] = psi_checked(rho, ph, err);
        } else if (active) {
            sm.psi[yl & 7][hx] = C(0);   // a solid cell: wall cells get their psi in phase B (not with SF)
        }
        int walls_now = 0;
        if constexpr (SOLID) {
            walls_now = __syncthreads_or(inner && (t & T_WALL) && yl >= yb - 1 && yl <= ye);
        } else {
            __syncthreads();
        }
        if (yl + AHEAD <= ylast) issue(yl + AHEAD);
        else cp_commit();

        // B. wall cells of row yl - 1
        if constexpr (SOLID) {
            if (walls_prev) {
                const int yw = yl - 1;
                // (the solid-fluid interaction scheme keeps psi = 0 on solids)
                if (inner && ph.wall_kind != 2 && (sm.type[yw & 7][ti] & T_WALL)) {
                    C rw;
                    if (ph.wall_kind == 1) {
                        rw = ph.wall_param;
                    } else {
                        // Eq. 17: weighted mean of the fluid neighbours' densities
                        C num = C(0), den = C(0);
#pragma unroll
                        for (int a = 1; a < Q; ++a) {
                            const int ex = L::ex(a), ey = L::ey(a);
                            if (!(sm.type[(yw + ey) & 7][ti + ex] & T_SOLID)) {
                                num += C(L::wf(a)) * sm.rho[(yw + ey) & 3][hx + ex];
                                den += C(L::wf(a));
                            }
                        }
                        const C rho_ave = cdiv(num, den);
                        if (ph.wall_kind == 3) {
                            // geometric formulation (Eqs. 10-15): crossings of the characteristic lines
                            const double* t = g.kappa_w + GF_STRIDE * g.wall_id[wy(yw) * nx + gx];
                            rw = gf_wall_density(t, rho_ave,
                                                 [&](int dx, int dy) { return sm.rho[(yw + dy) & 3][hx + dx]; });
                        } else {
                            const C kap = g.kappa_w ? C(g.kappa_w[g.wall_id[wy(yw) * nx + gx]]) : C(g.kappa);
                            // Eq. 16 (kappa >= 0: phi = 1 + kappa; kappa < 0: drho = -kappa) and the limiter
                            const C raw = (kap >= C(0)) ? (C(1) + kap) * rho_ave : rho_ave + kap;
                            rw = raw > ph.rho_l ? ph.rho_l : raw;
                            rw = rw < ph.rho_g ? ph.rho_g : rw;
                        }
                    }
                    sm.psi[yw & 7][hx] = psi_checked(rw, ph, err);
                }
                __syncthreads();
            }
            walls_prev = walls_now;
        }

        // C. collision of row yc
        const int yc = yl - LAG;
        bool fluid_c = true;
        if constexpr (SOLID) fluid_c = !(sm.type[yc & 7][ti] & T_SOLID);
        if (own && yc >= yb && fluid_c) {
            C f[Q];
            const S* fr = &sm.f[yc & 3][0][hx];
#pragma unroll
            for (int a = 0; a < Q; ++a) f[a] = C(fr[a * TW]);
            const C psi_c = sm.psi[yc & 7][hx];
            // sum_a w_a psi(x + e_a) e_a, taken over opposite pairs: w_a e_a (psi(x + e_a) - psi(x - e_a))
            C sx = C(0), sy = C(0);
#pragma unroll
            for (int a = 1; a < Q; ++a) {
                if (L::opp(a) < a) continue;
                const int ex = L::ex(a), ey = L::ey(a);
                const C wd = C(L::wf(a)) * (sm.psi[(yc + ey) & 7][hx + ex] - sm.psi[(yc - ey) & 7][hx - ex]);
                if (ex) sx += C(ex) * wd;
                if (ey) sy += C(ey) * wd;
            }
            // Eq. 5
            const C Fmx = -ph.G * psi_c * sx, Fmy = -ph.G * psi_c * sy;
            C drho = C(0), jx = C(0), jy = C(0);
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                drho += f[a];
                if (L::ex(a)) jx += C(L::ex(a)) * f[a];
                if (L::ey(a)) jy += C(L::ey(a)) * f[a];
            }
            const C rho = ph.rho_ref + drho;
            C Fx = Fmx + ph.fx, Fy = Fmy + ph.fy;
            // Eq. 8 (solid-fluid interaction scheme): F_ads = -G_w rho sum_a w_a s(x + e_a) e_a
            if constexpr (SOLID) {
                if (ph.wall_kind == 2 && !(sm.type[yc & 7][ti] & T_BULK)) {
                    C ax = C(0), ay = C(0);
#pragma unroll
                    for (int a = 1; a < Q; ++a) {
                        const int ex = L::ex(a), ey = L::ey(a);
                        if (sm.type[(yc + ey) & 7][ti + ex] & T_SOLID) {
                            if (ex) ax += C(L::wf(a) * ex);
                            if (ey) ay += C(L::wf(a) * ey);
                        }
                    }
                    const C gr = -ph.wall_param * rho;
                    Fx = (Fmx + gr * ax) + ph.fx;
                    Fy = (Fmy + gr * ay) + ph.fy;
                }
            }
            if (!(rho > C(0))) atomicOr(err, ERR_RHO);
            // Eq. 4: rho u = sum e f + F/2
            const C inv = cdiv(C(1), rho);
            const C ux = (jx + C(0.5) * Fx) * inv, uy = (jy + C(0.5) * Fy) * inv;
            const C X = cdiv(Fmx * Fmx + Fmy * Fmy, psi_c * psi_c);
            collide_d2q9<C>(f, drho, rho, ux, uy, Fx, Fy, X, ph.r);
            const int fi = yc * fp + gx;
#pragma unroll
            for (int a = 0; a < Q; ++a) fout[a * fs + fi] = S(f[a]);
        }
        load_types(yl + 3);
    }
    cp_wait<0>();
}

template <class S>
__global__ void __launch_bounds__(YShape<S>::TW, YShape<S>::MINB)
    ymarch_step(int parity, const BatchItem* __restrict__ items, const int* __restrict__ begin, Phys<S> ph,
                unsigned* err) {
    constexpr int TW = YShape<S>::TW;
    constexpr int WORDS = int(sizeof(BatchItem) / 4);
    static_assert(WORDS <= TW, "one lane per record word");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    YSmem<S, TW>& sm = *reinterpret_cast<YSmem<S, TW>*>(smem_raw);
    __shared__ BatchItem s_item[2];
    const int tid = threadIdx.x;
    const int i0 = begin[blockIdx.x], i1 = begin[blockIdx.x + 1];
    if (tid < WORDS && i0 < i1)
        reinterpret_cast<uint32_t*>(&s_item[0])[tid] = reinterpret_cast<const uint32_t*>(&items[i0])[tid];
    __syncthreads();
    int slot = 0;
    for (int it = i0; it < i1; ++it) {
        const BatchItem& item = s_item[slot];
        // fetch the next record during this run
        uint32_t w = 0;
        const bool fetch = tid < WORDS && it + 1 < i1;
        if (fetch) w = reinterpret_cast<const uint32_t*>(&items[it + 1])[tid];
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
        const int x0 = item.x0, y0 = item.y0, y1 = item.y1;
        if (item.solid) ymarch_run<S, true>(fin, fout, g, ph, x0, y0, y1, err, sm);
        else ymarch_run<S, false>(fin, fout, g, ph, x0, y0, y1, err, sm);
        if (fetch) reinterpret_cast<uint32_t*>(&s_item[slot ^ 1])[tid] = w;
        __syncthreads();
        slot ^= 1;
    }
}

template <class S>
cudaError_t ensure_smem_attr() {
    static bool done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!done[dev]) {
        cudaError_t e = cudaFuncSetAttribute(ymarch_step<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(sizeof(YSmem<S, YShape<S>::TW>)));
        if (e != cudaSuccess) return e;
        done[dev] = true;
    }
    return cudaSuccess;
}

template <class S>
int ymarch_occ() {
    if (ensure_smem_attr<S>() != cudaSuccess) return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ymarch_step<S>, YShape<S>::TW,
                                                      sizeof(YSmem<S, YShape<S>::TW>)) != cudaSuccess)
        n = 1;
    return n < 1 ? 1 : n;
}

template <class S>
cudaError_t launch_y(int parity, const DevParams& p, const BatchItem* items, const int* begin, int ctas,
                     cudaStream_t s) {
    cudaError_t e = ensure_smem_attr<S>();
    if (e != cudaSuccess) return e;
    ymarch_step<S><<<ctas, YShape<S>::TW, sizeof(YSmem<S, YShape<S>::TW>), s>>>(parity, items, begin,
                                                                                make_phys<S>(p), p.err);
    return cudaGetLastError();
}

}  // namespace

int ymarch_threads(int prec) { return prec == PREC_FP64 ? YShape<double>::TW : YShape<float>::TW; }

int ymarch_ctas_per_sm(int prec) { return prec == PREC_FP64 ? ymarch_occ<double>() : ymarch_occ<float>(); }

cudaError_t launch_ymarch(int prec, int parity, const DevParams& p, const BatchItem* items, const int* begin,
                          int ctas, cudaStream_t s) {
    return prec == PREC_FP64 ? launch_y<double>(parity, p, items, begin, ctas, s)
                             : launch_y<float>(parity, p, items, begin, ctas, s);
}

}  // namespace lbmwet
