// D2Q9 FP32 time step with two nodes per thread and packed FP32x2 arithmetic.
//
// A CTA of 32 x 8 threads owns a 32 x 16 tile; thread (lx, ly) owns the nodes (x0 + lx, y0 + ly)
// and (x0 + lx, y0 + ly + 8).  Every per-node quantity of the pair is one float2 and the arithmetic
// of the step (density, pseudopotential, force, velocity, MRT collision) runs on both nodes at once
// through the packed FP32 instructions (__fadd2_rn, __fmul2_rn, __ffma2_rn), which do two IEEE
// single-precision operations per instruction.  The phases are those of the scalar tile kernel:
//   0. node types of the tile + 3-node halo into shared memory (tiles holding a solid node; a batch
//      copies them during the previous tile);
//   1. pull (Eq. 3, halfway bounce-back of Fig. 3) of the two own nodes into registers and of the
//      tile's 1-node halo ring (one cell per thread of the first 100 threads, copied with cp.async
//      into shared memory so that its loads are in flight with the own nodes'); density (Eq. 4)
//      and psi (Eq. 6) into shared memory; wall cells queued; the 2-node ring where a wall needs it;
//   2. virtual wall densities (Eqs. 16-17 with the limiter, or the constant one) and their psi;
//   3. F_m (Eq. 5), u (Eq. 4), the MRT collision with the consistency source (Eqs. 2, 7) in the
//      increment form f += M^-1 (m* - m), and coalesced stores of f*.
// The arithmetic is the scalar kernels' (same operations, regrouped): results agree with them to
// FP32 rounding, not bit for bit.
#include <cmath>

#include "kernels.h"
#include "lattice.cuh"
#include "pack2.cuh"
#include "tile_common.cuh"

namespace lbmwet {

namespace {

constexpr int PTX = 32, PTY = 8, PNY = 16;   // threads x, threads y, tile rows (two per thread)

// Collision constants folded with the row norms of M: a_k = (m*_k - m_k) / |row_k|^2.
struct PairRates {
    float ke1, ke2, ke3;    // a1 = ke1 (m1 - e_eq) + ke2 u.F + ke3 X
    float kp1, kp2, kp3;    // a2 = kp1 (m2 - eps_eq) + kp2 u.F + kp3 X
    float kq1, kq2;         // a4 = kq1 (m4 + rho ux) + kq2 Fx (a6 likewise)
    float kn1, kn2;         // a7 = kn1 (m7 - rho (ux^2 - uy^2)) + kn2 (ux Fx - uy Fy); a8 = kn1 (m8 - rho ux uy) + kn2/2 (ux Fy + uy Fx)
};

PairRates make_pair_rates(const DevParams& p) {
    PairRates r;
    const double he = 1.0 - 0.5 * p.s_e, hp = 1.0 - 0.5 * p.s_eps, hq = 1.0 - 0.5 * p.s_q, hn = 1.0 - 0.5 * p.s_nu;
    // row norms |row|^2: e 36, eps 36, q 12, pxx 4, pxy 4
    r.ke1 = float(-p.s_e / 36.0);
    r.ke2 = float(6.0 * he / 36.0);
    r.ke3 = float(he * p.c_e / 36.0);
    r.kp1 = float(-p.s_eps / 36.0);
    r.kp2 = float(-6.0 * hp / 36.0);
    r.kp3 = float(-hp * p.c_eps / 36.0);
    r.kq1 = float(-p.s_q / 12.0);
    r.kq2 = float(-hq / 12.0);
    r.kn1 = float(-p.s_nu / 4.0);
    r.kn2 = float(2.0 * hn / 4.0);
    return r;
}

// MRT collision (Eq. 2 with the source of Eq. 7) of a pair in deviation variables; f += M^-1 (m* - m)
__device__ __forceinline__ void collide2(V2 (&f)[9], V2 drho, V2 rho, V2 ux, V2 uy, V2 Fx, V2 Fy, V2 X,
                                         const PairRates& k) {
    const V2 p13 = f[1] + f[3], p24 = f[2] + f[4], p57 = f[5] + f[7], p68 = f[6] + f[8];
    const V2 s14 = p13 + p24, s58 = p57 + p68;
    const V2 m7 = p13 - p24, m8 = p57 - p68;
    const V2 m1 = fma2(-4.0f, f[0], fma2(2.0f, s58, -s14));
    const V2 m2 = fma2(4.0f, f[0], fma2(-2.0f, s14, s58));
    const V2 q57 = f[5] - f[7], q86 = f[8] - f[6];
    const V2 m4 = fma2(2.0f, f[3] - f[1], q57 + q86);
    const V2 m6 = fma2(2.0f, f[4] - f[2], q57 - q86);
    // equilibria (deviation form) and sources
    const V2 uxx = ux * ux, uyy = uy * uy, uxy = ux * uy;
    const V2 rhou2 = rho * (uxx + uyy);
    const V2 uF = fma2(ux, Fx, uy * Fy);
    const V2 e_eq = fma2(3.0f, rhou2, -2.0f * drho);
    const V2 eps_eq = fma2(-3.0f, rhou2, drho);
    const V2 a1 = fma2(k.ke3, X, fma2(k.ke2, uF, k.ke1 * (m1 - e_eq)));
    const V2 a2 = fma2(k.kp3, X, fma2(k.kp2, uF, k.kp1 * (m2 - eps_eq)));
    const V2 a4 = fma2(k.kq2, Fx, k.kq1 * fma2(rho, ux, m4));
    const V2 a6 = fma2(k.kq2, Fy, k.kq1 * fma2(rho, uy, m6));
    const V2 a7 = fma2(k.kn2, fma2(ux, Fx, -(uy * Fy)), k.kn1 * (m7 - rho * (uxx - uyy)));
    const V2 a8 = fma2(0.5f * k.kn2, fma2(ux, Fy, uy * Fx), k.kn1 * (m8 - rho * uxy));
    const V2 a3 = (1.0f / 6.0f) * Fx, a5 = (1.0f / 6.0f) * Fy;
    // f += M^T diag(1/|row|^2) (m* - m)
    const V2 b = fma2(-2.0f, a2, -a1), c = fma2(2.0f, a1, a2);
    f[0] = fma2(4.0f, a2 - a1, f[0]);
    const V2 r3 = fma2(-2.0f, a4, a3), r5 = fma2(-2.0f, a6, a5);
    const V2 bp = b + a7, bm = b - a7;
    f[1] = f[1] + (bp + r3);
    f[3] = f[3] + (bp - r3);
    f[2] = f[2] + (bm + r5);
    f[4] = f[4] + (bm - r5);
    const V2 t1 = a3 + a4, t2 = a5 + a6;
    const V2 pp = t1 + t2, qq = t2 - t1;
    const V2 cu = c + a8, cv = c - a8;
    f[5] = f[5] + (cu + pp);
    f[7] = f[7] + (cu - pp);
    f[6] = f[6] + (cv + qq);
    f[8] = f[8] + (cv - qq);
}

// LBMWET_PAIR_BOX_RING2 = 1: the box also holds the rows the 2-node density ring of a wall tile pulls
// from, so that the ring comes from the box instead of global memory (2.9 KB more shared memory per
// CTA; 4 CTAs still fit the 164 KB shared-memory carveout, so L1 keeps 64 KB).  Measured on the
// 600 x 400 sweep: 0.759 of the HBM roofline against 0.751 without it.
#ifndef LBMWET_PAIR_BOX_RING2
#define LBMWET_PAIR_BOX_RING2 1
#endif

// The TMA box of a tile: every direction's values over x0 - 4 .. x0 + 35, y0 - Y0 .. y0 + 15 + Y0
// (the tile, its halo ring and the ring's upstream cells; with LBMWET_PAIR_BOX_RING2 the 2-node ring
// and its upstream cells), [a][y][x].
struct PairBox {
    static constexpr int BX = PTX + 8, BY = PNY + (LBMWET_PAIR_BOX_RING2 ? 6 : 4), X0 = 4,
                         Y0 = LBMWET_PAIR_BOX_RING2 ? 3 : 2;
    static constexpr int ELEMS = 9 * BY * BX;
    static_assert(PTX % 4 == 0, "x0 - 4 must be a 16-byte boundary");
};

struct NoHook {
    __device__ void operator()() const {}
};

struct PairSmem {
    static constexpr int RX = PTX + 4, RY = PNY + 4;   // density tile (2-node halo)
    static constexpr int PX = PTX + 2, PY = PNY + 2;   // psi tile (1-node halo)
    static constexpr int YX = PTX + 8, YY = PNY + 6;   // type tile: x0 - 4 .. x0 + 35, 3-node halo in y
    static constexpr int SHELL = 2 * PX + 2 * (PY - 2);
    uint8_t type[2][YY * YX];   // two buffers: a batch copies the next tile's types during this tile
    float rho[RY * RX];
    float psi[PY * PX];
    short wall[PY * PX];
    int nwall;
};

// The grid of a single-grid launch (kernel parameters); a batch passes its work record (shared
// memory) with the same member names.  Members are read where they are used, so that nothing of
// the grid needs a register across the tile's barriers.
struct PairGrid {
    int nx, ny, N;
    int fp, fs;   // distribution row pitch and direction stride
    const uint8_t* type;
    const int* wall_id;
    const double* kappa_w;
    double kappa;
    const void* f[2];
};

// One 32 x 16 tile with first node (x0, y0), reading g.f[parity] and writing g.f[parity ^ 1].
// SOLID = false: no solid node within the tile + 3-node halo.  WRAP as in the scalar tile kernel:
// 0 no periodic wrap, 1 a single wrap, 2 full modulo.
// box: the tile's PairBox already in shared memory, or null (pulls from global memory).  pre() runs
// once in every thread right after the halo ring's copies are issued; its own cp.async copies form
// the one commit group the phase does not wait for.  hook() runs once in every thread right after
// the barrier that ends phase 1 (the box and the halo staging are free from then on).
template <bool SOLID, int WRAP, class G, class Pre = NoHook, class Hook = NoHook>
__device__ __forceinline__ void pair_body(const G& g, int parity, const Phys<float>& ph, const PairRates& kr, int x0,
                                          int y0, unsigned* err, PairSmem& sm, float* hst, const float* box,
                                          int tbuf, bool ty_ready, const Pre& pre, const Hook& hook) {
    using L = D2Q9;
    constexpr int Q = 9, NT = PTX * PTY;
    using Sm = PairSmem;
    constexpr int RX = Sm::RX, PX = Sm::PX, PY = Sm::PY, YX = Sm::YX, YY = Sm::YY, SHELL = Sm::SHELL;
    const int nx = g.nx, ny = g.ny;
    const int fp = g.fp, fs = g.fs;   // distribution row pitch and direction stride
    const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * PTX + lx;
    const float* __restrict__ fin = static_cast<const float*>(g.f[parity]);
    auto wr = [](int v, int n) { return WRAP == 0 ? v : (WRAP == 1 ? wrap1(v, n) : wrap_full(v, n)); };
    auto tix = [](int cx, int cy) { return cy * YX + cx + 1; };   // type cell of tile-relative (cx - 3, cy - 3)
    uint8_t* const tyb = sm.type[tbuf];
    auto rix = [](int cx, int cy) { return cy * RX + cx; };   // density cell of (cx - 2, cy - 2)
    auto pix = [](int cx, int cy) { return cy * PX + cx; };   // psi cell of (cx - 1, cy - 1)

    // 0. node types of the tile + 3-node halo (unless already in tyb); does the 1-node halo region
    // hold a wall?
    if (tid == 0) sm.nwall = 0;
    bool tile_has_wall = false;
    if constexpr (SOLID) {
        int wall_seen = 0;
        for (int i = tid; i < YX * YY; i += NT) {
            const int cx = i % YX, cy = i / YX;   // node (x0 + cx - 4, y0 + cy - 3)
            uint8_t ty;
            if (ty_ready) {
                ty = tyb[i];
            } else {
                ty = g.type[wr(y0 + cy - 3, ny) * nx + wr(x0 + cx - 4, nx)];
                tyb[i] = ty;
            }
            if (cx >= 3 && cx < PTX + 5 && cy >= 2 && cy < PNY + 4 && (ty & T_WALL)) wall_seen = 1;
        }
        tile_has_wall = __syncthreads_or(wall_seen);
    }
    auto type_at = [&](int ti) -> uint8_t {
        if constexpr (!SOLID) return uint8_t(T_BULK);
        return tyb[ti];
    };
    // source of every distribution streaming into node (gx, gy), handed to sink(a, pointer)
    auto pull_src = [&](auto&& sink, int gx, int gy, int ti, uint8_t self) {
        if constexpr (WRAP == 0) {
            const float* p = fin + (gy * fp + gx);
            if (!SOLID || (self & T_BULK)) {
#pragma unroll
                for (int a = 0; a < Q; ++a) sink(a, p + (a * fs - L::ex(a) - L::ey(a) * fp));
            } else {
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    const bool bb = (tyb[ti - L::ex(a) - L::ey(a) * YX] & T_SOLID) != 0;
                    sink(a, p + (bb ? L::opp(a) * fs : a * fs - L::ex(a) - L::ey(a) * fp));
                }
            }
        } else {
            const int cx[3] = {wrap1(gx - 1, nx), gx, wrap1(gx + 1, nx)};
            const int ry[3] = {wrap1(gy - 1, ny) * fp, gy * fp, wrap1(gy + 1, ny) * fp};
            if (!SOLID || (self & T_BULK)) {
#pragma unroll
                for (int a = 0; a < Q; ++a) sink(a, fin + (a * fs + ry[1 - L::ey(a)] + cx[1 - L::ex(a)]));
            } else {
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    const bool bb = (tyb[ti - L::ex(a) - L::ey(a) * YX] & T_SOLID) != 0;
                    sink(a, fin + (bb ? L::opp(a) * fs + ry[1] + cx[1]
                                      : a * fs + ry[1 - L::ey(a)] + cx[1 - L::ex(a)]));
                }
            }
        }
    };

    // the same from the box: node at box cell (bx, by) of tile-relative type cell ti
    using B = PairBox;
    auto box_src = [&](auto&& sink, int bx, int by, int ti, uint8_t self) {
        if (!SOLID || (self & T_BULK)) {
#pragma unroll
            for (int a = 0; a < Q; ++a) sink(a, box[(a * B::BY + by - L::ey(a)) * B::BX + bx - L::ex(a)]);
        } else {
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const bool bb = (tyb[ti - L::ex(a) - L::ey(a) * YX] & T_SOLID) != 0;
                sink(a, bb ? box[(L::opp(a) * B::BY + by) * B::BX + bx]
                           : box[(a * B::BY + by - L::ey(a)) * B::BX + bx - L::ex(a)]);
            }
        }
    };

    // 1. the halo-ring cell of this thread: its loads go out first (cp.async into shared memory)
    using Ring = Shell<PX, PY, 1, 2>;
    static_assert(Ring::COUNT == SHELL && SHELL <= NT, "one ring cell per thread");
    const bool boxed = box != nullptr;
    const bool has_h = tid < SHELL;
    uint8_t hty = uint8_t(T_SOLID);
    int hpx = 0, hpy = 0;
    if (has_h) {
        int pz;
        Ring::cell(tid, hpx, hpy, pz);
        const int ti = tix(hpx + 2, hpy + 2);
        hty = type_at(ti);
        if (!boxed && !(hty & T_SOLID))
            pull_src([&](int a, const float* src) { cp_async(&hst[a * SHELL + tid], src); },
                     wr(x0 + hpx - 1, nx), wr(y0 + hpy - 1, ny), ti, hty);
    }
    cp_commit();
    pre();
    cp_commit();
    // the two own nodes: rows ly and ly + 8
    const int gx = wr(x0 + lx, nx);
    const int gya = wr(y0 + ly, ny), gyb = wr(y0 + ly + PTY, ny);
    const int tia = tix(lx + 3, ly + 3), tib = tix(lx + 3, ly + PTY + 3);
    const uint8_t ta = type_at(tia), tb = type_at(tib);
    const bool fa = !(ta & T_SOLID), fb = !(tb & T_SOLID);
    V2 f[Q];
    if (boxed && !SOLID) {
        // node (x, y), direction a: the value at (x - e_a, y - e_a) of the box
#pragma unroll
        for (int a = 0; a < Q; ++a)
            f[a] = mk(box[(a * B::BY + ly + B::Y0 - L::ey(a)) * B::BX + lx + B::X0 - L::ex(a)],
                      box[(a * B::BY + ly + PTY + B::Y0 - L::ey(a)) * B::BX + lx + B::X0 - L::ex(a)]);
    } else {
#pragma unroll
        for (int a = 0; a < Q; ++a) f[a] = bc(0.0f);
        if (boxed) {
            if (fa) box_src([&](int a, float v) { f[a].v.x = v; }, lx + B::X0, ly + B::Y0, tia, ta);
            if (fb) box_src([&](int a, float v) { f[a].v.y = v; }, lx + B::X0, ly + PTY + B::Y0, tib, tb);
        } else {
            if (fa) pull_src([&](int a, const float* src) { f[a].v.x = *src; }, gx, gya, tia, ta);
            if (fb) pull_src([&](int a, const float* src) { f[a].v.y = *src; }, gx, gyb, tib, tb);
        }
    }
    V2 drho = f[0];
#pragma unroll
    for (int a = 1; a < Q; ++a) drho = drho + f[a];
    {
        const V2 rho = bc(ph.rho_ref) + drho;
        const V2 ps = psi2(rho, ph, fa, fb, err);
        sm.psi[pix(lx + 1, ly + 1)] = fa ? ps.v.x : 0.0f;
        sm.psi[pix(lx + 1, ly + PTY + 1)] = fb ? ps.v.y : 0.0f;
        if constexpr (SOLID) {
            if (tile_has_wall) {
                sm.rho[rix(lx + 2, ly + 2)] = fa ? rho.v.x : 0.0f;
                sm.rho[rix(lx + 2, ly + PTY + 2)] = fb ? rho.v.y : 0.0f;
            }
            if (ta & T_WALL) sm.wall[atomicAdd(&sm.nwall, 1)] = short(pix(lx + 1, ly + 1));
            if (tb & T_WALL) sm.wall[atomicAdd(&sm.nwall, 1)] = short(pix(lx + 1, ly + PTY + 1));
        }
    }
    cp_wait<1>();   // the halo ring (and anything older), not pre()'s copies
    if (has_h) {
        const int hpi = pix(hpx, hpy);
        float hrho = 0.0f, hpsi = 0.0f;
        if (!(hty & T_SOLID)) {
            float h[Q];
            if (boxed) {
                // ring cell (x0 + hpx - 1, y0 + hpy - 1)
                box_src([&](int a, float v) { h[a] = v; }, hpx - 1 + B::X0, hpy - 1 + B::Y0, tix(hpx + 2, hpy + 2),
                        hty);
            } else {
#pragma unroll
                for (int a = 0; a < Q; ++a) h[a] = hst[a * SHELL + tid];
            }
            float d = h[0];
#pragma unroll
            for (int a = 1; a < Q; ++a) d += h[a];
            hrho = ph.rho_ref + d;
            hpsi = psi2(bc(hrho), ph, true, false, err).v.x;   // the own nodes' formula
        } else if (hty & T_WALL) {
            sm.wall[atomicAdd(&sm.nwall, 1)] = short(hpi);
        }
        if (SOLID && tile_has_wall) sm.rho[rix(hpx + 1, hpy + 1)] = hrho;
        sm.psi[hpi] = hpsi;
    }
    // the 2-node ring, only where Eq. 17 will need it
    if constexpr (SOLID) {
        if (tile_has_wall) {
            using Ring2 = Shell<RX, PNY + 4, 1, 2>;
            for (int k = tid; k < Ring2::COUNT; k += NT) {
                int rx, ry, rz;
                Ring2::cell(k, rx, ry, rz);
                const int ti = tix(rx + 1, ry + 1);
                const uint8_t ty = tyb[ti];
                float rho = 0.0f;
                if (!(ty & T_SOLID)) {
                    float d = 0.0f;
                    int first = 1;
                    if (LBMWET_PAIR_BOX_RING2 && boxed) {
                        box_src(
                            [&](int a, float v) {
                                (void)a;
                                d = first ? v : d + v;
                                first = 0;
                            },
                            rx - 2 + B::X0, ry - 2 + B::Y0, ti, ty);
                    } else {
                        pull_src(
                            [&](int a, const float* src) {
                                (void)a;
                                d = first ? *src : d + *src;
                                first = 0;
                            },
                            wr(x0 + rx - 2, nx), wr(y0 + ry - 2, ny), ti, ty);
                    }
                    rho = ph.rho_ref + d;
                }
                sm.rho[rix(rx, ry)] = rho;
            }
        }
    }
    __syncthreads();
    hook();

    // 2. wall cells of the tile + 1-node halo: virtual density and its psi
    if constexpr (SOLID) {
        const int nwall = sm.nwall;
        if (nwall > 0 && ph.wall_kind != 2) {   // the solid-fluid interaction scheme keeps psi = 0 on solids
            for (int k = tid; k < nwall; k += NT) {
                const int i = sm.wall[k];
                const int px = i % PX, py = i / PX;
                const int ti = tix(px + 2, py + 2);
                float rw;
                if (ph.wall_kind == 1) {
                    rw = ph.wall_param;
                } else {
                    // Eq. 17: weighted mean of the fluid neighbours' densities
                    float num = 0.0f, den = 0.0f;
#pragma unroll
                    for (int a = 1; a < Q; ++a) {
                        const int ex = L::ex(a), ey = L::ey(a);
                        if (!(tyb[ti + ex + ey * YX] & T_SOLID)) {
                            num += float(L::wf(a)) * sm.rho[rix(px + 1 + ex, py + 1 + ey)];
                            den += float(L::wf(a));
                        }
                    }
                    const float rho_ave = cdiv(num, den);
                    const int gw = wr(y0 + py - 1, ny) * nx + wr(x0 + px - 1, nx);
                    if (ph.wall_kind == 3) {
                        // geometric formulation (Eqs. 10-15): crossings of the characteristic lines
                        rw = gf_wall_density(g.kappa_w + GF_STRIDE * g.wall_id[gw], rho_ave, [&](int dx, int dy) {
                            return sm.rho[rix(px + 1 + dx, py + 1 + dy)];
                        });
                    } else {
                        const float kap = g.kappa_w ? float(g.kappa_w[g.wall_id[gw]]) : float(g.kappa);
                        // Eq. 16 (kappa >= 0: phi = 1 + kappa; kappa < 0: drho = -kappa) and the limiter
                        const float raw = (kap >= 0.0f) ? (1.0f + kap) * rho_ave : rho_ave + kap;
                        rw = raw > ph.rho_l ? ph.rho_l : raw;
                        rw = rw < ph.rho_g ? ph.rho_g : rw;
                    }
                }
                sm.psi[i] = psi2(bc(rw), ph, true, false, err).v.x;
            }
            __syncthreads();
        }
    }

    // 3. force, velocity, collision and store of the pair
    const bool va = x0 + lx < nx && y0 + ly < ny && fa;
    const bool vb = x0 + lx < nx && y0 + ly + PTY < ny && fb;
    if (!va && !vb) return;
    const int pca = pix(lx + 1, ly + 1), pcb = pix(lx + 1, ly + PTY + 1);
    auto psi_pair = [&](int off) { return mk(sm.psi[pca + off], sm.psi[pcb + off]); };
    const V2 psi_c = psi_pair(0);
    // sum_a w_a psi(x + e_a) e_a over opposite pairs: w_a e_a (psi(x + e_a) - psi(x - e_a))
    const V2 w1 = (1.0f / 3.0f) * (psi_pair(1) - psi_pair(-1));                  // e = (1, 0)
    const V2 w2 = (1.0f / 3.0f) * (psi_pair(PX) - psi_pair(-PX));                // e = (0, 1)
    const V2 w5 = (1.0f / 12.0f) * (psi_pair(PX + 1) - psi_pair(-PX - 1));       // e = (1, 1)
    const V2 w6 = (1.0f / 12.0f) * (psi_pair(PX - 1) - psi_pair(-PX + 1));       // e = (-1, 1)
    const V2 sx = (w1 + w5) - w6, sy = (w2 + w5) + w6;
    // Eq. 5
    const V2 gpsi = (-ph.G) * psi_c;
    const V2 Fmx = gpsi * sx, Fmy = gpsi * sy;
    V2 Fx = Fmx + bc(ph.fx), Fy = Fmy + bc(ph.fy);
    // Eq. 8 (solid-fluid interaction scheme): F_ads = -G_w rho sum_a w_a s(x + e_a) e_a
    if constexpr (SOLID) {
        if (ph.wall_kind == 2 && !((ta & tb) & T_BULK)) {
            float axa = 0.0f, aya = 0.0f, axb = 0.0f, ayb = 0.0f;
#pragma unroll
            for (int a = 1; a < Q; ++a) {
                const int ex = L::ex(a), ey = L::ey(a), off = ex + ey * YX;
                const float w = float(L::wf(a));
                if (tyb[tia + off] & T_SOLID) {
                    if (ex) axa += w * float(ex);
                    if (ey) aya += w * float(ey);
                }
                if (tyb[tib + off] & T_SOLID) {
                    if (ex) axb += w * float(ex);
                    if (ey) ayb += w * float(ey);
                }
            }
            const V2 gr = (-ph.wall_param) * (bc(ph.rho_ref) + drho);
            Fx = (Fmx + gr * mk(axa, axb)) + bc(ph.fx);
            Fy = (Fmy + gr * mk(aya, ayb)) + bc(ph.fy);
        }
    }
    const V2 jx = ((f[1] - f[3]) + (f[5] - f[7])) + (f[8] - f[6]);
    const V2 jy = ((f[2] - f[4]) + (f[5] - f[7])) + (f[6] - f[8]);
    const V2 rho = bc(ph.rho_ref) + drho;
    if ((va && !(rho.v.x > 0.0f)) || (vb && !(rho.v.y > 0.0f))) atomicOr(err, ERR_RHO);
    // Eq. 4: rho u = sum e f + F/2
    const V2 inv = div2(bc(1.0f), rho);
    const V2 ux = fma2(0.5f, Fx, jx) * inv, uy = fma2(0.5f, Fy, jy) * inv;
    const V2 X = div2(fma2(Fmx, Fmx, Fmy * Fmy), psi_c * psi_c);
    collide2(f, drho, rho, ux, uy, Fx, Fy, X, kr);
    const int gia = (y0 + ly) * fp + x0 + lx, gib = gia + PTY * fp;   // distribution indices
    float* __restrict__ fout = static_cast<float*>(const_cast<void*>(g.f[parity ^ 1]));
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        if (va) fout[a * fs + gia] = f[a].v.x;
        if (vb) fout[a * fs + gib] = f[a].v.y;
    }
}

__host__ __device__ __forceinline__ int pair_wrap(int x0, int y0, int nx, int ny) {
    if (nx < PTX + 8 || ny < PNY + 8) return 2;
    return (x0 >= 3 && x0 + PTX + 2 < nx && y0 >= 3 && y0 + PNY + 2 < ny) ? 0 : 1;
}

// hst: shared memory for the halo ring's pulled distributions, [a][ring cell] (9 * SHELL floats),
// used when box is null
template <bool SOLID, class G, class Pre = NoHook, class Hook = NoHook>
__device__ __forceinline__ void pair_tile(const G& g, int parity, const Phys<float>& ph, const PairRates& kr, int x0,
                                          int y0, unsigned* err, PairSmem& sm, float* hst, const float* box = nullptr,
                                          int tbuf = 0, bool ty_ready = false, const Pre& pre = Pre(),
                                          const Hook& hook = Hook()) {
    const int w = pair_wrap(x0, y0, g.nx, g.ny);
    if (w == 0) pair_body<SOLID, 0>(g, parity, ph, kr, x0, y0, err, sm, hst, box, tbuf, ty_ready, pre, hook);
    else if (w == 1) pair_body<SOLID, 1>(g, parity, ph, kr, x0, y0, err, sm, hst, box, tbuf, ty_ready, pre, hook);
    else pair_body<SOLID, 2>(g, parity, ph, kr, x0, y0, err, sm, hst, box, tbuf, ty_ready, pre, hook);
}

#ifndef LBMWET_PAIR_MINB
#define LBMWET_PAIR_MINB 4
#endif

__global__ void __launch_bounds__(PTX* PTY, LBMWET_PAIR_MINB)
    pair_step(PairGrid g, const uint8_t* __restrict__ tile_solid, Phys<float> ph, PairRates kr, unsigned* err) {
    __shared__ PairSmem sm;
    __shared__ float hst[9 * PairSmem::SHELL];
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    const bool solid = tile_solid ? tile_solid[tile] != 0 : true;
    if (solid) pair_tile<true>(g, 0, ph, kr, blockIdx.x * PTX, blockIdx.y * PNY, err, sm, hst);
    else pair_tile<false>(g, 0, ph, kr, blockIdx.x * PTX, blockIdx.y * PNY, err, sm, hst);
}

// Polls of an mbarrier before a wait gives up (flags ERR_TIMEOUT and goes on).  A poll
// (mbarrier.try_wait) suspends for about 3.8 us when the phase is incomplete (measured on GB300 by
// lbm_selftest_bounded_wait), so 2^18 polls bound a wait at about one second, far above any copy's
// latency.
constexpr unsigned MBAR_POLL_LIMIT = 1u << 18;

// Persistent form with dynamic tile scheduling.  CTA b starts with items b and b + gridDim.x; every
// further item is claimed from a global counter (sched[0]), so that a CTA slowed by costly tiles
// (walls, periodic edges, ragged columns) simply takes fewer of them, and items are taken in list
// order (the tiles in flight stay neighbours in memory).  Work records sit in a ring of three
// shared slots: the current tile's, the next tile's and the one after.  Thread 0 claims the one
// after at the end of the previous tile (few registers are live there), and early in phase 1 it
// publishes the index and copies that record with 16-byte cp.async copies that the next tile waits
// for.  Every tile away from the periodic edges of a grid with TMA tensor maps (every 2D grid: the
// distribution rows are padded to 128 bytes) pulls from a box that one TMA load brings into shared
// memory while the previous tile finishes (issued right after that tile's phase 1, when the box is
// free); such a tile holding a solid node also gets its node types copied (cp.async) into the other
// type buffer meanwhile, and takes its 2-node density ring from the box.  A tile without a box
// stages its halo ring in the box's memory, which keeps the CTA under the 40 KB that lets 4 CTAs
// share a 164 KB carveout.  One claim is made per tile processed; the last CTA to finish resets the
// counter for the next launch (sched[1] counts finished CTAs).
__global__ void __launch_bounds__(PTX* PTY, LBMWET_PAIR_MINB)
    pair_step_batched(int parity, const BatchItem* __restrict__ items, int n_items, Phys<float> ph, PairRates kr,
                      unsigned* err, unsigned* sched) {
    constexpr int WORDS = int(sizeof(BatchItem) / 4), CHUNKS = int(sizeof(BatchItem) / 16);
    static_assert(sizeof(BatchItem) % 16 == 0, "records are copied in 16-byte chunks");
    using B = PairBox;
    __shared__ PairSmem sm;
    __shared__ alignas(128) float box[B::ELEMS];
    static_assert(B::ELEMS >= 9 * PairSmem::SHELL, "the halo staging of unboxed tiles fits in the box");
    __shared__ alignas(8) uint64_t bar;
    __shared__ BatchItem s_item[3];
    __shared__ int s_idx[3];   // item index held by each record slot (n_items or more: none)
    const int tid = threadIdx.y * PTX + threadIdx.x;
    const int grid = gridDim.x;
    if (tid < WORDS) {
        if (blockIdx.x < n_items)
            reinterpret_cast<uint32_t*>(&s_item[0])[tid] = reinterpret_cast<const uint32_t*>(&items[blockIdx.x])[tid];
        if (blockIdx.x + grid < n_items)
            reinterpret_cast<uint32_t*>(&s_item[1])[tid] =
                reinterpret_cast<const uint32_t*>(&items[blockIdx.x + grid])[tid];
    }
    unsigned claim = 0;   // thread 0: the claim for the record two tiles ahead
    if (tid == 0) {
        s_idx[0] = blockIdx.x;
        s_idx[1] = blockIdx.x + grid;
        if (blockIdx.x < n_items) claim = atomicAdd(sched, 1u);
        mbar_init(&bar);
        fence_mbar_init();
    }
    __syncthreads();
    // 1: the tile pulls from a TMA box, 0: from global memory
    auto box_kind = [](const BatchItem& r) -> int {
        return r.tmap != nullptr && pair_wrap(r.x0, r.y0, r.nx, r.ny) == 0 ? 1 : 0;
    };
    auto issue = [&](const BatchItem& r) {
        fence_proxy_async();
        tma_load_box(box, static_cast<const char*>(r.tmap) + 128 * parity, r.x0 - B::X0, r.y0 - B::Y0, 0, &bar,
                     unsigned(B::ELEMS * sizeof(float)));
    };
    unsigned phase = 0;
    int cur_kind = blockIdx.x < n_items ? box_kind(s_item[0]) : 0;
    if (cur_kind == 1 && tid == 0) issue(s_item[0]);
    int s0 = 0, s1 = 1, s2 = 2;   // ring slots of the current, next and after-next records
    int tbuf = 0;                 // type buffer of the current tile
    bool ty_ready = false;        // its types were copied during the previous tile
    for (int it = blockIdx.x; it < n_items;) {
        const BatchItem& item = s_item[s0];
        const BatchItem& nxt = s_item[s1];
        auto pre = [&]() {
            if (tid == 0) {
                const int far = 2 * grid + int(claim);
                s_idx[s2] = far;
                if (far < n_items) {
#pragma unroll
                    for (int c = 0; c < CHUNKS; ++c)
                        cp_async16(reinterpret_cast<float*>(&s_item[s2]) + 4 * c,
                                   reinterpret_cast<const float*>(&items[far]) + 4 * c);
                }
            }
        };
        int next_kind = 0;
        bool next_types = false;
        auto hook = [&]() {
            next_kind = s_idx[s1] < n_items ? box_kind(nxt) : 0;
            if (next_kind == 1 && tid == 0) issue(nxt);
            // an interior tile holding a solid, of a grid whose rows are a multiple of 4 nodes: its node
            // types (rows y0 - 3 .. y0 + 18, columns x0 - 4 .. x0 + 35, all inside the grid; every row
            // segment starts on a 4-byte boundary) into the other type buffer, 4 bytes per copy
            next_types = next_kind == 1 && nxt.solid && (nxt.nx & 3) == 0;
            if (next_types) {
                constexpr int CW = PairSmem::YX / 4;
                if (tid < PairSmem::YY * CW) {
                    const int r = tid / CW, c = tid % CW;
                    cp_async(reinterpret_cast<float*>(&sm.type[tbuf ^ 1][r * PairSmem::YX + 4 * c]),
                             reinterpret_cast<const float*>(nxt.type + (size_t)(nxt.y0 - 3 + r) * nxt.nx + nxt.x0 -
                                                            4 + 4 * c));
                }
                cp_commit();
            }
        };
        if (cur_kind == 1) {
            if (!mbar_wait(&bar, phase, MBAR_POLL_LIMIT)) atomicOr(err, ERR_TIMEOUT);
            phase ^= 1u;
        }
        const float* bx = cur_kind != 0 ? box : nullptr;
        // a tile without a box stages its halo ring in the box's memory (no load targets it meanwhile:
        // the next tile's TMA load is issued after this tile's phase 1)
        if (item.solid)
            pair_tile<true>(item, parity, ph, kr, item.x0, item.y0, err, sm, box, bx, tbuf, ty_ready, pre, hook);
        else
            pair_tile<false>(item, parity, ph, kr, item.x0, item.y0, err, sm, box, bx, tbuf, ty_ready, pre, hook);
        it = s_idx[s1];
        if (tid == 0 && it < n_items) claim = atomicAdd(sched, 1u);   // for the tile after `it`'s next
        if (next_types) cp_wait<0>();   // the next tile's types (published by the barrier below)
        __syncthreads();   // this tile's threads are done with shared memory
        if (next_types) tbuf ^= 1;
        ty_ready = next_types;
        const int t = s0;
        s0 = s1;
        s1 = s2;
        s2 = t;
        cur_kind = next_kind;
    }
    cp_wait<0>();
    if (tid == 0) {
        // every claim of this CTA has returned; the last CTA to get here resets the counters
        __threadfence();
        if (atomicAdd(sched + 1, 1u) == unsigned(grid) - 1u) {
            atomicExch(sched, 0u);
            atomicExch(sched + 1, 0u);
        }
    }
}

// Self-test of the bounded waits: an mbarrier that no thread arrives on and no copy completes, waited
// on by every thread with `limit` polls.  Each wait must give up and flag ERR_TIMEOUT; nothing is in
// flight when the kernel returns.
__global__ void __launch_bounds__(128) wait_timeout_probe(unsigned* err, unsigned limit) {
    __shared__ alignas(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        fence_mbar_init();
    }
    __syncthreads();
    if (!mbar_wait(&bar, 0u, limit)) atomicOr(err, ERR_TIMEOUT);
}

}  // namespace

cudaError_t launch_wait_timeout_probe(unsigned* err, unsigned limit, cudaStream_t s) {
    wait_timeout_probe<<<1, 128, 0, s>>>(err, limit);
    return cudaGetLastError();
}

void pair_tile_shape(int* tx, int* ty) {
    *tx = PTX;
    *ty = PNY;
}

void pair_box_dims(int* bx, int* by) {
    *bx = PairBox::BX;
    *by = PairBox::BY;
}

int pair_ctas_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_step_batched, PTX * PTY, 0) != cudaSuccess) n = 1;
    return n < 1 ? 1 : n;
}

cudaError_t launch_pair_step(const void* fin, void* fout, const DevParams& p, cudaStream_t s) {
    PairGrid g;
    g.nx = p.nx;
    g.ny = p.ny;
    g.N = int(p.N);
    g.fp = p.fp;
    g.fs = int(p.fs);
    g.type = p.type;
    g.wall_id = p.wall_id;
    g.kappa_w = p.kappa_w;
    g.kappa = p.kappa;
    g.f[0] = fin;
    g.f[1] = fout;
    dim3 grid((p.nx + PTX - 1) / PTX, (p.ny + PNY - 1) / PNY, 1);
    pair_step<<<grid, dim3(PTX, PTY, 1), 0, s>>>(g, p.pair_solid, make_phys<float>(p), make_pair_rates(p), p.err);
    return cudaGetLastError();
}

cudaError_t launch_pair_batched(int parity, const DevParams& p, const BatchItem* items, int n_items, int ctas,
                                unsigned* sched, cudaStream_t s) {
    pair_step_batched<<<ctas, dim3(PTX, PTY, 1), 0, s>>>(parity, items, n_items, make_phys<float>(p),
                                                         make_pair_rates(p), p.err, sched);
    return cudaGetLastError();
}

}  // namespace lbmwet
