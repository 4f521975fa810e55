// D3Q19 FP32 time step as a z-pair march: the z-march of the scalar kernel with two planes per
// iteration, each thread carrying the same (x, y) cell on two consecutive planes, so that every
// per-node quantity is a float2 and the step's arithmetic runs on packed FP32x2 instructions.
//
// A CTA of TX x TY threads owns a TX x TY column and walks a chunk of z-planes.  For the lead pair
// of planes (zl, zl + 1) it
//   A. pulls (Eq. 3 with halfway bounce-back, Fig. 3) both planes of its own cells and of the 1-node
//      xy halo ring (the 2-node ring too where the chunk holds solids), stores rho (Eq. 4) and, at
//      fluid cells, psi (Eq. 6); wall cells are queued per plane;
//   B. gives the wall cells of planes zl - 1 and zl their virtual density (Eqs. 16-17 with the
//      limiter, or the constant one) from the densities of planes zl - 2 .. zl + 1, and its psi;
//   C. collides planes zl - 2 and zl - 1: F_m (Eq. 5), u (Eq. 4), the MRT collision with the
//      consistency source (Eqs. 2, 7) in the increment form f += M^-1 (m* - m), coalesced stores.
// Rings indexed by the absolute plane: densities 4 planes, psi 8, node types 8, wall queues 4 (and,
// with LBMWET_ZP_REPULL = 0, the own distributions, 4 planes).  Results equal the scalar z-march's up to FP32 rounding (operations regrouped).
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "kernels.h"
#include "lattice.cuh"
#include "maskscan.h"
#include "pack2.cuh"
#include "tile_common.cuh"

namespace lbmwet {

namespace {

// LBMWET_ZP_REPULL = 1: the collision pulls its pair of planes again (from L2, where the lead pull
// left them one iteration earlier) instead of keeping a 39 KB ring of them in shared memory; the
// smaller footprint leaves more of the SM's memory to L1 and one more CTA resident.  Measured on
// the 256^3 sphere: 22.4 GLUPS (4 CTAs per SM) against 22.1 for the ring (3 CTAs per SM).
#ifndef LBMWET_ZP_REPULL
#define LBMWET_ZP_REPULL 1
#endif
#ifndef LBMWET_ZP_MINB   // resident CTAs per SM of the z-pair march (chosen by measurement)
#define LBMWET_ZP_MINB (LBMWET_ZP_REPULL ? 4 : 3)
#endif
// column and chunk: the FP32 z-march's (the per-chunk solid flags are shared)
constexpr int ZTX = LBMWET_Z3F_X, ZTY = LBMWET_Z3F_Y, ZCH = LBMWET_Z3F_Z;
static_assert(ZCH % 2 == 0, "planes are marched in pairs");

// D3Q19 collision constants folded with the row norms of the d'Humieres basis:
// a_k = (m*_k - m_k) / |row_k|^2, |row|^2 = (19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24,
// 4, 4, 4, 8, 8, 8).
struct Rates3P {
    float k1e, k2e, k3e;     // a1 = k1e (m1 - e_eq) + k2e u.F + k3e X
    float k1p, k2p, k3p;     // a2 = k1p (m2 - eps_eq) + k2p u.F + k3p X
    float kq1, kq2;          // a4 = kq1 (m4 + 2/3 rho ux) + kq2 Fx (a6, a8 likewise)
    float kn9, kh9;          // a9 = kn9 (m9 - 3pxx_eq) + kh9 S3xx
    float kp10, kh10;        // a10 = kp10 (m10 + 3pxx_eq / 2) + kh10 S3xx
    float kn11, kh11;        // a11 = kn11 (m11 - pww_eq) + kh11 Sww
    float kp12, kh12;        // a12 = kp12 (m12 + pww_eq / 2) + kh12 Sww
    float kn13, kh13;        // a13 = kn13 (m13 - rho ux uy) + kh13 (ux Fy + uy Fx) (a14, a15 likewise)
    float km;                // a16 = km m16 (a17, a18 likewise)
};

Rates3P make_rates3p(const DevParams& p) {
    const double he = 1.0 - 0.5 * p.s_e, hp = 1.0 - 0.5 * p.s_eps, hq = 1.0 - 0.5 * p.s_q;
    const double hn = 1.0 - 0.5 * p.s_nu, hpi = 1.0 - 0.5 * p.s_pi;
    Rates3P r;
    r.k1e = float(-p.s_e / 2394.0);
    r.k2e = float(38.0 * he / 2394.0);
    r.k3e = float(he * p.c_e / 2394.0);
    r.k1p = float(-p.s_eps / 252.0);
    r.k2p = float(-11.0 * hp / 252.0);
    r.k3p = float(-hp * p.c_eps / 252.0);
    r.kq1 = float(-p.s_q / 40.0);
    r.kq2 = float(-hq * (2.0 / 3.0) / 40.0);
    r.kn9 = float(-p.s_nu / 36.0);
    r.kh9 = float(hn / 36.0);
    r.kp10 = float(-p.s_pi / 72.0);
    r.kh10 = float(-0.5 * hpi / 72.0);
    r.kn11 = float(-p.s_nu / 12.0);
    r.kh11 = float(hn / 12.0);
    r.kp12 = float(-p.s_pi / 24.0);
    r.kh12 = float(-0.5 * hpi / 24.0);
    r.kn13 = float(-p.s_nu / 4.0);
    r.kh13 = float(hn / 4.0);
    r.km = float(-p.s_m / 8.0);
    return r;
}

// MRT collision (d'Humieres D3Q19, source of Eq. 7 as in collide_d3q19) of a pair; f += M^-1 (m* - m)
__device__ __forceinline__ void collide3p(V2 (&f)[19], V2 drho, V2 rho, V2 ux, V2 uy, V2 uz, V2 Fx, V2 Fy, V2 Fz, V2 X,
                                          const Rates3P& k) {
    // moments of the non-conserved rows
    const V2 ax = f[1] + f[2], ay = f[3] + f[4], az = f[5] + f[6];
    const V2 d12 = f[1] - f[2], d34 = f[3] - f[4], d56 = f[5] - f[6];
    const V2 p78 = f[7] + f[8], p910 = f[9] + f[10], p1112 = f[11] + f[12], p1314 = f[13] + f[14];
    const V2 p1516 = f[15] + f[16], p1718 = f[17] + f[18];
    const V2 q78 = f[7] - f[8], q910 = f[9] - f[10], q1112 = f[11] - f[12], q1314 = f[13] - f[14];
    const V2 q1516 = f[15] - f[16], q1718 = f[17] - f[18];
    const V2 exy = p78 + p910, exz = p1112 + p1314, eyz = p1516 + p1718;
    const V2 s16 = (ax + ay) + az, s718 = (exy + exz) + eyz;
    const V2 m1 = fma2(-30.0f, f[0], fma2(8.0f, s718, -11.0f * s16));
    const V2 m2 = fma2(12.0f, f[0], fma2(-4.0f, s16, s718));
    const V2 m4 = fma2(-4.0f, d12, (q78 + q910) + (q1112 + q1314));
    const V2 m6 = fma2(-4.0f, d34, (q78 - q910) + (q1516 + q1718));
    const V2 m8 = fma2(-4.0f, d56, (q1112 - q1314) + (q1516 - q1718));
    const V2 exyz = exy + exz;
    const V2 ayz = ay + az;
    const V2 m9 = fma2(2.0f, ax, fma2(-2.0f, eyz, exyz - ayz));
    const V2 m10 = fma2(-4.0f, ax, fma2(2.0f, ayz, fma2(-2.0f, eyz, exyz)));
    const V2 m11 = (ay - az) + (exy - exz);
    const V2 m12 = fma2(2.0f, az - ay, exy - exz);
    const V2 m13 = p78 - p910, m14 = p1516 - p1718, m15 = p1112 - p1314;
    const V2 m16 = (q78 + q910) - (q1112 + q1314);
    const V2 m17 = (q910 - q78) + (q1516 + q1718);
    const V2 m18 = (q1112 - q1314) - (q1516 - q1718);
    // equilibria (deviation form) and sources
    const V2 uxx = ux * ux, uyy = uy * uy, uzz = uz * uz;
    const V2 u2 = (uxx + uyy) + uzz;
    const V2 rhou2 = rho * u2;
    const V2 uF = fma2(ux, Fx, fma2(uy, Fy, uz * Fz));
    const V2 e_eq = fma2(19.0f, rhou2, -11.0f * drho);
    const V2 eps_eq = fma2(-5.5f, rhou2, 3.0f * drho);
    const V2 a1 = fma2(k.k3e, X, fma2(k.k2e, uF, k.k1e * (m1 - e_eq)));
    const V2 a2 = fma2(k.k3p, X, fma2(k.k2p, uF, k.k1p * (m2 - eps_eq)));
    const V2 a4 = fma2(k.kq2, Fx, k.kq1 * fma2(2.0f / 3.0f, rho * ux, m4));
    const V2 a6 = fma2(k.kq2, Fy, k.kq1 * fma2(2.0f / 3.0f, rho * uy, m6));
    const V2 a8 = fma2(k.kq2, Fz, k.kq1 * fma2(2.0f / 3.0f, rho * uz, m8));
    const V2 p3xx = rho * fma2(3.0f, uxx, -u2);
    const V2 uyFy = uy * Fy, uzFz = uz * Fz;
    const V2 S3xx = 2.0f * fma2(2.0f * ux, Fx, -(uyFy + uzFz));
    const V2 a9 = fma2(k.kh9, S3xx, k.kn9 * (m9 - p3xx));
    const V2 a10 = fma2(k.kh10, S3xx, k.kp10 * fma2(0.5f, p3xx, m10));
    const V2 pww = rho * (uyy - uzz);
    const V2 Sww = 2.0f * (uyFy - uzFz);
    const V2 a11 = fma2(k.kh11, Sww, k.kn11 * (m11 - pww));
    const V2 a12 = fma2(k.kh12, Sww, k.kp12 * fma2(0.5f, pww, m12));
    const V2 a13 = fma2(k.kh13, fma2(ux, Fy, uy * Fx), k.kn13 * (m13 - rho * (ux * uy)));
    const V2 a14 = fma2(k.kh13, fma2(uy, Fz, uz * Fy), k.kn13 * (m14 - rho * (uy * uz)));
    const V2 a15 = fma2(k.kh13, fma2(ux, Fz, uz * Fx), k.kn13 * (m15 - rho * (ux * uz)));
    const V2 a16 = k.km * m16, a17 = k.km * m17, a18 = k.km * m18;
    const V2 a3 = 0.1f * Fx, a5 = 0.1f * Fy, a7 = 0.1f * Fz;
    // f += M^T diag(1/|row|^2) (m* - m), columns of M per velocity
    f[0] = fma2(-30.0f, a1, fma2(12.0f, a2, f[0]));
    const V2 axis = fma2(-11.0f, a1, -4.0f * a2);
    const V2 a910 = fma2(-2.0f, a10, a9);                       // a9 - 2 a10
    const V2 axx = fma2(2.0f, a910, axis);                      // axis + 2 a9 - 4 a10
    const V2 r34 = fma2(-4.0f, a4, a3), r56 = fma2(-4.0f, a6, a5), r78 = fma2(-4.0f, a8, a7);
    f[1] = f[1] + (axx + r34);
    f[2] = f[2] + (axx - r34);
    const V2 a1112 = fma2(-2.0f, a12, a11);                     // a11 - 2 a12
    const V2 ayy = (axis - a910) + a1112;
    const V2 azz = (axis - a910) - a1112;
    f[3] = f[3] + (ayy + r56);
    f[4] = f[4] + (ayy - r56);
    f[5] = f[5] + (azz + r78);
    f[6] = f[6] + (azz - r78);
    const V2 edge = fma2(8.0f, a1, a2);
    const V2 b910 = a9 + a10, b1112 = a11 + a12;
    const V2 exy0 = (edge + b910) + b1112, exz0 = (edge + b910) - b1112;
    const V2 eyz0 = fma2(-2.0f, b910, edge);
    const V2 t34 = a3 + a4, t56 = a5 + a6, t78 = a7 + a8;
    const V2 g1 = t34 + t56, g2 = t34 - t56;
    const V2 h1 = a16 - a17, h2 = a16 + a17;
    f[7] = f[7] + ((exy0 + a13) + (g1 + h1));
    f[8] = f[8] + ((exy0 + a13) - (g1 + h1));
    f[9] = f[9] + ((exy0 - a13) + (g2 + h2));
    f[10] = f[10] + ((exy0 - a13) - (g2 + h2));
    const V2 g3 = t34 + t78, g4 = t34 - t78;
    const V2 h3 = a18 - a16, h4 = a16 + a18;
    f[11] = f[11] + ((exz0 + a15) + (g3 + h3));
    f[12] = f[12] + ((exz0 + a15) - (g3 + h3));
    f[13] = f[13] + ((exz0 - a15) + (g4 - h4));
    f[14] = f[14] + ((exz0 - a15) - (g4 - h4));
    const V2 g5 = t56 + t78, g6 = t56 - t78;
    const V2 h5 = a17 - a18, h6 = a17 + a18;
    f[15] = f[15] + ((eyz0 + a14) + (g5 + h5));
    f[16] = f[16] + ((eyz0 + a14) - (g5 + h5));
    f[17] = f[17] + ((eyz0 - a14) + (g6 + h6));
    f[18] = f[18] + ((eyz0 - a14) - (g6 + h6));
}

template <int TX, int TY>
struct ZPSmem {
    static constexpr int YX = TX + 6, YY = TY + 6;   // type planes (3-node xy halo)
    static constexpr int RX = TX + 4, RY = TY + 4;   // density planes (2-node xy halo)
    static constexpr int PX = TX + 2, PY = TY + 2;   // psi planes (1-node xy halo)
    float f[LBMWET_ZP_REPULL ? 1 : 4][19][LBMWET_ZP_REPULL ? 1 : TY * TX];
    float rho[4][RY * RX];
    float psi[8][PY * PX];
    uint8_t type[8][YY * YX];
    short wq[4][PY * PX];
    int nw[4];
};

// SF: the solid-fluid interaction scheme (Eq. 8) in a chunk holding solids, compiled as its own
// body so that the adhesion force adds no registers to the other schemes' bodies
template <bool SOLID, bool SF = false>
__device__ __forceinline__ void zpair_chunk(const float* __restrict__ fin, float* __restrict__ fout, const Geo& g,
                                            const Phys<float>& ph, const Rates3P& kr, int x0, int y0, int zb,
                                            unsigned* err, ZPSmem<ZTX, ZTY>& sm) {
    using L = D3Q19;
    constexpr int Q = 19, TX = ZTX, TY = ZTY, NT = TX * TY;
    using Sm = ZPSmem<TX, TY>;
    constexpr int YX = Sm::YX, YY = Sm::YY, RX = Sm::RX, RY = Sm::RY, PX = Sm::PX, PY = Sm::PY;
    const int nx = g.nx, ny = g.ny, nz = g.nz, N = g.N, nxy = nx * ny;
    const int ze = min(zb + ZCH, nz);
    const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * TX + lx;
    const bool small = nx < TX + 8 || ny < TY + 8 || nz < 8;
    auto wx = [&](int v) { return small ? wrap_full(v, nx) : wrap1(v, nx); };
    auto wy = [&](int v) { return small ? wrap_full(v, ny) : wrap1(v, ny); };
    auto wz = [&](int v) { return small ? wrap_full(v, nz) : wrap1(v, nz); };

    auto load_types = [&](int z) {
        if constexpr (SOLID) {
            uint8_t* dst = sm.type[z & 7];
            const int gz = wz(z);
            for (int i = tid; i < YX * YY; i += NT) dst[i] = g.type[gz * nxy + wy(y0 + i / YX - 3) * nx + wx(x0 + i % YX - 3)];
        }
    };
    auto type_at = [&](int z, int ti) -> uint8_t {
        if constexpr (!SOLID) return uint8_t(T_BULK);
        return sm.type[z & 7][ti];
    };
    // sources of node (gx, gy, gz) of plane z (type cell ti): sink(a, pointer)
    auto pull_src = [&](auto&& sink, int gx, int gy, int gz, int z, int ti, uint8_t self) {
        const int cx[3] = {wrap1(gx - 1, nx), gx, wrap1(gx + 1, nx)};
        const int ry[3] = {wrap1(gy - 1, ny) * nx, gy * nx, wrap1(gy + 1, ny) * nx};
        const int pz[3] = {wrap1(gz - 1, nz) * nxy, gz * nxy, wrap1(gz + 1, nz) * nxy};
        if (!SOLID || (self & T_BULK)) {
#pragma unroll
            for (int a = 0; a < Q; ++a)
                sink(a, fin + (a * N + pz[1 - L::ez(a)] + ry[1 - L::ey(a)] + cx[1 - L::ex(a)]));
        } else {
            const uint8_t* tm = sm.type[(z - 1) & 7];
            const uint8_t* t0 = sm.type[z & 7];
            const uint8_t* tp = sm.type[(z + 1) & 7];
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
                const uint8_t* tz = ez > 0 ? tm : (ez < 0 ? tp : t0);   // upstream plane is z - ez
                const bool bb = (tz[ti - ex - ey * YX] & T_SOLID) != 0;
                sink(a, fin + (bb ? L::opp(a) * N + pz[1] + ry[1] + cx[1] : a * N + pz[1 - ez] + ry[1 - ey] + cx[1 - ex]));
            }
        }
    };
    // pull both planes (zl, zl + 1) of the xy cell (hx, hy) of the density plane; f0/f1: keep the
    // distributions of the own cell (index own) in the ring
    auto do_pair = [&](int zl, int hx, int hy, bool want_psi, int own, bool keep0, bool keep1) {
        const int gx = wx(x0 + hx - 2), gy = wy(y0 + hy - 2);
        const int ti = (hy + 1) * YX + hx + 1;
        const uint8_t t0 = type_at(zl, ti), t1 = type_at(zl + 1, ti);
        const bool fl0 = !(t0 & T_SOLID), fl1 = !(t1 & T_SOLID);
        V2 h[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) h[a] = bc(0.0f);
        if (fl0) pull_src([&](int a, const float* src) { h[a].v.x = *src; }, gx, gy, wz(zl), zl, ti, t0);
        if (fl1) pull_src([&](int a, const float* src) { h[a].v.y = *src; }, gx, gy, wz(zl + 1), zl + 1, ti, t1);
        V2 d = h[0];
#pragma unroll
        for (int a = 1; a < Q; ++a) d = d + h[a];
        const V2 rho = bc(ph.rho_ref) + d;
        if constexpr (!LBMWET_ZP_REPULL) {
            if (own >= 0) {
                if (keep0) {
#pragma unroll
                    for (int a = 0; a < Q; ++a) sm.f[zl & 3][a][own] = h[a].v.x;
                }
                if (keep1) {
#pragma unroll
                    for (int a = 0; a < Q; ++a) sm.f[(zl + 1) & 3][a][own] = h[a].v.y;
                }
            }
        }
        if constexpr (SOLID) {   // densities are read only by Eq. 17
            const int ri = hy * RX + hx;
            sm.rho[zl & 3][ri] = fl0 ? rho.v.x : 0.0f;
            sm.rho[(zl + 1) & 3][ri] = fl1 ? rho.v.y : 0.0f;
        }
        if (want_psi) {
            const int pi = (hy - 1) * PX + hx - 1;
            const V2 ps = psi2(rho, ph, fl0, fl1, err);
            sm.psi[zl & 7][pi] = fl0 ? ps.v.x : 0.0f;
            sm.psi[(zl + 1) & 7][pi] = fl1 ? ps.v.y : 0.0f;
            if (SOLID && (t0 & T_WALL)) sm.wq[zl & 3][atomicAdd(&sm.nw[zl & 3], 1)] = short(pi);
            if (SOLID && (t1 & T_WALL)) sm.wq[(zl + 1) & 3][atomicAdd(&sm.nw[(zl + 1) & 3], 1)] = short(pi);
        }
    };

    // prologue: type planes zb - 3 .. zb, empty wall queues of the first lead pair
    for (int z = zb - 3; z <= zb; ++z) load_types(z);
    if (tid == 0) sm.nw[(zb - 2) & 3] = sm.nw[(zb - 1) & 3] = 0;
    __syncthreads();

    for (int zl = zb - 2; zl <= ze + 1; zl += 2) {
        // A. the lead pair: own cells, the 1-node xy halo ring, the 2-node ring near solids.  One
        // loop over the thread's cells keeps a single copy of the pull code in the kernel.
        using Ring1 = Shell<PX, PY, 1, 2>;
        using Ring2 = Shell<RX, RY, 1, 2>;
        constexpr int N1 = (Ring1::COUNT + NT - 1) / NT, N2 = SOLID ? (Ring2::COUNT + NT - 1) / NT : 0;
#pragma unroll 1
        for (int c = 0; c < 1 + N1 + N2; ++c) {
            int hx, hy, own = -1;
            bool want_psi = true;
            if (c == 0) {
                hx = lx + 2;
                hy = ly + 2;
                own = tid;
            } else if (c <= N1) {
                const int k = tid + (c - 1) * NT;
                if (k >= Ring1::COUNT) continue;
                int px, py, pz;
                Ring1::cell(k, px, py, pz);
                hx = px + 1;
                hy = py + 1;
            } else {
                const int k = tid + (c - 1 - N1) * NT;
                if (k >= Ring2::COUNT) continue;
                int pz;
                Ring2::cell(k, hx, hy, pz);
                want_psi = false;
            }
            do_pair(zl, hx, hy, want_psi, own, own >= 0 && zl >= zb && zl < ze, own >= 0 && zl + 1 >= zb && zl + 1 < ze);
        }
        __syncthreads();

        // B. wall cells of planes zl - 1 and zl
        if constexpr (SOLID) {
            bool any = false;
            for (int zw = zl - 1; zw <= zl; ++zw) {
                const int nwb = sm.nw[zw & 3];
                // (the solid-fluid interaction scheme keeps psi = 0 on solids)
                if (zw < zb - 1 || zw > ze || nwb == 0 || ph.wall_kind == 2) continue;
                any = true;
                const short* q = sm.wq[zw & 3];
                for (int k = tid; k < nwb; k += NT) {
                    const int i = q[k];
                    const int px = i % PX, py = i / PX;
                    const int rc = (py + 1) * RX + px + 1, tc = (py + 2) * YX + px + 2;
                    float rw;
                    if (ph.wall_kind == 1) {
                        rw = ph.wall_param;
                    } else {
                        // Eq. 17: weighted mean of the fluid neighbours' densities
                        float num = 0.0f, den = 0.0f;
#pragma unroll
                        for (int a = 1; a < Q; ++a) {
                            const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
                            if (!(sm.type[(zw + ez) & 7][tc + ex + ey * YX] & T_SOLID)) {
                                num += float(L::wf(a)) * sm.rho[(zw + ez) & 3][rc + ex + ey * RX];
                                den += float(L::wf(a));
                            }
                        }
                        const float rho_ave = cdiv(num, den);
                        const float kap = g.kappa_w
                                              ? float(g.kappa_w[g.wall_id[wz(zw) * nxy + wy(y0 + py - 1) * nx + wx(x0 + px - 1)]])
                                              : float(g.kappa);
                        // Eq. 16 (kappa >= 0: phi = 1 + kappa; kappa < 0: drho = -kappa) and the limiter
                        const float raw = (kap >= 0.0f) ? (1.0f + kap) * rho_ave : rho_ave + kap;
                        rw = raw > ph.rho_l ? ph.rho_l : raw;
                        rw = rw < ph.rho_g ? ph.rho_g : rw;
                    }
                    sm.psi[zw & 7][i] = psi2(bc(rw), ph, true, false, err).v.x;
                }
            }
            if (any) __syncthreads();
        }

        // C. collide planes zl - 2 and zl - 1
        const int zc = zl - 2;
        const bool va0 = zc >= zb && zc < ze, va1 = zc + 1 >= zb && zc + 1 < ze;
        if ((va0 || va1) && x0 + lx < nx && y0 + ly < ny) {
            const int ti = (ly + 3) * YX + lx + 3;
            const bool fl0 = va0 && !(type_at(zc, ti) & T_SOLID), fl1 = va1 && !(type_at(zc + 1, ti) & T_SOLID);
            if (fl0 || fl1) {
                V2 f[Q];
#if LBMWET_ZP_REPULL
#pragma unroll
                for (int a = 0; a < Q; ++a) f[a] = bc(0.0f);
                {
                    const int gx = x0 + lx, gy = y0 + ly;
                    if (fl0) pull_src([&](int a, const float* src) { f[a].v.x = *src; }, gx, gy, zc, zc, ti, type_at(zc, ti));
                    if (fl1)
                        pull_src([&](int a, const float* src) { f[a].v.y = *src; }, gx, gy, zc + 1, zc + 1, ti,
                                 type_at(zc + 1, ti));
                }
#else
#pragma unroll
                for (int a = 0; a < Q; ++a) f[a] = mk(sm.f[zc & 3][a][tid], sm.f[(zc + 1) & 3][a][tid]);
#endif
                const int pc = (ly + 1) * PX + lx + 1;
                auto psi_at = [&](int dz, int off) {
                    return mk(sm.psi[(zc + dz) & 7][pc + off], sm.psi[(zc + 1 + dz) & 7][pc + off]);
                };
                const V2 psi_c = psi_at(0, 0);
                // sum_a w_a psi(x + e_a) e_a over opposite pairs: w_a e_a (psi(x + e_a) - psi(x - e_a))
                V2 sx = bc(0.0f), sy = bc(0.0f), sz = bc(0.0f);
#pragma unroll
                for (int a = 1; a < Q; ++a) {
                    if (L::opp(a) < a) continue;
                    const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
                    const int off = ex + ey * PX;
                    const V2 wd = float(L::wf(a)) * (psi_at(ez, off) - psi_at(-ez, -off));
                    if (ex) sx = ex > 0 ? sx + wd : sx - wd;
                    if (ey) sy = ey > 0 ? sy + wd : sy - wd;
                    if (ez) sz = ez > 0 ? sz + wd : sz - wd;
                }
                // Eq. 5
                const V2 gpsi = (-ph.G) * psi_c;
                const V2 Fmx = gpsi * sx, Fmy = gpsi * sy, Fmz = gpsi * sz;
                V2 Fx = Fmx + bc(ph.fx), Fy = Fmy + bc(ph.fy), Fz = Fmz + bc(ph.fz);
                V2 drho = f[0];
#pragma unroll
                for (int a = 1; a < Q; ++a) drho = drho + f[a];
                const V2 jx = ((f[1] - f[2]) + (f[7] - f[8])) + ((f[9] - f[10]) + (f[11] - f[12])) + (f[13] - f[14]);
                const V2 jy = ((f[3] - f[4]) + (f[7] - f[8])) + ((f[10] - f[9]) + (f[15] - f[16])) + (f[17] - f[18]);
                const V2 jz = ((f[5] - f[6]) + (f[11] - f[12])) + ((f[14] - f[13]) + (f[15] - f[16])) + (f[18] - f[17]);
                const V2 rho = bc(ph.rho_ref) + drho;
                // Eq. 8 (solid-fluid interaction scheme): F_ads = -G_w rho sum_a w_a s(x + e_a) e_a
                if constexpr (SOLID && SF) {
                    {
                        float ax0 = 0.0f, ay0 = 0.0f, az0 = 0.0f, ax1 = 0.0f, ay1 = 0.0f, az1 = 0.0f;
#pragma unroll
                        for (int a = 1; a < Q; ++a) {
                            const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a), off = ex + ey * YX;
                            const float w = float(L::wf(a));
                            if (sm.type[(zc + ez) & 7][ti + off] & T_SOLID) {
                                if (ex) ax0 += w * float(ex);
                                if (ey) ay0 += w * float(ey);
                                if (ez) az0 += w * float(ez);
                            }
                            if (sm.type[(zc + 1 + ez) & 7][ti + off] & T_SOLID) {
                                if (ex) ax1 += w * float(ex);
                                if (ey) ay1 += w * float(ey);
                                if (ez) az1 += w * float(ez);
                            }
                        }
                        const V2 gr = (-ph.wall_param) * rho;
                        Fx = (Fmx + gr * mk(ax0, ax1)) + bc(ph.fx);
                        Fy = (Fmy + gr * mk(ay0, ay1)) + bc(ph.fy);
                        Fz = (Fmz + gr * mk(az0, az1)) + bc(ph.fz);
                    }
                }
                if ((fl0 && !(rho.v.x > 0.0f)) || (fl1 && !(rho.v.y > 0.0f))) atomicOr(err, ERR_RHO);
                // Eq. 4: rho u = sum e f + F/2
                const V2 inv = div2(bc(1.0f), rho);
                const V2 ux = fma2(0.5f, Fx, jx) * inv, uy = fma2(0.5f, Fy, jy) * inv, uz = fma2(0.5f, Fz, jz) * inv;
                const V2 X = div2(fma2(Fmx, Fmx, fma2(Fmy, Fmy, Fmz * Fmz)), psi_c * psi_c);
                collide3p(f, drho, rho, ux, uy, uz, Fx, Fy, Fz, X, kr);
                const int gi = zc * nxy + (y0 + ly) * nx + x0 + lx;
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    if (fl0) fout[a * N + gi] = f[a].v.x;
                    if (fl1) fout[a * N + gi + nxy] = f[a].v.y;
                }
            }
        }
        // type planes of the next lead pair's pulls; empty its wall queues
        load_types(zl + 3);
        load_types(zl + 4);
        if (tid == 0) sm.nw[(zl + 2) & 3] = sm.nw[(zl + 3) & 3] = 0;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(ZTX* ZTY, LBMWET_ZP_MINB)
    zpair_step(const float* __restrict__ fin, float* __restrict__ fout, Geo g, Phys<float> ph, Rates3P kr,
               unsigned* err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    ZPSmem<ZTX, ZTY>& sm = *reinterpret_cast<ZPSmem<ZTX, ZTY>*>(smem_raw);
    const int tile = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const bool solid = g.tile_solid ? g.tile_solid[tile] != 0 : true;
    if (solid && ph.wall_kind == 2)
        zpair_chunk<true, true>(fin, fout, g, ph, kr, blockIdx.x * ZTX, blockIdx.y * ZTY, blockIdx.z * ZCH, err, sm);
    else if (solid)
        zpair_chunk<true>(fin, fout, g, ph, kr, blockIdx.x * ZTX, blockIdx.y * ZTY, blockIdx.z * ZCH, err, sm);
    else
        zpair_chunk<false>(fin, fout, g, ph, kr, blockIdx.x * ZTX, blockIdx.y * ZTY, blockIdx.z * ZCH, err, sm);
}


// ---------------------------------------------------------------------------------------------
// TMA-staged z-march (the default FP32 D3Q19 step).  A CTA of 32 x 4 threads owns a 32 x 8 column
// of a 32-plane chunk; thread (lx, ly) carries the cells (x0 + lx, y0 + ly) and (x0 + lx, y0 + ly + 4)
// as the two lanes of its FP32x2 values.  The chunk marches plane by plane through shared memory:
//   * every lead plane zl is staged by TMA: for each direction a, the box of f*_a on plane zl - ez(a)
//     over x0 - 4 .. x0 + 35 (x starts on a 16-byte boundary) and y0 - 2 .. y0 + 9 (y0 - 3 .. y0 + 10
//     in chunks holding solids, whose walls need densities two nodes out), so that the pull (Eq. 3)
//     of any cell of the column and of its halo reads its 19 values at constant offsets from one
//     shared-memory address; two stages on two mbarriers keep the next plane's 19 boxes in flight
//     while the current one is used;
//   * where the box crosses a periodic edge of the grid (TMA cannot wrap), the out-of-range columns
//     and rows it needs are loaded by the threads and written over the box's zero fill after its
//     wait (one plane ahead, from registers, in chunks without solids);
//   * phase A of lead plane zl: rho (Eq. 4) and psi (Eq. 6) of the column and its halo into rings of
//     planes; the column's own pulled values stay in registers;
//   * chunks holding solids: bounce-back (Fig. 3) replaces a pulled value whose source is solid by
//     the cell's own post-collision value in the opposite direction (from this plane's boxes when
//     e_z = 0, from the next plane's when e_z = -1, plain loads otherwise), and phase B
//     gives the wall cells of plane zl - 1 their virtual density (Eqs. 16-17 with the limiter, or the
//     constant one) from the densities of planes zl - 2 .. zl;
//   * phase C collides plane zl - 1 (zl - 2 in chunks holding solids) once its psi neighbours are
//     final: F_m (Eq. 5; plus Eq. 8 with the solid-fluid interaction scheme), u (Eq. 4), the MRT
//     collision with the consistency source (Eqs. 2, 7), coalesced stores.
// Ragged edge columns and small grids take the z-pair march on the column's two 32 x 4 halves.
// ---------------------------------------------------------------------------------------------
constexpr int TTX = 32, TTY = 8, TCH = ZCH;
static_assert(TTX == ZTX && TTY == 2 * ZTY, "a TMA column is two z-pair columns");
constexpr int TBX = TTX + 8;                  // box columns: x0 - 4 .. x0 + 35
constexpr int TBY = TTY + 4;                  // box rows: y0 - 2 .. y0 + 9
constexpr int TBSLOT = TBY * TBX;             // floats per direction and stage, chunks without solids (480)
static_assert((TBSLOT * 4) % 128 == 0, "every direction's box starts on a 128-byte boundary");
constexpr int TPX = TTX + 2, TPY = TTY + 2;   // psi window: the column + 1-node ring (box cols 3..36)
constexpr int TRX = TTX + 4, TRY = TTY + 4;   // density window (solid chunks): + 2-node ring
constexpr int TYX = TTX + 6, TYY = TTY + 6;   // node-type window (solid chunks): + 3-node ring
constexpr int TRING = 2 * TPX + 2 * (TPY - 2);                 // 84 cells of the 1-node ring
constexpr int TRING2 = 2 * TRX + 2 * (TRY - 2);                // 92 cells of the 2-node ring
constexpr int TTYPES = TYX * TYY;                              // 532 type cells per plane
constexpr unsigned TBYTES_BULK = 19u * TBY * TBX * 4u;
// the directions with ey = +1 (3, 7, 10, 15, 17) and ey = -1 (4, 8, 9, 16, 18), five bits each
constexpr unsigned XROW_UP = 3u | 7u << 5 | 10u << 10 | 15u << 15 | 17u << 20;
constexpr unsigned XROW_DN = 4u | 8u << 5 | 9u << 10 | 16u << 15 | 18u << 20;
__host__ __device__ constexpr int xrow_slot(int a) {   // position of a among its five directions
    return a == 3 || a == 4 ? 0 : a == 7 || a == 8 ? 1 : a == 10 || a == 9 ? 2 : a == 15 || a == 16 ? 3 : 4;
}

// Shared memory of the two kinds of chunk, overlaid: both keep two planes of boxes in flight (the
// same 12-row boxes); chunks holding solids add node types, a density ring and the two rows beyond
// the box that their 2-node density ring pulls from.  The CTA stays under 97 KB, so that two CTAs
// per SM leave the L1 at least 60 KB, which the loads of the periodic-edge patches need (with 107 KB
// CTAs the 256^3 step ran at 0.65 of the HBM roofline instead of 0.78).
struct ZTBulk {
    float stage[2][19][TBSLOT];
    float psi[4][TPY * TPX];
};
struct ZTSolid {
    float stage[2][19][TBSLOT];
    float xrow[2][2][5][TBX];   // by plane parity: row y0 - 3 (directions with ey = 1), row y0 + 10 (ey = -1)
    float psi[5][TPY * TPX];
    float rho[4][TRY * TRX];
    uint8_t type[8][TTYPES];
};
struct ZTSmem {
    union {
        ZTBulk b;
        ZTSolid s;
    };
    uint64_t bar[2];
};
constexpr size_t ZT_SMEM = sizeof(ZTSmem) > sizeof(ZPSmem<ZTX, ZTY>) ? sizeof(ZTSmem) : sizeof(ZPSmem<ZTX, ZTY>);

// Polls of an mbarrier before a wait gives up (about one second at ~3.8 us per unsuccessful poll).
constexpr unsigned ZT_POLL_LIMIT = 1u << 18;

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_box3(void* dst, const void* tmap, int cx, int cy, int cz, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(cx), "r"(cy), "r"(cz), "r"(smem_u32(bar))
        : "memory");
}

// z component of D3Q19 velocity a for a run-time index (bit tables instead of an indexed array)
__device__ __forceinline__ int ez_rt(int a) {
    constexpr unsigned PLUS = (1u << 5) | (1u << 11) | (1u << 14) | (1u << 15) | (1u << 18);
    constexpr unsigned MINUS = (1u << 6) | (1u << 12) | (1u << 13) | (1u << 16) | (1u << 17);
    return int((PLUS >> a) & 1u) - int((MINUS >> a) & 1u);
}

// Out-of-range part of a box's used window (rows [rw0, rw1), columns [cw0, cw1) of a box whose
// cell (0, 0) is the grid node (bx0, by0)): rows [r_lo, r_lo + nr) and columns [c_lo, c_lo + nc),
// each on one side at most (the grid is wider than the window).
struct OutBand {
    int r_lo, nr, c_lo, nc, rin_lo, rin, cells, wc;
    __device__ OutBand(int bx0, int by0, int nx, int ny, int rw0, int rw1, int cw0, int cw1) {
        r_lo = rw0;
        nr = 0;
        if (by0 + rw0 < 0) {
            nr = -(by0 + rw0);
        } else if (by0 + rw1 > ny) {
            nr = by0 + rw1 - ny;
            r_lo = rw1 - nr;
        }
        c_lo = cw0;
        nc = 0;
        if (bx0 + cw0 < 0) {
            nc = -(bx0 + cw0);
        } else if (bx0 + cw1 > nx) {
            nc = bx0 + cw1 - nx;
            c_lo = cw1 - nc;
        }
        wc = cw1 - cw0;
        rin = (rw1 - rw0) - nr;
        rin_lo = r_lo == rw0 ? rw0 + nr : rw0;
        cells = nr * wc + nc * rin;
    }
    // the k-th out-of-range cell (k < cells): whole rows first, then the columns of the other rows
    __device__ void cell(int k, int cw0, int& r, int& c) const {
        if (k < nr * wc) {
            r = r_lo + k / wc;
            c = cw0 + k % wc;
        } else {
            k -= nr * wc;
            c = c_lo + k / rin;
            r = rin_lo + k % rin;
        }
    }
};

// A chunk without solids within 3 nodes: no walls, no bounce-back; lag 1 between the lead plane
// and the collided plane.
__device__ __forceinline__ void ztma_chunk_bulk(const float* __restrict__ fin, float* __restrict__ fout,
                                                const void* tmap, const Geo& g, const Phys<float>& ph,
                                                const Rates3P& kr, int x0, int y0, int zb, int ze, unsigned* err,
                                                ZTBulk& S, uint64_t* bar) {
    using L = D3Q19;
    constexpr int Q = 19;
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
    const long long fs = g.fs;
    const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * TTX + lx;
    const int zlo = zb - 1, zhi = ze;   // lead planes zlo .. zhi, collided planes zb .. ze - 1
    const int nlead = zhi - zlo + 1;

    // out-of-range cells of the used window (rows 0 .. 11, columns 2 .. 37): at most
    // 2 * 36 + 2 * 10 = 92 < 128, one per thread, prefetched one plane ahead
    const OutBand ob_(x0 - 4, y0 - 2, nx, ny, 0, TBY, 2, TBX - 2);
    const bool edge = ob_.cells > 0;
    int fr = 0, fcl = 0, fsrc = 0;
    const bool fixer = tid < ob_.cells;
    if (fixer) {
        ob_.cell(tid, 2, fr, fcl);
        fsrc = wrap_full(y0 - 2 + fr, ny) * nx + wrap_full(x0 - 4 + fcl, nx);
    }
    float fix[Q];
    auto issue = [&](int zl, int s) {   // thread 0: the 19 boxes of lead plane zl into stage s
        fence_proxy_async();
        mbar_expect_tx(&bar[s], TBYTES_BULK);
#pragma unroll
        for (int a = 0; a < Q; ++a) tma_box3(S.stage[s][a], tmap, x0 - 4, y0 - 2, a * nz + wrap1(zl - L::ez(a), nz), &bar[s]);
    };

    if (tid == 0) {
        issue(zlo, 0);
        issue(zlo + 1, 1);
    }
    if (edge && fixer) {
#pragma unroll
        for (int a = 0; a < Q; ++a) fix[a] = fin[a * fs + (long long)wrap1(zlo - L::ez(a), nz) * nxy + fsrc];
    }

    // own cells in box and psi-window coordinates
    const int ob = (ly + 2) * TBX + lx + 4;
    const int pc = (ly + 1) * TPX + lx + 1;
    // this thread's halo-ring cell (threads 0 .. 83)
    int rb = 0, rp = 0;
    const bool ringer = tid < TRING;
    if (ringer) {
        int px, py, pz;
        Shell<TPX, TPY, 1, 2>::cell(tid, px, py, pz);
        rb = (py + 1) * TBX + px + 3;
        rp = py * TPX + px;
    }

    V2 fprev[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) fprev[a] = bc(0.0f);

#pragma unroll 1
    for (int i = 0; i < nlead; ++i) {
        const int zl = zlo + i, s = i & 1;
        if (!mbar_wait(&bar[s], unsigned(i >> 1) & 1u, ZT_POLL_LIMIT)) atomicOr(err, ERR_TIMEOUT);
        float* st = S.stage[s][0];
        if (edge) {
            if (fixer) {
#pragma unroll
                for (int a = 0; a < Q; ++a) st[a * TBSLOT + fr * TBX + fcl] = fix[a];
                fence_proxy_async();
            }
            if (fixer && zl + 1 <= zhi) {
#pragma unroll
                for (int a = 0; a < Q; ++a)
                    fix[a] = fin[a * fs + (long long)wrap1(zl + 1 - L::ez(a), nz) * nxy + fsrc];
            }
            __syncthreads();
        }
        // A. rho and psi of lead plane zl: the column (own values kept) and its halo ring
        V2 fcur[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const int off = a * TBSLOT - L::ey(a) * TBX - L::ex(a);
            fcur[a] = mk(st[ob + off], st[ob + 4 * TBX + off]);
        }
        {
            V2 d = fcur[0];
#pragma unroll
            for (int a = 1; a < Q; ++a) d = d + fcur[a];
            const V2 ps = psi2(bc(ph.rho_ref) + d, ph, true, true, err);
            float* pp = S.psi[zl & 3];
            pp[pc] = ps.v.x;
            pp[pc + 4 * TPX] = ps.v.y;
        }
        if (ringer) {
            float d = 0.0f;
#pragma unroll
            for (int a = 0; a < Q; ++a) d += st[rb + a * TBSLOT - L::ey(a) * TBX - L::ex(a)];
            S.psi[zl & 3][rp] = psi_checked(ph.rho_ref + d, ph, err);
        }
        __syncthreads();
        if (tid == 0 && zl + 2 <= zhi) issue(zl + 2, s);

        // C. collide plane zc = zl - 1
        const int zc = zl - 1;
        if (zc >= zb) {
            V2(&f)[Q] = fprev;
            auto psi_at = [&](int dz, int off) {
                const float* pp = S.psi[(zc + dz) & 3];
                return mk(pp[pc + off], pp[pc + 4 * TPX + off]);
            };
            const V2 psi_c = psi_at(0, 0);
            V2 sx = bc(0.0f), sy = bc(0.0f), sz = bc(0.0f);
#pragma unroll
            for (int a = 1; a < Q; ++a) {
                if (L::opp(a) < a) continue;
                const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
                const int off = ex + ey * TPX;
                const V2 wd = float(L::wf(a)) * (psi_at(ez, off) - psi_at(-ez, -off));
                if (ex) sx = ex > 0 ? sx + wd : sx - wd;
                if (ey) sy = ey > 0 ? sy + wd : sy - wd;
                if (ez) sz = ez > 0 ? sz + wd : sz - wd;
            }
            // Eq. 5
            const V2 gpsi = (-ph.G) * psi_c;
            const V2 Fmx = gpsi * sx, Fmy = gpsi * sy, Fmz = gpsi * sz;
            const V2 Fx = Fmx + bc(ph.fx), Fy = Fmy + bc(ph.fy), Fz = Fmz + bc(ph.fz);
            V2 drho = f[0];
#pragma unroll
            for (int a = 1; a < Q; ++a) drho = drho + f[a];
            const V2 jx = ((f[1] - f[2]) + (f[7] - f[8])) + ((f[9] - f[10]) + (f[11] - f[12])) + (f[13] - f[14]);
            const V2 jy = ((f[3] - f[4]) + (f[7] - f[8])) + ((f[10] - f[9]) + (f[15] - f[16])) + (f[17] - f[18]);
            const V2 jz = ((f[5] - f[6]) + (f[11] - f[12])) + ((f[14] - f[13]) + (f[15] - f[16])) + (f[18] - f[17]);
            const V2 rho = bc(ph.rho_ref) + drho;
            if (!(rho.v.x > 0.0f) || !(rho.v.y > 0.0f)) atomicOr(err, ERR_RHO);
            // Eq. 4: rho u = sum e f + F/2
            const V2 inv = div2(bc(1.0f), rho);
            const V2 ux = fma2(0.5f, Fx, jx) * inv, uy = fma2(0.5f, Fy, jy) * inv, uz = fma2(0.5f, Fz, jz) * inv;
            const V2 X = div2(fma2(Fmx, Fmx, fma2(Fmy, Fmy, Fmz * Fmz)), psi_c * psi_c);
            collide3p(f, drho, rho, ux, uy, uz, Fx, Fy, Fz, X, kr);
            float* o = fout + (long long)zc * nxy + (y0 + ly) * nx + x0 + lx;
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                o[a * fs] = f[a].v.x;
                o[a * fs + 4 * nx] = f[a].v.y;
            }
        }
#pragma unroll
        for (int a = 0; a < Q; ++a) fprev[a] = fcur[a];
    }
}

// A chunk holding solids within 3 nodes: node types of planes zl - 3 .. zl + 2 in a ring, bounce-back
// links, a 2-node density ring for the wall cells' Eq. 17, lag 2 between lead and collided plane.
// Coordinates (rb, c) are those of the box: row rb is grid row y0 - 2 + rb, column c is x0 - 4 + c.
template <bool SF>
__device__ __forceinline__ void ztma_chunk_solid(const float* __restrict__ fin, float* __restrict__ fout,
                                                 const void* tmap, const Geo& g, const Phys<float>& ph,
                                                 const Rates3P& kr, int x0, int y0, int zb, int ze, unsigned* err,
                                                 ZTSolid& S, uint64_t* bar) {
    using L = D3Q19;
    constexpr int Q = 19, NT = TTX * ZTY;
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
    const long long fs = g.fs;
    const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * TTX + lx;
    const int zlo = zb - 2, zhi = ze + 1;   // lead planes; collided planes zb .. ze - 1
    const int nlead = zhi - zlo + 1;
    auto wz = [&](int z) { return wrap1(wrap1(z, nz), nz); };
    auto ps5 = [](int z) { return (z + 10) % 5; };   // psi ring slot (z >= -10)
    // node types of plane z (rows -1 .. 12, columns 1 .. 38 of the box) into ring slot z & 7
    auto type_src = [&](int z, int k) {
        const int tr = k / TYX, tc = k % TYX;
        return g.type[(long long)wz(z) * nxy + wrap1(y0 - 3 + tr, ny) * nx + wrap1(x0 - 3 + tc, nx)];
    };
    // the rows beyond the box that the 2-node ring pulls from (box row -1 for ey = 1, row 12 for
    // ey = -1), columns 1 .. 38: item k < 380 of plane z
    auto xrow_src = [&](int z, int k) {
        const int row = k / 190, rem = k - row * 190, d = rem / 38, col = 1 + rem % 38;
        const int a = int(((row ? XROW_DN : XROW_UP) >> (5 * d)) & 31u);
        return fin[a * fs + (long long)wz(z - ez_rt(a)) * nxy + wrap1(row ? y0 + 10 : y0 - 3, ny) * nx +
                   wrap1(x0 - 4 + col, nx)];
    };
    auto xrow_dst = [&](int z, int k) -> float& {
        const int row = k / 190, rem = k - row * 190, d = rem / 38, col = 1 + rem % 38;
        return S.xrow[z & 1][row][d][col];
    };
    // out-of-range cells of the used window (rows 0 .. 11, columns 1 .. 38), written after each
    // wait from plain loads (chunks holding solids rarely touch the grid's edges)
    const OutBand band(x0 - 4, y0 - 2, nx, ny, 0, TBY, 1, TBX - 1);
    const bool edge = band.cells > 0;
    auto issue = [&](int zl, int s) {   // thread 0: the 19 boxes of lead plane zl into stage s
        fence_proxy_async();
        mbar_expect_tx(&bar[s], TBYTES_BULK);
#pragma unroll
        for (int a = 0; a < Q; ++a) tma_box3(S.stage[s][a], tmap, x0 - 4, y0 - 2, a * nz + wz(zl - L::ez(a)), &bar[s]);
    };
    if (tid == 0) {
        issue(zlo, 0);
        issue(zlo + 1, 1);
    }
    for (int z = zlo - 3; z <= zlo + 1; ++z)
        for (int k = tid; k < TTYPES; k += NT) S.type[z & 7][k] = type_src(z, k);
    for (int k = tid; k < 380; k += NT) xrow_dst(zlo, k) = xrow_src(zlo, k);
    __syncthreads();

    // post-collision value f*_{opp(a)} of box cell (rb, c) on plane z (bounce-back source)
    auto bb_src = [&](int a, int z, int rb, int c) {
        return fin[L::opp(a) * fs + (long long)wz(z) * nxy + wrap1(y0 - 2 + rb, ny) * nx + wrap1(x0 - 4 + c, nx)];
    };
    // pull of a fluid cell (rb, c) of plane zl with its type t; RING2: the cell may lie on box row 0
    // or 11, whose pulls reach the rows beyond the box
    // stn: the other stage (lead plane zl + 1, waited for) or null.  Bounce-back sources f*_abar of the
    // cell's own plane: for e_az = 0 in this stage's box of abar, for e_az = -1 in the next stage's
    // (its box of abar holds plane zl), otherwise plain loads.
    auto pull = [&](auto ring2, const float* st, const float* stn, int zl, int rb, int c, uint8_t t,
                    float (&v)[Q]) {
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const int ey = L::ey(a), sr = rb - ey;
            if (decltype(ring2)::value && ey != 0 && (sr < 0 || sr >= TBY))
                v[a] = S.xrow[zl & 1][sr < 0 ? 0 : 1][xrow_slot(a)][c - L::ex(a)];
            else
                v[a] = st[a * TBSLOT + sr * TBX + c - L::ex(a)];
        }
        if (!(t & T_BULK)) {
#pragma unroll
            for (int a = 1; a < Q; ++a) {
                const uint8_t tu = S.type[(zl - L::ez(a)) & 7][(rb - L::ey(a) + 1) * TYX + c - L::ex(a) - 1];
                if (tu & T_SOLID) {
                    if (L::ez(a) == 0)
                        v[a] = st[L::opp(a) * TBSLOT + rb * TBX + c];
                    else if (L::ez(a) < 0 && stn)
                        v[a] = stn[L::opp(a) * TBSLOT + rb * TBX + c];
                    else
                        v[a] = bb_src(a, zl, rb, c);
                }
            }
        }
    };
    using NoRing2 = std::integral_constant<bool, false>;
    using Ring2 = std::integral_constant<bool, true>;
    const int pc = (ly + 1) * TPX + lx + 1;   // own cell in the psi window
    const int rc = (ly + 2) * TRX + lx + 2;   // own cell in the density window
    const int tcl = (ly + 3) * TYX + lx + 3;  // own cell in the type window
    V2 f1[Q], f2[Q];                          // own values of planes zl - 1 and zl - 2
#pragma unroll
    for (int a = 0; a < Q; ++a) f1[a] = f2[a] = bc(0.0f);
    uint8_t tnext[5];                         // types of plane zl + 2 (this thread's cells)
    float xnext[3];                           // the rows beyond the box of plane zl + 1

#pragma unroll 1
    for (int i = 0; i < nlead; ++i) {
        const int zl = zlo + i, s = i & 1;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const int k = tid + j * NT;
            tnext[j] = k < TTYPES ? type_src(zl + 2, k) : uint8_t(0);
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int k = tid + j * NT;
            xnext[j] = (k < 380 && zl + 1 <= zhi) ? xrow_src(zl + 1, k) : 0.0f;
        }
        if (!mbar_wait(&bar[s], unsigned(i >> 1) & 1u, ZT_POLL_LIMIT)) atomicOr(err, ERR_TIMEOUT);
        float* st = S.stage[s][0];
        if (edge) {
            for (int k = tid; k < band.cells * Q; k += NT) {
                const int a = k / band.cells;
                int rb, c;
                band.cell(k - a * band.cells, 1, rb, c);
                st[a * TBSLOT + rb * TBX + c] =
                    fin[a * fs + (long long)wz(zl - ez_rt(a)) * nxy + wrap1(y0 - 2 + rb, ny) * nx + wrap1(x0 - 4 + c, nx)];
            }
            fence_proxy_async();
            __syncthreads();
        }
        // the next stage (lead plane zl + 1) for bounce-back sources, where it holds them unpatched
        const float* stn = nullptr;
        if (!edge && zl + 1 <= zhi) {
            if (!mbar_wait(&bar[s ^ 1], unsigned((i + 1) >> 1) & 1u, ZT_POLL_LIMIT)) atomicOr(err, ERR_TIMEOUT);
            stn = S.stage[s ^ 1][0];
        }
        // A. densities of the density window, psi of the psi window (fluid cells), own values kept
        const uint8_t* ty = S.type[zl & 7];
        float* rr = S.rho[zl & 3];
        float* pp = S.psi[ps5(zl)];
        V2 fcur[Q];
        {
            float v[Q];
            const uint8_t t0 = ty[tcl], t1 = ty[tcl + 4 * TYX];
            const bool fl0 = !(t0 & T_SOLID), fl1 = !(t1 & T_SOLID);
            float d0 = 0.0f, d1 = 0.0f;
            if (fl0) {
                pull(NoRing2{}, st, stn, zl, ly + 2, lx + 4, t0, v);
#pragma unroll
                for (int a = 0; a < Q; ++a) d0 += v[a];
            } else {
#pragma unroll
                for (int a = 0; a < Q; ++a) v[a] = 0.0f;
            }
#pragma unroll
            for (int a = 0; a < Q; ++a) fcur[a].v.x = v[a];
            if (fl1) {
                pull(NoRing2{}, st, stn, zl, ly + 6, lx + 4, t1, v);
#pragma unroll
                for (int a = 0; a < Q; ++a) d1 += v[a];
            } else {
#pragma unroll
                for (int a = 0; a < Q; ++a) v[a] = 0.0f;
            }
#pragma unroll
            for (int a = 0; a < Q; ++a) fcur[a].v.y = v[a];
            const V2 rho = mk(ph.rho_ref + d0, ph.rho_ref + d1);
            const V2 ps = psi2(rho, ph, fl0, fl1, err);
            rr[rc] = fl0 ? rho.v.x : 0.0f;
            rr[rc + 4 * TRX] = fl1 ? rho.v.y : 0.0f;
            pp[pc] = fl0 ? ps.v.x : 0.0f;
            pp[pc + 4 * TPX] = fl1 ? ps.v.y : 0.0f;
        }
        // halo cells: the 1-node ring (density and psi) and the 2-node ring (density)
        for (int k = tid; k < TRING + TRING2; k += NT) {
            int px, py, pz, rb, c;
            if (k < TRING) {
                Shell<TPX, TPY, 1, 2>::cell(k, px, py, pz);
                rb = py + 1;
                c = px + 3;
            } else {
                Shell<TRX, TRY, 1, 2>::cell(k - TRING, px, py, pz);
                rb = py;
                c = px + 2;
            }
            const uint8_t t = ty[(rb + 1) * TYX + c - 1];
            const bool fl = !(t & T_SOLID);
            float rho = 0.0f;
            if (fl) {
                float v[Q];
                pull(Ring2{}, st, stn, zl, rb, c, t, v);
                float d = 0.0f;
#pragma unroll
                for (int a = 0; a < Q; ++a) d += v[a];
                rho = ph.rho_ref + d;
            }
            rr[rb * TRX + c - 2] = rho;
            if (k < TRING) pp[(rb - 1) * TPX + c - 3] = fl ? psi_checked(rho, ph, err) : 0.0f;
        }
        __syncthreads();
        if (tid == 0 && zl + 2 <= zhi) issue(zl + 2, s);

        // B. wall cells of plane zw = zl - 1: virtual density and its psi (the solid-fluid interaction
        // scheme keeps psi = 0 on solids); node types of plane zl + 2 and the rows beyond the box of
        // plane zl + 1 into their rings
        const int zw = zl - 1;
        if (!SF && zw >= zb - 1) {
            const uint8_t* tw = S.type[zw & 7];
            for (int k = tid; k < TPX * TPY; k += NT) {
                const int c = k % TPX + 3, rb = k / TPX + 1;
                if (!(tw[(rb + 1) * TYX + c - 1] & T_WALL)) continue;
                float rw;
                if (ph.wall_kind == 1) {
                    rw = ph.wall_param;
                } else {
                    // Eq. 17: weighted mean of the fluid neighbours' densities
                    float num = 0.0f, den = 0.0f;
#pragma unroll
                    for (int a = 1; a < Q; ++a) {
                        const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
                        if (!(S.type[(zw + ez) & 7][(rb + ey + 1) * TYX + c + ex - 1] & T_SOLID)) {
                            num += float(L::wf(a)) * S.rho[(zw + ez) & 3][(rb + ey) * TRX + c + ex - 2];
                            den += float(L::wf(a));
                        }
                    }
                    const float rho_ave = cdiv(num, den);
                    const float kap =
                        g.kappa_w ? float(g.kappa_w[g.wall_id[(long long)wz(zw) * nxy + wrap1(y0 - 2 + rb, ny) * nx +
                                                              wrap1(x0 - 4 + c, nx)]])
                                  : float(g.kappa);
                    // Eq. 16 (kappa >= 0: phi = 1 + kappa; kappa < 0: drho = -kappa) and the limiter
                    const float raw = (kap >= 0.0f) ? (1.0f + kap) * rho_ave : rho_ave + kap;
                    rw = raw > ph.rho_l ? ph.rho_l : raw;
                    rw = rw < ph.rho_g ? ph.rho_g : rw;
                }
                S.psi[ps5(zw)][k] = psi_checked(rw, ph, err);
            }
        }
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const int k = tid + j * NT;
            if (k < TTYPES) S.type[(zl + 2) & 7][k] = tnext[j];
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int k = tid + j * NT;
            if (k < 380) xrow_dst(zl + 1, k) = xnext[j];
        }
        __syncthreads();

        // C. collide plane zc = zl - 2
        const int zc = zl - 2;
        if (zc >= zb) {
            const uint8_t* tc = S.type[zc & 7];
            const bool fl0 = !(tc[tcl] & T_SOLID), fl1 = !(tc[tcl + 4 * TYX] & T_SOLID);
            if (fl0 || fl1) {
                V2(&f)[Q] = f2;
                auto psi_at = [&](int dz, int off) {
                    const float* q = S.psi[ps5(zc + dz)];
                    return mk(q[pc + off], q[pc + 4 * TPX + off]);
                };
                const V2 psi_c = psi_at(0, 0);
                V2 sx = bc(0.0f), sy = bc(0.0f), sz = bc(0.0f);
#pragma unroll
                for (int a = 1; a < Q; ++a) {
                    if (L::opp(a) < a) continue;
                    const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
                    const int off = ex + ey * TPX;
                    const V2 wd = float(L::wf(a)) * (psi_at(ez, off) - psi_at(-ez, -off));
                    if (ex) sx = ex > 0 ? sx + wd : sx - wd;
                    if (ey) sy = ey > 0 ? sy + wd : sy - wd;
                    if (ez) sz = ez > 0 ? sz + wd : sz - wd;
                }
                // Eq. 5
                const V2 gpsi = (-ph.G) * psi_c;
                const V2 Fmx = gpsi * sx, Fmy = gpsi * sy, Fmz = gpsi * sz;
                V2 Fx = Fmx + bc(ph.fx), Fy = Fmy + bc(ph.fy), Fz = Fmz + bc(ph.fz);
                V2 drho = f[0];
#pragma unroll
                for (int a = 1; a < Q; ++a) drho = drho + f[a];
                const V2 jx = ((f[1] - f[2]) + (f[7] - f[8])) + ((f[9] - f[10]) + (f[11] - f[12])) + (f[13] - f[14]);
                const V2 jy = ((f[3] - f[4]) + (f[7] - f[8])) + ((f[10] - f[9]) + (f[15] - f[16])) + (f[17] - f[18]);
                const V2 jz = ((f[5] - f[6]) + (f[11] - f[12])) + ((f[14] - f[13]) + (f[15] - f[16])) + (f[18] - f[17]);
                const V2 rho = bc(ph.rho_ref) + drho;
                // Eq. 8 (solid-fluid interaction scheme): F_ads = -G_w rho sum_a w_a s(x + e_a) e_a
                if constexpr (SF) {
                    float ax0 = 0.0f, ay0 = 0.0f, az0 = 0.0f, ax1 = 0.0f, ay1 = 0.0f, az1 = 0.0f;
#pragma unroll
                    for (int a = 1; a < Q; ++a) {
                        const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a), off = ex + ey * TYX;
                        const float w = float(L::wf(a));
                        const uint8_t* tz = S.type[(zc + ez) & 7];
                        if (tz[tcl + off] & T_SOLID) {
                            if (ex) ax0 += w * float(ex);
                            if (ey) ay0 += w * float(ey);
                            if (ez) az0 += w * float(ez);
                        }
                        if (tz[tcl + 4 * TYX + off] & T_SOLID) {
                            if (ex) ax1 += w * float(ex);
                            if (ey) ay1 += w * float(ey);
                            if (ez) az1 += w * float(ez);
                        }
                    }
                    const V2 gr = (-ph.wall_param) * rho;
                    Fx = (Fmx + gr * mk(ax0, ax1)) + bc(ph.fx);
                    Fy = (Fmy + gr * mk(ay0, ay1)) + bc(ph.fy);
                    Fz = (Fmz + gr * mk(az0, az1)) + bc(ph.fz);
                }
                if ((fl0 && !(rho.v.x > 0.0f)) || (fl1 && !(rho.v.y > 0.0f))) atomicOr(err, ERR_RHO);
                // Eq. 4: rho u = sum e f + F/2
                const V2 inv = div2(bc(1.0f), rho);
                const V2 ux = fma2(0.5f, Fx, jx) * inv, uy = fma2(0.5f, Fy, jy) * inv, uz = fma2(0.5f, Fz, jz) * inv;
                const V2 X = div2(fma2(Fmx, Fmx, fma2(Fmy, Fmy, Fmz * Fmz)), psi_c * psi_c);
                collide3p(f, drho, rho, ux, uy, uz, Fx, Fy, Fz, X, kr);
                const int gi = zc * nxy + (y0 + ly) * nx + x0 + lx;
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    if (fl0) fout[a * fs + gi] = f[a].v.x;
                    if (fl1) fout[a * fs + gi + 4 * nx] = f[a].v.y;
                }
            }
        }
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            f2[a] = f1[a];
            f1[a] = fcur[a];
        }
    }
}

// Can the march box column (x0, y0) with TMA loads?  (Full 32 x 8 columns of grids at least 64 x 16 x 4;
// the host's work list uses the same test.)
__host__ __device__ __forceinline__ bool ztma_boxed(int x0, int y0, int nx, int ny, int nz) {
    return x0 + TTX <= nx && y0 + TTY <= ny && nx >= 64 && ny >= 16 && nz >= 4;
}

__global__ void __launch_bounds__(TTX* ZTY, 2)
    ztma_step(const float* __restrict__ fin, float* __restrict__ fout, const void* tmap, Geo g, Phys<float> ph,
              Rates3P kr, unsigned* err, const ZItem* __restrict__ items) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const ZItem it = items[blockIdx.x];
    const int x0 = it.bx * TTX, y0 = it.by * TTY, zb = it.z0, ze = it.z1;
    const bool boxed = tmap != nullptr && ztma_boxed(x0, y0, g.nx, g.ny, g.nz);
    const bool sf = ph.wall_kind == 2;
    if (boxed) {
        ZTSmem& S = *reinterpret_cast<ZTSmem*>(smem_raw);
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            mbar_init(&S.bar[0]);
            mbar_init(&S.bar[1]);
            fence_mbar_init();
        }
        __syncthreads();
        // tmap: the input buffer's map (box TBX x TBY x 1)
        if (!it.solid)
            ztma_chunk_bulk(fin, fout, tmap, g, ph, kr, x0, y0, zb, ze, err, S.b, S.bar);
        else if (sf)
            ztma_chunk_solid<true>(fin, fout, tmap, g, ph, kr, x0, y0, zb, ze, err, S.s, S.bar);
        else
            ztma_chunk_solid<false>(fin, fout, tmap, g, ph, kr, x0, y0, zb, ze, err, S.s, S.bar);
        return;
    }
    // a column the march cannot box: its 32-plane chunk by the z-pair march on the two 32 x 4 halves,
    // with their chunk flags
    const int ty4 = (g.ny + ZTY - 1) / ZTY, tx = (g.nx + ZTX - 1) / ZTX;
    const int h0 = ((zb / ZCH) * ty4 + 2 * it.by) * tx + it.bx;
    const bool has1 = y0 + ZTY < g.ny;
    const bool s0 = g.tile_solid ? g.tile_solid[h0] != 0 : true;
    const bool s1 = has1 && (g.tile_solid ? g.tile_solid[h0 + tx] != 0 : true);
    ZPSmem<ZTX, ZTY>& sm = *reinterpret_cast<ZPSmem<ZTX, ZTY>*>(smem_raw);
    for (int h = 0; h < (has1 ? 2 : 1); ++h) {
        const bool solid = h ? s1 : s0;
        if (h) __syncthreads();   // the first half is done with shared memory
        if (solid && sf)
            zpair_chunk<true, true>(fin, fout, g, ph, kr, x0, y0 + h * ZTY, zb, err, sm);
        else if (solid)
            zpair_chunk<true>(fin, fout, g, ph, kr, x0, y0 + h * ZTY, zb, err, sm);
        else
            zpair_chunk<false>(fin, fout, g, ph, kr, x0, y0 + h * ZTY, zb, err, sm);
    }
}

}  // namespace

void zpair_tile_shape(int* tx, int* ty, int* tz) {
    *tx = ZTX;
    *ty = ZTY;
    *tz = ZCH;
}

cudaError_t launch_zpair_step(const void* fin, void* fout, const Geo& g, const DevParams& p, cudaStream_t s) {
    constexpr size_t bytes = sizeof(ZPSmem<ZTX, ZTY>);
    static bool attr[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr[dev]) {
        cudaError_t e = cudaFuncSetAttribute(zpair_step, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    dim3 grid((p.nx + ZTX - 1) / ZTX, (p.ny + ZTY - 1) / ZTY, (p.nz + ZCH - 1) / ZCH);
    zpair_step<<<grid, dim3(ZTX, ZTY, 1), bytes, s>>>(static_cast<const float*>(fin), static_cast<float*>(fout), g,
                                                      make_phys<float>(p), make_rates3p(p), p.err);
    return cudaGetLastError();
}

cudaError_t launch_ztma_step(const void* fin, void* fout, const void* tmap, const Geo& g, const DevParams& p,
                             cudaStream_t s) {
    static bool attr[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr[dev]) {
        cudaError_t e = cudaFuncSetAttribute(ztma_step, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ZT_SMEM));
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    if (!p.zitems || p.nzitems < 1) return cudaErrorInvalidValue;
    ztma_step<<<p.nzitems, dim3(TTX, ZTY, 1), ZT_SMEM, s>>>(static_cast<const float*>(fin), static_cast<float*>(fout),
                                                           tmap, g, make_phys<float>(p), make_rates3p(p), p.err,
                                                           p.zitems);
    return cudaGetLastError();
}

void ztma_box_dims(int* bx, int* by) {
    *bx = TBX;
    *by = TBY;
}

#ifndef LBMWET_ZWL_MIN_RUN   // shortest bulk run kept on the bulk path, and shortest piece (planes)
#define LBMWET_ZWL_MIN_RUN 8
#endif

std::vector<ZItem> ztma_work_list(const uint8_t* mask, int nx, int ny, int nz) {
    constexpr int HALO = 3, MIN_RUN = LBMWET_ZWL_MIN_RUN;
    const int gx = (nx + TTX - 1) / TTX, gy = (ny + TTY - 1) / TTY;
    // per plane and column: a solid within 3 nodes of the column's cells in x and y (periodic)
    const int t[3] = {TTX, TTY, 1};
    const std::vector<uint8_t> col = tile_solid_flags(mask, nx, ny, nz, t, 2, scan_threads((long long)nx * ny * nz));
    std::vector<ZItem> items;
    std::vector<uint8_t> need(nz);
    for (int by = 0; by < gy; ++by)
        for (int bx = 0; bx < gx; ++bx) {
            if (!ztma_boxed(bx * TTX, by * TTY, nx, ny, nz)) {
                for (int z0 = 0; z0 < nz; z0 += ZCH) items.push_back(ZItem{bx, by, z0, std::min(z0 + ZCH, nz), 1});
                continue;
            }
            // planes within 3 planes (periodic) of a plane with a solid near the column
            for (int z = 0; z < nz; ++z) {
                uint8_t n = 0;
                for (int d = -HALO; d <= HALO && !n; ++d) {
                    const int zz = ((z + d) % nz + nz) % nz;
                    n = col[((size_t)zz * gy + by) * gx + bx];
                }
                need[z] = n;
            }
            // runs of equal need; short bulk runs join the solid path
            std::vector<ZItem> runs;
            for (int z0 = 0; z0 < nz;) {
                int z1 = z0 + 1;
                while (z1 < nz && need[z1] == need[z0]) ++z1;
                runs.push_back(ZItem{bx, by, z0, z1, need[z0] ? 1 : 0});
                z0 = z1;
            }
            for (ZItem& r : runs)
                if (!r.solid && r.z1 - r.z0 < MIN_RUN && runs.size() > 1) r.solid = 1;
            std::vector<ZItem> merged;
            for (const ZItem& r : runs) {
                if (!merged.empty() && merged.back().solid == r.solid) merged.back().z1 = r.z1;
                else merged.push_back(r);
            }
            // pieces cut at the multiples of TCH planes, so that items of neighbouring columns start
            // on the same planes and share their halo reads in L2; a first or last piece shorter than
            // MIN_RUN joins its neighbour (items of up to TCH + MIN_RUN - 1 planes)
            for (const ZItem& r : merged) {
                std::vector<int> cuts{r.z0};
                for (int z = (r.z0 / TCH + 1) * TCH; z < r.z1; z += TCH) cuts.push_back(z);
                cuts.push_back(r.z1);
                if (cuts.size() > 2 && cuts[1] - cuts[0] < MIN_RUN) cuts.erase(cuts.begin() + 1);
                if (cuts.size() > 2 && cuts[cuts.size() - 1] - cuts[cuts.size() - 2] < MIN_RUN)
                    cuts.erase(cuts.end() - 2);
                for (size_t k = 0; k + 1 < cuts.size(); ++k)
                    items.push_back(ZItem{bx, by, cuts[k], cuts[k + 1], r.solid});
            }
        }
    std::stable_sort(items.begin(), items.end(), [](const ZItem& a, const ZItem& b) {
        return a.z0 != b.z0 ? a.z0 < b.z0 : (a.by != b.by ? a.by < b.by : a.bx < b.bx);
    });
    return items;
}

}  // namespace lbmwet
