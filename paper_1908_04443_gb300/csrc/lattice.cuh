// Lattice tables and the hand-expanded MRT collision of the GPU path.
//
// D2Q9 velocities: e0=(0,0); e1..e4=(1,0),(0,1),(-1,0),(0,-1); e5..e8=(1,1),(-1,1),(-1,-1),(1,-1).
// Moment order (rho, e, eps, jx, qx, jy, qy, pxx, pxy): the diagonal of Lambda in Sec. II.A and the
// rows of S in Eq. 7.  M is the Lallemand-Luo basis (the paper defers M and m^eq = M f^eq to its
// Ref. [34]); its rows are orthogonal, so M^-1 = M^T diag(1/|row|^2).
//
// D3Q19 velocities: e0=0; +-x, +-y, +-z; then (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0),(1,0,1),(-1,0,-1),
// (1,0,-1),(-1,0,1),(0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1).  Moment order of the d'Humieres basis:
// (rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww, pxy, pyz, pxz, mx, my, mz).
// The paper defers its 3D model to Refs. [32,33,39]: the source S is the Guo source projected on M
// plus the consistency terms on e and eps scaled to give the same isotropic pressure-tensor change
// per dimension as Eq. 7 (coefficients 114 and -33 in place of 12 and -12).
#pragma once

#include <cstdint>

namespace lbmwet {

enum : uint8_t { T_SOLID = 1, T_WALL = 2, T_NEARWALL = 4, T_BULK = 8 };  // BULK: fluid, all neighbours fluid
enum : unsigned { ERR_PSI = 1u, ERR_RHO = 2u, ERR_NONFINITE = 4u, ERR_TIMEOUT = 8u };

struct D2Q9 {
    static constexpr int Q = 9, D = 2;
    __host__ __device__ static constexpr int ex(int a) {
        constexpr int t[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
        return t[a];
    }
    __host__ __device__ static constexpr int ey(int a) {
        constexpr int t[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
        return t[a];
    }
    __host__ __device__ static constexpr int ez(int a) {
        constexpr int t[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        return t[a];
    }
    __host__ __device__ static constexpr int opp(int a) {
        constexpr int t[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
        return t[a];
    }
    __host__ __device__ static constexpr double w(int a) {
        constexpr double t[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                                    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
        return t[a];
    }
    // Eq. 5 weights: 1/3 for |e|^2 = 1, 1/12 for |e|^2 = 2
    __host__ __device__ static constexpr double wf(int a) {
        constexpr double t[9] = {0.0, 1.0 / 3, 1.0 / 3, 1.0 / 3, 1.0 / 3,
                                     1.0 / 12, 1.0 / 12, 1.0 / 12, 1.0 / 12};
        return t[a];
    }
};

struct D3Q19 {
    static constexpr int Q = 19, D = 3;
    __host__ __device__ static constexpr int ex(int a) {
        constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
        return t[a];
    }
    __host__ __device__ static constexpr int ey(int a) {
        constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
        return t[a];
    }
    __host__ __device__ static constexpr int ez(int a) {
        constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
        return t[a];
    }
    __host__ __device__ static constexpr int opp(int a) {
        constexpr int t[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
        return t[a];
    }
    __host__ __device__ static constexpr double w(int a) {
        constexpr double t[19] = {1.0 / 3,
                                     1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
                                     1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                                     1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
        return t[a];
    }
    // force weights 1/6 (|e|^2 = 1) and 1/12 (|e|^2 = 2): sum_a w_a e_ax^2 = 1 as in 2D
    __host__ __device__ static constexpr double wf(int a) {
        constexpr double t[19] = {0.0,
                                      1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6,
                                      1.0 / 12, 1.0 / 12, 1.0 / 12, 1.0 / 12, 1.0 / 12, 1.0 / 12,
                                      1.0 / 12, 1.0 / 12, 1.0 / 12, 1.0 / 12, 1.0 / 12, 1.0 / 12};
        return t[a];
    }
};

// Collision constants in compute precision C.
template <class C>
struct Rates {
    C s_e, s_eps, s_q, s_nu, s_pi, s_m;
    C c_e, c_eps;     // consistency coefficients: 12 sigma/(tau_e - 1/2), 12 sigma/(tau_eps - 1/2) (2D)
};

// MRT collision (Eq. 2) of one D2Q9 node in deviation variables: f holds f_a - w_a rho_ref, drho =
// rho - rho_ref.  S is Eq. 7 with F the total force and X = |F_m|^2 / psi^2.  On return f holds
// the post-collision deviations f*_a - w_a rho_ref.
template <class C>
__host__ __device__ __forceinline__ void collide_d2q9(C (&f)[9], C drho, C rho, C ux, C uy, C Fx, C Fy, C X,
                                             const Rates<C>& r) {
    const C s14 = f[1] + f[2] + f[3] + f[4];
    const C s58 = f[5] + f[6] + f[7] + f[8];
    const C m1 = -C(4) * f[0] - s14 + C(2) * s58;
    const C m2 = C(4) * f[0] - C(2) * s14 + s58;
    const C m4 = -C(2) * f[1] + C(2) * f[3] + f[5] - f[6] - f[7] + f[8];
    const C m6 = -C(2) * f[2] + C(2) * f[4] + f[5] + f[6] - f[7] - f[8];
    const C m7 = f[1] - f[2] + f[3] - f[4];
    const C m8 = f[5] - f[6] + f[7] - f[8];
    const C u2 = ux * ux + uy * uy;
    const C uF = ux * Fx + uy * Fy;
    // increments m* - m; equilibria in deviation form: e^eq = -2 rho + 3 rho u^2, eps^eq = rho - 3 rho u^2
    const C e_eq = -C(2) * drho + C(3) * rho * u2;
    const C eps_eq = drho - C(3) * rho * u2;
    const C d1 = -r.s_e * (m1 - e_eq) + (C(1) - C(0.5) * r.s_e) * (C(6) * uF + r.c_e * X);
    const C d2 = -r.s_eps * (m2 - eps_eq) + (C(1) - C(0.5) * r.s_eps) * (-C(6) * uF - r.c_eps * X);
    const C d4 = -r.s_q * (m4 + rho * ux) - (C(1) - C(0.5) * r.s_q) * Fx;
    const C d6 = -r.s_q * (m6 + rho * uy) - (C(1) - C(0.5) * r.s_q) * Fy;
    const C d7 = -r.s_nu * (m7 - rho * (ux * ux - uy * uy)) + (C(1) - C(0.5) * r.s_nu) * C(2) * (ux * Fx - uy * Fy);
    const C d8 = -r.s_nu * (m8 - rho * ux * uy) + (C(1) - C(0.5) * r.s_nu) * (ux * Fy + uy * Fx);
    // conserved: the density increment is zero, j* - j = F (independent of s_rho and s_j).  Adding
    // M^-1 (m* - m) to f, rather than rebuilding f from m*, keeps the mass of the stored deviations
    // exact up to unbiased rounding: rebuilding scales drho by 9 * round(1/9) every step.
    const C a1 = d1 * C(1.0 / 36);
    const C a2 = d2 * C(1.0 / 36);
    const C a3 = Fx * C(1.0 / 6);
    const C a4 = d4 * C(1.0 / 12);
    const C a5 = Fy * C(1.0 / 6);
    const C a6 = d6 * C(1.0 / 12);
    const C a7 = d7 * C(0.25);
    const C a8 = d8 * C(0.25);
    // f += M^T diag(1/|row|^2) (m* - m)
    const C b = -a1 - C(2) * a2;
    const C c = C(2) * a1 + a2;
    f[0] += C(4) * (a2 - a1);
    f[1] += b + a3 - C(2) * a4 + a7;
    f[2] += b + a5 - C(2) * a6 - a7;
    f[3] += b - a3 + C(2) * a4 + a7;
    f[4] += b - a5 + C(2) * a6 - a7;
    f[5] += c + a3 + a4 + a5 + a6 + a8;
    f[6] += c - a3 - a4 + a5 + a6 - a8;
    f[7] += c - a3 - a4 - a5 - a6 + a8;
    f[8] += c + a3 + a4 - a5 - a6 - a8;
}

// MRT collision of one D3Q19 node (d'Humieres basis) in deviation variables.
// Equilibria (deviation form): e = -11 drho + 19 rho u^2, eps = 3 drho - 11/2 rho u^2,
// q = -2/3 rho u, 3pxx = rho (3ux^2 - u^2), 3pixx = -1/2 3pxx, pww = rho (uy^2 - uz^2), piww = -1/2 pww,
// p_ab = rho u_a u_b, m = 0.
// Guo source moments: S_e = 38 u.F, S_eps = -11 u.F, S_q = -2/3 F, S_3pxx = 2(2uxFx - uyFy - uzFz),
// S_3pixx = -1/2 S_3pxx, S_pww = 2(uyFy - uzFz), S_piww = -1/2 S_pww, S_pab = ua Fb + ub Fa, S_m = 0;
// plus the consistency terms c_e X on e and -c_eps X on eps.
template <class C>
__host__ __device__ __forceinline__ void collide_d3q19(C (&f)[19], C drho, C rho, C ux, C uy, C uz, C Fx, C Fy,
                                              C Fz, C X, const Rates<C>& r) {
    // sums over the velocity groups
    const C s16 = f[1] + f[2] + f[3] + f[4] + f[5] + f[6];
    const C s718 = f[7] + f[8] + f[9] + f[10] + f[11] + f[12] + f[13] + f[14] + f[15] + f[16] + f[17] + f[18];
    // e = 19|e|^2 - 30:  -30 f0 - 11 (axis) + 8 (edges)
    const C m1 = -C(30) * f[0] - C(11) * s16 + C(8) * s718;
    // eps = (21|e|^4 - 53|e|^2 + 24)/2:  12 f0 - 4 (axis) + 1 (edges)
    const C m2 = C(12) * f[0] - C(4) * s16 + s718;
    // q = (5|e|^2 - 9) e:  -4 on axis links, +1 on edges
    const C ex_edges = (f[7] - f[8]) + (f[9] - f[10]) + (f[11] - f[12]) + (f[13] - f[14]);
    const C ey_edges = (f[7] - f[8]) - (f[9] - f[10]) + (f[15] - f[16]) + (f[17] - f[18]);
    const C ez_edges = (f[11] - f[12]) - (f[13] - f[14]) + (f[15] - f[16]) - (f[17] - f[18]);
    const C m4 = -C(4) * (f[1] - f[2]) + ex_edges;
    const C m6 = -C(4) * (f[3] - f[4]) + ey_edges;
    const C m8 = -C(4) * (f[5] - f[6]) + ez_edges;
    // 3pxx = 3ex^2 - |e|^2 and 3pixx = (3|e|^2 - 5)(3ex^2 - |e|^2)
    const C ax = f[1] + f[2], ay = f[3] + f[4], az = f[5] + f[6];
    const C exy = f[7] + f[8] + f[9] + f[10];     // edges in the xy plane
    const C exz = f[11] + f[12] + f[13] + f[14];  // edges in the xz plane
    const C eyz = f[15] + f[16] + f[17] + f[18];  // edges in the yz plane
    const C m9 = C(2) * ax - ay - az + exy + exz - C(2) * eyz;
    const C m10 = -C(4) * ax + C(2) * ay + C(2) * az + exy + exz - C(2) * eyz;
    const C m11 = ay - az + exy - exz;
    const C m12 = -C(2) * ay + C(2) * az + exy - exz;
    const C m13 = (f[7] + f[8]) - (f[9] + f[10]);
    const C m14 = (f[15] + f[16]) - (f[17] + f[18]);
    const C m15 = (f[11] + f[12]) - (f[13] + f[14]);
    const C m16 = (f[7] - f[8]) + (f[9] - f[10]) - (f[11] - f[12]) - (f[13] - f[14]);
    const C m17 = -(f[7] - f[8]) + (f[9] - f[10]) + (f[15] - f[16]) + (f[17] - f[18]);
    const C m18 = (f[11] - f[12]) - (f[13] - f[14]) - (f[15] - f[16]) + (f[17] - f[18]);

    const C u2 = ux * ux + uy * uy + uz * uz;
    const C uF = ux * Fx + uy * Fy + uz * Fz;
    const C h_e = C(1) - C(0.5) * r.s_e, h_eps = C(1) - C(0.5) * r.s_eps, h_q = C(1) - C(0.5) * r.s_q;
    const C h_nu = C(1) - C(0.5) * r.s_nu, h_pi = C(1) - C(0.5) * r.s_pi;
    // increments m* - m of the non-conserved moments
    const C d1 = -r.s_e * (m1 - (-C(11) * drho + C(19) * rho * u2)) + h_e * (C(38) * uF + r.c_e * X);
    const C d2 = -r.s_eps * (m2 - (C(3) * drho - C(5.5) * rho * u2)) + h_eps * (-C(11) * uF - r.c_eps * X);
    const C c23 = C(2.0 / 3.0);
    const C d4 = -r.s_q * (m4 + c23 * rho * ux) - h_q * c23 * Fx;
    const C d6 = -r.s_q * (m6 + c23 * rho * uy) - h_q * c23 * Fy;
    const C d8 = -r.s_q * (m8 + c23 * rho * uz) - h_q * c23 * Fz;
    const C p3xx_eq = rho * (C(3) * ux * ux - u2);
    const C S3xx = C(2) * (C(2) * ux * Fx - uy * Fy - uz * Fz);
    const C d9 = -r.s_nu * (m9 - p3xx_eq) + h_nu * S3xx;
    const C d10 = -r.s_pi * (m10 + C(0.5) * p3xx_eq) - h_pi * C(0.5) * S3xx;
    const C pww_eq = rho * (uy * uy - uz * uz);
    const C Sww = C(2) * (uy * Fy - uz * Fz);
    const C d11 = -r.s_nu * (m11 - pww_eq) + h_nu * Sww;
    const C d12 = -r.s_pi * (m12 + C(0.5) * pww_eq) - h_pi * C(0.5) * Sww;
    const C d13 = -r.s_nu * (m13 - rho * ux * uy) + h_nu * (ux * Fy + uy * Fx);
    const C d14 = -r.s_nu * (m14 - rho * uy * uz) + h_nu * (uy * Fz + uz * Fy);
    const C d15 = -r.s_nu * (m15 - rho * ux * uz) + h_nu * (ux * Fz + uz * Fx);
    const C d16 = -r.s_m * m16;
    const C d17 = -r.s_m * m17;
    const C d18 = -r.s_m * m18;

    // scale by 1/|row|^2: (19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8).
    // The density increment is zero and j* - j = F; adding M^-1 (m* - m) to f keeps the stored
    // deviations' mass exact up to unbiased rounding.
    const C a1 = d1 * C(1.0 / 2394);
    const C a2 = d2 * C(1.0 / 252);
    const C a3 = Fx * C(0.1);
    const C a4 = d4 * C(1.0 / 40);
    const C a5 = Fy * C(0.1);
    const C a6 = d6 * C(1.0 / 40);
    const C a7 = Fz * C(0.1);
    const C a8 = d8 * C(1.0 / 40);
    const C a9 = d9 * C(1.0 / 36);
    const C a10 = d10 * C(1.0 / 72);
    const C a11 = d11 * C(1.0 / 12);
    const C a12 = d12 * C(1.0 / 24);
    const C a13 = d13 * C(0.25);
    const C a14 = d14 * C(0.25);
    const C a15 = d15 * C(0.25);
    const C a16 = d16 * C(0.125);
    const C a17 = d17 * C(0.125);
    const C a18 = d18 * C(0.125);

    // f_a += sum_k M[k][a] a_k; columns of M written per velocity
    f[0] += -C(30) * a1 + C(12) * a2;
    const C axis = -C(11) * a1 - C(4) * a2;
    // x axis: 3pxx = 2, 3pixx = -4, pww = piww = 0
    const C axx = axis + C(2) * a9 - C(4) * a10;
    f[1] += axx + a3 - C(4) * a4;
    f[2] += axx - a3 + C(4) * a4;
    // y axis: 3pxx = -1, 3pixx = 2, pww = 1, piww = -2
    const C ayy = axis - a9 + C(2) * a10 + a11 - C(2) * a12;
    f[3] += ayy + a5 - C(4) * a6;
    f[4] += ayy - a5 + C(4) * a6;
    // z axis: 3pxx = -1, 3pixx = 2, pww = -1, piww = 2
    const C azz = axis - a9 + C(2) * a10 - a11 + C(2) * a12;
    f[5] += azz + a7 - C(4) * a8;
    f[6] += azz - a7 + C(4) * a8;
    const C edge = C(8) * a1 + a2;
    // xy edges: 3pxx = 1, 3pixx = 1, pww = 1, piww = 1
    const C exy0 = edge + a9 + a10 + a11 + a12;
    f[7] += exy0 + (a3 + a4) + (a5 + a6) + a13 + (a16 - a17);
    f[8] += exy0 - (a3 + a4) - (a5 + a6) + a13 - (a16 - a17);
    f[9] += exy0 + (a3 + a4) - (a5 + a6) - a13 + (a16 + a17);
    f[10] += exy0 - (a3 + a4) + (a5 + a6) - a13 - (a16 + a17);
    // xz edges: 3pxx = 1, 3pixx = 1, pww = -1, piww = -1
    const C exz0 = edge + a9 + a10 - a11 - a12;
    f[11] += exz0 + (a3 + a4) + (a7 + a8) + a15 + (-a16 + a18);
    f[12] += exz0 - (a3 + a4) - (a7 + a8) + a15 - (-a16 + a18);
    f[13] += exz0 + (a3 + a4) - (a7 + a8) - a15 + (-a16 - a18);
    f[14] += exz0 - (a3 + a4) + (a7 + a8) - a15 - (-a16 - a18);
    // yz edges: 3pxx = -2, 3pixx = -2, pww = 0, piww = 0
    const C eyz0 = edge - C(2) * a9 - C(2) * a10;
    f[15] += eyz0 + (a5 + a6) + (a7 + a8) + a14 + (a17 - a18);
    f[16] += eyz0 - (a5 + a6) - (a7 + a8) + a14 - (a17 - a18);
    f[17] += eyz0 + (a5 + a6) - (a7 + a8) - a14 + (a17 + a18);
    f[18] += eyz0 - (a5 + a6) + (a7 + a8) - a14 - (a17 + a18);
}

// Reverse of collide_d2q9: given mu = dL/df* at one node, the adjoints of its inputs.  f holds the
// post-streaming deviations, F = F_m + F_body the total force and psi_c the node's psi; on return
// fbar[a] = dL/df_a (through the moments, u, rho and the equilibria), Fmbar = dL/dF_m (through F and
// the consistency term X = |F_m|^2/psi_c^2) and psibar = dL/dpsi_c (through X only; F_m's own
// dependence on psi is handled by the caller).
template <class C>
__host__ __device__ __forceinline__ void collide_d2q9_adjoint(const C (&f)[9], const C (&mu)[9], C rho, C ux, C uy,
                                                              C Fx, C Fy, C Fmx, C Fmy, C psi_c, const Rates<C>& r,
                                                              C (&fbar)[9], C& Fmbar_x, C& Fmbar_y, C& psibar) {
    (void)f;
    // dL/dm* = diag(1/|row|^2) M mu
    const C u14 = mu[1] + mu[2] + mu[3] + mu[4];
    const C u58 = mu[5] + mu[6] + mu[7] + mu[8];
    const C ms0 = (mu[0] + u14 + u58) * C(1.0 / 9);
    const C ms1 = (-C(4) * mu[0] - u14 + C(2) * u58) * C(1.0 / 36);
    const C ms2 = (C(4) * mu[0] - C(2) * u14 + u58) * C(1.0 / 36);
    const C ms3 = (mu[1] - mu[3] + mu[5] - mu[6] - mu[7] + mu[8]) * C(1.0 / 6);
    const C ms4 = (-C(2) * mu[1] + C(2) * mu[3] + mu[5] - mu[6] - mu[7] + mu[8]) * C(1.0 / 12);
    const C ms5 = (mu[2] - mu[4] + mu[5] + mu[6] - mu[7] - mu[8]) * C(1.0 / 6);
    const C ms6 = (-C(2) * mu[2] + C(2) * mu[4] + mu[5] + mu[6] - mu[7] - mu[8]) * C(1.0 / 12);
    const C ms7 = (mu[1] - mu[2] + mu[3] - mu[4]) * C(0.25);
    const C ms8 = (mu[5] - mu[6] + mu[7] - mu[8]) * C(0.25);
    const C h_e = C(1) - C(0.5) * r.s_e, h_eps = C(1) - C(0.5) * r.s_eps;
    const C h_q = C(1) - C(0.5) * r.s_q, h_nu = C(1) - C(0.5) * r.s_nu;
    const C u2 = ux * ux + uy * uy;
    // adjoints of rho (= rho_ref + sum f), j, u and F
    C Rb = ms0, jbx = ms3, jby = ms5, Fbx = ms3, Fby = ms5, ubx = C(0), uby = C(0);
    // rows e, eps: relaxation towards -2 drho + 3 rho u^2 and drho - 3 rho u^2, source 6 u.F +- c X
    const C a_e = r.s_e * ms1, a_eps = r.s_eps * ms2;
    Rb += -C(2) * a_e + a_eps + C(3) * u2 * (a_e - a_eps);
    ubx += C(6) * rho * ux * (a_e - a_eps);
    uby += C(6) * rho * uy * (a_e - a_eps);
    const C t_uF = C(6) * (h_e * ms1 - h_eps * ms2);
    ubx += t_uF * Fx;
    uby += t_uF * Fy;
    Fbx += t_uF * ux;
    Fby += t_uF * uy;
    const C Xb = h_e * r.c_e * ms1 - h_eps * r.c_eps * ms2;
    // rows qx, qy: relaxation towards -rho u, source -F
    Rb += -r.s_q * (ms4 * ux + ms6 * uy);
    ubx += -r.s_q * ms4 * rho;
    uby += -r.s_q * ms6 * rho;
    Fbx += -h_q * ms4;
    Fby += -h_q * ms6;
    // pxx: rho (ux^2 - uy^2), source 2 (ux Fx - uy Fy); pxy: rho ux uy, source ux Fy + uy Fx
    const C a7 = r.s_nu * ms7, b7 = C(2) * h_nu * ms7, a8 = r.s_nu * ms8, b8 = h_nu * ms8;
    Rb += a7 * (ux * ux - uy * uy) + a8 * ux * uy;
    ubx += C(2) * a7 * rho * ux + b7 * Fx + a8 * rho * uy + b8 * Fy;
    uby += -C(2) * a7 * rho * uy - b7 * Fy + a8 * rho * ux + b8 * Fx;
    Fbx += b7 * ux + b8 * uy;
    Fby += -b7 * uy + b8 * ux;
    // u = (j + F/2) / rho
    const C inv = C(1) / rho;
    jbx += ubx * inv;
    jby += uby * inv;
    Fbx += C(0.5) * ubx * inv;
    Fby += C(0.5) * uby * inv;
    Rb += -(ubx * ux + uby * uy) * inv;
    // X = |F_m|^2 / psi_c^2;  F = F_m + F_body
    const C ip2 = C(1) / (psi_c * psi_c);
    const C X = (Fmx * Fmx + Fmy * Fmy) * ip2;
    Fmbar_x = Fbx + C(2) * Xb * Fmx * ip2;
    Fmbar_y = Fby + C(2) * Xb * Fmy * ip2;
    psibar = -C(2) * Xb * X / psi_c;
    // f: rows e, eps, qx, qy, pxx, pxy of M (m-bar = (1 - s) m*-bar), plus rho and j
    const C mb1 = (C(1) - r.s_e) * ms1, mb2 = (C(1) - r.s_eps) * ms2, mb4 = (C(1) - r.s_q) * ms4;
    const C mb6 = (C(1) - r.s_q) * ms6, mb7 = (C(1) - r.s_nu) * ms7, mb8 = (C(1) - r.s_nu) * ms8;
    const C b = -mb1 - C(2) * mb2 + Rb;
    const C c = C(2) * mb1 + mb2 + Rb;
    fbar[0] = -C(4) * mb1 + C(4) * mb2 + Rb;
    fbar[1] = b - C(2) * mb4 + mb7 + jbx;
    fbar[2] = b - C(2) * mb6 - mb7 + jby;
    fbar[3] = b + C(2) * mb4 + mb7 - jbx;
    fbar[4] = b + C(2) * mb6 - mb7 - jby;
    fbar[5] = c + mb4 + mb6 + mb8 + jbx + jby;
    fbar[6] = c - mb4 + mb6 - mb8 - jbx + jby;
    fbar[7] = c - mb4 - mb6 + mb8 - jbx - jby;
    fbar[8] = c + mb4 - mb6 - mb8 + jbx - jby;
}

}  // namespace lbmwet
