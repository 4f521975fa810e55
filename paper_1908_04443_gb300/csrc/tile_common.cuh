// Device helpers shared by the step kernels: physics constants in compute precision, grid
// geometry, the equation of state and pseudopotential (Eq. 6 with Eq. 18 or Carnahan-Starling),
// periodic wrapping and the enumeration of halo shells.
#pragma once

#include "kernels.h"
#include "lattice.cuh"
#include "wall_gf.h"

namespace lbmwet {

// physics constants in compute precision
template <class C>
struct Phys {
    int eos_kind, wall_kind;
    C RT, a, b, b4, aphi, two_over_G, G;
    C rho_l, rho_g, rho_ref, fx, fy, fz;
    C wall_param;   // VD: the constant virtual density; SF: the adhesion parameter G_w of Eq. 8
    Rates<C> r;
};

template <class C>
Phys<C> make_phys(const DevParams& p) {
    Phys<C> h;
    h.eos_kind = p.eos_kind;
    h.wall_kind = p.wall_kind;
    h.RT = C(p.RT);
    h.a = C(p.a);
    h.b = C(p.b);
    h.b4 = C(0.25 * p.b);
    h.aphi = C(p.aphi);
    h.two_over_G = C(p.two_over_G);
    h.G = C(p.G);
    h.rho_l = C(p.rho_l);
    h.rho_g = C(p.rho_g);
    h.rho_ref = C(p.rho_ref);
    h.fx = C(p.fx);
    h.fy = C(p.fy);
    h.fz = C(p.fz);
    h.wall_param = C(p.wall_kind == 2 ? p.Gw : p.rho_w_const);
    h.r.s_e = C(p.s_e);
    h.r.s_eps = C(p.s_eps);
    h.r.s_q = C(p.s_q);
    h.r.s_nu = C(p.s_nu);
    h.r.s_pi = C(p.s_pi);
    h.r.s_m = C(p.s_m);
    h.r.c_e = C(p.c_e);
    h.r.c_eps = C(p.c_eps);
    return h;
}

// geometry of one grid
struct Geo {
    int nx, ny, nz, N;
    int fp, fs;   // distributions: row pitch (>= nx) and stride between directions (>= fp * ny * nz)
    const uint8_t* type;
    const uint8_t* tile_solid;   // per tile (single-grid kernel) or null
    const int* wall_id;
    const double* kappa_w;   // per wall node or null
    double kappa;
};

// Division in compute precision: FP64 keeps IEEE division (parity with the FP64 oracle); the FP32
// path uses the fast hardware approximation (relative error of a few ulp, below the rounding of the
// FP32 state).
__device__ __forceinline__ float cdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double cdiv(double a, double b) { return a / b; }

// Virtual density of the geometric-formulation scheme at a wall node (Eq. 11) from its table entry
// t = {lambda_1, lambda_2, code} (see wall_gf.h) and rho_at(dx, dy), the same-step density of the
// neighbour at offset (dx, dy); rho_ave (Eq. 17) where neither crossing is usable.
template <typename C, typename F>
__device__ __forceinline__ C gf_wall_density(const double* t, C rho_ave, F rho_at) {
    const unsigned code = unsigned(t[2]);
    if (!(code & (GF_USE1 | GF_USE2))) return rho_ave;
    auto crossing = [&](int d) {
        const unsigned a = (code >> (8 * d)) & 15u, b = (code >> (8 * d + 4)) & 15u;
        const C ra = rho_at(int(a & 3u) - 1, int(a >> 2) - 1);
        const C rb = rho_at(int(b & 3u) - 1, int(b >> 2) - 1);
        return ra + C(t[d]) * (rb - ra);
    };
    const C r1 = (code & GF_USE1) ? crossing(0) : crossing(1);
    const C r2 = (code & GF_USE2) ? crossing(1) : r1;
    return (code & GF_MAX) ? (r1 > r2 ? r1 : r2) : (r1 < r2 ? r1 : r2);
}

template <class C>
__device__ __forceinline__ C psi_arg(C rho, const Phys<C>& e) {
    C p;
    if (e.eos_kind == 1) {  // Carnahan-Starling
        const C eta = e.b4 * rho;
        const C om = C(1) - eta;
        p = cdiv(rho * e.RT * (C(1) + eta + eta * eta - eta * eta * eta), om * om * om) - e.a * rho * rho;
    } else {                // Peng-Robinson, Eq. 18
        p = cdiv(rho * e.RT, C(1) - e.b * rho) - cdiv(e.aphi * rho * rho, C(1) + C(2) * e.b * rho - e.b * e.b * rho * rho);
    }
    return e.two_over_G * (p - rho * C(1.0 / 3.0));   // Eq. 6 argument: 2 (p - rho c_s^2) / (G c^2)
}

// Square root in compute precision: IEEE in FP64; in FP32 x * rsqrt(x) (a few ulp, below the
// rounding of the FP32 state; x > 0 here).
__device__ __forceinline__ float csqrt(float x) { return x * rsqrtf(x); }
__device__ __forceinline__ double csqrt(double x) { return sqrt(x); }

template <class C>
__device__ __forceinline__ C psi_checked(C rho, const Phys<C>& e, unsigned* err) {
    const C arg = psi_arg(rho, e);
    if (!(arg > C(0))) {
        atomicOr(err, ERR_PSI);
        return C(0);
    }
    return csqrt(arg);
}

// The k-th cell of the one-cell-thick shell of an AX x AY (x AZ) box, enumerated so that
// consecutive k are neighbouring cells (warps stay coherent).
template <int AX, int AY, int AZ, int D>
struct Shell {
    static constexpr int COUNT = D == 2 ? 2 * AX + 2 * (AY - 2) : 2 * AX * AY + (AZ - 2) * (2 * AX + 2 * (AY - 2));
    __device__ static __forceinline__ void cell(int k, int& x, int& y, int& z) {
        if (D == 2) {
            z = 0;
            if (k < 2 * AX) {
                y = k < AX ? 0 : AY - 1;
                x = k < AX ? k : k - AX;
            } else {
                const int j = k - 2 * AX;
                y = 1 + (j >> 1);
                x = (j & 1) ? AX - 1 : 0;
            }
        } else {
            constexpr int plane = AX * AY, per = 2 * AX + 2 * (AY - 2);
            if (k < 2 * plane) {
                z = k < plane ? 0 : AZ - 1;
                const int r = k < plane ? k : k - plane;
                x = r % AX;
                y = r / AX;
            } else {
                const int j = k - 2 * plane;
                z = 1 + j / per;
                const int r = j % per;
                if (r < 2 * AX) {
                    y = r < AX ? 0 : AY - 1;
                    x = r < AX ? r : r - AX;
                } else {
                    const int t = r - 2 * AX;
                    y = 1 + (t >> 1);
                    x = (t & 1) ? AX - 1 : 0;
                }
            }
        }
    }
};

// Asynchronous global -> shared copies (cp.async) of one element (4 or 8 bytes) or of 16 bytes,
// their commit groups and the wait for all but PENDING of the thread's groups.
__device__ __forceinline__ void cp_async(float* dst, const float* src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async(double* dst, const double* src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
// 16 bytes (both addresses 16-byte aligned), not kept in L1
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory"); }

// TMA (cp.async.bulk.tensor) loads into shared memory completed on an mbarrier, and a bounded wait.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
// orders this thread's (and, after a barrier, the CTA's) generic accesses to shared memory before
// later asynchronous-proxy writes (TMA) to it
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// one 3D box (x, y, direction) of a tensor map into dst; the barrier expects `bytes`
__device__ __forceinline__ void tma_load_box(void* dst, const void* tmap, int cx, int cy, int cz, uint64_t* bar,
                                             unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(cx), "r"(cy), "r"(cz), "r"(smem_u32(bar))
        : "memory");
}
// wait for the barrier's phase `parity` to complete; false after `limit` unsuccessful polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned limit) {
    for (unsigned i = 0; i < limit; ++i) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ int wrap_full(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}
__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

}  // namespace lbmwet
