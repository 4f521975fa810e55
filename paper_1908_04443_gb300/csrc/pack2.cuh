// Packed pair arithmetic: two FP32 values of two lattice nodes held in one float2 and combined by
// the FP32x2 instructions of sm_100+ (__fadd2_rn, __fmul2_rn, __ffma2_rn: two IEEE single-precision
// operations per instruction), and the pseudopotential of a pair.
#pragma once

#include "kernels.h"
#include "lattice.cuh"
#include "tile_common.cuh"

namespace lbmwet {

struct V2 {
    float2 v;
};
__device__ __forceinline__ V2 bc(float a) { return {make_float2(a, a)}; }
__device__ __forceinline__ V2 mk(float a, float b) { return {make_float2(a, b)}; }
__device__ __forceinline__ V2 operator+(V2 a, V2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ V2 operator*(V2 a, V2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ V2 operator*(float s, V2 b) { return {__fmul2_rn(make_float2(s, s), b.v)}; }
__device__ __forceinline__ V2 fma2(V2 a, V2 b, V2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ V2 fma2(float s, V2 b, V2 c) { return {__ffma2_rn(make_float2(s, s), b.v, c.v)}; }
__device__ __forceinline__ V2 operator-(V2 a, V2 b) { return fma2(-1.0f, b, a); }
__device__ __forceinline__ V2 operator-(V2 a) { return -1.0f * a; }
__device__ __forceinline__ V2 div2(V2 a, V2 b) { return mk(__fdividef(a.v.x, b.v.x), __fdividef(a.v.y, b.v.y)); }

// psi of a pair (Eq. 6 with the C-S or PR pressure); a non-positive argument flags ERR_PSI on
// the lanes in `check` and gives psi 0
__device__ __forceinline__ V2 psi2(V2 rho, const Phys<float>& e, bool check_a, bool check_b, unsigned* err) {
    V2 p;
    if (e.eos_kind == 1) {
        const V2 eta = e.b4 * rho;
        const V2 om = bc(1.0f) - eta;
        const V2 eta2 = eta * eta;
        const V2 poly = fma2(eta2, bc(1.0f) - eta, bc(1.0f) + eta);   // 1 + eta + eta^2 - eta^3
        const V2 num = (e.RT * rho) * poly;
        const V2 den = (om * om) * om;
        p = div2(num, den) - e.a * (rho * rho);
    } else {
        const V2 br = e.b * rho;
        const V2 den2 = fma2(br, bc(2.0f) - br, bc(1.0f));           // 1 + 2 b rho - b^2 rho^2
        p = div2(e.RT * rho, bc(1.0f) - br) - div2(e.aphi * (rho * rho), den2);
    }
    const V2 arg = e.two_over_G * fma2(-1.0f / 3.0f, rho, p);
    V2 out;
    out.v.x = arg.v.x > 0.0f ? arg.v.x * rsqrtf(arg.v.x) : 0.0f;
    out.v.y = arg.v.y > 0.0f ? arg.v.y * rsqrtf(arg.v.y) : 0.0f;
    if ((check_a && !(arg.v.x > 0.0f)) || (check_b && !(arg.v.y > 0.0f))) atomicOr(err, ERR_PSI);
    return out;
}


}  // namespace lbmwet
