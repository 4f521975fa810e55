// Geometry tables of the curved geometric-formulation contact-angle scheme (2D, Sec. III.A,
// Eqs. 10-15), shared by the host builder and the step kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

namespace lbmwet {

// One wall node's entry: three doubles {lambda_1, lambda_2, code}.  The code packs, for each
// crossing d = 1, 2 (byte d - 1), the end nodes A (bits 0-3) and B (bits 4-7) of its mesh segment
// as (dx + 1) | (dy + 1) << 2, offsets from the wall node; rho_D = rho(A) + lambda (rho(B) - rho(A)).
// Flags: crossing d usable, and Eq. 11's max (theta_a <= 90 degrees) rather than min.
constexpr unsigned GF_USE1 = 1u << 16;
constexpr unsigned GF_USE2 = 1u << 17;
constexpr unsigned GF_MAX = 1u << 18;
constexpr int GF_STRIDE = 3;

// Fills out[3 * k .. 3 * k + 2] for the wall nodes wall[0 .. nw) (linear indices y * nx + x of a
// periodic nx x ny grid with the given solid mask).  Returns false (with a message) when a wall
// node has no normal.
bool gf_tables(const uint8_t* solid, int nx, int ny, const int64_t* wall, size_t nw, double theta_a_deg,
               double* out, std::string* err);

}  // namespace lbmwet
