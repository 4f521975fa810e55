// Static geometry of the curved geometric-formulation contact-angle scheme (2D, Sec. III.A).
//
// Per wall node P the scheme needs the densities at two points D1, D2 where the characteristic
// lines through P cross the mesh.  The lines depend on the solid mask and the prescribed angle
// only, so the host finds them once: the unit normal of Eq. 13 (eighth-order isotropic weights of
// Eq. 14, switch s = 1 on solid nodes), the two directions of Eq. 15, and for each the first mesh
// line it crosses (the boundary of the square of half-width 1 around P) with the two lattice nodes
// of that mesh segment and the linear-interpolation weight.  The step kernels then evaluate
// rho_D = rho(A) + lambda (rho(B) - rho(A)) from densities they already hold, and Eq. 11.
//
// Crossings within 1e-12 of a node are taken at the node; an end node that is solid is dropped
// (the other end carries rho_D); a crossing with no fluid end is unusable; a node with no usable
// crossing falls back to the mean of Eq. 17.  A wall node whose Eq. 13 sum vanishes has no normal
// and the geometry is rejected.
#include "wall_gf.h"

#include <cmath>
#include <string>

namespace lbmwet {

namespace {

// Eq. 14 weight of a vector with squared length e2 (0 for lengths outside the stencil)
double eq14_weight(int e2) {
    switch (e2) {
        case 1: return 4.0 / 21.0;
        case 2: return 4.0 / 45.0;
        case 4: return 1.0 / 60.0;
        case 5: return 2.0 / 315.0;
        case 8: return 1.0 / 5040.0;
        default: return 0.0;
    }
}

constexpr double kSnap = 1e-12;

struct End {
    int dx, dy;   // offset of the lattice node from P
    double w;     // its interpolation weight
};

// The crossing of the ray from P along the unit vector (vx, vy) with the square's boundary: one or
// two end nodes with weights summing to 1.
int crossing(double vx, double vy, End out[2]) {
    const double ax = std::fabs(vx), ay = std::fabs(vy);
    int n = 0;
    auto add = [&](int dx, int dy, double w) {
        if (w > 1.0 - kSnap) {
            out[0] = End{dx, dy, 1.0};
            n = -1;   // a node: the only end
        } else if (n >= 0 && w >= kSnap) {
            out[n++] = End{dx, dy, w};
        }
    };
    if (ax >= ay) {
        const int X = vx > 0.0 ? 1 : -1;
        const double t = vy / ax;   // where the vertical mesh line x = X is crossed
        const double lo = std::floor(t);
        const double lam = t - lo;
        add(X, int(lo), 1.0 - lam);
        if (n >= 0) add(X, int(lo) + 1, lam);
    } else {
        const int Y = vy > 0.0 ? 1 : -1;
        const double t = vx / ay;   // the horizontal mesh line y = Y
        const double lo = std::floor(t);
        const double lam = t - lo;
        add(int(lo), Y, 1.0 - lam);
        if (n >= 0) add(int(lo) + 1, Y, lam);
    }
    return n < 0 ? 1 : n;
}

unsigned code_of(int dx, int dy) { return unsigned(dx + 1) | (unsigned(dy + 1) << 2); }

}  // namespace

bool gf_tables(const uint8_t* solid, int nx, int ny, const int64_t* wall, size_t nw, double theta_a_deg,
               double* out, std::string* err) {
    const double pi = 3.14159265358979323846;
    const double tp = pi / 2.0 - theta_a_deg * (pi / 180.0);   // theta' of Eq. 15
    const double c = std::cos(tp), s = std::sin(tp);
    auto is_solid = [&](int x, int y) {
        return solid[(long long)((y % ny + ny) % ny) * nx + ((x % nx + nx) % nx)] != 0;
    };
    for (size_t k = 0; k < nw; ++k) {
        const int x = int(wall[k] % nx), y = int(wall[k] / nx);
        // Eq. 13
        double gx = 0.0, gy = 0.0;
        for (int ex = -2; ex <= 2; ++ex)
            for (int ey = -2; ey <= 2; ++ey) {
                const double w = eq14_weight(ex * ex + ey * ey);
                if (w == 0.0) continue;
                const double sw = is_solid(x + ex, y + ey) ? 1.0 : 0.0;
                gx += w * sw * ex;
                gy += w * sw * ey;
            }
        const double norm = std::hypot(gx, gy);
        if (norm < 1e-9) {   // the weights are multiples of 1/5040: below this the sum cancels
            if (err)
                *err = "geometric-formulation scheme: wall node (" + std::to_string(x) + ", " + std::to_string(y) +
                       ") has no surface normal (Eq. 13 sums to zero)";
            return false;
        }
        const double nsx = -gx / norm, nsy = -gy / norm;
        // Eq. 15: n_1 and n_2
        const double dir[2][2] = {{nsx * c - nsy * s, nsx * s + nsy * c}, {nsx * c + nsy * s, -nsx * s + nsy * c}};
        unsigned code = theta_a_deg <= 90.0 ? GF_MAX : 0u;
        for (int d = 0; d < 2; ++d) {
            End ends[2];
            const int ne = crossing(dir[d][0], dir[d][1], ends);
            End fl[2];
            int nf = 0;
            for (int i = 0; i < ne; ++i)
                if (!is_solid(x + ends[i].dx, y + ends[i].dy)) fl[nf++] = ends[i];
            double lam = 0.0;
            unsigned a, b;
            if (nf == 0) {
                out[3 * k + d] = 0.0;
                continue;   // D unusable
            } else if (nf == 1) {
                a = b = code_of(fl[0].dx, fl[0].dy);
            } else {
                a = code_of(fl[0].dx, fl[0].dy);
                b = code_of(fl[1].dx, fl[1].dy);
                lam = fl[1].w;   // weights of two fluid ends sum to 1
            }
            code |= (a | (b << 4)) << (8 * d);
            code |= d == 0 ? GF_USE1 : GF_USE2;
            out[3 * k + d] = lam;
        }
        out[3 * k + 2] = double(code);
    }
    return true;
}

}  // namespace lbmwet
