// Host-side thermodynamics of the C ABI: critical temperature and coexistence densities by the
// Maxwell equal-area rule, used for the limiter bounds of Sec. III.B (rho_g <= rho_w <= rho_l).
//
// Equations of state: Peng-Robinson (Eq. 18) and Carnahan-Starling.  The equal-area rule reads
// p(rho_g) = p(rho_l) = p* and integral_{rho_g}^{rho_l} (p(rho) - p*) / rho^2 d rho = 0, i.e. equal
// areas on the p-v plane (v = 1/rho).  Roots are bracketed by the spinodals and found by bisection;
// the area integral is a composite Gauss-Legendre rule in s = ln(rho).
#include <cmath>

#include "eos_host.h"

namespace lbmwet {

namespace {

double pr_phi(const EosHost& e) {
    const double tc = critical_temperature(e);
    const double k = 0.37464 + 1.54226 * e.omega - 0.26992 * e.omega * e.omega;
    const double t = 1.0 + k * (1.0 - std::sqrt(e.T / tc));
    return t * t;
}

double max_density(const EosHost& e) { return e.kind == 0 ? 1.0 / e.b : 4.0 / e.b; }

double pressure_T(const EosHost& e, double rho, double T, double aphi) {
    if (e.kind == 1) {
        const double eta = e.b * rho / 4.0;
        const double om = 1.0 - eta;
        return rho * e.R * T * (1.0 + eta + eta * eta - eta * eta * eta) / (om * om * om) - e.a * rho * rho;
    }
    return rho * e.R * T / (1.0 - e.b * rho) - aphi * rho * rho / (1.0 + 2.0 * e.b * rho - e.b * e.b * rho * rho);
}

double dpdrho(const EosHost& e, double rho, double T, double aphi) {
    const double h = 1e-7 * max_density(e);
    return (pressure_T(e, rho + h, T, aphi) - pressure_T(e, rho - h, T, aphi)) / (2.0 * h);
}

// minimum of dp/drho over (0, rho_max): grid scan then golden-section refinement
double min_dp(const EosHost& e, double T, double aphi, double* at) {
    const double rmax = max_density(e);
    const int n = 4000;
    double best = 1e300, br = 0;
    int bi = 1;
    for (int i = 1; i < n; ++i) {
        const double r = rmax * 0.95 * i / n;
        const double d = dpdrho(e, r, T, aphi);
        if (d < best) {
            best = d;
            br = r;
            bi = i;
        }
    }
    double lo = rmax * 0.95 * (bi - 1) / n, hi = rmax * 0.95 * (bi + 1) / n;
    const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
    for (int it = 0; it < 200; ++it) {
        const double c = hi - gr * (hi - lo), d = lo + gr * (hi - lo);
        if (dpdrho(e, c, T, aphi) < dpdrho(e, d, T, aphi)) hi = d;
        else lo = c;
    }
    br = 0.5 * (lo + hi);
    if (at) *at = br;
    return dpdrho(e, br, T, aphi);
}

template <class F>
double bisect(F f, double lo, double hi) {
    double flo = f(lo);
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        const double fm = f(mid);
        if ((fm < 0) == (flo < 0)) {
            lo = mid;
            flo = fm;
        } else {
            hi = mid;
        }
    }
    return 0.5 * (lo + hi);
}

// 16-point Gauss-Legendre nodes/weights on [-1, 1] (positive half)
const double GL_X[8] = {0.0950125098376374, 0.2816035507792589, 0.4580167776572274, 0.6178762444026438,
                        0.7554044083550030, 0.8656312023878318, 0.9445750230732326, 0.9894009349916499};
const double GL_W[8] = {0.1894506104550685, 0.1826034150449236, 0.1691565193950025, 0.1495959888165767,
                        0.1246289712555339, 0.0951585116824928, 0.0622535239386479, 0.0271524594117541};

}  // namespace

double critical_temperature(const EosHost& e) {
    if (e.kind == 0) return 0.0778 * e.a / (0.45724 * e.b * e.R);
    // C-S: the temperature at which min_rho dp/drho = 0, a few milliseconds of scans and bisection;
    // remembered for the last (a, b, R) of this thread, since a batch initialises many grids with
    // one equation of state
    thread_local double last_a = -1.0, last_b = -1.0, last_R = -1.0, last_tc = 0.0;
    if (e.a == last_a && e.b == last_b && e.R == last_R) return last_tc;
    double lo = 1e-12, hi = 1.0;
    while (min_dp(e, hi, 0.0, nullptr) < 0) hi *= 2.0;
    const double tc = bisect([&](double T) { return min_dp(e, T, 0.0, nullptr); }, lo, hi);
    last_a = e.a;
    last_b = e.b;
    last_R = e.R;
    last_tc = tc;
    return tc;
}

double eos_pressure(const EosHost& e, double rho) {
    const double aphi = e.kind == 0 ? e.a * pr_phi(e) : 0.0;
    return pressure_T(e, rho, e.T, aphi);
}

double eos_aphi(const EosHost& e) { return e.kind == 0 ? e.a * pr_phi(e) : e.a; }

namespace {
bool coexistence_solve(const EosHost& e, double* rho_g, double* rho_l);
}

// The Maxwell construction is tens of milliseconds of root finding and quadrature: remembered for
// the last EOS (kind and every constant) of this thread, since a batch initialises many grids with
// one equation of state.
bool coexistence(const EosHost& e, double* rho_g, double* rho_l) {
    thread_local bool have = false, last_ok = false;
    thread_local EosHost last{};
    thread_local double last_g = 0.0, last_l = 0.0;
    if (!(have && e.kind == last.kind && e.a == last.a && e.b == last.b && e.R == last.R && e.T == last.T &&
          e.omega == last.omega)) {
        last_ok = coexistence_solve(e, &last_g, &last_l);
        last = e;
        have = true;
    }
    *rho_g = last_g;
    *rho_l = last_l;
    return last_ok;
}

namespace {

bool coexistence_solve(const EosHost& e, double* rho_g, double* rho_l) {
    const double T = e.T;
    const double aphi = e.kind == 0 ? e.a * pr_phi(e) : 0.0;
    double rm;
    if (!(min_dp(e, T, aphi, &rm) < 0)) return false;
    auto dp = [&](double r) { return dpdrho(e, r, T, aphi); };
    auto p = [&](double r) { return pressure_T(e, r, T, aphi); };
    const double rmax = max_density(e);
    const double r1 = bisect(dp, 1e-12, rm);            // gas spinodal (local max of p)
    double hi = rm;
    while (dp(hi) < 0) hi += 0.5 * (0.999 * rmax - hi);
    const double r2 = bisect(dp, rm, hi);               // liquid spinodal (local min of p)
    const double pmax = p(r1), pmin = p(r2);
    auto roots = [&](double ps, double* g, double* l) {
        const double lo_r = 1e-3 * ps / (e.R * T);
        *g = bisect([&](double r) { return p(r) - ps; }, lo_r, r1);
        double h2 = r2;
        while (p(h2) - ps < 0) h2 += 0.5 * (0.999999 * rmax - h2);
        *l = bisect([&](double r) { return p(r) - ps; }, r2, h2);
    };
    auto area = [&](double ps) {
        double g, l;
        roots(ps, &g, &l);
        const double s0 = std::log(g), s1 = std::log(l);
        const int panels = 400;
        const double hs = (s1 - s0) / panels;
        double acc = 0.0;
        for (int k = 0; k < panels; ++k) {
            const double c = s0 + (k + 0.5) * hs;
            for (int j = 0; j < 8; ++j) {
                for (int sgn = -1; sgn <= 1; sgn += 2) {
                    const double s = c + sgn * GL_X[j] * 0.5 * hs;
                    const double r = std::exp(s);
                    acc += GL_W[j] * 0.5 * hs * (p(r) - ps) / r;   // (p - p*)/rho^2 d rho = (p - p*)/rho ds
                }
            }
        }
        return acc;
    };
    double lo = (pmin > 0 ? pmin : 0.0) + 1e-13 * std::fabs(pmax);
    double hp = pmax - 1e-13 * std::fabs(pmax);
    const double ps = bisect(area, lo, hp);
    roots(ps, rho_g, rho_l);
    return std::isfinite(*rho_g) && std::isfinite(*rho_l) && *rho_g < *rho_l;
}

}  // namespace

}  // namespace lbmwet
