// Host thermodynamics helpers of the C ABI (critical temperature, coexistence densities).
#pragma once

namespace lbmwet {

struct EosHost {
    int kind;        // 0 Peng-Robinson (Eq. 18), 1 Carnahan-Starling
    double a, b, R, T, omega;
};

double critical_temperature(const EosHost& e);
double eos_pressure(const EosHost& e, double rho);
// a*phi(T) for PR (the attraction coefficient of Eq. 18); a for C-S
double eos_aphi(const EosHost& e);
// Maxwell equal-area coexistence densities; false if T is not below the critical temperature
bool coexistence(const EosHost& e, double* rho_g, double* rho_l);

}  // namespace lbmwet
