// Gas constants, host side.
#pragma once
#include <cmath>

namespace mlvs {

// Reference viscosity of a Knudsen number.  The paper gives only the temperature law
// mu = mu_ref (T/T_ref)^omega (Sec. 4); the library reads Kn through the standard VHS/VSS
// mean-free-path relation with alpha = 1:
//   mu_ref = 5 (alpha+1)(alpha+2) sqrt(pi) / (4 alpha (5-2 omega)(7-2 omega)) Kn rho_ref sqrt(2 R T_ref) L_ref.
inline double vhs_mu_ref(double Kn, double omega, double rho_ref, double R, double T_ref, double L_ref) {
  const double alpha = 1.0;
  const double c = 5.0 * (alpha + 1.0) * (alpha + 2.0) * std::sqrt(M_PI) /
                   (4.0 * alpha * (5.0 - 2.0 * omega) * (7.0 - 2.0 * omega));
  return c * Kn * rho_ref * std::sqrt(2.0 * R * T_ref) * L_ref;
}

}  // namespace mlvs
