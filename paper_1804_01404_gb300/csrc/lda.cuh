// Adiabatic LDA potential of the spin-unpolarised electron gas (Sec. 3.1: the xc potential is
// evaluated with the instantaneous density), Hartree units.
//   xc = 1: Slater exchange, V_x = -(3 rho / pi)^(1/3);
//   xc = 2: exchange plus the Perdew-Zunger parametrisation of the correlation energy per electron,
//           with r_s = (3 / (4 pi rho))^(1/3):
//             eps_c = g / (1 + b1 sqrt(r_s) + b2 r_s)                 for r_s >= 1,
//             eps_c = A ln r_s + B + C r_s ln r_s + D r_s              for r_s < 1,
//           and V_c = d(rho eps_c)/d rho = eps_c - (r_s / 3) d eps_c / d r_s.
//   xc = 3: the correlation of xc = 2 alone (the TB-mBJ exchange is added by its own kernel);
//   xc = 0: nothing.
#pragma once

#include <cuda_runtime.h>

namespace tdks {

__device__ __forceinline__ double lda_vxc(double rho, int xc) {
  if (xc == 0) return 0.0;
  const double r = fmax(rho, 0.0);
  double v = xc == 3 ? 0.0 : -cbrt(3.0 * r / 3.14159265358979323846);
  if ((xc == 2 || xc == 3) && r > 1e-30) {
    constexpr double g = -0.1423, b1 = 1.0529, b2 = 0.3334;
    constexpr double A = 0.0311, B = -0.048, C = 0.0020, D = -0.0116;
    const double rs = cbrt(3.0 / (4.0 * 3.14159265358979323846 * r));
    if (rs >= 1.0) {
      const double sq = sqrt(rs);
      const double den = 1.0 + b1 * sq + b2 * rs;
      v += (g / den) * (1.0 + (7.0 / 6.0) * b1 * sq + (4.0 / 3.0) * b2 * rs) / den;
    } else {
      const double l = log(rs);
      v += A * l + (B - A / 3.0) + (2.0 / 3.0) * C * rs * l + (2.0 * D - C) * rs / 3.0;
    }
  }
  return v;
}

}  // namespace tdks
