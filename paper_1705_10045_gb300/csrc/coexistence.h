// Coexistence densities of the reduced van der Waals fluid, for the
// latent-heat source (Sec. 5).  Host code.
#pragma once

namespace lbm {

// Temperature grid of the coexistence table: T_j = kCoexT0 + j / kCoexPerT,
// j = 0..kCoexIntervals; the last point is the critical point T = 1.
constexpr double kCoexT0 = 0.5;
constexpr double kCoexPerT = 1024.0;
constexpr int kCoexIntervals = 512;

// rho_v(T) and rho_l(T) on the Maxwell coexistence curve for 0 < T < 1
// (equal pressure and chemical potential); false outside that range.
bool coexistence(double T, double* rho_v, double* rho_l);

// rho_v and rho_l at every grid temperature (kCoexIntervals + 1 entries each).
void coexistence_table(double* rho_v, double* rho_l);

}  // namespace lbm
