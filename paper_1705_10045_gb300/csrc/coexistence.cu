// Coexistence curve of the reduced van der Waals fluid (Sec. 3), computed on
// the host for the latent-heat source of Sec. 5, which releases or absorbs
// heat only inside the transition layer rho_v(T) < rho < rho_l(T).
//
// At coexistence the two phases have equal pressure and equal chemical
// potential.  Per particle, the reduced vdW fluid has the free energy
//   f(rho, T) = -(8T/3) ln(3/rho - 1) - 3 rho   (+ a function of T alone),
// whence p = rho^2 df/drho = 8 rho T/(3 - rho) - 3 rho^2 and
//   mu = f + p/rho = -(8T/3) ln((3 - rho)/rho) + 8T/(3 - rho) - 6 rho.
// For a trial pressure P between the two spinodal pressures the vapour root
// (below the vapour spinodal) and the liquid root (above the liquid spinodal)
// of p(rho) = P are found by bisection, and P is bisected until the two
// chemical potentials agree.
#include <cmath>

#include "coexistence.h"

namespace lbm {
namespace {

double p_red(double r, double T) { return 8.0 * r * T / (3.0 - r) - 3.0 * r * r; }

double mu_red(double r, double T) {
    return -(8.0 * T / 3.0) * std::log((3.0 - r) / r) + 8.0 * T / (3.0 - r) - 6.0 * r;
}

// root of f on [a, b] where f(a) and f(b) differ in sign
template <typename F> double bisect(F f, double a, double b) {
    const bool neg_a = f(a) < 0.0;
    for (int i = 0; i < 200; ++i) {
        const double m = 0.5 * (a + b);
        if (m <= a || m >= b) break;
        if ((f(m) < 0.0) == neg_a) a = m; else b = m;
    }
    return 0.5 * (a + b);
}

}  // namespace

bool coexistence(double T, double* rho_v, double* rho_l) {
    if (!(T > 0.0 && T < 1.0)) return false;
    // spinodals, where dp/drho = 24T/(3 - rho)^2 - 6 rho = 0, i.e. rho (3 - rho)^2 = 4T:
    // the left side rises on (0, 1) and falls on (1, 3)
    auto h = [T](double r) { return r * (3.0 - r) * (3.0 - r) - 4.0 * T; };
    const double s_v = bisect(h, 0.0, 1.0), s_l = bisect(h, 1.0, 3.0);
    const double p_hi = p_red(s_v, T);
    double p_lo = p_red(s_l, T);
    if (p_lo < 0.0) p_lo = 0.0;
    auto roots = [&](double P, double* rv, double* rl) {
        *rv = bisect([&](double r) { return p_red(r, T) - P; }, 0.0, s_v);
        *rl = bisect([&](double r) { return p_red(r, T) - P; }, s_l, 3.0 - 1e-12);
    };
    auto gap = [&](double P) {
        double rv, rl;
        roots(P, &rv, &rl);
        return mu_red(rl, T) - mu_red(rv, T);
    };
    const double lo = p_lo + 1e-300, hi = p_hi;
    const double P = bisect(gap, lo, hi);
    roots(P, rho_v, rho_l);
    return true;
}

void coexistence_table(double* rho_v, double* rho_l) {
    for (int j = 0; j <= kCoexIntervals; ++j) {
        const double T = kCoexT0 + j / kCoexPerT;
        if (j == kCoexIntervals || !coexistence(T, &rho_v[j], &rho_l[j])) {
            rho_v[j] = 1.0;   // the critical point: both branches meet at rho = 1
            rho_l[j] = 1.0;
        }
    }
}

}  // namespace lbm
