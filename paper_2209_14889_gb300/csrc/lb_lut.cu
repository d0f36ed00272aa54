// lb_lut.cu -- host-side FP64 construction of the C~(P) table used by the lattice kernel.
//
// The stiffness tensor of App. B depends on |P| only through r2 = I2(k)/I0(k) and
// r4 = I4(k)/I0(k), where k solves I1(k)/I0(k) = min(|P|, P_cap) (Eq. Pk).  The table stores
// a2 = r2/q and a4 = r4/q^2 against q = |P|^2, both smooth on [0, q_cap] with a2(0) = 1/2 and
// a4(0) = 1/24, so that the kernel forms r2 cos 2theta_P = a2 (Px^2 - Py^2), etc., without
// trigonometry, Bessel functions or a division by |P|.
//
// Bessel ratios come from the integral representation
//   I_n(k) = (1/pi) int_0^pi exp(k cos t) cos(n t) dt,
// evaluated with the trapezoid rule (spectrally accurate for this periodic, even integrand)
// with the factor exp(-k) taken out so that nothing overflows.
#include <cmath>

#include "lb_internal.h"

namespace vlb {

namespace {

constexpr int M_TRAP = 256;   // spectrally accurate: the integrand is smooth and periodic

// I_n(k) e^{-k} * pi (the common factor cancels in the ratios)
double scaled_in(int n, double k)
{
    const double h = M_PI / M_TRAP;
    double s = 0.0;
    for (int j = 0; j <= M_TRAP; ++j) {
        double t = j * h;
        double w = (j == 0 || j == M_TRAP) ? 0.5 : 1.0;
        s += w * std::exp(k * (std::cos(t) - 1.0)) * std::cos(n * t);
    }
    return s * h;
}

double ratio(int n, double k) { return scaled_in(n, k) / scaled_in(0, k); }

// Invert P = I1(k)/I0(k) (monotone increasing, P'(k) = 1 - P/k - P^2) by safeguarded Newton,
// starting from k0 (the previous table entry).
double invert_P(double P, double k0)
{
    if (P <= 0.0) return 0.0;
    double lo = 0.0, hi = 4.0;
    while (ratio(1, hi) < P) { lo = hi; hi *= 2.0; }
    double k = (k0 > lo && k0 < hi) ? k0 : 0.5 * (lo + hi);
    for (int it = 0; it < 100; ++it) {
        double r = ratio(1, k);
        if (r > P) hi = k; else lo = k;
        double d = 1.0 - r / k - r * r;
        double kn = k - (r - P) / d;
        if (!(kn > lo && kn < hi)) kn = 0.5 * (lo + hi);
        if (std::fabs(kn - k) < 1e-14 * (1.0 + k)) return kn;
        k = kn;
    }
    return k;
}

}  // namespace

void build_lut(double P_cap, float* lut)
{
    const double q_cap = P_cap * P_cap;
    double k = 0.0;
    for (int i = 0; i <= LUT_N; ++i) {
        double a2, a4;
        if (i == 0) {
            a2 = 0.5;            // r2 ~ k^2/8, q ~ k^2/4
            a4 = 1.0 / 24.0;     // r4 ~ k^4/384, q^2 ~ k^4/16
        } else {
            double q = q_cap * i / LUT_N;
            k = invert_P(std::sqrt(q), k);
            a2 = ratio(2, k) / q;
            a4 = ratio(4, k) / (q * q);
        }
        lut[2 * i] = (float)a2;
        lut[2 * i + 1] = (float)a4;
    }
}

}  // namespace vlb
