// derived.cpp -- quantities derived from estimated frame potentials (host):
// epsilon_max of the design bound and the layer count for an eps-approximate
// k-design from an exponential fit over depths (paper: Sec. "Frame potential",
// Eqs. epsilonmax, exponential and layers; fitting region from the
// supplementary "Choice of curve fitting region").
#include <cmath>
#include <vector>

#include "fp.h"

namespace fpk {
fp_status api_fail(fp_status s, const char *msg);
}

namespace {
double factorial(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
}
}  // namespace

extern "C" fp_status fp_epsilon_max(double F, int32_t k, int32_t n, int32_t q, double *log10_eps) {
    if (!log10_eps) return fpk::api_fail(FP_ERR_ARG, "null argument");
    if (k < 1 || n < 1 || q < 2) return fpk::api_fail(FP_ERR_ARG, "need k >= 1, n >= 1, q >= 2");
    const double dev = F - factorial(k);
    // d^k sqrt(F - k!) with d = q^n, in log10 (d^k overflows a double at n = 50)
    *log10_eps = dev > 0 ? k * n * std::log10((double)q) + 0.5 * std::log10(dev) : NAN;
    return FP_OK;
}

extern "C" fp_status fp_design_layers(int32_t n_depths, const double *depths, const double *F, int32_t k, int32_t n,
                                      int32_t q, double eps, double dev_max, double *l_eps, double *A, double *C) {
    if (!depths || !F || !l_eps || n_depths < 0) return fpk::api_fail(FP_ERR_ARG, "null argument");
    if (k < 1 || n < 1 || q < 2 || !(eps > 0) || !(dev_max > 0))
        return fpk::api_fail(FP_ERR_ARG, "need k >= 1, n >= 1, q >= 2, eps > 0, dev_max > 0");
    const double fh = factorial(k);
    std::vector<double> x, y;
    for (int i = 0; i < n_depths; ++i) {
        const double rel = (F[i] - fh) / fh;
        if (rel > 0 && rel < dev_max) {
            x.push_back(depths[i]);
            y.push_back(std::log(F[i] - fh));
        }
    }
    *l_eps = NAN;
    if (A) *A = NAN;
    if (C) *C = NAN;
    if (x.size() < 2) return FP_OK;
    double xm = 0, ym = 0;
    for (size_t i = 0; i < x.size(); ++i) { xm += x[i]; ym += y[i]; }
    xm /= (double)x.size();
    ym /= (double)x.size();
    double sxy = 0, sxx = 0;
    for (size_t i = 0; i < x.size(); ++i) {
        sxy += (x[i] - xm) * (y[i] - ym);
        sxx += (x[i] - xm) * (x[i] - xm);
    }
    if (!(sxx > 0)) return FP_OK;
    const double slope = sxy / sxx, a = ym - slope * xm;
    if (!(slope < 0)) return FP_OK;
    const double c = -2.0 / slope, lnA = 0.5 * a;
    *l_eps = c * (k * n * std::log((double)q) + lnA + std::log(1.0 / eps));
    if (A) *A = std::exp(lnA);
    if (C) *C = c;
    return FP_OK;
}
