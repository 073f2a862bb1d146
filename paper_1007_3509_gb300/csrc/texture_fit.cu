// Texture fit of Eq. (10) (Sec. 5): the Gaussian width g of the misorientation
// density of a 90-bin one-degree texture histogram, host FP64.
#include <math.h>

#include <vector>

#include "common.cuh"

namespace hp {
namespace {

// folded orientation of a 1-degree angle bin: bins 0..45 -> phi = b + 1/2,
// bins 46..89 are represented by negative angles phi = b + 1/2 - 90 (Sec. 5)
double folded_centre(int b) {
    const double c = b + 0.5;
    return c > 45.0 ? c - 90.0 : c;
}

double fit_residual(const double* dens, int nb, double g) {
    const double k = 1.0 / (g * sqrt(2.0 * 3.14159265358979323846));
    double r = 0.0;
    for (int b = 0; b < nb; ++b) {
        const double phi = folded_centre(b);
        const double d = dens[b] - k * exp(-phi * phi / (2.0 * g * g));
        r += d * d;
    }
    return r;
}

}  // namespace
}  // namespace hp

using namespace hp;

extern "C" int hp_texture_fit(const int64_t* hist, int32_t n_bins, double* g_out, double* residual_out) {
    if (!hist || n_bins != 90 || !g_out) return set_error(HP_ERR_ARG, "hp_texture_fit: needs the 90 one-degree bins");
    double tot = 0.0;
    for (int b = 0; b < n_bins; ++b) tot += (double)hist[b];
    if (!(tot > 0.0)) return set_error(HP_ERR_ARG, "hp_texture_fit: empty histogram");
    std::vector<double> dens(n_bins);
    for (int b = 0; b < n_bins; ++b) dens[b] = (double)hist[b] / tot;  // per degree
    // golden-section search of the least-squares residual over log g
    double lo = log(0.5), hi = log(2000.0);
    const double phi = 0.5 * (sqrt(5.0) - 1.0);
    double x1 = hi - phi * (hi - lo), x2 = lo + phi * (hi - lo);
    double f1 = fit_residual(dens.data(), n_bins, exp(x1)), f2 = fit_residual(dens.data(), n_bins, exp(x2));
    for (int it = 0; it < 200; ++it) {
        if (f1 < f2) { hi = x2; x2 = x1; f2 = f1; x1 = hi - phi * (hi - lo); f1 = fit_residual(dens.data(), n_bins, exp(x1)); }
        else { lo = x1; x1 = x2; f1 = f2; x2 = lo + phi * (hi - lo); f2 = fit_residual(dens.data(), n_bins, exp(x2)); }
    }
    const double g = exp(0.5 * (lo + hi));
    *g_out = g;
    if (residual_out) *residual_out = fit_residual(dens.data(), n_bins, g);
    return HP_OK;
}
