// tables.cpp -- host-side tables of the FDTD library: shower profiles and
// lateral weights (Sec. III.B) and CPML grading coefficients.
#include <cmath>
#include <vector>

#include "../../include/cyl.h"
#include "../../include/fdtd.h"

namespace {
constexpr double kC = 299792458.0;
constexpr double kMu0 = 1.25663706212e-6;
constexpr double kE = 1.602176634e-19;
constexpr double kPi = 3.14159265358979323846;
}  // namespace

namespace fdtd {

// Roden-Gedney convolutional PML, kappa = 1, cubic conductivity grading with a
// design reflection of 1e-6, complex-frequency shift alpha falling linearly
// from 2 pi 50 MHz eps at the interface to 0 at the PEC wall behind the layer.
// psi^{new} = b psi + a d, with b = exp(-(sigma + alpha) dt / eps) and
// a = sigma (b - 1) / (sigma + alpha).  aE/bE are indexed by the integer
// position i (0..n), aH/bH by the half-integer position i + 1/2 (0..n-1);
// positions outside the layer get a = b = 0 (psi stays zero there).
void cpml_coefficients(int n, int P, double dx, double dt, double eps_r, float *aE, float *bE,
                       float *aH, float *bH) {
    const double eps = eps_r / (kMu0 * kC * kC);
    const double eta = kMu0 * kC / std::sqrt(eps_r);
    const double order = 3.0;
    const double sigma_max = -(order + 1.0) * std::log(1e-6) / (2.0 * eta * P * dx);
    const double alpha_max = 2.0 * kPi * 50e6 * eps;
    auto coef = [&](double depth, float *a, float *b) {
        double x = depth / P;
        double sg = sigma_max * std::pow(x, order);
        double al = alpha_max * (1.0 - x);
        double bb = std::exp(-(sg + al) * dt / eps);
        *b = (float)bb;
        *a = (sg + al) > 0.0 ? (float)(sg * (bb - 1.0) / (sg + al)) : 0.0f;
    };
    for (int i = 0; i <= n; ++i) {
        aE[i] = bE[i] = 0.0f;
        if (i >= 1 && i <= P) coef((double)(P - i), &aE[i], &bE[i]);
        else if (i >= n - P && i <= n - 1) coef((double)(i - (n - P)), &aE[i], &bE[i]);
    }
    for (int i = 0; i < n; ++i) {
        aH[i] = bH[i] = 0.0f;
        if (i <= P - 1) coef(P - i - 0.5, &aH[i], &bH[i]);
        else if (i >= n - P) coef(i + 0.5 - (n - P), &aH[i], &bH[i]);
    }
}

}  // namespace fdtd

extern "C" {

int fdtd_profile_gaussian(double z0, double bin_dz, int n_bins, double z_peak, double l,
                          double q_max, double *out) {
    if (!out || n_bins < 1 || !(l > 0.0)) return FDTD_ERR_ARG;
    for (int b = 0; b < n_bins; ++b) {
        double d = z0 + b * bin_dz - z_peak;
        out[b] = q_max * std::exp(-0.5 * d * d / (l * l));
    }
    return FDTD_OK;
}

int fdtd_profile_greisen(double bin_dz, int n_bins, double E0, double Ec, double X0,
                         double frac, double *out) {
    if (!out || n_bins < 1 || !(E0 > Ec) || !(Ec > 0.0) || !(X0 > 0.0)) return FDTD_ERR_ARG;
    const double beta0 = std::log(E0 / Ec);
    const double pre = 0.31 / std::sqrt(beta0);
    for (int b = 0; b < n_bins; ++b) {
        double t = b * bin_dz / X0;  // depth in radiation lengths
        double ne = 0.0;
        if (t > 0.0) {
            double age = 3.0 * t / (t + 2.0 * beta0);
            ne = pre * std::exp(t * (1.0 - 1.5 * std::log(age)));
        }
        out[b] = -kE * frac * ne;
    }
    return FDTD_OK;
}

int fdtd_profile_gaisser_hillas(double z0, double bin_dz, int n_bins, int n_sub,
                                const double *z1, const double *zmax, const double *lambda,
                                const double *nmax, double frac, double *out) {
    if (!out || n_bins < 1 || n_sub < 0 || (n_sub > 0 && (!z1 || !zmax || !lambda || !nmax)))
        return FDTD_ERR_ARG;
    for (int b = 0; b < n_bins; ++b) {
        double z = z0 + b * bin_dz;
        double n = 0.0;
        for (int s = 0; s < n_sub; ++s) {
            double rise = zmax[s] - z1[s];
            if (z <= z1[s] || !(rise > 0.0)) continue;
            n += nmax[s] * std::pow((z - z1[s]) / rise, rise / lambda[s]) *
                 std::exp((zmax[s] - z) / lambda[s]);
        }
        out[b] = -kE * frac * n;
    }
    return FDTD_OK;
}

int fdtd_lateral_gaussian(int L, double sigma_cells, double *w) {
    if (!w || L < 0 || !(sigma_cells > 0.0)) return FDTD_ERR_ARG;
    const int n = 2 * L + 1;
    double tot = 0.0;
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            double di = c - L, dj = r - L;
            double v = std::exp(-(di * di + dj * dj) / (2.0 * sigma_cells * sigma_cells));
            w[r * n + c] = v;
            tot += v;
        }
    for (int t = 0; t < n * n; ++t) w[t] /= tot;
    return FDTD_OK;
}

int cyl_rings_gaussian(int n_rings, double d, double sigma_r, double *w) {
    if (!w || n_rings < 1 || !(d > 0.0) || !(sigma_r > 0.0)) return FDTD_ERR_ARG;
    // fraction of a radial Gaussian inside radius r: 1 - exp(-r^2 / (2 sigma_r^2))
    auto inside = [&](double r) { return -std::expm1(-0.5 * (r / sigma_r) * (r / sigma_r)); };
    double tot = 0.0, lo = 0.0;
    for (int i = 0; i < n_rings; ++i) {
        const double hi = (i + 0.5) * d;
        w[i] = inside(hi) - inside(lo);
        tot += w[i];
        lo = hi;
    }
    if (!(tot > 0.0)) return FDTD_ERR_ARG;
    for (int i = 0; i < n_rings; ++i) w[i] /= tot;
    return FDTD_OK;
}

int fdtd_lateral_nkg(int L, double dx, double r_m, double s, int nsub, double r_cut, double *w) {
    if (!w || L < 0 || nsub < 1 || !(dx > 0.0) || !(r_m > 0.0)) return FDTD_ERR_ARG;
    const int n = 2 * L + 1;
    double tot = 0.0;
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            double acc = 0.0;
            for (int sb = 0; sb < nsub; ++sb)
                for (int sa = 0; sa < nsub; ++sa) {
                    double x = (c - L + (sa + 0.5) / nsub - 0.5) * dx;
                    double y = (r - L + (sb + 0.5) / nsub - 0.5) * dx;
                    double rr = std::sqrt(x * x + y * y);
                    if (rr <= 0.0 || rr > r_cut) continue;
                    double u = rr / r_m;
                    acc += std::pow(u, s - 2.0) * std::pow(1.0 + u, s - 4.5);
                }
            w[r * n + c] = acc;
            tot += acc;
        }
    if (!(tot > 0.0)) return FDTD_ERR_ARG;
    for (int t = 0; t < n * n; ++t) w[t] /= tot;
    return FDTD_OK;
}

}  // extern "C"
