// Eigenvalue counts of a window from Chebyshev moments (kernel polynomial
// method): the moments the filter records (Algorithm 1, lines 10-11) monitor
// the number of eigenstates in the search interval (Sect. 2).  Host code.
#include <cmath>

#include "common.cuh"

namespace cfd {
namespace {

// sum_m g_m c_m mu_m for one vector: Jackson kernel over M = n_mom moments,
// window [xl, xr] on the scaled axis.
double damped_window_sum(const double *mu, int n_mom, double xl, double xr) {
    const double pi = 3.141592653589793238462643383279502884;
    const double tl = std::acos(std::fmin(std::fmax(xl, -1.0), 1.0));
    const double tr = std::acos(std::fmin(std::fmax(xr, -1.0), 1.0));
    const double M = n_mom;
    const double q = pi / (M + 1.0);
    const double cotq = std::cos(q) / std::sin(q);
    double s = 0.0;
    for (int m = 0; m < n_mom; ++m) {
        double c = (m == 0) ? (tl - tr) / pi : 2.0 * (std::sin(m * tl) - std::sin(m * tr)) / (m * pi);
        double g = ((M - m + 1.0) * std::cos(q * m) + std::sin(q * m) * cotq) / (M + 1.0);
        s += g * c * mu[m];
    }
    return s;
}

double count_of(const double *mu, int n_vec, int n_mom, int64_t N, double alpha, double beta, double lam_l,
                double lam_r) {
    double xl = alpha * (lam_l - beta), xr = alpha * (lam_r - beta);
    double acc = 0.0;
    for (int r = 0; r < n_vec; ++r) {
        const double *m = mu + (int64_t)r * n_mom;
        if (m[0] > 0) acc += damped_window_sum(m, n_mom, xl, xr) / m[0];
    }
    return (double)N * acc / n_vec;
}

}  // namespace
}  // namespace cfd

using namespace cfd;

extern "C" {

cfd_status cfd_kpm_count(const double *mu, int n_vec, int n_mom, int64_t N, double lmin, double lmax,
                         double lam_l, double lam_r, double *count) {
    clear_error();
    if (!mu || !count || n_vec < 1 || n_mom < 2 || N < 1) return fail(CFD_ERR_ARG, "bad arguments");
    if (!(lmin < lmax) || !(lam_l <= lam_r)) return fail(CFD_ERR_ARG, "bad interval");
    *count = count_of(mu, n_vec, n_mom, N, 2.0 / (lmax - lmin), 0.5 * (lmax + lmin), lam_l, lam_r);
    return CFD_OK;
}

cfd_status cfd_kpm_window(const double *mu, int n_vec, int n_mom, int64_t N, double lmin, double lmax,
                          double center, double target, double *lam_l, double *lam_r) {
    clear_error();
    if (!mu || !lam_l || !lam_r || n_vec < 1 || n_mom < 2 || N < 1) return fail(CFD_ERR_ARG, "bad arguments");
    if (!(lmin < center && center < lmax) || !(target > 0)) return fail(CFD_ERR_ARG, "bad centre or target");
    const double alpha = 2.0 / (lmax - lmin), beta = 0.5 * (lmax + lmin);
    double lo = 0.0, hi = std::fmin(center - lmin, lmax - center);
    if (count_of(mu, n_vec, n_mom, N, alpha, beta, center - hi, center + hi) < target)
        return fail(CFD_ERR_ARG, "the whole interval holds fewer than %g states", target);
    for (int it = 0; it < 200 && hi - lo > 1e-15 * (1.0 + std::fabs(center)); ++it) {
        double mid = 0.5 * (lo + hi);
        if (count_of(mu, n_vec, n_mom, N, alpha, beta, center - mid, center + mid) < target) lo = mid;
        else hi = mid;
    }
    *lam_l = center - hi;
    *lam_r = center + hi;
    return CFD_OK;
}

}  // extern "C"
