// Host-side analysis of sampled titration curves (no device code).
//
// The paper fits pKa with eq (1), f_prot(pH) = 1 / (1 + 10^(n (pH - pKa))),
// and E0 with eq (2), f_red(E) = 1 / (1 + exp(n v F (E - E0) / (kB T))), to the
// fractions gathered at every condition of the grid (results of the
// "E,pH-REMD at 300 K" section and the following ones).  Both are the logistic
// function f = 1 / (1 + e^u) of u = c n (x - x0), with c = ln 10 for eq (1) and
// c = v F / (kB T) for eq (2), so one least-squares routine serves both.
//
// Start: the linear Hill plot, ln((1 - f) / f) / c = n x - n x0, regressed over
// the points strictly inside (0, 1).  Refinement: Levenberg-Marquardt on the
// residuals f_i - f(x_i) in (x0, n), with the 2 x 2 normal equations solved
// directly and Marquardt's diagonal scaling.
#include <cmath>
#include <string>
#include <vector>

#include "../../include/cphremd.h"
#include "cph_device.cuh"

void cph_internal_set_error(const std::string& m);

namespace {

int afail(const std::string& m) {
    cph_internal_set_error(m);
    return CPH_E_INVALID;
}

// logistic model value and its derivative with respect to u, overflow-free
inline void logistic(double u, double* f, double* dfdu) {
    double v;
    if (u > 0) {
        const double e = std::exp(-u);
        v = e / (1.0 + e);
    } else {
        v = 1.0 / (1.0 + std::exp(u));
    }
    *f = v;
    *dfdu = -v * (1.0 - v);
}

double rss_at(const std::vector<double>& x, const std::vector<double>& f, double c, double x0,
              double m) {
    double s = 0.0;
    for (size_t i = 0; i < x.size(); ++i) {
        double fi, d;
        logistic(c * m * (x[i] - x0), &fi, &d);
        const double r = f[i] - fi;
        s += r * r;
    }
    return s;
}

} // namespace

extern "C" int cph_fit_hill(int kind, int n_pts, const double* x, const double* f, double T,
                            double v, double* x0_out, double* n_out, double* rss_out) {
    if ((kind != CPH_FIT_PH && kind != CPH_FIT_REDOX) || n_pts < 2 || !x || !f || !x0_out || !n_out)
        return afail("cph_fit_hill: bad arguments");
    double c = cph::kLn10;
    if (kind == CPH_FIT_REDOX) {
        if (!(T > 0.0) || !(v > 0.0) || !std::isfinite(T) || !std::isfinite(v))
            return afail("cph_fit_hill: redox fit needs T > 0 and v > 0");
        c = v * cph::kFaraday / (cph::kBoltzmann * T);
    }
    std::vector<double> X(x, x + n_pts), F(f, f + n_pts);
    bool distinct = false, inside = false;
    for (int i = 0; i < n_pts; ++i) {
        if (!std::isfinite(X[i]) || !(F[i] >= 0.0 && F[i] <= 1.0))
            return afail("cph_fit_hill: x must be finite and f in [0, 1]");
        if (X[i] != X[0]) distinct = true;
        if (F[i] > 0.0 && F[i] < 1.0) inside = true;
    }
    if (!distinct) return afail("cph_fit_hill: needs at least two distinct x");
    if (!inside) return afail("cph_fit_hill: no fraction strictly inside (0, 1)");

    // Hill-plot start over the interior points (all points, clipped, if the
    // interior ones share one x)
    auto regress = [&](bool interior_only, double* a, double* b) {
        double sw = 0, sx = 0, sz = 0, sxx = 0, sxz = 0;
        for (int i = 0; i < n_pts; ++i) {
            double fi = F[i];
            if (interior_only && !(fi > 0.0 && fi < 1.0)) continue;
            fi = std::fmin(std::fmax(fi, 1e-6), 1.0 - 1e-6);
            const double z = std::log((1.0 - fi) / fi) / c;
            sw += 1;
            sx += X[i];
            sz += z;
            sxx += X[i] * X[i];
            sxz += X[i] * z;
        }
        const double den = sw * sxx - sx * sx;
        if (sw < 2 || !(std::fabs(den) > 0.0)) return false;
        *a = (sw * sxz - sx * sz) / den;
        *b = (sz - *a * sx) / sw;
        return std::isfinite(*a) && std::isfinite(*b);
    };
    double a = 0, b = 0;
    if (!regress(true, &a, &b) && !regress(false, &a, &b)) return afail("cph_fit_hill: degenerate data");
    double m = a, x0;
    if (std::fabs(m) < 1e-12) {
        m = 1.0;
        x0 = 0.0;
        for (double xi : X) x0 += xi / n_pts;
    } else {
        x0 = -b / m;
    }

    double S = rss_at(X, F, c, x0, m);
    double lambda = 1e-3;
    bool converged = false;
    for (int it = 0; it < 500 && !converged; ++it) {
        // J = d f_model / d(x0, m); the Gauss-Newton step solves J^T J d = J^T r
        double a11 = 0, a12 = 0, a22 = 0, g1 = 0, g2 = 0;
        for (int i = 0; i < n_pts; ++i) {
            double fi, d;
            const double dx = X[i] - x0;
            logistic(c * m * dx, &fi, &d);
            const double j1 = -d * c * m, j2 = d * c * dx, r = F[i] - fi;
            a11 += j1 * j1;
            a12 += j1 * j2;
            a22 += j2 * j2;
            g1 += j1 * r;
            g2 += j2 * r;
        }
        if (!(a11 > 0.0 || a22 > 0.0)) return afail("cph_fit_hill: degenerate Jacobian");
        for (;;) {
            const double b11 = a11 * (1.0 + lambda), b22 = a22 * (1.0 + lambda);
            const double det = b11 * b22 - a12 * a12;
            if (!(std::fabs(det) > 0.0) || lambda > 1e16) {
                converged = true; // no descent direction left: a minimum to rounding
                break;
            }
            const double d1 = (b22 * g1 - a12 * g2) / det, d2 = (b11 * g2 - a12 * g1) / det;
            const double nx0 = x0 + d1, nm = m + d2;
            const double nS = rss_at(X, F, c, nx0, nm);
            if (std::isfinite(nS) && nS <= S) {
                const bool small = std::fabs(d1) <= 1e-14 * (1.0 + std::fabs(x0)) &&
                                   std::fabs(d2) <= 1e-14 * (1.0 + std::fabs(m));
                x0 = nx0;
                m = nm;
                S = nS;
                lambda = std::fmax(lambda * 0.1, 1e-12);
                if (small || S == 0.0) converged = true;
                break;
            }
            lambda *= 10.0;
        }
    }
    if (!converged || !std::isfinite(x0) || !std::isfinite(m))
        return afail("cph_fit_hill: Levenberg-Marquardt did not converge in 500 iterations");
    *x0_out = x0;
    *n_out = m;
    if (rss_out) *rss_out = S;
    return CPH_OK;
}

// ---------------------------------------------------------------------------
// Predictions of eqs (6)-(8) ("Temperature dependence in predicting E0 vs pH
// and pKa vs redox potential": Figure 6's solid lines come from eqs (7) and (8)
// with parameters taken from the simulation).  A redox-active group couples to
// n_sites pH-active groups; pKa_red / pKa_oxi of site i are its pKa with the
// redox group reduced / oxidised, E0_prot / E0_deprot the redox group's E0
// with every pH site protonated / deprotonated.
//   eq (6): v F (E0_prot - E0_deprot) = kB T ln 10 sum_i (pKa_red,i - pKa_oxi,i)
//   eq (7): E0(pH) = E0_prot + kB T / (v F) sum_i ln((10^-pKa_red,i + 10^-pH)
//                                                    / (10^-pKa_oxi,i + 10^-pH))
//   eq (8): sum_i pKa_i(E) = sum_i pKa_red,i + log10((e^(-v F E0_prot / kB T)
//                    + e^(-F E / kB T)) / (e^(-v F E0_deprot / kB T) + e^(-F E / kB T)))
// The logarithm in eq (8) is read as base 10 (it adds to a sum of pKa values);
// v multiplies the E0 terms and not the E term, as printed.  Sums of
// exponentials are taken in log space (log(a + b) = max + log1p(exp(-|d|)))
// so no term under- or overflows.
namespace {

inline double log_add(double a, double b) { // ln(e^a + e^b)
    const double m = std::fmax(a, b);
    return m + std::log1p(std::exp(-std::fabs(a - b)));
}

bool finite_all(const double* p, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

} // namespace

extern "C" int cph_predict_delta_e0(int n_sites, const double* pka_red, const double* pka_oxi,
                                    double T, double v, double* delta_e0) {
    if (n_sites < 0 || (n_sites > 0 && (!pka_red || !pka_oxi)) || !delta_e0)
        return afail("cph_predict_delta_e0: bad arguments");
    if (!(T > 0.0) || !(v > 0.0) || !std::isfinite(T) || !std::isfinite(v))
        return afail("cph_predict_delta_e0: needs T > 0 and v > 0");
    if (!finite_all(pka_red, n_sites) || !finite_all(pka_oxi, n_sites))
        return afail("cph_predict_delta_e0: non-finite pKa");
    double s = 0.0;
    for (int i = 0; i < n_sites; ++i) s += pka_red[i] - pka_oxi[i];
    *delta_e0 = cph::kBoltzmann * T * cph::kLn10 * s / (v * cph::kFaraday);
    return CPH_OK;
}

extern "C" int cph_predict_e0(int n_pts, const double* pH, double e0_prot, int n_sites,
                              const double* pka_red, const double* pka_oxi, double T, double v,
                              double* e0) {
    if (n_pts < 0 || (n_pts > 0 && (!pH || !e0)) || n_sites < 0 ||
        (n_sites > 0 && (!pka_red || !pka_oxi)))
        return afail("cph_predict_e0: bad arguments");
    if (!(T > 0.0) || !(v > 0.0) || !std::isfinite(T) || !std::isfinite(v) || !std::isfinite(e0_prot))
        return afail("cph_predict_e0: needs T > 0, v > 0 and a finite E0_prot");
    if (!finite_all(pH, n_pts) || !finite_all(pka_red, n_sites) || !finite_all(pka_oxi, n_sites))
        return afail("cph_predict_e0: non-finite pH or pKa");
    const double scale = cph::kBoltzmann * T / (v * cph::kFaraday);
    for (int k = 0; k < n_pts; ++k) {
        const double lp = -cph::kLn10 * pH[k];
        double s = 0.0;
        for (int i = 0; i < n_sites; ++i)
            s += log_add(-cph::kLn10 * pka_red[i], lp) - log_add(-cph::kLn10 * pka_oxi[i], lp);
        e0[k] = e0_prot + scale * s;
    }
    return CPH_OK;
}

extern "C" int cph_predict_sum_pka(int n_pts, const double* E, double e0_prot, double e0_deprot,
                                   int n_sites, const double* pka_red, double T, double v,
                                   double* sum_pka) {
    if (n_pts < 0 || (n_pts > 0 && (!E || !sum_pka)) || n_sites < 0 || (n_sites > 0 && !pka_red))
        return afail("cph_predict_sum_pka: bad arguments");
    if (!(T > 0.0) || !(v > 0.0) || !std::isfinite(T) || !std::isfinite(v) ||
        !std::isfinite(e0_prot) || !std::isfinite(e0_deprot))
        return afail("cph_predict_sum_pka: needs T > 0, v > 0 and finite E0 values");
    if (!finite_all(E, n_pts) || !finite_all(pka_red, n_sites))
        return afail("cph_predict_sum_pka: non-finite E or pKa");
    const double b = cph::kFaraday / (cph::kBoltzmann * T);
    double base = 0.0;
    for (int i = 0; i < n_sites; ++i) base += pka_red[i];
    for (int k = 0; k < n_pts; ++k) {
        const double le = -b * E[k];
        sum_pka[k] = base + (log_add(-v * b * e0_prot, le) - log_add(-v * b * e0_deprot, le)) / cph::kLn10;
    }
    return CPH_OK;
}
