// qmc_fit.cpp -- variance-reduction fit on the host (Sec. 2.4).
//
// Per integration variable j the histogram row hist[j][0..bins) of |f| (one shifted
// lattice, no transform) gives the CDF at the bin edges x_b = b/bins.  The PolySingular
// map p (Eq. (ISfit), |a2| and |a3| as in the fit-function table of App. A.5) is fitted to
// the inverse CDF: p(CDF(x_b)) ~ x_b on every stepsize-th edge, by Levenberg-Marquardt
// with the parameter bounds a0 >= 1.001, a1 <= -0.001 of Sec. 2.4 enforced by projection.
// The paper uses GSL's nonlinear least squares with maxiter/xtol/gtol/ftol; the same
// stopping tests are used here (xtol: |delta_i| <= xtol (|a_i| + xtol) for all i;
// gtol: max |J^T r| <= gtol max(1, cost); ftol: relative cost decrease <= ftol).
#include <cmath>
#include <cstring>
#include <vector>

#include "qmc_gb300.h"

namespace {

struct Model {
    double a[6];
};

inline double sgn1(double v) { return v < 0.0 ? -1.0 : 1.0; }

// p(y) and dp/da_k
void model(const double *a, double y, double &p, double *grad) {
    const double A2 = std::fabs(a[2]), A3 = std::fabs(a[3]);
    const double a6 = 1.0 - A2 - A3 - a[4] - a[5];
    const double d0 = a[0] - y, d1 = a[1] - y;
    const double t0 = y * (a[0] - 1.0) / d0;
    const double t1 = y * (a[1] - 1.0) / d1;
    const double y2 = y * y, y3 = y2 * y;
    p = A2 * t0 + A3 * t1 + y * (a[4] + y * (a[5] + y * a6));
    if (grad) {
        grad[0] = A2 * y * (1.0 - y) / (d0 * d0);
        grad[1] = A3 * y * (1.0 - y) / (d1 * d1);
        grad[2] = sgn1(a[2]) * (t0 - y3);
        grad[3] = sgn1(a[3]) * (t1 - y3);
        grad[4] = y - y3;
        grad[5] = y2 - y3;
    }
}

double cost_of(const double *a, const std::vector<double> &ys, const std::vector<double> &xs,
               std::vector<double> *r = nullptr) {
    double c = 0.0;
    for (size_t i = 0; i < ys.size(); ++i) {
        double p;
        model(a, ys[i], p, nullptr);
        double ri = p - xs[i];
        if (r) (*r)[i] = ri;
        c += ri * ri;
    }
    return c;
}

void project(double *a) {
    if (a[0] < 1.001) a[0] = 1.001;
    if (a[1] > -0.001) a[1] = -0.001;
}

// Solve (6x6) M x = b by Gaussian elimination with partial pivoting; false if singular.
bool solve6(double M[6][6], double b[6], double x[6]) {
    double A[6][7];
    for (int i = 0; i < 6; ++i) {
        for (int j = 0; j < 6; ++j) A[i][j] = M[i][j];
        A[i][6] = b[i];
    }
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        for (int r = c + 1; r < 6; ++r)
            if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return false;
        if (piv != c)
            for (int j = 0; j < 7; ++j) std::swap(A[c][j], A[piv][j]);
        for (int r = c + 1; r < 6; ++r) {
            double f = A[r][c] / A[c][c];
            for (int j = c; j < 7; ++j) A[r][j] -= f * A[c][j];
        }
    }
    for (int i = 5; i >= 0; --i) {
        double s = A[i][6];
        for (int j = i + 1; j < 6; ++j) s -= A[i][j] * x[j];
        x[i] = s / A[i][i];
    }
    return true;
}

void fit_one(const std::vector<double> &ys, const std::vector<double> &xs, int maxiter, double xtol,
             double gtol, double ftol, double *out) {
    double a[6] = {1.1, -0.1, 0.0, 0.0, 1.0, 0.0};   // the identity map p(y) = y
    const size_t N = ys.size();
    std::vector<double> r(N);
    double cost = cost_of(a, ys, xs, &r);
    double lambda = 1e-3;
    for (int it = 0; it < maxiter; ++it) {
        double JtJ[6][6] = {{0}};
        double g[6] = {0};
        for (size_t i = 0; i < N; ++i) {
            double p, gr[6];
            model(a, ys[i], p, gr);
            for (int u = 0; u < 6; ++u) {
                g[u] += gr[u] * r[i];
                for (int v = 0; v < 6; ++v) JtJ[u][v] += gr[u] * gr[v];
            }
        }
        double gmax = 0.0;
        for (int u = 0; u < 6; ++u) gmax = std::fmax(gmax, std::fabs(g[u]));
        if (gmax <= gtol * std::fmax(1.0, cost)) break;
        bool accepted = false;
        for (int tries = 0; tries < 12 && !accepted; ++tries) {
            double M[6][6], b[6], delta[6];
            for (int u = 0; u < 6; ++u) {
                for (int v = 0; v < 6; ++v) M[u][v] = JtJ[u][v];
                M[u][u] += lambda * std::fmax(JtJ[u][u], 1e-12);
                b[u] = -g[u];
            }
            if (!solve6(M, b, delta)) {
                lambda *= 10.0;
                continue;
            }
            double an[6];
            for (int u = 0; u < 6; ++u) an[u] = a[u] + delta[u];
            project(an);
            double cn = cost_of(an, ys, xs, nullptr);
            if (cn < cost) {
                bool small = true;
                for (int u = 0; u < 6; ++u)
                    if (std::fabs(an[u] - a[u]) > xtol * (std::fabs(a[u]) + xtol)) small = false;
                double dec = cost - cn;
                std::memcpy(a, an, sizeof(a));
                cost = cost_of(a, ys, xs, &r);
                lambda = std::fmax(lambda * 0.1, 1e-12);
                accepted = true;
                if (small || dec <= ftol * cost) it = maxiter;   // converged
            } else {
                lambda *= 10.0;
            }
        }
        if (!accepted) break;
    }
    std::memcpy(out, a, sizeof(a));
}

}  // namespace

extern "C" int qmc_fit_polysingular(const double *hist, int dim, int bins, const qmc_fit_opts *opts,
                                    double *params) {
    if (!hist || !params) return QMC_ERR_ARG;
    if (dim < 1 || dim > QMC_MAX_DIM) return QMC_ERR_DIM;
    if (bins < 2) return QMC_ERR_RANGE;
    int maxiter = 40, stepsize = 10;
    double xtol = 3e-3, gtol = 1e-8, ftol = 1e-8;
    if (opts) {
        if (opts->maxiter > 0) maxiter = opts->maxiter;
        if (opts->stepsize > 0) stepsize = opts->stepsize;
        if (opts->xtol > 0) xtol = opts->xtol;
        if (opts->gtol > 0) gtol = opts->gtol;
        if (opts->ftol > 0) ftol = opts->ftol;
    }
    for (int j = 0; j < dim; ++j) {
        const double *h = hist + (size_t)j * bins;
        std::vector<double> cdf(bins + 1, 0.0);
        for (int b = 0; b < bins; ++b) cdf[b + 1] = cdf[b] + std::fabs(h[b]);
        double tot = cdf[bins];
        double *out = params + 6 * j;
        if (!(tot > 0.0) || !std::isfinite(tot)) {
            const double ident[6] = {1.1, -0.1, 0.0, 0.0, 1.0, 0.0};
            std::memcpy(out, ident, sizeof(ident));
            continue;
        }
        std::vector<double> ys, xs;
        for (int b = 0; b <= bins; b += stepsize) {
            ys.push_back(cdf[b] / tot);
            xs.push_back((double)b / bins);
        }
        if (bins % stepsize != 0) {
            ys.push_back(1.0);
            xs.push_back(1.0);
        }
        fit_one(ys, xs, maxiter, xtol, gtol, ftol, out);
    }
    return QMC_OK;
}
