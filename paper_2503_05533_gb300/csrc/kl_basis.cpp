// Host construction of the KL basis of log a (A2's second operand).
//
// Field kinds (mlmc_field.kind):
//  0  separable exponential covariance sigma^2 exp(-|x1-y1|/lam - |x2-y2|/lam).
//     The paper's own field is Eq. (5.2); this covariance is the one the
//     workloads name.  1D eigenpairs of exp(-|s-t|/lam) on [0,1]:
//       theta = 2 lam / (1 + lam^2 w^2),  b(t) = sin(w t) + lam w cos(w t),
//       (lam^2 w^2 - 1) sin w = 2 lam w cos w,
//     with exactly one root w_i in (i pi, (i+1) pi), i = 0, 1, ...  Each root is
//     found by bisection on that bracket and polished by Newton steps; the
//     L^2(0,1) norm of b is the closed form
//       1/2 - sin(2w)/(4w) + lam sin^2 w + lam^2 w^2 (1/2 + sin(2w)/(4w)).
//     2D modes are products b_i(x1) b_j(x2) with eigenvalue sigma^2 theta_i theta_j,
//     ordered by theta_i theta_j descending; values within a relative 1e-12 of a
//     run's first value are ties, ordered by i + j, then i (ascending).
//  1  Eq. (5.2): Phi_j = sigma j^-q sin(2 pi j x1) cos(2 pi j x2), j = 1..K.
//  2  a single constant mode Phi_0 = sigma.
// Every mode is separable, Phi_k(x_i, y_j) = c_k bx_k(x_i) by_k(y_j); the
// tables (c, bx, by) are built here and expanded on the device.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace mlmc {
namespace {

double char_eq(double w, double lam) {
    return (lam * lam * w * w - 1.0) * std::sin(w) - 2.0 * lam * w * std::cos(w);
}
double char_eq_dw(double w, double lam) {
    return 2.0 * lam * lam * w * std::sin(w) + (lam * lam * w * w - 1.0) * std::cos(w) -
           2.0 * lam * std::cos(w) + 2.0 * lam * w * std::sin(w);
}

double root_in_bracket(int i, double lam) {
    double lo = (i == 0) ? 1e-12 : i * M_PI;
    double hi = (i + 1) * M_PI;
    double flo = char_eq(lo, lam);
    for (int it = 0; it < 200 && hi - lo > 4e-16 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        const double fm = char_eq(mid, lam);
        if ((fm < 0.0) == (flo < 0.0)) {
            lo = mid;
            flo = fm;
        } else {
            hi = mid;
        }
    }
    double w = 0.5 * (lo + hi);
    for (int it = 0; it < 3; ++it) {
        const double d = char_eq_dw(w, lam);
        if (d == 0.0) break;
        const double step = char_eq(w, lam) / d;
        if (std::fabs(step) > 1e-10 * w) break;   // bisection already converged
        w -= step;
    }
    return w;
}

}  // namespace

Basis1D expcov_1d(double lam, int count) {
    Basis1D b;
    b.w.resize(count);
    b.theta.resize(count);
    b.norm.resize(count);
    for (int i = 0; i < count; ++i) {
        const double w = root_in_bracket(i, lam);
        b.w[i] = w;
        b.theta[i] = 2.0 * lam / (1.0 + lam * lam * w * w);
        const double s2w = std::sin(2.0 * w) / (4.0 * w);
        const double sw = std::sin(w);
        const double nn = 0.5 - s2w + lam * sw * sw + lam * lam * w * w * (0.5 + s2w);
        b.norm[i] = std::sqrt(nn);
    }
    return b;
}

void expcov_modes(double sigma2, double lam, int K, std::vector<int>& mi, std::vector<int>& mj,
                  std::vector<double>& eig, Basis1D& b1) {
    const int m1 = std::max(K, 8);
    b1 = expcov_1d(lam, m1);
    struct Cand {
        double v;
        int i, j;
    };
    std::vector<Cand> cand;
    cand.reserve((size_t)m1 * m1);
    for (int i = 0; i < m1; ++i)
        for (int j = 0; j < m1; ++j) cand.push_back({b1.theta[i] * b1.theta[j], i, j});
    std::stable_sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) { return a.v > b.v; });
    // Runs of values within kTieRtol of the run's first value are ties (theta_i theta_j and
    // theta_j theta_i are equal eigenvalues); a run is ordered by (i + j, i).
    const double kTieRtol = 1e-12;
    size_t start = 0;
    while (start < cand.size()) {
        size_t end = start + 1;
        while (end < cand.size() && cand[start].v - cand[end].v <= kTieRtol * cand[start].v) ++end;
        std::sort(cand.begin() + start, cand.begin() + end, [](const Cand& a, const Cand& b) {
            return (a.i + a.j != b.i + b.j) ? (a.i + a.j < b.i + b.j) : (a.i < b.i);
        });
        start = end;
    }
    mi.resize(K);
    mj.resize(K);
    eig.resize(K);
    for (int k = 0; k < K; ++k) {
        eig[k] = sigma2 * cand[k].v;
        mi[k] = cand[k].i;
        mj[k] = cand[k].j;
    }
}

// Separable tables: coef[K], bx[K][n+1], by[K][n+1], so that
// Phi[k][j (n+1) + i] = coef[k] * bx[k][i] * by[k][j].
bool build_separable(const mlmc_field& f, int n, std::vector<double>& coef, std::vector<double>& bx,
                     std::vector<double>& by, std::string& err) {
    const int K = f.K;
    coef.assign(K, 0.0);
    bx.assign((size_t)K * (n + 1), 0.0);
    by.assign((size_t)K * (n + 1), 0.0);
    if (f.kind == 0) {
        std::vector<int> mi, mj;
        std::vector<double> eig;
        Basis1D b1;
        expcov_modes(f.sigma2, f.corr_len, K, mi, mj, eig, b1);
        for (int k = 0; k < K; ++k) {
            coef[k] = std::sqrt(eig[k]);
            const double wi = b1.w[mi[k]], wj = b1.w[mj[k]];
            for (int t = 0; t <= n; ++t) {
                const double x = (double)t / n;
                bx[(size_t)k * (n + 1) + t] =
                    (std::sin(wi * x) + f.corr_len * wi * std::cos(wi * x)) / b1.norm[mi[k]];
                by[(size_t)k * (n + 1) + t] =
                    (std::sin(wj * x) + f.corr_len * wj * std::cos(wj * x)) / b1.norm[mj[k]];
            }
        }
        return true;
    }
    if (f.kind == 1) {
        const double sigma = std::sqrt(f.sigma2);
        for (int k = 0; k < K; ++k) {
            const int j = k + 1;
            coef[k] = sigma * std::pow((double)j, -f.q);
            for (int t = 0; t <= n; ++t) {
                const double x = (double)t / n;
                bx[(size_t)k * (n + 1) + t] = std::sin(2.0 * M_PI * j * x);
                by[(size_t)k * (n + 1) + t] = std::cos(2.0 * M_PI * j * x);
            }
        }
        return true;
    }
    if (f.kind == 2) {
        if (K != 1) {
            err = "field kind 2 (constant) needs K = 1";
            return false;
        }
        coef[0] = std::sqrt(f.sigma2);
        std::fill(bx.begin(), bx.end(), 1.0);
        std::fill(by.begin(), by.end(), 1.0);
        return true;
    }
    err = "unknown field kind";
    return false;
}

}  // namespace mlmc
