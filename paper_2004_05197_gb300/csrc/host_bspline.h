// Host-side B-spline numerics of libiga (tables, index sets, interpolation set-up).
//
// Own implementations of published methods:
//  * knot span search by bisection and the triangular Cox-de Boor evaluation of
//    the deg+1 non-zero B-splines and their first derivatives on a span
//    (de Boor, "A Practical Guide to Splines", Ch. X);
//  * Gauss-Legendre nodes by Newton's method on P_n from its three-term recurrence;
//  * de Boor's knot averaging for interpolation knots;
//  * LU factorisation of the banded collocation matrix without pivoting (the
//    matrix is totally positive, so no pivoting is needed: de Boor, Ch. XIII).
#pragma once

#include <cmath>
#include <vector>

namespace hb {

inline std::vector<double> open_uniform_knots(int n_el, int p) {
    std::vector<double> t;
    for (int i = 0; i <= p; ++i) t.push_back(0.0);
    for (int i = 1; i < n_el; ++i) t.push_back((double)i / n_el);
    for (int i = 0; i <= p; ++i) t.push_back(1.0);
    return t;
}

inline void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));   // initial guess for root i
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;                         // P_0, P_1
            if (n == 1) p1 = z;
            double pn = (n == 0) ? 1.0 : p1, pm = p0;
            for (int k = 2; k <= n; ++k) {
                const double pk = ((2.0 * k - 1.0) * z * pn - (k - 1.0) * pm) / k;
                pm = pn;
                pn = pk;
            }
            dp = n * (z * pn - pm) / (z * z - 1.0);
            const double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        // recompute derivative at the converged root
        double pm = 1.0, pn = z;
        for (int k = 2; k <= n; ++k) {
            const double pk = ((2.0 * k - 1.0) * z * pn - (k - 1.0) * pm) / k;
            pm = pn;
            pn = pk;
        }
        dp = n * (z * pn - pm) / (z * z - 1.0);
        // map [-1,1] -> [0,1]: node (1 - z)/2 keeps ascending order for descending z
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);               // 2/((1-z^2)P'^2) times 1/2
    }
}

// Index mu with t[mu] <= x < t[mu+1], deg <= mu <= nbasis-1; the right end
// point belongs to the last span.
inline int find_span(const std::vector<double>& t, int deg, double x) {
    const int nb = (int)t.size() - deg - 1;
    if (x >= t[nb]) return nb - 1;
    if (x <= t[deg]) return deg;
    int lo = deg, hi = nb;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (x < t[mid]) hi = mid; else lo = mid;
    }
    return lo;
}

// Values N[a] and derivatives dN[a] of B_{mu-deg+a, deg} at x, a = 0..deg.
inline void basis_and_derivative(const std::vector<double>& t, int deg, int mu, double x, double* N,
                                 double* dN) {
    // lower-degree table: B[r][a] = B_{mu-r+a, r}(x)
    std::vector<double> prev(1, 1.0), cur;
    std::vector<double> lowdeg;   // degree deg-1 values, kept for the derivative
    for (int r = 1; r <= deg; ++r) {
        if (r == deg) lowdeg = prev;
        cur.assign(r + 1, 0.0);
        for (int a = 0; a <= r; ++a) {
            const int k = mu - r + a;   // function B_{k, r}
            double v = 0.0;
            if (a > 0) {   // term with B_{k, r-1} = prev[a-1]
                const double den = t[k + r] - t[k];
                if (den > 0) v += (x - t[k]) / den * prev[a - 1];
            }
            if (a < r) {   // term with B_{k+1, r-1} = prev[a]
                const double den = t[k + r + 1] - t[k + 1];
                if (den > 0) v += (t[k + r + 1] - x) / den * prev[a];
            }
            cur[a] = v;
        }
        prev.swap(cur);
    }
    for (int a = 0; a <= deg; ++a) N[a] = prev[a];
    if (!dN) return;
    if (deg == 0) {
        dN[0] = 0.0;
        return;
    }
    for (int a = 0; a <= deg; ++a) {
        const int k = mu - deg + a;
        double v = 0.0;
        if (a > 0) {
            const double den = t[k + deg] - t[k];
            if (den > 0) v += deg / den * lowdeg[a - 1];
        }
        if (a < deg) {
            const double den = t[k + deg + 1] - t[k + 1];
            if (den > 0) v -= deg / den * lowdeg[a];
        }
        dN[a] = v;
    }
}

// Knots of order q+1 for interpolation at abscissae xs: q+1-fold end knots at
// xs[0] and xs[n-1], interior knots by de Boor averaging of q consecutive
// abscissae.
inline std::vector<double> averaged_knots(const std::vector<double>& xs, int q) {
    const int n = (int)xs.size();
    std::vector<double> t;
    for (int i = 0; i <= q; ++i) t.push_back(xs[0]);
    for (int j = 0; j < n - q - 1; ++j) {
        double s = 0.0;
        for (int l = 1; l <= q; ++l) s += xs[j + l];
        t.push_back(s / q);
    }
    for (int i = 0; i <= q; ++i) t.push_back(xs[n - 1]);
    return t;
}

// Dense inverse of the n x n collocation matrix A[r][c] = beta_c(xs_r), by a
// banded LU factorisation without pivoting followed by n forward/backward
// substitutions.  Returns Ainv row-major.
inline bool collocation_inverse(const std::vector<double>& t, int q, const std::vector<double>& xs,
                                std::vector<double>& Ainv) {
    const int n = (int)xs.size();
    // band storage: row r holds columns lo[r] .. lo[r]+q (span - q .. span)
    std::vector<double> A((size_t)n * n, 0.0);
    std::vector<double> Nv(q + 1);
    for (int r = 0; r < n; ++r) {
        const int mu = find_span(t, q, xs[r]);
        basis_and_derivative(t, q, mu, xs[r], Nv.data(), nullptr);
        for (int a = 0; a <= q; ++a) A[(size_t)r * n + (mu - q + a)] = Nv[a];
    }
    // LU without pivoting restricted to the band |r - c| <= q
    for (int k = 0; k < n; ++k) {
        const double piv = A[(size_t)k * n + k];
        if (!(std::fabs(piv) > 0.0)) return false;
        const int rmax = std::min(n - 1, k + q);
        const int cmax = std::min(n - 1, k + q);
        for (int r = k + 1; r <= rmax; ++r) {
            const double l = A[(size_t)r * n + k] / piv;
            A[(size_t)r * n + k] = l;
            for (int c = k + 1; c <= cmax; ++c) A[(size_t)r * n + c] -= l * A[(size_t)k * n + c];
        }
    }
    Ainv.assign((size_t)n * n, 0.0);
    std::vector<double> y(n);
    for (int col = 0; col < n; ++col) {
        for (int r = 0; r < n; ++r) {
            double v = (r == col) ? 1.0 : 0.0;
            for (int c = std::max(0, r - q); c < r; ++c) v -= A[(size_t)r * n + c] * y[c];
            y[r] = v;
        }
        for (int r = n - 1; r >= 0; --r) {
            double v = y[r];
            for (int c = r + 1; c <= std::min(n - 1, r + q); ++c) v -= A[(size_t)r * n + c] * y[c];
            y[r] = v / A[(size_t)r * n + r];
        }
        for (int r = 0; r < n; ++r) Ainv[(size_t)r * n + col] = y[r];
    }
    return true;
}

}  // namespace hb
