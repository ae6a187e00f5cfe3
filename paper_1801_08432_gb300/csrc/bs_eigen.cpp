// Dense symmetric eigensolver (FP64, host) for the Lanczos matrix T.
//
// The paper hands the (block-)tridiagonal Lanczos matrix to LAPACK's DSYEV.
// Here, only the lowest eigenvectors are needed, so:
//   1. Householder reduction to tridiagonal form, A = Q T Q^T, with the
//      rank-two update A <- A - v q^T - q v^T (p = tau A v, q = p - (tau/2)
//      (v^T p) v) of Golub & Van Loan, Sec. 8.3;
//   2. every eigenvalue of T by bisection on the Sturm count (the number of
//      negative pivots of the LDL^T factorization of T - x I equals the
//      number of eigenvalues below x);
//   3. eigenvectors of the lowest ones by inverse iteration on T - lambda I
//      (tridiagonal Gaussian elimination with partial pivoting), orthogonalized
//      against earlier vectors of nearby eigenvalues, then back-transformed
//      by Q.
#include <algorithm>
#include <cmath>
#include <vector>

#include "bs_internal.h"

namespace bs {

namespace {

void householder_tridiag(int n, std::vector<double> &A, std::vector<double> &d, std::vector<double> &e,
                         std::vector<double> &Q)
{
    Q.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
    std::vector<double> v(n), p(n), q(n);
    for (int k = 0; k + 2 < n; ++k) {
        double below = 0.0;   // the column is already tridiagonal when this is zero
        for (int i = k + 2; i < n; ++i) below += A[(size_t)i * n + k] * A[(size_t)i * n + k];
        if (below == 0.0) continue;
        double norm2 = below + A[(size_t)(k + 1) * n + k] * A[(size_t)(k + 1) * n + k];
        const double alpha = std::sqrt(norm2);
        if (alpha == 0.0) continue;
        const double a1 = A[(size_t)(k + 1) * n + k];
        const double target = a1 >= 0.0 ? -alpha : alpha;   // the value A[k+1][k] takes
        std::fill(v.begin(), v.end(), 0.0);
        v[k + 1] = a1 - target;
        for (int i = k + 2; i < n; ++i) v[i] = A[(size_t)i * n + k];
        double vv = 0.0;
        for (int i = k + 1; i < n; ++i) vv += v[i] * v[i];
        if (vv == 0.0) continue;
        const double tau = 2.0 / vv;
        for (int i = k; i < n; ++i) {
            double t = 0.0;
            for (int j = k + 1; j < n; ++j) t += A[(size_t)i * n + j] * v[j];
            p[i] = tau * t;
        }
        double vp = 0.0;
        for (int i = k + 1; i < n; ++i) vp += v[i] * p[i];
        const double half = 0.5 * tau * vp;
        for (int i = k; i < n; ++i) q[i] = p[i] - half * v[i];
        for (int i = k; i < n; ++i)
            for (int j = k; j < n; ++j) A[(size_t)i * n + j] -= v[i] * q[j] + q[i] * v[j];
        for (int i = 0; i < n; ++i) {   // Q <- Q (I - tau v v^T)
            double t = 0.0;
            for (int j = k + 1; j < n; ++j) t += Q[(size_t)i * n + j] * v[j];
            t *= tau;
            for (int j = k + 1; j < n; ++j) Q[(size_t)i * n + j] -= t * v[j];
        }
    }
    d.resize(n);
    e.assign(n, 0.0);
    for (int i = 0; i < n; ++i) d[i] = A[(size_t)i * n + i];
    for (int i = 0; i + 1 < n; ++i) e[i] = A[(size_t)(i + 1) * n + i];
}

// number of eigenvalues of the tridiagonal (d, e) below x
int sturm_below(int n, const std::vector<double> &d, const std::vector<double> &e, double x, double tiny)
{
    int neg = 0;
    double piv = 1.0;
    for (int i = 0; i < n; ++i) {
        const double off = i > 0 ? e[i - 1] * e[i - 1] / piv : 0.0;
        piv = d[i] - x - off;
        if (std::fabs(piv) < tiny) piv = -tiny;
        if (piv < 0.0) ++neg;
    }
    return neg;
}

// solve (T - lam I) y = b in place (b -> y), Gaussian elimination with row
// pivoting on the tridiagonal band
void tridiag_solve(int n, const std::vector<double> &d, const std::vector<double> &e, double lam, double tiny,
                   std::vector<double> &b)
{
    // rows: sub l[i] (col i-1), diag m[i], sup u[i] (col i+1), fill f[i] (col i+2)
    std::vector<double> l(n, 0.0), m(n), u(n, 0.0), f(n, 0.0);
    for (int i = 0; i < n; ++i) {
        m[i] = d[i] - lam;
        if (i > 0) l[i] = e[i - 1];
        if (i + 1 < n) u[i] = e[i];
    }
    for (int i = 0; i + 1 < n; ++i) {
        // pivot between row i (entries m[i], u[i], f[i]) and row i+1 (l[i+1], m[i+1], u[i+1])
        if (std::fabs(l[i + 1]) > std::fabs(m[i])) {
            std::swap(m[i], l[i + 1]);
            std::swap(u[i], m[i + 1]);
            std::swap(f[i], u[i + 1]);
            std::swap(b[i], b[i + 1]);
        }
        if (std::fabs(m[i]) < tiny) m[i] = tiny;
        const double r = l[i + 1] / m[i];
        m[i + 1] -= r * u[i];
        u[i + 1] -= r * f[i];
        b[i + 1] -= r * b[i];
        l[i + 1] = 0.0;
    }
    if (std::fabs(m[n - 1]) < tiny) m[n - 1] = tiny;
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        if (i + 1 < n) s -= u[i] * b[i + 1];
        if (i + 2 < n) s -= f[i] * b[i + 2];
        b[i] = s / m[i];
    }
}

}  // namespace

// Symmetric n x n matrix A (row-major): all eigenvalues ascending in w[n];
// the eigenvectors of the lowest nvec in the columns of Z (n x nvec,
// row-major).  Returns false on failure.
bool host_eigh(int n, const double *A, double *w, double *Z, int nvec)
{
    if (n <= 0) return true;
    nvec = std::min(nvec, n);
    std::vector<double> M(A, A + (size_t)n * n), d, e, Q;
    householder_tridiag(n, M, d, e, Q);
    double lo = 1e300, hi = -1e300, scale = 0.0;
    for (int i = 0; i < n; ++i) {
        const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(e[i]) : 0.0);
        lo = std::min(lo, d[i] - r);
        hi = std::max(hi, d[i] + r);
        scale = std::max(scale, std::fabs(d[i]) + r);
    }
    if (scale == 0.0) scale = 1.0;
    const double tiny = 1e-300 + 1e-30 * scale;
    lo -= 1e-12 * scale;
    hi += 1e-12 * scale;
    // eigenvalue j: smallest x with sturm_below(x) > j
    for (int j = 0; j < n; ++j) {
        double a = lo, b = hi;
        for (int it = 0; it < 200 && b - a > 4e-16 * scale; ++it) {
            const double mid = 0.5 * (a + b);
            if (sturm_below(n, d, e, mid, tiny) > j) b = mid;
            else a = mid;
        }
        w[j] = 0.5 * (a + b);
    }
    // inverse iteration for the lowest nvec
    std::vector<double> y(n), Yt((size_t)nvec * n);
    for (int j = 0; j < nvec; ++j) {
        for (int i = 0; i < n; ++i) y[i] = 1.0 + 0.1 * std::sin(1.0 + 7.0 * i + 13.0 * j);
        const double lam = w[j] + 1e-13 * scale;
        for (int it = 0; it < 4; ++it) {
            tridiag_solve(n, d, e, lam, tiny, y);
            // keep orthogonal to earlier vectors of close eigenvalues
            for (int p = 0; p < j; ++p) {
                if (std::fabs(w[p] - w[j]) > 1e-6 * scale) continue;
                double dot = 0.0;
                for (int i = 0; i < n; ++i) dot += Yt[(size_t)p * n + i] * y[i];
                for (int i = 0; i < n; ++i) y[i] -= dot * Yt[(size_t)p * n + i];
            }
            double nrm = 0.0;
            for (int i = 0; i < n; ++i) nrm += y[i] * y[i];
            nrm = std::sqrt(nrm);
            if (nrm == 0.0) return false;
            for (int i = 0; i < n; ++i) y[i] /= nrm;
        }
        std::copy(y.begin(), y.end(), Yt.begin() + (size_t)j * n);
    }
    // back-transform: Z = Q Y
    for (int r = 0; r < n; ++r)
        for (int j = 0; j < nvec; ++j) {
            double s = 0.0;
            for (int i = 0; i < n; ++i) s += Q[(size_t)r * n + i] * Yt[(size_t)j * n + i];
            Z[(size_t)r * nvec + j] = s;
        }
    return true;
}

// Banded symmetric matrix (half-bandwidth bw, row-major full n x n storage):
// the lowest nval eigenvalues by bisection on inertia counts and the
// eigenvectors of the lowest nvec by inverse iteration, without forming a
// tridiagonal matrix.  The inertia count of A - x I is the number of negative
// pivots of its elimination without pivoting (Sylvester's law of inertia);
// fill stays inside the band, so a count costs O(n bw^2).  Inverse iteration
// solves (A - lambda I) y = b by Gaussian elimination with row pivoting on
// the band (upper bandwidth grows to 2 bw).
bool host_eigh_banded(int n, int bw, const double *A, int nval, double *w, double *Z, int nvec)
{
    if (n <= 0) return true;
    nval = std::min(nval, n);
    nvec = std::min(nvec, nval);
    const int W = 2 * bw + 1;   // band storage: B[i][bw + j - i] = A[i][j]
    std::vector<double> band((size_t)n * W, 0.0);
    double scale = 0.0, lo = 1e300, hi = -1e300;
    for (int i = 0; i < n; ++i) {
        double r = 0.0;
        for (int j = std::max(0, i - bw); j <= std::min(n - 1, i + bw); ++j) {
            band[(size_t)i * W + bw + j - i] = A[(size_t)i * n + j];
            if (j != i) r += std::fabs(A[(size_t)i * n + j]);
        }
        const double d = A[(size_t)i * n + i];
        lo = std::min(lo, d - r);
        hi = std::max(hi, d + r);
        scale = std::max(scale, std::fabs(d) + r);
    }
    if (scale == 0.0) scale = 1.0;
    const double tiny = 1e-300 + 1e-30 * scale;
    lo -= 1e-12 * scale;
    hi += 1e-12 * scale;
    std::vector<double> M((size_t)n * W);
    auto below = [&](double x) {
        // elimination without pivoting on the band of A - x I
        std::copy(band.begin(), band.end(), M.begin());
        for (int i = 0; i < n; ++i) M[(size_t)i * W + bw] -= x;
        int neg = 0;
        for (int k = 0; k < n; ++k) {
            double piv = M[(size_t)k * W + bw];
            if (std::fabs(piv) < tiny) piv = M[(size_t)k * W + bw] = -tiny;
            if (piv < 0.0) ++neg;
            for (int i = k + 1; i <= std::min(n - 1, k + bw); ++i) {
                const double f = M[(size_t)i * W + bw + k - i] / piv;
                if (f == 0.0) continue;
                for (int j = k + 1; j <= std::min(n - 1, k + bw); ++j)
                    M[(size_t)i * W + bw + j - i] -= f * M[(size_t)k * W + bw + j - k];
            }
        }
        return neg;
    };
    for (int j = 0; j < nval; ++j) {
        double a = lo, b = hi;
        for (int it = 0; it < 200 && b - a > 4e-16 * scale; ++it) {
            const double mid = 0.5 * (a + b);
            if (below(mid) > j) b = mid;
            else a = mid;
        }
        w[j] = 0.5 * (a + b);
    }
    // inverse iteration; LU with row pivoting in a band of upper width 2 bw
    const int U = 2 * bw, LW = bw + U + 1;   // columns i-bw .. i+U
    std::vector<double> L((size_t)n * LW), y(n), Y((size_t)nvec * n);
    std::vector<int> perm(n);
    for (int v = 0; v < nvec; ++v) {
        const double lam = w[v] + 1e-13 * scale;
        // factor: row i of L holds A[i][i-bw .. i+U] at offset (j - i + bw)
        std::fill(L.begin(), L.end(), 0.0);
        for (int i = 0; i < n; ++i)
            for (int j = std::max(0, i - bw); j <= std::min(n - 1, i + bw); ++j)
                L[(size_t)i * LW + j - i + bw] = A[(size_t)i * n + j] - (i == j ? lam : 0.0);
        auto at = [&](int i, int j) -> double & { return L[(size_t)i * LW + j - i + bw]; };
        std::vector<double> mult((size_t)n * bw, 0.0);   // multipliers of column k for rows k+1..k+bw
        for (int k = 0; k < n; ++k) {
            int p = k;
            for (int i = k + 1; i <= std::min(n - 1, k + bw); ++i)
                if (std::fabs(at(i, k)) > std::fabs(at(p, k))) p = i;
            perm[k] = p;
            if (p != k)
                for (int j = k; j <= std::min(n - 1, k + U); ++j) {
                    // rows k and p share the column range k..k+U inside the band (p <= k+bw)
                    if (j - p + bw < 0 || j - p + bw >= LW) continue;
                    std::swap(at(k, j), at(p, j));
                }
            if (std::fabs(at(k, k)) < tiny) at(k, k) = tiny;
            for (int i = k + 1; i <= std::min(n - 1, k + bw); ++i) {
                const double f = at(i, k) / at(k, k);
                mult[(size_t)k * bw + (i - k - 1)] = f;
                at(i, k) = 0.0;
                if (f == 0.0) continue;
                for (int j = k + 1; j <= std::min(n - 1, k + U); ++j)
                    if (j - i + bw < LW) at(i, j) -= f * at(k, j);
            }
        }
        for (int i = 0; i < n; ++i) y[i] = 1.0 + 0.1 * std::sin(1.0 + 7.0 * i + 13.0 * v);
        for (int it = 0; it < 4; ++it) {
            // forward: apply the row swaps and multipliers in order
            for (int k = 0; k < n; ++k) {
                if (perm[k] != k) std::swap(y[k], y[perm[k]]);
                for (int i = k + 1; i <= std::min(n - 1, k + bw); ++i) y[i] -= mult[(size_t)k * bw + (i - k - 1)] * y[k];
            }
            for (int i = n - 1; i >= 0; --i) {
                double s = y[i];
                for (int j = i + 1; j <= std::min(n - 1, i + U); ++j) s -= at(i, j) * y[j];
                y[i] = s / at(i, i);
            }
            for (int p = 0; p < v; ++p) {
                if (std::fabs(w[p] - w[v]) > 1e-6 * scale) continue;
                double dot = 0.0;
                for (int i = 0; i < n; ++i) dot += Y[(size_t)p * n + i] * y[i];
                for (int i = 0; i < n; ++i) y[i] -= dot * Y[(size_t)p * n + i];
            }
            double nrm = 0.0;
            for (int i = 0; i < n; ++i) nrm += y[i] * y[i];
            nrm = std::sqrt(nrm);
            if (!(nrm > 0.0)) return false;
            for (int i = 0; i < n; ++i) y[i] /= nrm;
        }
        std::copy(y.begin(), y.end(), Y.begin() + (size_t)v * n);
    }
    for (int r = 0; r < n; ++r)
        for (int v = 0; v < nvec; ++v) Z[(size_t)r * nvec + v] = Y[(size_t)v * n + r];
    return true;
}

}  // namespace bs

extern "C" int bs_debug_eigh_banded(int n, int bw, const double *A, int nval, double *w, double *Z, int nvec)
{
    if (n < 0 || bw < 0 || nval < 0 || nvec < 0 || nvec > nval || (n > 0 && (!A || !w || (nvec > 0 && !Z))))
        return BS_EINVAL;
    return bs::host_eigh_banded(n, bw, A, nval, w, Z, nvec) ? BS_OK : BS_EBREAKDOWN;
}

extern "C" int bs_debug_eigh(int n, const double *A, double *w, double *Z, int nvec)
{
    if (n < 0 || nvec < 0 || (n > 0 && (!A || !w || (nvec > 0 && !Z)))) return BS_EINVAL;
    return bs::host_eigh(n, A, w, Z, nvec) ? BS_OK : BS_EBREAKDOWN;
}
