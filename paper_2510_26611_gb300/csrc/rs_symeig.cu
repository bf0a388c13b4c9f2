// Host FP64 symmetric eigen-decomposition for the Rayleigh-Ritz step of the RHOSVD
// build (TEP step 4): Householder reduction to tridiagonal form with the
// transformations accumulated, then the implicit QL iteration with Wilkinson shifts
// on the tridiagonal matrix (Golub & Van Loan, "Matrix Computations", 4th ed.,
// sections 8.3.1 and 8.3.3).  The matrices are p x p with p <= 48: the host solves
// them in microseconds, while on the GPU one SM's FP64 pipe would spend ~1 ms.
// Also the thin QR of stacked factor matrices used by add-and-compress.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "rs_common.cuh"

namespace rs {

// A: n x n row-major (its symmetric part is used).  lam: n eigenvalues, descending.
// W: n x n row-major, column c the unit eigenvector of lam[c].  Returns false if the
// QL iteration did not converge (60 sweeps per eigenvalue).
bool symeig_host(int n, const double* A, double* lam, double* W) {
    std::vector<double> a((size_t)n * n), z((size_t)n * n, 0.0), d(n), e(n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) a[(size_t)i * n + j] = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
    for (int i = 0; i < n; ++i) z[(size_t)i * n + i] = 1.0;
    // work on A / max|a_ij| so that squares neither underflow nor overflow
    double amax = 0.0;
    for (double x : a) amax = std::max(amax, std::fabs(x));
    if (amax > 0.0)
        for (double& x : a) x /= amax;
    // Householder: for each column k, reflect a[k+1.., k] onto a multiple of e_{k+1}.
    std::vector<double> v(n), pv(n), q(n);
    for (int k = 0; k + 2 < n; ++k) {
        double norm2 = 0.0;
        for (int i = k + 1; i < n; ++i) norm2 += a[(size_t)i * n + k] * a[(size_t)i * n + k];
        if (norm2 == 0.0) continue;
        double alpha = std::sqrt(norm2);
        if (a[(size_t)(k + 1) * n + k] > 0.0) alpha = -alpha;
        std::fill(v.begin(), v.end(), 0.0);
        for (int i = k + 1; i < n; ++i) v[i] = a[(size_t)i * n + k];
        v[k + 1] -= alpha;
        double vn = 0.0;
        for (int i = k + 1; i < n; ++i) vn += v[i] * v[i];
        vn = std::sqrt(vn);
        if (vn == 0.0) continue;
        for (int i = k + 1; i < n; ++i) v[i] /= vn;
        // A <- H A H, H = I - 2 v v^T:  p = A v, K = v^T p, q = p - K v, A -= 2 (v q^T + q v^T)
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = k + 1; j < n; ++j) s += a[(size_t)i * n + j] * v[j];
            pv[i] = s;
        }
        double K = 0.0;
        for (int i = k + 1; i < n; ++i) K += v[i] * pv[i];
        for (int i = 0; i < n; ++i) q[i] = pv[i] - K * v[i];
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) a[(size_t)i * n + j] -= 2.0 * (v[i] * q[j] + q[i] * v[j]);
        // Z <- Z H
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = k + 1; j < n; ++j) s += z[(size_t)i * n + j] * v[j];
            for (int j = k + 1; j < n; ++j) z[(size_t)i * n + j] -= 2.0 * s * v[j];
        }
    }
    for (int i = 0; i < n; ++i) d[i] = a[(size_t)i * n + i];
    for (int i = 0; i + 1 < n; ++i) e[i] = a[(size_t)(i + 1) * n + i];  // couples i and i+1
    // Implicit QL with shifts from the leading 2 x 2 block of the unreduced part.
    bool ok = true;
    for (int l = 0; l < n; ++l) {
        int iter = 0;
        for (;;) {
            int m = l;
            for (; m + 1 < n; ++m) {
                // negligible against its neighbours; after 30 sweeps also against the
                // matrix (scaled to max |a_ij| = 1): the couplings between the (near-)zero
                // eigenvalues of a rank-deficient matrix stay at rounding level, where
                // the relative test never holds
                double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
                if (std::fabs(e[m]) <= 1e-16 * dd || (iter > 30 && std::fabs(e[m]) <= 4e-16 * n)) break;
            }
            if (m == l) break;
            if (++iter > 60) {
                ok = false;
                break;
            }
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = std::hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + std::copysign(r, g));
            double s = 1.0, c = 1.0, p = 0.0;
            int i = m - 1;
            bool split = false;
            for (; i >= l; --i) {
                double f = s * e[i], b = c * e[i];
                r = std::hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {  // the rotation decoupled the matrix: restart on the part above
                    d[i + 1] -= p;
                    e[m] = 0.0;
                    split = true;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * c * b;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - b;
                for (int k = 0; k < n; ++k) {
                    double zf = z[(size_t)k * n + i + 1];
                    z[(size_t)k * n + i + 1] = s * z[(size_t)k * n + i] + c * zf;
                    z[(size_t)k * n + i] = c * z[(size_t)k * n + i] - s * zf;
                }
            }
            if (split) continue;
            d[l] -= p;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    // descending order, ties by index
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return d[x] > d[y]; });
    for (int c = 0; c < n; ++c) {
        lam[c] = d[order[c]] * amax;
        for (int i = 0; i < n; ++i) W[(size_t)i * n + c] = z[(size_t)i * n + order[c]];
    }
    return ok;
}

// Thin QR of the n x k matrix A (column j at A + j n), FP64 on the host, for the
// add-and-compress of Tucker tensors (Algorithm TEP step 4): classical Gram-Schmidt with
// re-orthogonalisation: a column is projected out against the previous ones again
// while a pass removes more than half of what is left (at most three passes), the
// coefficients of all passes summed into R (k x k, upper triangular, row-major); Q
// overwrites A.  A column whose remainder is at most 1e-12 of its norm lies in the span
// of the previous ones (a molecule given twice, or sharing factor directions with
// another): its Q column is set to zero and R[j][j] = 0, since normalising rounding
// noise would give a direction that is not orthogonal to the others.
void gs_qr_host(int n, int k, double* A, double* R) {
    std::fill(R, R + (size_t)k * k, 0.0);
    std::vector<double> c(k);
    auto norm = [n](const double* v) {
        double s = 0.0;
        for (int t = 0; t < n; ++t) s += v[t] * v[t];
        return std::sqrt(s);
    };
    for (int j = 0; j < k; ++j) {
        double* aj = A + (size_t)j * n;
        const double n0 = norm(aj);
        double prev = n0, cur = n0;
        for (int pass = 0; pass < 3 && j > 0; ++pass) {
            for (int i = 0; i < j; ++i) {
                const double* qi = A + (size_t)i * n;
                double d = 0.0;
                for (int t = 0; t < n; ++t) d += qi[t] * aj[t];
                c[i] = d;
            }
            for (int i = 0; i < j; ++i) {
                const double* qi = A + (size_t)i * n;
                for (int t = 0; t < n; ++t) aj[t] -= c[i] * qi[t];
                R[(size_t)i * k + j] += c[i];
            }
            prev = cur;
            cur = norm(aj);
            if (cur >= 0.5 * prev) break;
        }
        if (cur <= 1e-12 * n0 || cur == 0.0) {
            for (int t = 0; t < n; ++t) aj[t] = 0.0;
            R[(size_t)j * k + j] = 0.0;
        } else {
            R[(size_t)j * k + j] = cur;
            for (int t = 0; t < n; ++t) aj[t] /= cur;
        }
    }
}

}  // namespace rs

extern "C" rs_status rs_symeig_host(int32_t n, const double* A, double* lam, double* W) {
    rs::clear_error();
    if (n < 1 || n > 4096 || !A || !lam || !W) {
        rs::set_error("rs_symeig_host: bad argument");
        return RS_ERR_INVALID;
    }
    if (!rs::symeig_host(n, A, lam, W)) {
        rs::set_error("rs_symeig_host: QL iteration did not converge");
        return RS_ERR_UNSUPPORTED;
    }
    return RS_OK;
}

extern "C" rs_status rs_qr_host(int32_t n, int32_t k, double* A, double* R) {
    rs::clear_error();
    if (n < 1 || k < 1 || k > 4096 || !A || !R) {
        rs::set_error("rs_qr_host: bad argument");
        return RS_ERR_INVALID;
    }
    rs::gs_qr_host(n, k, A, R);
    return RS_OK;
}
