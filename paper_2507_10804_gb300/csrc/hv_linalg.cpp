// hv_linalg.cpp -- small dense linear algebra on the host for the PSF+ build:
// the eigen-decomposition of a Hermitian matrix (cyclic complex Jacobi) and
// the inverse of a small Hermitian positive definite matrix.
#include "hv_internal.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <vector>

namespace hvi {

using cd = std::complex<double>;

// Eigenvalues (descending) and eigenvectors (columns of V, row-major) of the
// Hermitian matrix A (n x n, row-major).  Each rotation zeroes one
// off-diagonal pair: a diagonal phase makes A_pq real, then the real 2 x 2
// Jacobi rotation diagonalises the (p, q) block.
int hermitian_eig(int n, std::vector<cd> A, std::vector<double> &w, std::vector<cd> &V)
{
    V.assign((size_t)n * n, cd(0.0, 0.0));
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    auto at = [&](int i, int j) -> cd & { return A[(size_t)i * n + j]; };
    double fro = 0.0;
    for (const cd &x : A) fro += std::norm(x);
    const double stop = 1e-30 * fro;
    int sweep = 0;
    for (; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += std::norm(at(p, q));
        if (off <= stop) break;
        for (int p = 0; p < n; ++p) {
            for (int q = p + 1; q < n; ++q) {
                const cd g = at(p, q);
                const double m = std::abs(g);
                if (m == 0.0) continue;
                const cd e = g / m, ec = std::conj(e);
                const double a = at(p, p).real(), b = at(q, q).real();
                const double cot2 = (b - a) / (2.0 * m);
                const double t = (cot2 >= 0 ? 1.0 : -1.0) / (std::fabs(cot2) + std::sqrt(cot2 * cot2 + 1.0));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                // A <- A J with J = [[c, s], [-s conj(e), c conj(e)]] on columns p, q
                for (int k = 0; k < n; ++k) {
                    const cd akp = at(k, p), akq = at(k, q);
                    at(k, p) = akp * c - akq * (s * ec);
                    at(k, q) = akp * s + akq * (c * ec);
                }
                // A <- J^H A on rows p, q (J^H = [[c, -s e], [s, c e]])
                for (int k = 0; k < n; ++k) {
                    const cd apk = at(p, k), aqk = at(q, k);
                    at(p, k) = apk * c - aqk * (s * e);
                    at(q, k) = apk * s + aqk * (c * e);
                }
                at(p, q) = at(q, p) = 0.0;
                at(p, p) = at(p, p).real();
                at(q, q) = at(q, q).real();
                for (int k = 0; k < n; ++k) {
                    const cd vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = vkp * c - vkq * (s * ec);
                    V[(size_t)k * n + q] = vkp * s + vkq * (c * ec);
                }
            }
        }
    }
    if (sweep == 100) return fail(HV_EINVAL, "Hermitian eigen-decomposition did not converge");
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int i, int j) { return at(i, i).real() > at(j, j).real(); });
    w.resize(n);
    std::vector<cd> Vs((size_t)n * n);
    for (int j = 0; j < n; ++j) {
        w[j] = at(order[j], order[j]).real();
        for (int i = 0; i < n; ++i) Vs[(size_t)i * n + j] = V[(size_t)i * n + order[j]];
    }
    V.swap(Vs);
    return HV_OK;
}

// Inverse of a small nonsingular matrix (Gauss-Jordan with partial pivoting).
int small_inverse(int n, std::vector<cd> M, std::vector<cd> &inv)
{
    inv.assign((size_t)n * n, cd(0.0, 0.0));
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::abs(M[(size_t)r * n + c]) > std::abs(M[(size_t)piv * n + c])) piv = r;
        if (std::abs(M[(size_t)piv * n + c]) == 0.0) return fail(HV_EINVAL, "singular matrix in the PSF+ refinement");
        if (piv != c)
            for (int k = 0; k < n; ++k) {
                std::swap(M[(size_t)c * n + k], M[(size_t)piv * n + k]);
                std::swap(inv[(size_t)c * n + k], inv[(size_t)piv * n + k]);
            }
        const cd d = M[(size_t)c * n + c];
        for (int k = 0; k < n; ++k) {
            M[(size_t)c * n + k] /= d;
            inv[(size_t)c * n + k] /= d;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const cd f = M[(size_t)r * n + c];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                M[(size_t)r * n + k] -= f * M[(size_t)c * n + k];
                inv[(size_t)r * n + k] -= f * inv[(size_t)c * n + k];
            }
        }
    }
    return HV_OK;
}

}  // namespace hvi

extern "C" int hv_util_hermitian_eig(int n, const double *A, double *w, double *V)
{
    if (n < 1 || n > 4096 || !A || !w || !V) return hvi::fail(HV_EINVAL, "hv_util_hermitian_eig: bad arguments");
    std::vector<hvi::cd> a((size_t)n * n);
    for (size_t i = 0; i < a.size(); ++i) a[i] = hvi::cd(A[2 * i], A[2 * i + 1]);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (std::abs(a[(size_t)i * n + j] - std::conj(a[(size_t)j * n + i])) >
                1e-12 * (1.0 + std::abs(a[(size_t)i * n + j])))
                return hvi::fail(HV_EINVAL, "hv_util_hermitian_eig: matrix is not Hermitian");
    std::vector<double> ww;
    std::vector<hvi::cd> vv;
    HV_RT_INTERNAL(hvi::hermitian_eig(n, a, ww, vv));
    for (int i = 0; i < n; ++i) w[i] = ww[i];
    for (size_t i = 0; i < vv.size(); ++i) {
        V[2 * i] = vv[i].real();
        V[2 * i + 1] = vv[i].imag();
    }
    return HV_OK;
}
