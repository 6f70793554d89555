// Host FP64 linear algebra for plan time: Householder QR (R factor only), its tall-skinny
// pairwise reduction, and the one-sided Jacobi SVD (Hestenes' method: rotate column pairs
// until all columns are mutually orthogonal; the column norms are the singular values).
#include "linalg.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace m2l {

// In-place Householder QR of the column-major m x n matrix A (m >= n); the upper triangle of
// the first n rows holds R afterwards.
static void householder_qr(double *A, long m, int n) {
    std::vector<double> v(m);
    for (int j = 0; j < n && j < m; ++j) {
        double *a = A + (size_t)j * m;
        double norm2 = 0.0;
        for (long i = j; i < m; ++i) norm2 += a[i] * a[i];
        double norm = std::sqrt(norm2);
        if (norm == 0.0) continue;
        double alpha = a[j] > 0 ? -norm : norm;
        long len = m - j;
        for (long i = 0; i < len; ++i) v[i] = a[j + i];
        v[0] -= alpha;
        double vnorm2 = norm2 - a[j] * a[j] + v[0] * v[0];
        if (vnorm2 == 0.0) continue;
        for (int c = j + 1; c < n; ++c) {
            double *col = A + (size_t)c * m + j;
            double dot = 0.0;
            for (long i = 0; i < len; ++i) dot += v[i] * col[i];
            double f = 2.0 * dot / vnorm2;
            for (long i = 0; i < len; ++i) col[i] -= f * v[i];
        }
        a[j] = alpha;
        for (long i = j + 1; i < m; ++i) a[i] = 0.0;
    }
}

static std::vector<double> r_of(std::vector<double> A, long m, int n) {
    householder_qr(A.data(), m, n);
    std::vector<double> R((size_t)n * n, 0.0);
    for (int c = 0; c < n; ++c)
        for (int r = 0; r <= c && r < m; ++r) R[(size_t)c * n + r] = A[(size_t)c * m + r];
    return R;
}

std::vector<double> stacked_r_factor(std::vector<std::vector<double>> blocks, int n) {
    if (blocks.empty()) return std::vector<double>((size_t)n * n, 0.0);
    while (blocks.size() > 1) {
        size_t npairs = (blocks.size() + 1) / 2;
        std::vector<std::vector<double>> next(npairs);
#pragma omp parallel for schedule(dynamic, 1)
        for (long k = 0; k < (long)npairs; ++k) {
            size_t a = 2 * k, b = 2 * k + 1;
            if (b >= blocks.size()) {
                long m = (long)(blocks[a].size() / n);
                next[k] = m >= n ? r_of(blocks[a], m, n) : blocks[a];
                continue;
            }
            long ma = (long)(blocks[a].size() / n), mb = (long)(blocks[b].size() / n);
            long m = ma + mb;
            std::vector<double> S((size_t)m * n);
            for (int c = 0; c < n; ++c) {
                std::copy(blocks[a].begin() + (size_t)c * ma, blocks[a].begin() + (size_t)(c + 1) * ma,
                          S.begin() + (size_t)c * m);
                std::copy(blocks[b].begin() + (size_t)c * mb, blocks[b].begin() + (size_t)(c + 1) * mb,
                          S.begin() + (size_t)c * m + ma);
            }
            next[k] = m >= n ? r_of(std::move(S), m, n) : S;
        }
        blocks.swap(next);
    }
    long m = (long)(blocks[0].size() / n);
    if (m == n) {
        // make sure the single remaining block is triangular
        return r_of(blocks[0], m, n);
    }
    return r_of(blocks[0], m, n);
}

void jacobi_svd(const std::vector<double> &A, int m, int n, std::vector<double> &U,
                std::vector<double> &s, std::vector<double> &V) {
    std::vector<double> W(A);
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    // Round-robin ordering: every sweep visits each column pair once, in n-1 (or n) rounds of
    // disjoint pairs that can be rotated concurrently.
    int np = n + (n & 1);
    std::vector<int> ring(np);
    std::iota(ring.begin(), ring.end(), 0);
    const double tol = 1e-15;
    for (int sweep = 0; sweep < 80; ++sweep) {
        double off = 0.0;
        for (int round = 0; round < np - 1; ++round) {
#pragma omp parallel for schedule(static) reduction(max : off)
            for (int k = 0; k < np / 2; ++k) {
                int i = ring[k], j = ring[np - 1 - k];
                if (i >= n || j >= n) continue;
                if (i > j) std::swap(i, j);
                double *wi = W.data() + (size_t)i * m, *wj = W.data() + (size_t)j * m;
                double a = 0, b = 0, g = 0;
                for (int r = 0; r < m; ++r) {
                    a += wi[r] * wi[r];
                    b += wj[r] * wj[r];
                    g += wi[r] * wj[r];
                }
                if (a == 0.0 || b == 0.0) continue;
                double rel = std::fabs(g) / std::sqrt(a * b);
                off = std::max(off, rel);
                if (rel <= tol) continue;
                double zeta = (b - a) / (2.0 * g);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
                for (int r = 0; r < m; ++r) {
                    double x = wi[r], y = wj[r];
                    wi[r] = c * x - sn * y;
                    wj[r] = sn * x + c * y;
                }
                double *vi = V.data() + (size_t)i * n, *vj = V.data() + (size_t)j * n;
                for (int r = 0; r < n; ++r) {
                    double x = vi[r], y = vj[r];
                    vi[r] = c * x - sn * y;
                    vj[r] = sn * x + c * y;
                }
            }
            // rotate the ring, keeping position 0 fixed
            int last = ring[np - 1];
            for (int k = np - 1; k > 1; --k) ring[k] = ring[k - 1];
            ring[1] = last;
        }
        if (off <= tol) break;
    }
    std::vector<double> norms(n);
    for (int c = 0; c < n; ++c) {
        double a = 0;
        for (int r = 0; r < m; ++r) a += W[(size_t)c * m + r] * W[(size_t)c * m + r];
        norms[c] = std::sqrt(a);
    }
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return norms[x] > norms[y]; });
    s.assign(n, 0.0);
    U.assign((size_t)m * n, 0.0);
    std::vector<double> Vs((size_t)n * n);
    for (int k = 0; k < n; ++k) {
        int c = order[k];
        s[k] = norms[c];
        if (norms[c] > 0)
            for (int r = 0; r < m; ++r) U[(size_t)k * m + r] = W[(size_t)c * m + r] / norms[c];
        std::copy(V.begin() + (size_t)c * n, V.begin() + (size_t)(c + 1) * n, Vs.begin() + (size_t)k * n);
    }
    V.swap(Vs);
}

void orthonormalize_columns(double *M, int rows, int cols) {
    for (int c = 0; c < cols; ++c) {
        double *vc = M + (size_t)c * rows;
        for (int pass = 0; pass < 2; ++pass)
            for (int b = 0; b < c; ++b) {
                const double *vb = M + (size_t)b * rows;
                double d = 0.0;
                for (int r = 0; r < rows; ++r) d += vb[r] * vc[r];
                for (int r = 0; r < rows; ++r) vc[r] -= d * vb[r];
            }
        double nr = 0.0;
        for (int r = 0; r < rows; ++r) nr += vc[r] * vc[r];
        nr = std::sqrt(nr);
        if (nr > 0)
            for (int r = 0; r < rows; ++r) vc[r] /= nr;
    }
}

}  // namespace m2l
