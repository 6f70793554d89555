// Plan construction (host, FP64): surfaces, M2L operators, pseudo-inverse, SVD compression,
// kernel spectra and the per-level box tables; upload of the device copies.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <random>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>

#include "internal.h"
#include "linalg.h"

namespace m2l {

static thread_local std::string g_err;

void set_error(const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}
void clear_error() { g_err.clear(); }
const char *last_error() { return g_err.c_str(); }

// ---------------------------------------------------------------------------------------------
// Transfer vectors: [-3,3]^3 minus [-1,1]^3, x slowest (Sec. 3.1). Built once, on first use from
// any thread (a function-local static is initialised exactly once, with the other threads
// waiting for it).
namespace {
struct TransferTables {
    int idx[7][7][7];
    int vec[kNumTransfer][3];
    TransferTables() {
        int k = 0;
        for (int x = -3; x <= 3; ++x)
            for (int y = -3; y <= 3; ++y)
                for (int z = -3; z <= 3; ++z) {
                    int m = std::max(std::abs(x), std::max(std::abs(y), std::abs(z)));
                    if (m >= 2) {
                        idx[x + 3][y + 3][z + 3] = k;
                        vec[k][0] = x; vec[k][1] = y; vec[k][2] = z;
                        ++k;
                    } else {
                        idx[x + 3][y + 3][z + 3] = -1;
                    }
                }
    }
};
const TransferTables &transfer_tables() {
    static const TransferTables t;
    return t;
}
}  // namespace

int transfer_index(int x, int y, int z) {
    if (x < -3 || x > 3 || y < -3 || y > 3 || z < -3 || z > 3) return -1;
    return transfer_tables().idx[x + 3][y + 3][z + 3];
}

void transfer_vector(int idx, int &x, int &y, int &z) {
    const TransferTables &t = transfer_tables();
    x = t.vec[idx][0]; y = t.vec[idx][1]; z = t.vec[idx][2];
}

// ---------------------------------------------------------------------------------------------
// Surfaces (Sec. 2.1.1; App. A.3 point count): boundary points of the p^3 lattice, x slowest.
// `check` selects the downward check surface, of order pc (M2L_OPT_CHECK_ORDER); every other
// surface has order p.
static void surface(const m2l_plan_t *pl, double cx, double cy, double cz, double alpha,
                    std::vector<double> &pts, bool check = false) {
    const std::vector<int> &lat = check ? pl->lattice_c : pl->lattice;
    const int n = (int)lat.size() / 3, p = check ? pl->pc : pl->p;
    pts.resize((size_t)3 * n);
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            double c = a == 0 ? cx : (a == 1 ? cy : cz);
            pts[3 * i + a] = c + alpha * 0.5 * (-1.0 + 2.0 * lat[3 * i + a] / (p - 1));
        }
    }
}

static inline double laplace(const double *x, const double *y) {
    double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    return 1.0 / (4.0 * M_PI * std::sqrt(d0 * d0 + d1 * d1 + d2 * d2));
}

// K_t (nc x n, row-major [i][j]): downward-check of the unit target at the origin against the
// upward-equivalent points of the unit source at t (Sec. 2.2).
static void m2l_matrix(const m2l_plan_t *pl, int t, std::vector<double> &K) {
    int x, y, z;
    transfer_vector(t, x, y, z);
    std::vector<double> xs, ys;
    surface(pl, 0, 0, 0, kAlphaInner, xs, true);
    surface(pl, x, y, z, kAlphaInner, ys);
    const int n = pl->n, nc = pl->nc;
    K.resize((size_t)nc * n);
    for (int i = 0; i < nc; ++i)
        for (int j = 0; j < n; ++j) K[(size_t)i * n + j] = laplace(&xs[3 * i], &ys[3 * j]);
}

static inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Pseudo-inverse of the downward check -> equivalent matrix (Eqs. 7-10), kept as V_eps and
// Ut_eps = Sigma_eps^-1 U_eps^T (the two-factor storage of the Sec. 2.1.1 footnote), with the
// threshold eps = (alpha + max(M, N) eps_mach) s_0 of Eq. 10:
//   alpha = 0     for the FP64 paths (the paper's choice);
//   alpha = 1e-9  for the paths that compute and store in single precision. Their check
//                 potentials carry ~1e-7..1e-6 relative rounding, which the pseudo-inverse
//                 amplifies along singular directions down to eps; once stored in FP32 that noise
//                 swamps the locals when K_tau is worse conditioned than ~1e10 (p >= 7).
//                 Dropping the directions below 1e-9 s_0 keeps single-precision locals at the
//                 rounding level of their check potential for p = 4..10.
static constexpr double kPinvAlphaSingle = 1e-9;

// For the m x n (m >= n) matrix A = U diag(s) V^T (column-major factors): Veps [n][r] and
// Uteps [r][m] of the singular values above (alpha + max(m, n) eps_mach) s_0.
void pinv_truncation(int m, int n, const std::vector<double> &U, const std::vector<double> &s,
                            const std::vector<double> &V, double alpha, int &r, std::vector<double> &Veps,
                            std::vector<double> &Uteps) {
    const double thresh = (alpha + std::max(m, n) * 2.220446049250313e-16) * s[0];
    r = 0;
    while (r < n && s[r] > thresh) ++r;
    Veps.assign((size_t)n * r, 0.0);
    Uteps.assign((size_t)r * m, 0.0);
    for (int a = 0; a < r; ++a) {
        for (int i = 0; i < n; ++i) Veps[(size_t)i * r + a] = V[(size_t)a * n + i];
        for (int i = 0; i < m; ++i) Uteps[(size_t)a * m + i] = U[(size_t)a * m + i] / s[a];
    }
}

// Process-wide table of the host operators by their parameters. It holds weak references: an
// entry lives while a plan uses it, so plans alive together share one build (64 uneven instances
// of four orders build four operator sets, not 64) and memory goes with the last plan. Two plans
// that miss at the same time both build; the first to publish wins.
template <class Ops, class Key>
class OpCache {
  public:
    std::shared_ptr<const Ops> find(const Key &key) {
        std::lock_guard<std::mutex> lock(mu_);
        auto it = map_.find(key);
        if (it == map_.end()) return nullptr;
        std::shared_ptr<const Ops> sp = it->second.lock();
        if (!sp) map_.erase(it);
        return sp;
    }
    std::shared_ptr<const Ops> publish(const Key &key, std::shared_ptr<const Ops> ops) {
        std::lock_guard<std::mutex> lock(mu_);
        std::weak_ptr<const Ops> &slot = map_[key];
        if (std::shared_ptr<const Ops> sp = slot.lock()) return sp;
        slot = ops;
        return ops;
    }

  private:
    std::mutex mu_;
    std::map<Key, std::weak_ptr<const Ops>> map_;
};

// keys: (kernel, p, p_c[, rank_tol[, dir_tol]]) and (kernel, p, grid)
static OpCache<PinvOps, std::tuple<int, int, int>> g_pinv_cache;
static OpCache<BlasOps, std::tuple<int, int, int, double, int>> g_blas_cache;   // last: SVD mode
static OpCache<DirOps, std::tuple<int, int, int, double, double, int>> g_dir_cache;
static OpCache<FftOps, std::tuple<int, int, int>> g_fft_cache;

// The full SVD bases of the stacked operators (Eqs. 12-13) for one (kernel, p, p_c): every rank
// threshold truncates the same factorisation, so the tuner can try several ranks for the cost of
// one SVD. Columns are re-orthonormalised (orthonormalize_columns) in order of the singular values,
// so the leading k columns of each basis are orthonormal for every k.
struct SvdBasis {
    std::vector<double> Uf;      // nc x nc, column-major: left singular vectors of K_fat
    std::vector<double> Sb;      // n x n, column-major: right singular vectors of K_thin
    std::vector<double> s_fat, s_thin;
};
static OpCache<SvdBasis, std::tuple<int, int, int>> g_svd_cache;
// randomised bases, by (kernel, p, p_c, rank threshold): their width depends on the threshold
static OpCache<SvdBasis, std::tuple<int, int, int, double>> g_rsvd_cache;

// One-shot randomised SVD (Sec. 3.1; Halko, Martinsson and Tropp, SIAM Review 2011, Alg. 4.1 and
// 5.1) of the wide stacked matrix A = [A_1 ... A_T] (m rows), A_t = K_t (m = nc, the fat stack) or
// A_t = K_t^T (m = n, the transposed thin stack): Y = A Omega with a Gaussian Omega of width l,
// Q = orth(Y), then the SVD of B = Q^T A through the R factor of B^T (tall-skinny QR of the blocks
// A_t^T Q, then Jacobi on l x l); the left singular vectors are Q times those of B. No power
// iterations. The width starts at 0.6 m + 10 (ten oversamples beyond the ranks the thresholds of
// interest keep: 143 of 152 at p = 6, 173 of 296 at p = 8 for 1e-7) and grows by half while the
// smallest sketched singular value is still at or above rank_tol times the largest, so every
// singular value the threshold keeps lies inside the sketch; at l = m it spans the column space.
static void rsvd_left(const std::vector<std::vector<double>> &Ks, int nc, int n, bool transpose, double rank_tol,
                      std::vector<double> &U, std::vector<double> &sv) {
    const int m = transpose ? n : nc, w = transpose ? nc : n;  // A_t is m x w
    auto at = [&](int t, int i, int j) {                        // A_t[i][j]
        return transpose ? Ks[t][(size_t)j * n + i] : Ks[t][(size_t)i * n + j];
    };
    int l = std::min(m, (3 * m) / 5 + 10);
    for (;;) {
        std::vector<double> Y((size_t)m * l, 0.0);  // column-major m x l
#pragma omp parallel
        {
            std::vector<double> Yp((size_t)m * l, 0.0), om((size_t)w * l);
#pragma omp for schedule(static)
            for (int t = 0; t < kNumTransfer; ++t) {
                std::mt19937_64 gen(0x5eed0000ULL + (uint64_t)t * 7919ULL + (uint64_t)l);
                std::normal_distribution<double> g(0.0, 1.0);
                for (auto &v : om) v = g(gen);
                for (int i = 0; i < m; ++i)
                    for (int j = 0; j < w; ++j) {
                        const double a = at(t, i, j);
                        const double *o = &om[(size_t)j * l];
                        for (int c = 0; c < l; ++c) Yp[(size_t)c * m + i] += a * o[c];
                    }
            }
#pragma omp critical
            for (size_t e = 0; e < Y.size(); ++e) Y[e] += Yp[e];
        }
        orthonormalize_columns(Y.data(), m, l);  // Q
        // blocks of B^T: A_t^T Q (w x l, column-major)
        std::vector<std::vector<double>> blocks(kNumTransfer);
#pragma omp parallel for schedule(static)
        for (int t = 0; t < kNumTransfer; ++t) {
            std::vector<double> &b = blocks[t];
            b.assign((size_t)w * l, 0.0);
            for (int c = 0; c < l; ++c)
                for (int i = 0; i < m; ++i) {
                    const double qv = Y[(size_t)c * m + i];
                    if (qv == 0.0) continue;
                    for (int j = 0; j < w; ++j) b[(size_t)c * w + j] += at(t, i, j) * qv;
                }
        }
        std::vector<double> R = stacked_r_factor(std::move(blocks), l);
        std::vector<double> Ur, Vr;
        jacobi_svd(R, l, l, Ur, sv, Vr);  // B = R^T Q2^T: left singular vectors of B = Vr
        const bool complete = l == m || sv[l - 1] < rank_tol * sv[0];
        if (complete) {
            U.assign((size_t)m * l, 0.0);
            for (int c = 0; c < l; ++c)
                for (int a = 0; a < l; ++a) {
                    const double v = Vr[(size_t)c * l + a];
                    for (int i = 0; i < m; ++i) U[(size_t)c * m + i] += Y[(size_t)a * m + i] * v;
                }
            orthonormalize_columns(U.data(), m, l);
            return;
        }
        l = std::min(m, l + l / 2);
    }
}

static std::shared_ptr<const SvdBasis> rsvd_basis(const m2l_plan_t *pl, const std::vector<std::vector<double>> &Ks,
                                                  double rank_tol) {
    const auto key = std::make_tuple(pl->kernel, pl->p, pl->pc, rank_tol);
    std::shared_ptr<const SvdBasis> b = g_rsvd_cache.find(key);
    if (b) return b;
    auto o = std::make_shared<SvdBasis>();
    rsvd_left(Ks, pl->nc, pl->n, false, rank_tol, o->Uf, o->s_fat);  // left singular vectors of K_fat
    rsvd_left(Ks, pl->nc, pl->n, true, rank_tol, o->Sb, o->s_thin);  // right singular vectors of K_thin
    return g_rsvd_cache.publish(key, std::move(o));
}

static std::shared_ptr<const SvdBasis> svd_basis(const m2l_plan_t *pl, const std::vector<std::vector<double>> &Ks) {
    const auto key = std::make_tuple(pl->kernel, pl->p, pl->pc);
    std::shared_ptr<const SvdBasis> b = g_svd_cache.find(key);
    if (b) return b;
    auto o = std::make_shared<SvdBasis>();
    const int n = pl->n, nc = pl->nc;
    // K_thin = [K_1; ...; K_316] (316 nc x n): stack the column-major K_t. K_fat^T =
    // [K_1^T; ...] (316 n x nc): a row-major K_t read as column-major is K_t^T.
    std::vector<std::vector<double>> thin(kNumTransfer), fatT(kNumTransfer);
    for (int t = 0; t < kNumTransfer; ++t) {
        fatT[t] = Ks[t];
        thin[t].resize((size_t)nc * n);
        for (int i = 0; i < nc; ++i)
            for (int j = 0; j < n; ++j) thin[t][(size_t)j * nc + i] = Ks[t][(size_t)i * n + j];
    }
    std::vector<double> Rf = stacked_r_factor(std::move(fatT), nc);
    std::vector<double> Rt = stacked_r_factor(std::move(thin), n);
    std::vector<double> Uf_, Ut_;
    // left singular vectors of K_fat = right singular vectors of K_fat^T (and of Rf)
    jacobi_svd(Rf, nc, nc, Uf_, o->s_fat, o->Uf);
    jacobi_svd(Rt, n, n, Ut_, o->s_thin, o->Sb);
    orthonormalize_columns(o->Uf.data(), nc, nc);
    orthonormalize_columns(o->Sb.data(), n, n);
    return g_svd_cache.publish(key, std::move(o));
}

static double rank_key(double rank_tol) { return rank_tol > 0 ? rank_tol : 0.0; }

int build_pinv(m2l_plan_t *pl) {
    if (pl->pinv) return M2L_OK;
    const auto key = std::make_tuple(pl->kernel, pl->p, pl->pc);
    std::shared_ptr<const PinvOps> ops = g_pinv_cache.find(key);
    if (!ops) {
        auto o = std::make_shared<PinvOps>();
        const int n = pl->n, nc = pl->nc;
        std::vector<double> xs, ys;
        surface(pl, 0, 0, 0, kAlphaInner, xs, true);   // downward check (order pc)
        surface(pl, 0, 0, 0, kAlphaOuter, ys);         // downward equivalent
        std::vector<double> K((size_t)nc * n);         // column-major, nc x n (nc >= n)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < nc; ++i) K[(size_t)j * nc + i] = laplace(&xs[3 * i], &ys[3 * j]);
        std::vector<double> U, sv, V;
        jacobi_svd(K, nc, n, U, sv, V);
        pinv_truncation(nc, n, U, sv, V, 0.0, o->r, o->Veps, o->Uteps);
        pinv_truncation(nc, n, U, sv, V, kPinvAlphaSingle, o->r32, o->Veps32, o->Uteps32);
        ops = g_pinv_cache.publish(key, std::move(o));
    }
    pl->pinv = ops;
    pl->r = ops->r;
    pl->r32 = ops->r32;
    pl->rp = round_up(pl->r, 16);
    return M2L_OK;
}

// SVD compression of Sec. 3.1 (Eqs. 12-14). Full rank (rank_tol <= 0) uses U = S = I: the
// compressed form is then exact for any orthonormal bases, so no SVD is needed.
// The compressed operators at rank threshold `rank_tol` for the plan's kernel and orders, from the
// shared table (built on a miss). Needs the plan's pseudo-inverse.
static std::shared_ptr<const BlasOps> make_blas(const m2l_plan_t *pl, double rank_tol) {
    const auto key = std::make_tuple(pl->kernel, pl->p, pl->pc, rank_key(rank_tol), pl->svd_mode);
    std::shared_ptr<const BlasOps> ops = g_blas_cache.find(key);
    if (!ops) {
        auto o = std::make_shared<BlasOps>();
        const int n = pl->n, nc = pl->nc;
        std::vector<std::vector<double>> Ks(kNumTransfer);
#pragma omp parallel for schedule(dynamic, 4)
        for (int t = 0; t < kNumTransfer; ++t) m2l_matrix(pl, t, Ks[t]);
        int k, kc;
        if (rank_tol <= 0) {
            k = n;
            kc = nc;
            o->U.assign((size_t)nc * kc, 0.0);
            for (int i = 0; i < nc; ++i) o->U[(size_t)i * kc + i] = 1.0;
            o->S.assign((size_t)n * k, 0.0);
            for (int i = 0; i < n; ++i) o->S[(size_t)i * k + i] = 1.0;
        } else {
            std::shared_ptr<const SvdBasis> B = pl->svd_mode ? rsvd_basis(pl, Ks, rank_tol) : svd_basis(pl, Ks);
            o->s_fat = B->s_fat;
            o->s_thin = B->s_thin;
            int kf = 0, kt = 0;
            const int lf = (int)o->s_fat.size(), lt = (int)o->s_thin.size();  // sketch widths (rSVD)
            while (kf < lf && o->s_fat[kf] / o->s_fat[0] >= rank_tol) ++kf;
            while (kt < lt && o->s_thin[kt] / o->s_thin[0] >= rank_tol) ++kt;
            if (nc == n) {
                // equal orders: one k (Sec. 3.1), within both sketches when they are randomised
                k = kc = std::min(std::max(std::max(kf, kt), 1), std::min(lf, lt));
            } else {
                kc = std::max(kf, 1);                    // check and equivalent spaces of different sizes
                k = std::max(kt, 1);
            }
            // U, S: the leading columns of the (re-orthonormalised) bases, stored row-major
            o->U.assign((size_t)nc * kc, 0.0);
            o->S.assign((size_t)n * k, 0.0);
            for (int c = 0; c < kc; ++c)
                for (int i = 0; i < nc; ++i) o->U[(size_t)i * kc + c] = B->Uf[(size_t)c * nc + i];
            for (int c = 0; c < k; ++c)
                for (int i = 0; i < n; ++i) o->S[(size_t)i * k + c] = B->Sb[(size_t)c * n + i];
        }
        o->k = k;
        o->kc = kc;
        // C_t = U^T K_t S  (kc x k, row-major)
        o->C.assign((size_t)kNumTransfer * kc * k, 0.0);
#pragma omp parallel for schedule(dynamic, 2)
        for (int t = 0; t < kNumTransfer; ++t) {
            std::vector<double> KS((size_t)nc * k, 0.0);
            const double *K = Ks[t].data();
            for (int i = 0; i < nc; ++i)
                for (int j = 0; j < n; ++j) {
                    double kij = K[(size_t)i * n + j];
                    const double *srow = &o->S[(size_t)j * k];
                    double *dst = &KS[(size_t)i * k];
                    for (int c = 0; c < k; ++c) dst[c] += kij * srow[c];
                }
            double *C = &o->C[(size_t)t * kc * k];
            for (int i = 0; i < nc; ++i) {
                const double *urow = &o->U[(size_t)i * kc];
                const double *ks = &KS[(size_t)i * k];
                for (int a = 0; a < kc; ++a) {
                    double u = urow[a];
                    if (u == 0.0) continue;
                    for (int c = 0; c < k; ++c) C[(size_t)a * k + c] += u * ks[c];
                }
            }
        }
        // A = Ut_eps U  (r x kc): the scaled factor of the pseudo-inverse times the uncompression.
        auto fold = [&](const std::vector<double> &Ut, int r, std::vector<double> &A) {
            A.assign((size_t)r * kc, 0.0);
            for (int a = 0; a < r; ++a)
                for (int i = 0; i < nc; ++i) {
                    double u = Ut[(size_t)a * nc + i];
                    for (int c = 0; c < kc; ++c) A[(size_t)a * kc + c] += u * o->U[(size_t)i * kc + c];
                }
        };
        fold(pl->pinv->Uteps, pl->pinv->r, o->Aop);
        fold(pl->pinv->Uteps32, pl->pinv->r32, o->Aop32);
        ops = g_blas_cache.publish(key, std::move(o));
    }
    return ops;
}

int build_blas_host(m2l_plan_t *pl) {
    if (pl->blas) return M2L_OK;
    int rc = build_pinv(pl);
    if (rc) return rc;
    std::shared_ptr<const BlasOps> ops = make_blas(pl, pl->rank_tol);
    pl->blas = ops;
    pl->k = ops->k;
    pl->kp = round_up(ops->k, 16);
    pl->kc = ops->kc;
    pl->kcp = round_up(ops->kc, 16);
    return M2L_OK;
}

// Directional recompression (Eq. 15): C_t ~ Ubar_t Sigmabar_t Vbar_t^T = Ubar_t Vbar'_t^T with the
// k_t singular values of C_t at or above dir_tol s_0(C_t). Packed as the contraction reads them:
// Ubar_t as [kc_pad][k_t8] (one row per output component) and Vbar'_t^T as [k_t8][k_pad], k_t
// rounded up to 8 with zero padding.
// The directional factors at threshold dir_tol of the compressed operators `B` (rank threshold
// rank_tol), from the shared table (built on a miss).
static std::shared_ptr<const DirOps> make_dir(const m2l_plan_t *pl, const BlasOps &B, double rank_tol, double dir_tol) {
    const auto key = std::make_tuple(pl->kernel, pl->p, pl->pc, rank_key(rank_tol), dir_tol, pl->svd_mode);
    std::shared_ptr<const DirOps> ops = g_dir_cache.find(key);
    if (!ops) {
        auto o = std::make_shared<DirOps>();
        const int k = B.k, kp = round_up(B.k, 16), kc = B.kc, kcp = round_up(B.kc, 16);
        const std::vector<double> &Call = B.C;
        std::vector<int> kt(kNumTransfer);
        std::vector<std::vector<double>> ub(kNumTransfer), vt(kNumTransfer);
#pragma omp parallel for schedule(dynamic, 2)
        for (int t = 0; t < kNumTransfer; ++t) {
            // C_t is row-major kc x k; the SVD routine takes a column-major matrix with at least as
            // many rows as columns, so a wide C_t is factored through its transpose
            const double *C = &Call[(size_t)t * kc * k];
            const bool tall = kc >= k;
            const int m = tall ? kc : k, nn = tall ? k : kc;
            std::vector<double> A((size_t)m * nn), U, sv, V;
            for (int a = 0; a < kc; ++a)
                for (int c = 0; c < k; ++c) {
                    if (tall)
                        A[(size_t)c * kc + a] = C[(size_t)a * k + c];
                    else
                        A[(size_t)a * k + c] = C[(size_t)a * k + c];
                }
            jacobi_svd(A, m, nn, U, sv, V);
            // left singular vectors of C_t (check side, kc values)
            auto left = [&](int j, int a) { return tall ? U[(size_t)j * kc + a] : V[(size_t)j * kc + a]; };
            int r = 0;
            while (r < nn && sv[r] >= dir_tol * sv[0]) ++r;
            if (r < 1) r = 1;
            const int r8 = round_up(r, 8);
            kt[t] = r;
            // Ubar_t: the r leading left singular vectors, re-orthonormalised; Vbar'_t^T =
            // Ubar_t^T C_t, so that Ubar_t Vbar'_t^T is the projection of C_t onto that subspace
            // (the same product as Ubar_t Sigmabar_t Vbar_t^T, without the drift of accumulated
            // rotations)
            std::vector<double> Ub((size_t)kc * r);
            for (int j = 0; j < r; ++j)
                for (int a = 0; a < kc; ++a) Ub[(size_t)j * kc + a] = left(j, a);
            orthonormalize_columns(Ub.data(), kc, r);
            ub[t].assign((size_t)kcp * r8, 0.0);
            vt[t].assign((size_t)r8 * kp, 0.0);
            for (int j = 0; j < r; ++j) {
                for (int a = 0; a < kc; ++a) ub[t][(size_t)a * r8 + j] = Ub[(size_t)j * kc + a];  // Ubar_t[a][j]
                for (int c = 0; c < k; ++c) {
                    double v = 0.0;
                    for (int a = 0; a < kc; ++a) v += Ub[(size_t)j * kc + a] * C[(size_t)a * k + c];
                    vt[t][(size_t)j * kp + c] = v;                                               // Vbar'_t^T[j][c]
                }
            }
        }
        o->kt = kt;
        o->meta.assign((size_t)kNumTransfer * 4, 0);
        for (int t = 0; t < kNumTransfer; ++t) {
            const int m8 = round_up(kt[t], 8);
            o->meta[4 * t + 0] = (int)o->ub.size();
            o->meta[4 * t + 1] = (int)o->vt.size();
            o->meta[4 * t + 2] = kt[t];
            o->meta[4 * t + 3] = m8;
            o->kt8_max = std::max(o->kt8_max, m8);
            o->ub.insert(o->ub.end(), ub[t].begin(), ub[t].end());
            o->vt.insert(o->vt.end(), vt[t].begin(), vt[t].end());
        }
        ops = g_dir_cache.publish(key, std::move(o));
    }
    return ops;
}

int build_directional(m2l_plan_t *pl) {
    if (pl->dirop) return M2L_OK;
    int rc = build_blas_host(pl);
    if (rc) return rc;
    std::shared_ptr<const DirOps> ops = make_dir(pl, *pl->blas, pl->rank_tol, pl->dir_tol);
    pl->dirop = ops;
    pl->dir_kt8_max = ops->kt8_max;
    return M2L_OK;
}

// Relative error (Eq. 16) that truncating the compressed operators at rank threshold rank_tol adds to
// the check potential of one target box of octant 0 with all 189 of its transfer vectors, against
// the full K_t: U_k U_k^T K_t S_k S_k^T q summed over the transfer vectors, for four seeded draws
// of the source densities (two uniform in [-1, 1], two uniform in [0, 1)), the largest of the
// four. A directional threshold dir_tol > 0 adds 10 dir_tol, the size of the error a directional
// cut was measured to add (p = 4..10). Only the SVD bases are needed, so trying many ranks costs
// one SVD. FP64, on the host.
double truncation_estimate(m2l_plan_t *pl, double rank_tol, double dir_tol) {
    if (build_pinv(pl)) return 1.0;
    const int n = pl->n, nc = pl->nc;
    int k = n, kc = nc;
    std::shared_ptr<const SvdBasis> B;
    if (rank_tol > 0) {
        B = g_svd_cache.find(std::make_tuple(pl->kernel, pl->p, pl->pc));
        if (!B) {
            std::vector<std::vector<double>> Ks(kNumTransfer);
#pragma omp parallel for schedule(dynamic, 4)
            for (int t = 0; t < kNumTransfer; ++t) m2l_matrix(pl, t, Ks[t]);
            B = svd_basis(pl, Ks);
        }
        pl->svd_hold = B;
        int kf = 0, kt = 0;
        while (kf < nc && B->s_fat[kf] / B->s_fat[0] >= rank_tol) ++kf;
        while (kt < n && B->s_thin[kt] / B->s_thin[0] >= rank_tol) ++kt;
        k = nc == n ? std::max(std::max(kf, kt), 1) : std::max(kt, 1);
        kc = nc == n ? k : std::max(kf, 1);
    }
    std::vector<int> ts;
    for (int x = -2; x <= 3; ++x)
        for (int y = -2; y <= 3; ++y)
            for (int z = -2; z <= 3; ++z) {
                const int t = transfer_index(x, y, z);
                if (t >= 0) ts.push_back(t);
            }
    std::vector<std::vector<double>> Kp(ts.size());
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < (int)ts.size(); ++i) m2l_matrix(pl, ts[i], Kp[i]);
    double worst = 0.0;
    std::mt19937_64 gen(24080);
    std::uniform_real_distribution<double> u11(-1.0, 1.0), u01(0.0, 1.0);
    std::vector<double> phi((size_t)nc), apx((size_t)nc), q((size_t)n), sq((size_t)n), w((size_t)nc), c((size_t)std::max(k, kc));
    for (int draw = 0; draw < 4; ++draw) {
        std::fill(phi.begin(), phi.end(), 0.0);
        std::fill(apx.begin(), apx.end(), 0.0);
        for (size_t it = 0; it < ts.size(); ++it) {
            for (int j = 0; j < n; ++j) q[j] = draw < 2 ? u11(gen) : u01(gen);
            const std::vector<double> &K = Kp[it];
            // S_k S_k^T q (the full q at full rank)
            if (B) {
                for (int a = 0; a < k; ++a) {
                    double v = 0.0;
                    for (int j = 0; j < n; ++j) v += B->Sb[(size_t)a * n + j] * q[j];
                    c[a] = v;
                }
                for (int j = 0; j < n; ++j) {
                    double v = 0.0;
                    for (int a = 0; a < k; ++a) v += B->Sb[(size_t)a * n + j] * c[a];
                    sq[j] = v;
                }
            } else {
                sq = q;
            }
            for (int i = 0; i < nc; ++i) {
                double a = 0.0, b = 0.0;
                for (int j = 0; j < n; ++j) {
                    a += K[(size_t)i * n + j] * q[j];
                    b += K[(size_t)i * n + j] * sq[j];
                }
                phi[i] += a;
                w[i] = b;
            }
            // U_k U_k^T (K_t S_k S_k^T q)
            if (B) {
                for (int a = 0; a < kc; ++a) {
                    double v = 0.0;
                    for (int i = 0; i < nc; ++i) v += B->Uf[(size_t)a * nc + i] * w[i];
                    c[a] = v;
                }
                for (int i = 0; i < nc; ++i) {
                    double v = 0.0;
                    for (int a = 0; a < kc; ++a) v += B->Uf[(size_t)a * nc + i] * c[a];
                    apx[i] += v;
                }
            } else {
                for (int i = 0; i < nc; ++i) apx[i] += w[i];
            }
        }
        double num = 0.0, den = 0.0;
        for (int i = 0; i < nc; ++i) {
            num += (apx[i] - phi[i]) * (apx[i] - phi[i]);
            den += phi[i] * phi[i];
        }
        worst = std::max(worst, den > 0 ? std::sqrt(num / den) : 0.0);
    }
    return worst + (dir_tol > 0 ? 10.0 * dir_tol : 0.0);
}

// Algorithmic flops of the BLAS contraction for one right-hand side at `level` (-1: levels
// 2..depth): 2 kc k per (target, source) pair, or 2 k_t (kc + k) for a pair with transfer vector t when
// the directional factors are used (the two products of Sec. 3.2 step 4): with M2L_OPT_DIR_TOL
// set and a precision whose contraction applies them (FP64, FP32, or AUTO).
int contract_flops(m2l_plan_t *pl, int level, double *out) {
    const bool dir = pl->dir_tol > 0 && pl->precision != M2L_PREC_TF32X3 && pl->precision != M2L_PREC_BF16X3;
    int rc = build_level_tables(pl);
    if (!rc) rc = build_blas_host(pl);
    if (!rc && dir) rc = build_directional(pl);
    if (rc) return rc;
    double w[kNumTransfer];
    for (int t = 0; t < kNumTransfer; ++t)
        w[t] = dir ? 2.0 * pl->dirop->kt[t] * (pl->kc + pl->k) : 2.0 * pl->kc * pl->k;
    double total = 0.0;
    const int l0 = level < 0 ? 2 : level, l1 = level < 0 ? pl->depth : level;
    for (int l = l0; l <= l1; ++l) {
        const LevelDev &L = pl->ldev[l];
        const long long N = 1LL << l;
        double sum = 0.0;
#pragma omp parallel for reduction(+ : sum) schedule(static)
        for (long long b = 0; b < L.nboxes; ++b) {
            const uint32_t p = L.h_xyz[b];
            const int x = p & 1023, y = (p >> 10) & 1023, z = (p >> 20) & 1023;
            for (int tx = -3; tx <= 3; ++tx)
                for (int ty = -3; ty <= 3; ++ty)
                    for (int tz = -3; tz <= 3; ++tz) {
                        const int ti = transfer_index(tx, ty, tz);
                        if (ti < 0) continue;
                        const int sx = x + tx, sy = y + ty, sz = z + tz;
                        // the source must lie in the target's interaction list: parents adjacent
                        if ((sx >> 1) - (x >> 1) < -1 || (sx >> 1) - (x >> 1) > 1 || (sy >> 1) - (y >> 1) < -1 ||
                            (sy >> 1) - (y >> 1) > 1 || (sz >> 1) - (z >> 1) < -1 || (sz >> 1) - (z >> 1) > 1)
                            continue;
                        if (sx < 0 || sy < 0 || sz < 0 || sx >= N || sy >= N || sz >= N) continue;
                        if (L.h_slot[((size_t)sz * N + sy) * N + sx] >= 0) sum += w[ti];
                    }
        }
        total += sum;
    }
    *out = total;
    return M2L_OK;
}

// Kernel spectra (App. A.1 step 1): for each transfer vector the kernel sequence
// G_t(m) = K(-t + h m), h = alpha_inner / (p - 1), m in [-(p-1), p-1]^3, placed at m mod g on the
// g^3 grid, then its 3D real DFT keeping kz in [0, g/2] (f = (kx g + ky)(g/2+1) + kz).
int build_fft_host(m2l_plan_t *pl) {
    if (pl->fft) return M2L_OK;
    int rc = build_pinv(pl);
    if (rc) return rc;
    int p = pl->p;
    int g = pl->fft_grid_opt ? pl->fft_grid_opt : 2 * p;
    const auto key = std::make_tuple(pl->kernel, p, g);
    std::shared_ptr<const FftOps> ops = g_fft_cache.find(key);
    if (ops) {
        pl->fft = ops;
        pl->g = ops->g;
        pl->F = ops->F;
        return M2L_OK;
    }
    auto o = std::make_shared<FftOps>();
    int H = g / 2 + 1;
    o->g = g;
    o->F = g * g * H;
    o->twiddle.resize((size_t)2 * g);
    for (int m = 0; m < g; ++m) {
        o->twiddle[2 * m] = std::cos(2.0 * M_PI * m / g);
        o->twiddle[2 * m + 1] = -std::sin(2.0 * M_PI * m / g);
    }
    const double h = kAlphaInner / (p - 1);
    o->Khat.assign((size_t)kNumTransfer * o->F * 2, 0.0);
    const double *w = o->twiddle.data();
#pragma omp parallel for schedule(dynamic, 2)
    for (int t = 0; t < kNumTransfer; ++t) {
        int tx, ty, tz;
        transfer_vector(t, tx, ty, tz);
        std::vector<double> grid((size_t)g * g * g, 0.0);
        for (int mx = -(p - 1); mx <= p - 1; ++mx)
            for (int my = -(p - 1); my <= p - 1; ++my)
                for (int mz = -(p - 1); mz <= p - 1; ++mz) {
                    double d0 = -tx + h * mx, d1 = -ty + h * my, d2 = -tz + h * mz;
                    double v = 1.0 / (4.0 * M_PI * std::sqrt(d0 * d0 + d1 * d1 + d2 * d2));
                    int a = ((mx % g) + g) % g, b = ((my % g) + g) % g, c = ((mz % g) + g) % g;
                    grid[((size_t)a * g + b) * g + c] = v;
                }
        // along z (real -> half spectrum)
        std::vector<double> Y1((size_t)g * g * H * 2, 0.0);
        for (int a = 0; a < g; ++a)
            for (int b = 0; b < g; ++b)
                for (int kz = 0; kz < H; ++kz) {
                    double re = 0, im = 0;
                    for (int c = 0; c < g; ++c) {
                        double v = grid[((size_t)a * g + b) * g + c];
                        int m = (c * kz) % g;
                        re += v * w[2 * m];
                        im += v * w[2 * m + 1];
                    }
                    size_t o = (((size_t)a * g + b) * H + kz) * 2;
                    Y1[o] = re; Y1[o + 1] = im;
                }
        // along y
        std::vector<double> Y2((size_t)g * g * H * 2, 0.0);
        for (int a = 0; a < g; ++a)
            for (int ky = 0; ky < g; ++ky)
                for (int kz = 0; kz < H; ++kz) {
                    double re = 0, im = 0;
                    for (int b = 0; b < g; ++b) {
                        size_t o = (((size_t)a * g + b) * H + kz) * 2;
                        int m = (b * ky) % g;
                        double xr = Y1[o], xi = Y1[o + 1], wr = w[2 * m], wi = w[2 * m + 1];
                        re += xr * wr - xi * wi;
                        im += xr * wi + xi * wr;
                    }
                    size_t o = (((size_t)a * g + ky) * H + kz) * 2;
                    Y2[o] = re; Y2[o + 1] = im;
                }
        // along x
        double *out = &o->Khat[(size_t)t * o->F * 2];
        for (int kx = 0; kx < g; ++kx)
            for (int ky = 0; ky < g; ++ky)
                for (int kz = 0; kz < H; ++kz) {
                    double re = 0, im = 0;
                    for (int a = 0; a < g; ++a) {
                        size_t o = (((size_t)a * g + ky) * H + kz) * 2;
                        int m = (a * kx) % g;
                        double xr = Y2[o], xi = Y2[o + 1], wr = w[2 * m], wi = w[2 * m + 1];
                        re += xr * wr - xi * wi;
                        im += xr * wi + xi * wr;
                    }
                    size_t f = ((size_t)kx * g + ky) * H + kz;
                    out[2 * f] = re; out[2 * f + 1] = im;
                }
    }
    ops = g_fft_cache.publish(key, std::move(o));
    pl->fft = ops;
    pl->g = ops->g;
    pl->F = ops->F;
    return M2L_OK;
}

// ---------------------------------------------------------------------------------------------
// Box tables per level.

static inline uint64_t spread3(uint32_t v) {
    uint64_t out = 0;
    for (int b = 0; b < 21; ++b) out |= (uint64_t)((v >> b) & 1u) << (3 * b);
    return out;
}
static inline uint32_t compact3(uint64_t v) {
    uint32_t out = 0;
    for (int b = 0; b < 21; ++b) out |= (uint32_t)((v >> (3 * b)) & 1u) << b;
    return out;
}

template <class T>
static int dev_upload(T *&dst, const std::vector<T> &src) {
    if (dst) cudaFree(dst);
    dst = nullptr;
    size_t bytes = std::max<size_t>(src.size(), 1) * sizeof(T);
    if (cudaMalloc((void **)&dst, bytes) != cudaSuccess) {
        set_error("cudaMalloc of %zu bytes failed", bytes);
        return M2L_ENOMEM;
    }
    if (!src.empty() && cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("cudaMemcpy to device failed: %s", cudaGetErrorString(cudaGetLastError()));
        return M2L_ECUDA;
    }
    return M2L_OK;
}

static void free_level(LevelDev &L) {
    void *ptrs[] = {L.slot, L.xyz, L.perm, L.cslot, L.cxyz, L.cchild, L.cperm};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    L.slot = nullptr; L.xyz = nullptr; L.perm = nullptr;
    L.cslot = nullptr; L.cxyz = nullptr; L.cchild = nullptr; L.cperm = nullptr;
}

int build_level_tables(m2l_plan_t *pl) {
    if (!pl->levels_dirty) return M2L_OK;
    long long base = 0, cbase = 0;
    for (int l = 2; l <= pl->depth; ++l) {
        LevelDev &L = pl->ldev[l];
        free_level(L);
        L.on_device = false;
        const LevelSet &S = pl->levels[l];
        uint32_t N = 1u << l;
        long long B = S.dense ? (1LL << (3 * l)) : (long long)S.keys.size();
        std::vector<uint64_t> keys(B);
        if (S.dense) std::iota(keys.begin(), keys.end(), 0ull);
        else keys = S.keys;
        std::vector<uint32_t> &xyz = L.h_xyz;
        std::vector<int> &slot = L.h_slot;
        xyz.assign(B, 0);
        slot.assign((size_t)N * N * N, -1);
        for (long long b = 0; b < B; ++b) {
            uint32_t x = compact3(keys[b]), y = compact3(keys[b] >> 1), z = compact3(keys[b] >> 2);
            xyz[b] = x | (y << 10) | (z << 20);
            slot[((size_t)z * N + y) * N + x] = (int)b;
        }
        // targets grouped by octant (the low three bits of the key); inside an octant by the
        // domain-boundary class of the parent (per axis: first plane, last plane, neither), Morton
        // order inside a class. A target's interaction list loses the transfer vectors that leave
        // the domain exactly by its class, so contraction tiles cut from this order hold targets
        // with the same live vectors and rows without a source stay rare.
        const uint32_t Np = N / 2;
        auto boundary_class = [&](long long b) {
            int c = 0;
            for (int a = 0; a < 3; ++a) {
                const uint32_t pv = ((xyz[b] >> (10 * a)) & 1023) >> 1;
                c |= ((pv == 0 ? 1 : 0) | (pv == Np - 1 ? 2 : 0)) << (2 * a);
            }
            return c;
        };
        std::vector<int> &perm = L.h_perm;
        perm.clear();
        perm.reserve(B);
        for (int c = 0; c < 8; ++c) {
            L.oct_start[c] = (long long)perm.size();
            for (long long b = 0; b < B; ++b)
                if ((int)(keys[b] & 7) == c) perm.push_back((int)b);
            std::stable_sort(perm.begin() + L.oct_start[c], perm.end(),
                             [&](int x, int y) { return boundary_class(x) < boundary_class(y); });
        }
        L.oct_start[8] = (long long)perm.size();
        // clusters: non-empty parents (App. A.1), Morton order
        std::vector<uint64_t> pk;
        for (long long b = 0; b < B; ++b)
            if (pk.empty() || pk.back() != (keys[b] >> 3)) pk.push_back(keys[b] >> 3);
        std::vector<int> &cslot = L.h_cslot, &cchild = L.h_cchild;
        std::vector<uint32_t> &cxyz = L.h_cxyz;
        cslot.assign((size_t)Np * Np * Np, -1);
        cchild.assign(pk.size() * 8, -1);
        cxyz.assign(pk.size(), 0);
        for (size_t c = 0; c < pk.size(); ++c) {
            uint32_t x = compact3(pk[c]), y = compact3(pk[c] >> 1), z = compact3(pk[c] >> 2);
            cxyz[c] = x | (y << 10) | (z << 20);
            cslot[((size_t)z * Np + y) * Np + x] = (int)c;
        }
        {
            size_t c = 0;
            for (long long b = 0; b < B; ++b) {
                while (pk[c] != (keys[b] >> 3)) ++c;
                cchild[c * 8 + (keys[b] & 7)] = (int)b;
            }
        }
        // clusters in the same grouping as the targets above: the Hadamard product works on a few
        // consecutive clusters per warp, which then miss the same neighbour directions
        std::vector<int> &cperm = L.h_cperm;
        cperm.resize(pk.size());
        std::iota(cperm.begin(), cperm.end(), 0);
        auto cluster_class = [&](int c) {
            int k = 0;
            for (int a = 0; a < 3; ++a) {
                const uint32_t v = (cxyz[c] >> (10 * a)) & 1023;
                k |= ((v == 0 ? 1 : 0) | (v == Np - 1 ? 2 : 0)) << (2 * a);
            }
            return k;
        };
        std::stable_sort(cperm.begin(), cperm.end(), [&](int x, int y) { return cluster_class(x) < cluster_class(y); });
        // pairs: targets x sources that exist, over the 189 transfer vectors of each octant
        long long pairs = 0;
#pragma omp parallel for reduction(+ : pairs) schedule(static)
        for (long long b = 0; b < B; ++b) {
            int x = xyz[b] & 1023, y = (xyz[b] >> 10) & 1023, z = (xyz[b] >> 20) & 1023;
            int cx = x & 1, cy = y & 1, cz = z & 1;
            for (int tx = -2 - cx; tx <= 3 - cx; ++tx)
                for (int ty = -2 - cy; ty <= 3 - cy; ++ty)
                    for (int tz = -2 - cz; tz <= 3 - cz; ++tz) {
                        if (std::max(std::abs(tx), std::max(std::abs(ty), std::abs(tz))) < 2) continue;
                        int sx = x + tx, sy = y + ty, sz = z + tz;
                        if (sx < 0 || sy < 0 || sz < 0 || sx >= (int)N || sy >= (int)N || sz >= (int)N) continue;
                        if (slot[((size_t)sz * N + sy) * N + sx] >= 0) ++pairs;
                    }
        }
        L.level = l;
        L.nboxes = B;
        L.base = base;
        L.nclusters = (long long)pk.size();
        L.cbase = cbase;
        L.pairs = pairs;
        base += B;
        cbase += (long long)pk.size();
    }
    pl->total_rows = base;
    pl->total_clusters = cbase;
    pl->levels_dirty = false;
    pl->levels_version++;  // tile lists and graphs depend on the box sets
    return M2L_OK;
}

int upload_level_tables(m2l_plan_t *pl) {
    int rc = build_level_tables(pl);
    if (rc) return rc;
    for (int l = 2; l <= pl->depth; ++l) {
        LevelDev &L = pl->ldev[l];
        if (L.on_device) continue;
        if ((rc = dev_upload(L.slot, L.h_slot)) || (rc = dev_upload(L.xyz, L.h_xyz)) ||
            (rc = dev_upload(L.perm, L.h_perm)) || (rc = dev_upload(L.cslot, L.h_cslot)) ||
            (rc = dev_upload(L.cxyz, L.h_cxyz)) || (rc = dev_upload(L.cchild, L.h_cchild)) ||
            (rc = dev_upload(L.cperm, L.h_cperm)))
            return rc;
        L.on_device = true;
    }
    return M2L_OK;
}

// ---------------------------------------------------------------------------------------------
// Device copies of the operators.

template <class T>
static std::vector<T> pad2(const std::vector<double> &src, int rows, int cols, int prow, int pcol) {
    std::vector<T> out((size_t)prow * pcol, T(0));
    for (int i = 0; i < rows; ++i)
        for (int j = 0; j < cols; ++j) out[(size_t)i * pcol + j] = (T)src[(size_t)i * cols + j];
    return out;
}

template <class T>
static int upload_vec(void *&dst, const std::vector<T> &v) {
    T *d = nullptr;
    int rc = dev_upload(d, v);
    if (dst) cudaFree(dst);
    dst = d;
    return rc;
}

int split_tc_operators(m2l_plan_t *pl, int precision);  // kernels_tc.cu
int build_hadamard_tc_operand(m2l_plan_t *pl, DevOps &D);  // hadamard_tc.cu
int build_pinv_tc_operand(m2l_plan_t *pl, DevOps &D);      // pinv_tc.cu

// The directional factors, when the plan asks for them and they are not on the device yet.
template <class T>
static int upload_directional(m2l_plan_t *pl, DevOps &D) {
    if (pl->dir_tol <= 0 || D.Ub) return M2L_OK;
    int rc = build_directional(pl);
    if (rc) return rc;
    const DirOps &dop = *pl->dirop;
    std::vector<T> ub(dop.ub.begin(), dop.ub.end()), vt(dop.vt.begin(), dop.vt.end());
    if ((rc = upload_vec(D.Ub, ub)) || (rc = upload_vec(D.Vt, vt)) || (rc = upload_vec(D.dir_meta, dop.meta))) return rc;
    return M2L_OK;
}

template <class T>
static int upload_typed(m2l_plan_t *pl, DevOps &D, int form) {
    // single-precision paths take the pseudo-inverse truncated with alpha = 1e-9 (build_pinv)
    const bool single = sizeof(T) == 4;
    const int n = pl->n, k = pl->k, kp = pl->kp, r = single ? pl->r32 : pl->r, rp = pl->rp;
    const int nc = pl->nc, kc = pl->kc, kcp = pl->kcp;
    const std::vector<double> &Veps = single ? pl->pinv->Veps32 : pl->pinv->Veps;
    const std::vector<double> &Uteps = single ? pl->pinv->Uteps32 : pl->pinv->Uteps;
    int rc = M2L_OK;
    if (form == M2L_FORM_BLAS) {
        const BlasOps &B = *pl->blas;
        const std::vector<double> &Aop = single ? B.Aop32 : B.Aop;
        // S^T  [kp][n]
        std::vector<double> St((size_t)k * n);
        for (int c = 0; c < k; ++c)
            for (int i = 0; i < n; ++i) St[(size_t)c * n + i] = B.S[(size_t)i * k + c];
        // C_t  [316][kcp][kp]
        std::vector<T> Cp((size_t)kNumTransfer * kcp * kp, T(0));
        for (int t = 0; t < kNumTransfer; ++t)
            for (int a = 0; a < kc; ++a)
                for (int c = 0; c < k; ++c)
                    Cp[((size_t)t * kcp + a) * kp + c] = (T)B.C[((size_t)t * kc + a) * k + c];
        if ((rc = upload_vec(D.St, pad2<T>(St, k, n, kp, n)))) return rc;
        if ((rc = upload_vec(D.C, Cp))) return rc;
        if ((rc = upload_vec(D.A, pad2<T>(Aop, r, kc, rp, kcp)))) return rc;
        if ((rc = upload_vec(D.Uc, pad2<T>(B.U, nc, kc, nc, kcp)))) return rc;
        if ((rc = upload_directional<T>(pl, D))) return rc;
    } else {
        const FftOps &Fo = *pl->fft;
        int F = Fo.F;
        std::vector<T> K((size_t)(kNumTransfer + 1) * F * 2, T(0));
        for (size_t i = 0; i < (size_t)kNumTransfer * F * 2; ++i) K[i] = (T)Fo.Khat[i];
        std::vector<T> tw(Fo.twiddle.size());
        for (size_t i = 0; i < tw.size(); ++i) tw[i] = (T)Fo.twiddle[i];
        if ((rc = upload_vec(D.Khat, K))) return rc;
        if ((rc = upload_vec(D.tw, tw))) return rc;
        if ((rc = upload_vec(D.Ut, pad2<T>(Uteps, r, n, rp, n)))) return rc;
    }
    // the second pseudo-inverse factor, shared by both forms; single-precision plans also keep the
    // part of V_eps below its FP32 rounding for the compensated product
    if (!D.V) {
        if ((rc = upload_vec(D.V, pad2<T>(Veps, n, r, n, rp)))) return rc;
        if (single) {
            std::vector<double> lo(Veps.size());
            for (size_t i = 0; i < lo.size(); ++i) lo[i] = Veps[i] - (double)(float)Veps[i];
            if ((rc = upload_vec(D.Vlo, pad2<T>(lo, n, r, n, rp)))) return rc;
        }
    }
    return rc;
}

int upload_ops(m2l_plan_t *pl, int precision, int form) {
    int slot = precision * 2 + (form == M2L_FORM_FFT ? 1 : 0);
    (void)slot;
    DevOps &D = pl->dev[precision];
    // one DevOps per precision holds both forms; track readiness per form with the pointers
    bool have = form == M2L_FORM_BLAS ? (D.C != nullptr) : (D.Khat != nullptr);
    if (have) {
        if (form != M2L_FORM_BLAS || pl->dir_tol <= 0 || D.Ub) return M2L_OK;
        return precision == M2L_PREC_FP64 ? upload_directional<double>(pl, D) : upload_directional<float>(pl, D);
    }
    int rc = form == M2L_FORM_BLAS ? build_blas_host(pl) : build_fft_host(pl);
    if (rc) return rc;
    if (precision == M2L_PREC_FP64) {
        D.elt = 8;
        rc = upload_typed<double>(pl, D, form);
    } else {
        D.elt = 4;
        rc = upload_typed<float>(pl, D, form);
        if (!rc && form == M2L_FORM_BLAS && (precision == M2L_PREC_TF32X3 || precision == M2L_PREC_BF16X3))
            rc = split_tc_operators(pl, precision);
        if (!rc && form == M2L_FORM_BLAS && (precision == M2L_PREC_TF32X3 || precision == M2L_PREC_BF16X3))
            rc = build_blas_sliced_operands(pl, D);
        if (!rc && form == M2L_FORM_FFT && precision == M2L_PREC_TF32X3) rc = build_hadamard_tc_operand(pl, D);
        if (!rc && form == M2L_FORM_FFT && precision == M2L_PREC_TF32X3) rc = build_pinv_tc_operand(pl, D);
    }
    D.ready = rc == M2L_OK;
    return rc;
}

// Device copies of the operators (every precision), for options that change them.
void release_operators(m2l_plan_t *pl) {
    for (auto &D : pl->dev) {
        void **ptrs[] = {&D.St, &D.C, &D.A, &D.V, &D.Vlo, &D.Uc, &D.C_hi, &D.C_lo, &D.Ub, &D.Vt, &D.dir_meta,
                         &D.Khat, &D.Ut, &D.tw, &D.Bhad, &D.Us.sl, &D.Us.scale, &D.Vs.sl, &D.Vs.scale,
                         &D.Ss.sl, &D.Ss.scale, &D.As.sl, &D.As.scale, &D.Ucs.sl, &D.Ucs.scale};
        for (void **pp : ptrs) {
            if (*pp) cudaFree(*pp);
            *pp = nullptr;
        }
        D.Us.kp = D.Vs.kp = D.Ss.kp = D.As.kp = D.Ucs.kp = 0;
        D.ready = false;
    }
}

void free_device(m2l_plan_t *pl) {
    for (auto &D : pl->dev) {
        void **ptrs[] = {&D.St, &D.C, &D.A, &D.V, &D.Vlo, &D.Uc, &D.C_hi, &D.C_lo, &D.Ub, &D.Vt, &D.dir_meta,
                         &D.Khat, &D.Ut, &D.tw, &D.Bhad, &D.Us.sl, &D.Us.scale, &D.Vs.sl, &D.Vs.scale,
                         &D.Ss.sl, &D.Ss.scale, &D.As.sl, &D.As.scale, &D.Ucs.sl, &D.Ucs.scale};
        for (void **pp : ptrs) {
            if (*pp) cudaFree(*pp);
            *pp = nullptr;
        }
        D.Us.kp = D.Vs.kp = D.Ss.kp = D.As.kp = D.Ucs.kp = 0;
        D.ready = false;
    }
    for (int l = 0; l <= kMaxDepth; ++l) free_level(pl->ldev[l]);
    if (pl->ws.buf) cudaFree(pl->ws.buf);
    if (pl->stage_in.buf) cudaFree(pl->stage_in.buf);
    if (pl->spec.buf) cudaFree(pl->spec.buf);
    pl->spec = {};
    if (pl->batch_ws.buf) cudaFree(pl->batch_ws.buf);
    pl->batch_ws = {};
    if (pl->stage_out.buf) cudaFree(pl->stage_out.buf);
    free_exec(pl);
    if (pl->lattice_dev) cudaFree(pl->lattice_dev);
    pl->lattice_dev = nullptr;
    if (pl->dev_status) cudaFree(pl->dev_status);
    pl->dev_status = nullptr;
    for (cudaEvent_t e : pl->event_pool) cudaEventDestroy(e);
    pl->event_pool.clear();
    pl->events.clear();
    pl->events_used = 0;
    pl->ws = {};
    pl->stage_in = {};
    pl->stage_out = {};
}

}  // namespace m2l
