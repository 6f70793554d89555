// A whole FMM around the M2L plan (the m2l_fmm_* entry points of include/m2l.h): the octree of
// the given points, the scale-free upward and downward operators of the kiFMM (Sec. 2.1-2.2),
// and the stage sequence P2M, M2M (fmm_kernels.cu), M2L (the M2L plan on the occupied boxes of
// every level), L2L, L2P and P2P (fmm_kernels.cu).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "fmm_internal.h"
#include "linalg.h"

using namespace m2l;

struct m2l_fmm_s {
    int depth = 0, p = 0, n = 0;
    double origin[3] = {0, 0, 0}, width = 1.0;
    long long N = 0;
    std::vector<long long> perm;       // sorted position -> given index
    std::vector<double> pts;           // sorted points
    std::vector<uint64_t> keys[kMaxDepth + 1];
    std::vector<uint32_t> xyz[kMaxDepth + 1];
    std::vector<int> child[kMaxDepth + 1], parent[kMaxDepth + 1];
    std::vector<long long> leaf_start, nbr_start;
    std::vector<int> nbr;
    long long nboxes[kMaxDepth + 1] = {0}, base[kMaxDepth + 1] = {0}, rows = 0;
    int r_up = 0;
    std::vector<double> unit, v_up, ut_up, m2m, l2l;
    m2l_plan_t *m2l = nullptr;
    std::vector<void *> dev;           // every device allocation
    double *d_in = nullptr, *d_out = nullptr;  // staging for host charges / potentials
    long long *d_perm = nullptr;               // sorted position -> given index, on the device
    FmmArgs args;
};

namespace {

constexpr double kFourPi = 12.566370614359172953850573533118;

uint64_t morton(uint32_t x, uint32_t y, uint32_t z, int level) {
    uint64_t k = 0;
    for (int b = 0; b < level; ++b)
        k |= ((uint64_t)((x >> b) & 1) << (3 * b)) | ((uint64_t)((y >> b) & 1) << (3 * b + 1)) |
             ((uint64_t)((z >> b) & 1) << (3 * b + 2));
    return k;
}

uint32_t unmorton(uint64_t k, int level) {
    uint32_t x = 0, y = 0, z = 0;
    for (int b = 0; b < level; ++b) {
        x |= (uint32_t)((k >> (3 * b)) & 1) << b;
        y |= (uint32_t)((k >> (3 * b + 1)) & 1) << b;
        z |= (uint32_t)((k >> (3 * b + 2)) & 1) << b;
    }
    return x | (y << 10) | (z << 20);
}

int find(const std::vector<uint64_t> &v, uint64_t k) {
    auto it = std::lower_bound(v.begin(), v.end(), k);
    return (it != v.end() && *it == k) ? (int)(it - v.begin()) : -1;
}

double green(const double *x, const double *y) {
    const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    return 1.0 / (kFourPi * std::sqrt(d0 * d0 + d1 * d1 + d2 * d2));
}

// Surface points of a box of width w centred at c on radius alpha (box half-widths).
std::vector<double> surface(const std::vector<double> &unit, int n, const double *c, double w, double alpha) {
    std::vector<double> pts((size_t)3 * n);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) pts[3 * i + a] = c[a] + alpha * 0.5 * w * unit[3 * i + a];
    return pts;
}

// Pseudo-inverse factors (Eqs. 7-10, alpha = 0) of the n x n matrix K(x_i, y_j).
void pinv_of(const std::vector<double> &x, const std::vector<double> &y, int n, int &r, std::vector<double> &V,
             std::vector<double> &Ut) {
    std::vector<double> K((size_t)n * n), U, s, W;  // column-major
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) K[(size_t)j * n + i] = green(&x[3 * i], &y[3 * j]);
    jacobi_svd(K, n, n, U, s, W);
    pinv_truncation(n, n, U, s, W, 0.0, r, V, Ut);
}

// Y = V (Ut K): the n x n operator pinv(check -> equivalent) applied after K(check, sources).
std::vector<double> apply_pinv(const std::vector<double> &V, const std::vector<double> &Ut, int r,
                               const std::vector<double> &x, const std::vector<double> &y, int n) {
    std::vector<double> K((size_t)n * n), T((size_t)r * n, 0.0), out((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) K[(size_t)i * n + j] = green(&x[3 * i], &y[3 * j]);
    for (int a = 0; a < r; ++a)
        for (int i = 0; i < n; ++i) {
            const double u = Ut[(size_t)a * n + i];
            for (int j = 0; j < n; ++j) T[(size_t)a * n + j] += u * K[(size_t)i * n + j];
        }
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < r; ++a) {
            const double v = V[(size_t)i * r + a];
            for (int j = 0; j < n; ++j) out[(size_t)i * n + j] += v * T[(size_t)a * n + j];
        }
    return out;
}

template <class T>
int upload(m2l_fmm_t *f, const std::vector<T> &v, T **dst) {
    *dst = nullptr;
    if (v.empty()) return M2L_OK;
    void *d = nullptr;
    if (cudaMalloc(&d, v.size() * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        set_error("FMM device allocation failed");
        return M2L_ENOMEM;
    }
    f->dev.push_back(d);
    if (cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("FMM upload failed: %s", cudaGetErrorString(cudaGetLastError()));
        return M2L_ECUDA;
    }
    *dst = (T *)d;
    return M2L_OK;
}

int alloc(m2l_fmm_t *f, size_t bytes, double **dst) {
    void *d = nullptr;
    if (cudaMalloc(&d, std::max<size_t>(bytes, 8)) != cudaSuccess) {
        cudaGetLastError();
        set_error("FMM device allocation failed");
        return M2L_ENOMEM;
    }
    f->dev.push_back(d);
    *dst = (double *)d;
    return M2L_OK;
}

// Octree of the points: leaves at `depth`, occupied boxes of every level, children, parents,
// leaf point ranges and the P2P neighbour lists (leaves within one box in max norm).
void build_tree(m2l_fmm_t *f, const double *points) {
    const int d = f->depth;
    const uint32_t M = 1u << d;
    std::vector<uint64_t> leaf(f->N);
    for (long long i = 0; i < f->N; ++i) {
        uint32_t c[3];
        for (int a = 0; a < 3; ++a) {
            double t = (points[3 * i + a] - f->origin[a]) / f->width * M;
            long long v = (long long)std::floor(t);
            c[a] = (uint32_t)std::min<long long>(std::max<long long>(v, 0), M - 1);
        }
        leaf[i] = morton(c[0], c[1], c[2], d);
    }
    f->perm.resize(f->N);
    std::iota(f->perm.begin(), f->perm.end(), 0LL);
    std::stable_sort(f->perm.begin(), f->perm.end(), [&](long long a, long long b) { return leaf[a] < leaf[b]; });
    f->pts.resize((size_t)3 * f->N);
    for (long long i = 0; i < f->N; ++i)
        for (int a = 0; a < 3; ++a) f->pts[3 * i + a] = points[3 * f->perm[i] + a];
    f->keys[d].clear();
    f->leaf_start.clear();
    for (long long i = 0; i < f->N; ++i) {
        const uint64_t k = leaf[f->perm[i]];
        if (f->keys[d].empty() || f->keys[d].back() != k) {
            f->keys[d].push_back(k);
            f->leaf_start.push_back(i);
        }
    }
    f->leaf_start.push_back(f->N);
    for (int l = d - 1; l >= 2; --l) {
        f->keys[l].clear();
        for (uint64_t k : f->keys[l + 1])
            if (f->keys[l].empty() || f->keys[l].back() != (k >> 3)) f->keys[l].push_back(k >> 3);
    }
    long long base = 0;
    for (int l = 2; l <= d; ++l) {
        f->nboxes[l] = (long long)f->keys[l].size();
        f->base[l] = base;
        base += f->nboxes[l];
        f->xyz[l].resize(f->nboxes[l]);
        for (long long b = 0; b < f->nboxes[l]; ++b) f->xyz[l][b] = unmorton(f->keys[l][b], l);
        if (l < d) {
            f->child[l].assign((size_t)f->nboxes[l] * 8, -1);
            for (long long b = 0; b < f->nboxes[l]; ++b)
                for (int o = 0; o < 8; ++o) f->child[l][b * 8 + o] = find(f->keys[l + 1], (f->keys[l][b] << 3) | (uint64_t)o);
        }
        if (l > 2) {
            f->parent[l].resize(f->nboxes[l]);
            for (long long b = 0; b < f->nboxes[l]; ++b) f->parent[l][b] = find(f->keys[l - 1], f->keys[l][b] >> 3);
        }
    }
    f->rows = base;
    f->nbr_start.assign(1, 0);
    f->nbr.clear();
    for (long long b = 0; b < f->nboxes[d]; ++b) {
        const uint32_t p = f->xyz[d][b];
        const int x = p & 1023, y = (p >> 10) & 1023, z = (p >> 20) & 1023;
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dz = -1; dz <= 1; ++dz) {
                    const int sx = x + dx, sy = y + dy, sz = z + dz;
                    if (sx < 0 || sy < 0 || sz < 0 || sx >= (int)M || sy >= (int)M || sz >= (int)M) continue;
                    const int nb = find(f->keys[d], morton(sx, sy, sz, d));
                    if (nb >= 0) f->nbr.push_back(nb);
                }
        f->nbr_start.push_back((long long)f->nbr.size());
    }
}

// Scale-free upward and downward operators at unit parent width (the Laplace kernel has degree
// -1, so K scales as 1/w and its pseudo-inverse as w; M2M and L2L combine one of each).
void build_operators(m2l_fmm_t *f) {
    const int n = f->n;
    f->unit.resize((size_t)3 * n);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) f->unit[3 * i + a] = -1.0 + 2.0 * f->m2l->lattice[3 * i + a] / (f->p - 1);
    const double zero[3] = {0, 0, 0};
    // P2M: upward check (outer radius) -> upward equivalent (inner radius), unit width
    pinv_of(surface(f->unit, n, zero, 1.0, kAlphaOuter), surface(f->unit, n, zero, 1.0, kAlphaInner), n, f->r_up,
            f->v_up, f->ut_up);
    f->m2m.assign((size_t)8 * n * n, 0.0);
    f->l2l.assign((size_t)8 * n * n, 0.0);
    const std::vector<double> par_uc = surface(f->unit, n, zero, 1.0, kAlphaOuter);
    const std::vector<double> par_de = surface(f->unit, n, zero, 1.0, kAlphaOuter);
    for (int o = 0; o < 8; ++o) {
        const double cc[3] = {((o & 1) - 0.5) * 0.5, (((o >> 1) & 1) - 0.5) * 0.5, (((o >> 2) & 1) - 0.5) * 0.5};
        // M2M: parent upward check <- child upward equivalent, then the parent's pseudo-inverse
        std::vector<double> M = apply_pinv(f->v_up, f->ut_up, f->r_up, par_uc, surface(f->unit, n, cc, 0.5, kAlphaInner), n);
        std::copy(M.begin(), M.end(), f->m2m.begin() + (size_t)o * n * n);
        // L2L: child downward check <- parent downward equivalent, then the child's pseudo-inverse
        const std::vector<double> ch_dc = surface(f->unit, n, cc, 0.5, kAlphaInner);
        int r;
        std::vector<double> V, Ut;
        pinv_of(ch_dc, surface(f->unit, n, cc, 0.5, kAlphaOuter), n, r, V, Ut);
        std::vector<double> Lo = apply_pinv(V, Ut, r, ch_dc, par_de, n);
        std::copy(Lo.begin(), Lo.end(), f->l2l.begin() + (size_t)o * n * n);
    }
}

void release(m2l_fmm_t *f) {
    for (void *d : f->dev) cudaFree(d);
    f->dev.clear();
    if (f->m2l) m2l_destroy(f->m2l);
    f->m2l = nullptr;
}

}  // namespace

extern "C" {

m2l_fmm_t *m2l_fmm_plan(const double *points, long long n_points, int depth, int p, double rank_tol,
                        const double *origin, double width) {
    clear_error();
    if (!points || n_points < 1 || !(width > 0) || !std::isfinite(width)) {
        set_error("invalid points, count or width");
        return nullptr;
    }
    m2l_fmm_t *f = new (std::nothrow) m2l_fmm_t;
    if (!f) {
        set_error("out of host memory");
        return nullptr;
    }
    f->m2l = m2l_plan(depth, p, M2L_LAPLACE3D, rank_tol);
    if (!f->m2l) {
        delete f;
        return nullptr;  // error set by m2l_plan
    }
    if (f->m2l->device < 0) {
        set_error("the FMM needs a GPU");
        release(f);
        delete f;
        return nullptr;
    }
    f->depth = depth;
    f->p = p;
    f->n = f->m2l->n;
    f->N = n_points;
    f->width = width;
    for (int a = 0; a < 3; ++a) f->origin[a] = origin ? origin[a] : 0.0;
    build_tree(f, points);
    int rc = M2L_OK;
    for (int l = 2; l <= depth && !rc; ++l) rc = m2l_set_boxes(f->m2l, l, f->keys[l].data(), f->nboxes[l]);
    if (!rc) build_operators(f);
    FmmArgs &A = f->args;
    A.depth = depth;
    A.n = f->n;
    A.r_up = f->r_up;
    for (int a = 0; a < 3; ++a) A.origin[a] = f->origin[a];
    if (!rc) rc = upload(f, f->pts, (double **)&A.pts);
    if (!rc) rc = upload(f, f->perm, &f->d_perm);
    if (!rc) rc = upload(f, f->leaf_start, (long long **)&A.leaf_start);
    if (!rc) rc = upload(f, f->nbr_start, (long long **)&A.nbr_start);
    if (!rc) rc = upload(f, f->nbr, (int **)&A.nbr);
    if (!rc) rc = upload(f, f->unit, (double **)&A.unit);
    if (!rc) rc = upload(f, f->v_up, (double **)&A.v_up);
    if (!rc) rc = upload(f, f->ut_up, (double **)&A.ut_up);
    if (!rc) rc = upload(f, f->m2m, (double **)&A.m2m);
    if (!rc) rc = upload(f, f->l2l, (double **)&A.l2l);
    for (int l = 2; l <= depth && !rc; ++l) {
        FmmLevel &L = A.levels[l];
        L.base = f->base[l];
        L.width = width / (double)(1LL << l);
        rc = upload(f, f->xyz[l], (uint32_t **)&L.xyz);
        if (!rc && l < depth) rc = upload(f, f->child[l], (int **)&L.child);
        if (!rc && l > 2) rc = upload(f, f->parent[l], (int **)&L.parent);
    }
    double *q = nullptr, *pot = nullptr;
    if (!rc) rc = alloc(f, sizeof(double) * f->N, &q);
    if (!rc) rc = alloc(f, sizeof(double) * f->N, &pot);
    if (!rc) rc = alloc(f, sizeof(double) * f->rows * f->n, &A.Q);
    if (!rc) rc = alloc(f, sizeof(double) * f->rows * f->n, &A.L);
    if (!rc) rc = alloc(f, sizeof(double) * f->N, &f->d_in);
    if (!rc) rc = alloc(f, sizeof(double) * f->N, &f->d_out);
    A.q = q;
    A.pot = pot;
    if (rc) {
        release(f);
        delete f;
        return nullptr;
    }
    return f;
}

int m2l_fmm_set_m2l_option(m2l_fmm_t *f, int key, long long value) {
    clear_error();
    if (!f) {
        set_error("NULL FMM");
        return M2L_EINVAL;
    }
    if ((key == M2L_OPT_PRECISION && value != M2L_PREC_FP64) || key == M2L_OPT_CHECK_ORDER ||
        key == M2L_OPT_OUTPUT || key == M2L_OPT_ACCUMULATE) {
        set_error("the FMM runs M2L in FP64 on locals with equal orders");
        return M2L_EINVAL;
    }
    return m2l_set_option(f->m2l, key, value);
}

m2l_plan_t *m2l_fmm_m2l_plan(m2l_fmm_t *f) { return f ? f->m2l : nullptr; }

int m2l_fmm_evaluate(m2l_fmm_t *f, const double *charges, double *potentials) {
    clear_error();
    if (!f || !charges || !potentials) {
        set_error("NULL FMM or buffer");
        return M2L_EINVAL;
    }
    cudaPointerAttributes a;
    auto on_device = [&](const void *p) {
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
    };
    const bool qdev = on_device(charges), pdev = on_device(potentials);
    cudaStream_t s = f->m2l->stream;
    const long long *perm = f->d_perm;
    const double *src = charges;
    if (!qdev) {
        if (cudaMemcpyAsync(f->d_in, charges, sizeof(double) * f->N, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            set_error("copying the charges failed: %s", cudaGetErrorString(cudaGetLastError()));
            return M2L_ECUDA;
        }
        src = f->d_in;
    }
    FmmArgs &A = f->args;
    int rc = fmm_gather(src, perm, f->N, (double *)A.q, s);
    if (!rc && cudaMemsetAsync(A.pot, 0, sizeof(double) * f->N, s) != cudaSuccess) rc = M2L_ECUDA;
    if (!rc) rc = fmm_upward(A, f->nboxes, s);
    if (!rc) rc = m2l_set_option(f->m2l, M2L_OPT_PRECISION, M2L_PREC_FP64);
    if (!rc) rc = m2l_apply(f->m2l, A.Q, A.L, -1, 1);
    if (!rc) rc = fmm_downward(A, f->nboxes, s);
    double *dst = pdev ? potentials : f->d_out;
    if (!rc) rc = fmm_scatter(A.pot, perm, f->N, dst, s);
    if (!rc && !pdev &&
        cudaMemcpyAsync(potentials, f->d_out, sizeof(double) * f->N, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        rc = M2L_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("FMM evaluation failed: %s", cudaGetErrorString(cudaGetLastError()));
        return M2L_ECUDA;
    }
    return rc;
}

void m2l_fmm_destroy(m2l_fmm_t *f) {
    if (!f) return;
    release(f);
    delete f;
}

}  // extern "C"
