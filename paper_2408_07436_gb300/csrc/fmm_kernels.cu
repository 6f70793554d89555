// The kiFMM stages around M2L (Sec. 2.1-2.2, Fig. 2): P2M, M2M, L2L, L2P and the near-field
// P2P, in FP64, one CTA per box. Points are sorted by leaf; a leaf's points are a contiguous
// range. Multipoles and locals of every level live in one array of rows [box][n] per level,
// levels 2..depth concatenated (the layout the M2L plan reads and writes).
#include <cuda_runtime.h>

#include <algorithm>

#include "fmm_internal.h"

namespace m2l {

namespace {

constexpr double kFourPi = 12.566370614359172953850573533118;  // 4 pi

__device__ __forceinline__ double green(double x0, double x1, double x2, double y0, double y1, double y2) {
    const double d0 = x0 - y0, d1 = x1 - y1, d2 = x2 - y2;
    return 1.0 / (kFourPi * sqrt(d0 * d0 + d1 * d1 + d2 * d2));
}

__device__ __forceinline__ void box_centre(const FmmLevel &L, long long b, double origin0, double origin1,
                                           double origin2, double &c0, double &c1, double &c2) {
    const uint32_t p = L.xyz[b];
    c0 = origin0 + ((p & 1023) + 0.5) * L.width;
    c1 = origin1 + (((p >> 10) & 1023) + 0.5) * L.width;
    c2 = origin2 + (((p >> 20) & 1023) + 0.5) * L.width;
}

__global__ void gather_kernel(const double *__restrict__ src, const long long *__restrict__ perm, long long n,
                              double *__restrict__ dst) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[perm[i]];
}

__global__ void scatter_kernel(const double *__restrict__ src, const long long *__restrict__ perm, long long n,
                               double *__restrict__ dst) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[perm[i]] = src[i];
}

// P2M (Eq. 6 solved by Eq. 9): the upward check potential of the leaf's points at its upward
// check surface, then q = w (V_up (Ut_up phi)) with the unit-width pseudo-inverse (K scales as
// 1/w, so its pseudo-inverse as w).
__global__ void p2m_kernel(FmmArgs A) {
    extern __shared__ double sm[];
    double *phi = sm;            // n
    double *tmp = sm + A.n;      // r_up
    const FmmLevel &L = A.levels[A.depth];
    const long long b = blockIdx.x;
    double c0, c1, c2;
    box_centre(L, b, A.origin[0], A.origin[1], A.origin[2], c0, c1, c2);
    const double h = kAlphaOuter * 0.5 * L.width;
    const long long s = A.leaf_start[b], e = A.leaf_start[b + 1];
    for (int i = threadIdx.x; i < A.n; i += blockDim.x) {
        const double x0 = c0 + h * A.unit[3 * i], x1 = c1 + h * A.unit[3 * i + 1], x2 = c2 + h * A.unit[3 * i + 2];
        double acc = 0.0;
        for (long long j = s; j < e; ++j)
            acc += A.q[j] * green(x0, x1, x2, A.pts[3 * j], A.pts[3 * j + 1], A.pts[3 * j + 2]);
        phi[i] = acc;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < A.r_up; a += blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < A.n; ++i) acc += A.ut_up[(long long)a * A.n + i] * phi[i];
        tmp[a] = acc;
    }
    __syncthreads();
    double *out = A.Q + (L.base + b) * A.n;
    for (int j = threadIdx.x; j < A.n; j += blockDim.x) {
        double acc = 0.0;
        for (int a = 0; a < A.r_up; ++a) acc += A.v_up[(long long)j * A.r_up + a] * tmp[a];
        out[j] = L.width * acc;
    }
}

// M2M: q_parent = sum over the existing children o of M_o q_child (M_o = pinv_up K(parent upward
// check, child upward equivalent), scale free).
__global__ void m2m_kernel(FmmArgs A, int level) {
    const FmmLevel &P = A.levels[level], &C = A.levels[level + 1];
    const long long b = blockIdx.x;
    double *out = A.Q + (P.base + b) * A.n;
    for (int j = threadIdx.x; j < A.n; j += blockDim.x) {
        double acc = 0.0;
        for (int o = 0; o < 8; ++o) {
            const int ch = P.child[b * 8 + o];
            if (ch < 0) continue;
            const double *qc = A.Q + (C.base + ch) * A.n;
            const double *M = A.m2m + ((long long)o * A.n + j) * A.n;
            for (int i = 0; i < A.n; ++i) acc += M[i] * qc[i];
        }
        out[j] = acc;
    }
}

// L2L: L_child += L_o L_parent (L_o = pinv_down K(child downward check, parent downward
// equivalent), scale free; o the child's octant).
__global__ void l2l_kernel(FmmArgs A, int level) {
    const FmmLevel &C = A.levels[level], &P = A.levels[level - 1];
    const long long b = blockIdx.x;
    const uint32_t xyz = C.xyz[b];
    const int o = (xyz & 1) | (((xyz >> 10) & 1) << 1) | (((xyz >> 20) & 1) << 2);
    const double *lp = A.L + (P.base + C.parent[b]) * A.n;
    double *out = A.L + (C.base + b) * A.n;
    for (int j = threadIdx.x; j < A.n; j += blockDim.x) {
        const double *M = A.l2l + ((long long)o * A.n + j) * A.n;
        double acc = 0.0;
        for (int i = 0; i < A.n; ++i) acc += M[i] * lp[i];
        out[j] += acc;
    }
}

// L2P: the potential of the leaf's local expansion (downward equivalent densities) at its points.
__global__ void l2p_kernel(FmmArgs A) {
    extern __shared__ double sm[];
    double *y = sm;              // 3 n: downward equivalent points
    double *lv = sm + 3 * A.n;   // n
    const FmmLevel &L = A.levels[A.depth];
    const long long b = blockIdx.x;
    double c0, c1, c2;
    box_centre(L, b, A.origin[0], A.origin[1], A.origin[2], c0, c1, c2);
    const double h = kAlphaOuter * 0.5 * L.width;
    for (int j = threadIdx.x; j < A.n; j += blockDim.x) {
        y[3 * j] = c0 + h * A.unit[3 * j];
        y[3 * j + 1] = c1 + h * A.unit[3 * j + 1];
        y[3 * j + 2] = c2 + h * A.unit[3 * j + 2];
        lv[j] = A.L[(L.base + b) * A.n + j];
    }
    __syncthreads();
    for (long long i = A.leaf_start[b] + threadIdx.x; i < A.leaf_start[b + 1]; i += blockDim.x) {
        const double x0 = A.pts[3 * i], x1 = A.pts[3 * i + 1], x2 = A.pts[3 * i + 2];
        double acc = 0.0;
        for (int j = 0; j < A.n; ++j) acc += lv[j] * green(x0, x1, x2, y[3 * j], y[3 * j + 1], y[3 * j + 2]);
        A.pot[i] += acc;
    }
}

// P2P: direct interactions of the leaf's points with the points of its neighbour leaves (itself
// included, the point itself excluded), sources staged through shared memory in tiles.
__global__ void p2p_kernel(FmmArgs A) {
    constexpr int TILE = 256;
    __shared__ double ys[TILE][4];
    const long long b = blockIdx.x;
    const long long s = A.leaf_start[b], e = A.leaf_start[b + 1];
    for (long long i0 = s; i0 < e; i0 += blockDim.x) {
        const long long i = i0 + threadIdx.x;
        const bool active = i < e;
        double x0 = 0, x1 = 0, x2 = 0, acc = 0.0;
        if (active) {
            x0 = A.pts[3 * i];
            x1 = A.pts[3 * i + 1];
            x2 = A.pts[3 * i + 2];
        }
        for (long long k = A.nbr_start[b]; k < A.nbr_start[b + 1]; ++k) {
            const int nb = A.nbr[k];
            const long long ns = A.leaf_start[nb], ne = A.leaf_start[nb + 1];
            for (long long t0 = ns; t0 < ne; t0 += TILE) {
                __syncthreads();
                for (int t = threadIdx.x; t < TILE && t0 + t < ne; t += blockDim.x) {
                    ys[t][0] = A.pts[3 * (t0 + t)];
                    ys[t][1] = A.pts[3 * (t0 + t) + 1];
                    ys[t][2] = A.pts[3 * (t0 + t) + 2];
                    ys[t][3] = A.q[t0 + t];
                }
                __syncthreads();
                const int cnt = (int)(ne - t0 < TILE ? ne - t0 : TILE);
                if (active) {
                    for (int t = 0; t < cnt; ++t) {
                        if (t0 + t == i) continue;
                        acc += ys[t][3] * green(x0, x1, x2, ys[t][0], ys[t][1], ys[t][2]);
                    }
                }
            }
        }
        if (active) A.pot[i] += acc;
    }
}

int launched(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s launch failed: %s", what, cudaGetErrorString(e));
        return M2L_ECUDA;
    }
    return M2L_OK;
}

}  // namespace

int fmm_gather(const double *src, const long long *perm, long long n, double *dst, cudaStream_t s) {
    if (n <= 0) return M2L_OK;
    gather_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, s>>>(src, perm, n, dst);
    return launched("gather");
}

int fmm_scatter(const double *src, const long long *perm, long long n, double *dst, cudaStream_t s) {
    if (n <= 0) return M2L_OK;
    scatter_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, s>>>(src, perm, n, dst);
    return launched("scatter");
}

int fmm_upward(const FmmArgs &A, const long long *nboxes, cudaStream_t s) {
    const size_t smem = sizeof(double) * (size_t)(A.n + A.r_up);
    p2m_kernel<<<(unsigned)nboxes[A.depth], 128, smem, s>>>(A);
    if (int rc = launched("p2m")) return rc;
    for (int l = A.depth - 1; l >= 2; --l) {
        m2m_kernel<<<(unsigned)nboxes[l], 128, 0, s>>>(A, l);
        if (int rc = launched("m2m")) return rc;
    }
    return M2L_OK;
}

int fmm_downward(const FmmArgs &A, const long long *nboxes, cudaStream_t s) {
    for (int l = 3; l <= A.depth; ++l) {
        l2l_kernel<<<(unsigned)nboxes[l], 128, 0, s>>>(A, l);
        if (int rc = launched("l2l")) return rc;
    }
    const size_t smem = sizeof(double) * (size_t)(4 * A.n);
    l2p_kernel<<<(unsigned)nboxes[A.depth], 128, smem, s>>>(A);
    if (int rc = launched("l2p")) return rc;
    p2p_kernel<<<(unsigned)nboxes[A.depth], 128, 0, s>>>(A);
    return launched("p2p");
}

}  // namespace m2l
