// CUDA-core kernels of the M2L library (FP64 and FP32): the small GEMMs of the BLAS form
// (compress S^T q, uncompress + pseudo-inverse), the gathered contraction over the 189
// transfer vectors of each target octant, and the three stages of the FFT form.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <type_traits>

#include "internal.h"
#include "kernels.cuh"

namespace m2l {

// ----------------------------------------------------------------------------------------------
// Constant tables.
//   c_tidx[x+3][y+3][z+3]: index of transfer vector (x, y, z) in [-3,3]^3 \ [-1,1]^3 (x slowest), or -1.
//   c_clu[d][8 i + j]:     transfer vector from child j of the source cluster in direction d to
//                          child i of the target cluster, or -1 when the two boxes are adjacent
//                          (App. A.1 cluster formulation: 26 directions x 64 pairs).
//   c_dir[d]:              the 26 parent offsets in [-1,1]^3 \ {0}, x slowest.
__constant__ short c_tidx[7][7][7];
__constant__ short c_clu[26][64];
__constant__ signed char c_dir[26][3];
// exp(-2 pi i m / g) for m in [0, g), for the grid sides of the FP32 transforms specialised on
// (p, g): g = 2p - 1 and 2p for p = 4, 6, 8, 10, stored one after another (twiddle_offset).
__constant__ float2 c_twf[108];
constexpr int kTwiddleSides[8] = {7, 8, 11, 12, 15, 16, 19, 20};
__host__ __device__ constexpr int twiddle_offset(int g) {
    int off = 0;
    for (int i = 0; i < 8; ++i) {
        if (kTwiddleSides[i] == g) return off;
        off += kTwiddleSides[i];
    }
    return -1;
}

static void cache_launch_shapes();

int ensure_constants(int device) {
    static bool done[64] = {false};
    if (device < 0 || device >= 64) return M2L_EINVAL;
    if (done[device]) return M2L_OK;
    cache_launch_shapes();  // before any launch, so never inside a stream capture
    short tidx[7][7][7];
    for (int x = -3; x <= 3; ++x)
        for (int y = -3; y <= 3; ++y)
            for (int z = -3; z <= 3; ++z) tidx[x + 3][y + 3][z + 3] = (short)transfer_index(x, y, z);
    short clu[26][64];
    signed char dir[26][3];
    int d = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                if (!dx && !dy && !dz) continue;
                dir[d][0] = (signed char)dx; dir[d][1] = (signed char)dy; dir[d][2] = (signed char)dz;
                for (int i = 0; i < 8; ++i)
                    for (int j = 0; j < 8; ++j) {
                        int tx = 2 * dx + (j & 1) - (i & 1);
                        int ty = 2 * dy + ((j >> 1) & 1) - ((i >> 1) & 1);
                        int tz = 2 * dz + ((j >> 2) & 1) - ((i >> 2) & 1);
                        clu[d][8 * i + j] = (short)transfer_index(tx, ty, tz);
                    }
                ++d;
            }
    float2 twf[108];
    for (int i = 0, off = 0; i < 8; off += kTwiddleSides[i], ++i)
        for (int m = 0; m < kTwiddleSides[i]; ++m) {
            const double a = -2.0 * M_PI * m / kTwiddleSides[i];
            twf[off + m] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
    if (cudaMemcpyToSymbol(c_twf, twf, sizeof twf) != cudaSuccess ||
        cudaMemcpyToSymbol(c_tidx, tidx, sizeof tidx) != cudaSuccess ||
        cudaMemcpyToSymbol(c_clu, clu, sizeof clu) != cudaSuccess ||
        cudaMemcpyToSymbol(c_dir, dir, sizeof dir) != cudaSuccess) {
        set_error("uploading constant tables failed: %s", cudaGetErrorString(cudaGetLastError()));
        return M2L_ECUDA;
    }
    done[device] = true;
    return M2L_OK;
}

// Streaming multiprocessors of the current device (launch shapes are sized in waves of CTAs).
static int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!cached[dev]) {
        int n = 0;
        cached[dev] = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0 ? n : 152;
    }
    return cached[dev];
}

static int check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s launch failed: %s", what, cudaGetErrorString(e));
        return M2L_ECUDA;
    }
    return M2L_OK;
}

// ----------------------------------------------------------------------------------------------
// Columns per thread for a rank: the fewest column blocks of at most 16 * max_tn columns, then
// the narrowest blocks that still cover k_pad.
inline int contract_tn(int kp, int max_tn) {
    const int units = (kp + 15) / 16;
    const int blocks = (units + max_tn - 1) / max_tn;
    return (units + blocks - 1) / blocks;
}

// Y = X W^T (+ Y): 64 rows x 16 TN columns per CTA, 4 x TN per thread, K in steps of 16 (one
// type for X, W and accumulation, written as TY). TN is picked per output width so the column
// blocks cover it with little padding (as in the contraction).
template <class TX, class TW, class TY, int TN>
__global__ void __launch_bounds__(256) gemm_xwt_kernel(const TX *__restrict__ X, long long ldx,
                                                       const TW *__restrict__ W, long long ldw,
                                                       TY *__restrict__ Y, long long ldy, long long rows,
                                                       int O, int K, int acc) {
    constexpr int BM = 64, BN = 16 * TN, BK = 16;
    __shared__ TW Xs[BK][BM + 4];
    __shared__ TW Ws[BK][BN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const long long row0 = (long long)blockIdx.x * BM;
    const int col0 = blockIdx.y * BN;
    // In single precision each block of BK terms is summed on its own and then added to the
    // running sum: the rounding of a K-term sum grows with the length of the sequential chain, and
    // this takes it from K to about BK + K / BK additions (3e-7 -> 1e-7 relative at K = 296 for
    // densities of both signs). FP64 keeps one chain.
    constexpr bool kBlocked = sizeof(TW) == 4;
    TW a[4][TN];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) a[i][j] = TW(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += 256) {
            const int r = e / BK, kk = e % BK;
            const long long gr = row0 + r;
            const int gk = k0 + kk;
            Xs[kk][r] = (gr < rows && gk < K) ? (TW)X[gr * ldx + gk] : TW(0);
        }
        for (int e = tid; e < BN * BK; e += 256) {
            const int c = e / BK, kk = e % BK, gc = col0 + c, gk = k0 + kk;
            Ws[kk][c] = (gc < O && gk < K) ? W[(long long)gc * ldw + gk] : TW(0);
        }
        __syncthreads();
        TW bl[4][TN];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) bl[i][j] = TW(0);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            TW xa[4], wb[TN];
#pragma unroll
            for (int i = 0; i < 4; ++i) xa[i] = Xs[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < TN; ++j) wb[j] = Ws[kk][tx * TN + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    if (kBlocked)
                        bl[i][j] = fma(xa[i], wb[j], bl[i][j]);
                    else
                        a[i][j] = fma(xa[i], wb[j], a[i][j]);
                }
        }
        if (kBlocked) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) a[i][j] += bl[i][j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        long long r = row0 + ty * 4 + i;
        if (r >= rows) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int c = col0 + tx * TN + j;
            if (c < O) {
                TW v = a[i][j];
                if (acc) v += (TW)Y[r * ldy + c];
                Y[r * ldy + c] = (TY)v;
            }
        }
    }
}

template <class T, int TN>
static void launch_gemm_tn(const T *X, long long ldx, const T *W, long long ldw, T *Y, long long ldy, long long rows,
                           int O, int K, int acc, cudaStream_t s) {
    dim3 grid((unsigned)((rows + 63) / 64), (unsigned)((O + 16 * TN - 1) / (16 * TN)));
    gemm_xwt_kernel<T, T, T, TN><<<grid, 256, 0, s>>>(X, ldx, W, ldw, Y, ldy, rows, O, K, acc);
}

// Y = X (W_hi + W_lo)^T (+ Y) for FP32 data with about twice FP32's precision in the sum: every
// product x w_hi is split exactly into p + e with one FMA, the running sum is an unevaluated
// pair s + c updated by Knuth's TwoSum, and c also gathers e and the small term x w_lo (the
// compensated dot product of Ogita, Rump and Oishi, "Accurate sum and dot product", 2005).
// W_lo is the part of an FP64 operator below its FP32 rounding. Used for the second factor of
// the pseudo-inverse (Eq. 9), whose sum cancels heavily: its terms reach 1 / (alpha s_0) times
// the check potential while the result is of the size of the check potential.
__global__ void __launch_bounds__(256) gemm_xwt_ff_kernel(const float *__restrict__ X, long long ldx,
                                                          const float *__restrict__ Wh, const float *__restrict__ Wl,
                                                          long long ldw, float *__restrict__ Y, long long ldy,
                                                          long long rows, int O, int K, int acc) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ float Xs[BK][BM + 4];
    __shared__ float Whs[BK][BN + 4];
    __shared__ float Wls[BK][BN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const long long row0 = (long long)blockIdx.x * BM;
    const int col0 = blockIdx.y * BN;
    float sh[4][4], sl[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) sh[i][j] = sl[i][j] = 0.f;
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += 256) {
            const int r = e / BK, kk = e % BK;
            const long long gr = row0 + r;
            const int gk = k0 + kk, gc = col0 + r;
            Xs[kk][r] = (gr < rows && gk < K) ? X[gr * ldx + gk] : 0.f;
            const bool w = gc < O && gk < K;
            Whs[kk][r] = w ? Wh[(long long)gc * ldw + gk] : 0.f;
            Wls[kk][r] = w ? Wl[(long long)gc * ldw + gk] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            float xa[4], wh[4], wl[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                xa[i] = Xs[kk][ty * 4 + i];
                wh[i] = Whs[kk][tx * 4 + i];
                wl[i] = Wls[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float p = __fmul_rn(xa[i], wh[j]);
                    const float e = __fmaf_rn(xa[i], wh[j], -p);  // x w_hi = p + e exactly
                    const float t = __fadd_rn(sh[i][j], p);
                    const float z = __fsub_rn(t, sh[i][j]);
                    const float d = __fadd_rn(__fsub_rn(sh[i][j], __fsub_rn(t, z)), __fsub_rn(p, z));  // s + p = t + d
                    sh[i][j] = t;
                    sl[i][j] = __fmaf_rn(xa[i], wl[j], __fadd_rn(sl[i][j], __fadd_rn(d, e)));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long r = row0 + ty * 4 + i;
        if (r >= rows) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = col0 + tx * 4 + j;
            if (c < O) {
                float v = __fadd_rn(sh[i][j], sl[i][j]);
                if (acc) v = __fadd_rn(Y[r * ldy + c], v);
                Y[r * ldy + c] = v;
            }
        }
    }
}

// gemm_xwt_ff_kernel on 128 x 64 tiles with 16-byte loads (as gemm_xwt_f32v_kernel): a thread
// 8 rows x 4 columns, operands one K block ahead in registers. Same compensated arithmetic, term
// for term in the same order, so results equal gemm_xwt_ff_kernel's. Needs K, ldx, ldw multiples
// of 4 and 16-byte aligned X, Wh, Wl.
__global__ void __launch_bounds__(256) gemm_xwt_ff_v_kernel(const float *__restrict__ X, long long ldx,
                                                            const float *__restrict__ Wh, const float *__restrict__ Wl,
                                                            long long ldw, float *__restrict__ Y, long long ldy,
                                                            long long rows, int O, int K, int acc) {
    constexpr int BM = 128, BN = 64, BK = 16;
    __shared__ __align__(16) float Xs[BK][BM + 4];
    __shared__ __align__(16) float Whs[BK][BN + 4];
    __shared__ __align__(16) float Wls[BK][BN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const long long row0 = (long long)blockIdx.x * BM;
    const int col0 = blockIdx.y * BN;
    const int lr = tid >> 2, lk = (tid & 3) * 4;
    float4 xr[2], hr, lr4;
    auto load = [&](int k0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long long gr = row0 + lr + 64 * h;
            xr[h] = (gr < rows && k0 + lk < K) ? *reinterpret_cast<const float4 *>(X + gr * ldx + k0 + lk)
                                               : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const int gc = col0 + lr;
        const bool w = gc < O && k0 + lk < K;
        hr = w ? *reinterpret_cast<const float4 *>(Wh + (long long)gc * ldw + k0 + lk) : make_float4(0.f, 0.f, 0.f, 0.f);
        lr4 = w ? *reinterpret_cast<const float4 *>(Wl + (long long)gc * ldw + k0 + lk) : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    float sh[8][4], sl[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) sh[i][j] = sl[i][j] = 0.f;
    load(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            Xs[lk + 0][lr + 64 * h] = xr[h].x;
            Xs[lk + 1][lr + 64 * h] = xr[h].y;
            Xs[lk + 2][lr + 64 * h] = xr[h].z;
            Xs[lk + 3][lr + 64 * h] = xr[h].w;
        }
        Whs[lk + 0][lr] = hr.x; Whs[lk + 1][lr] = hr.y; Whs[lk + 2][lr] = hr.z; Whs[lk + 3][lr] = hr.w;
        Wls[lk + 0][lr] = lr4.x; Wls[lk + 1][lr] = lr4.y; Wls[lk + 2][lr] = lr4.z; Wls[lk + 3][lr] = lr4.w;
        __syncthreads();
        if (k0 + BK < K) load(k0 + BK);
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            const float4 x0 = *reinterpret_cast<const float4 *>(&Xs[kk][ty * 4]);
            const float4 x1 = *reinterpret_cast<const float4 *>(&Xs[kk][64 + ty * 4]);
            const float4 wh4 = *reinterpret_cast<const float4 *>(&Whs[kk][tx * 4]);
            const float4 wl4 = *reinterpret_cast<const float4 *>(&Wls[kk][tx * 4]);
            const float xa[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
            const float wh[4] = {wh4.x, wh4.y, wh4.z, wh4.w}, wl[4] = {wl4.x, wl4.y, wl4.z, wl4.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float p = __fmul_rn(xa[i], wh[j]);
                    const float e = __fmaf_rn(xa[i], wh[j], -p);  // x w_hi = p + e exactly
                    const float t = __fadd_rn(sh[i][j], p);
                    const float z = __fsub_rn(t, sh[i][j]);
                    const float d = __fadd_rn(__fsub_rn(sh[i][j], __fsub_rn(t, z)), __fsub_rn(p, z));  // s + p = t + d
                    sh[i][j] = t;
                    sl[i][j] = __fmaf_rn(xa[i], wl[j], __fadd_rn(sl[i][j], __fadd_rn(d, e)));
                }
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const long long r = row0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
        if (r >= rows) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = col0 + tx * 4 + j;
            if (c < O) {
                float v = __fadd_rn(sh[i][j], sl[i][j]);
                if (acc) v = __fadd_rn(Y[r * ldy + c], v);
                Y[r * ldy + c] = v;
            }
        }
    }
}

int launch_gemm_xwt_ff(const float *X, long long ldx, const float *Wh, const float *Wl, long long ldw, float *Y,
                       long long ldy, long long rows, int O, int K, int acc, cudaStream_t s) {
    if (rows <= 0 || O <= 0) return M2L_OK;
    if (K % 4 == 0 && ldx % 4 == 0 && ldw % 4 == 0 && ((uintptr_t)X & 15) == 0 && ((uintptr_t)Wh & 15) == 0 &&
        ((uintptr_t)Wl & 15) == 0) {
        dim3 grid((unsigned)((rows + 127) / 128), (unsigned)((O + 63) / 64));
        gemm_xwt_ff_v_kernel<<<grid, 256, 0, s>>>(X, ldx, Wh, Wl, ldw, Y, ldy, rows, O, K, acc);
        return check_launch("gemm_ff");
    }
    dim3 grid((unsigned)((rows + 63) / 64), (unsigned)((O + 63) / 64));
    gemm_xwt_ff_kernel<<<grid, 256, 0, s>>>(X, ldx, Wh, Wl, ldw, Y, ldy, rows, O, K, acc);
    return check_launch("gemm_ff");
}

// Y = X W^T (+ Y) in FP32 with 16-byte loads: 128 rows x 64 columns per CTA, a thread 8 rows x
// 4 columns (two groups of 4 consecutive rows, 64 apart, read as two 16-byte shared loads), K in
// blocks of 16 loaded into registers one block ahead of their use and stored to shared memory
// transposed. Each block of 16 terms is summed on its own, then added to the running sum (the
// same blocked accumulation as gemm_xwt_kernel). Needs K, ldx and ldw multiples of 4 and 16-byte
// aligned X and W.
__global__ void __launch_bounds__(256) gemm_xwt_f32v_kernel(const float *__restrict__ X, long long ldx,
                                                            const float *__restrict__ W, long long ldw,
                                                            float *__restrict__ Y, long long ldy, long long rows,
                                                            int O, int K, int acc) {
    constexpr int BM = 128, BN = 64, BK = 16;
    __shared__ __align__(16) float Xs[BK][BM + 4];
    __shared__ __align__(16) float Ws[BK][BN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const long long row0 = (long long)blockIdx.x * BM;
    const int col0 = blockIdx.y * BN;
    // loaders: X rows tid / 4 and 64 + tid / 4, W row tid / 4, K offset (tid % 4) * 4
    const int lr = tid >> 2, lk = (tid & 3) * 4;
    float4 xr[2], wr;
    auto load = [&](int k0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long long gr = row0 + lr + 64 * h;
            xr[h] = (gr < rows && k0 + lk < K) ? *reinterpret_cast<const float4 *>(X + gr * ldx + k0 + lk)
                                               : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const int gc = col0 + lr;
        wr = (gc < O && k0 + lk < K) ? *reinterpret_cast<const float4 *>(W + (long long)gc * ldw + k0 + lk)
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    float a[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) a[i][j] = 0.f;
    load(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
        __syncthreads();  // the previous block's operands are consumed
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            Xs[lk + 0][lr + 64 * h] = xr[h].x;
            Xs[lk + 1][lr + 64 * h] = xr[h].y;
            Xs[lk + 2][lr + 64 * h] = xr[h].z;
            Xs[lk + 3][lr + 64 * h] = xr[h].w;
        }
        Ws[lk + 0][lr] = wr.x;
        Ws[lk + 1][lr] = wr.y;
        Ws[lk + 2][lr] = wr.z;
        Ws[lk + 3][lr] = wr.w;
        __syncthreads();
        if (k0 + BK < K) load(k0 + BK);  // in flight while this block is summed
        float bl[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) bl[i][j] = 0.f;
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 x0 = *reinterpret_cast<const float4 *>(&Xs[kk][ty * 4]);
            const float4 x1 = *reinterpret_cast<const float4 *>(&Xs[kk][64 + ty * 4]);
            const float4 w = *reinterpret_cast<const float4 *>(&Ws[kk][tx * 4]);
            const float xa[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
            const float wb[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) bl[i][j] = fmaf(xa[i], wb[j], bl[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) a[i][j] += bl[i][j];
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const long long r = row0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
        if (r >= rows) continue;
        const int c = col0 + tx * 4;
        float *y = Y + r * ldy + c;
        if (c + 3 < O && (ldy & 3) == 0) {
            float4 v = make_float4(a[i][0], a[i][1], a[i][2], a[i][3]);
            if (acc) {
                const float4 o = *reinterpret_cast<const float4 *>(y);
                v.x += o.x; v.y += o.y; v.z += o.z; v.w += o.w;
            }
            *reinterpret_cast<float4 *>(y) = v;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (c + j < O) y[j] = acc ? y[j] + a[i][j] : a[i][j];
        }
    }
}

template <class T>
int launch_gemm_xwt(const T *X, long long ldx, const T *W, long long ldw, T *Y, long long ldy,
                    long long rows, int O, int K, int acc, cudaStream_t s) {
    if (rows <= 0 || O <= 0) return M2L_OK;
    if constexpr (sizeof(T) == 4) {
        const bool vec = K % 4 == 0 && ldx % 4 == 0 && ldw % 4 == 0 && ((uintptr_t)X & 15) == 0 && ((uintptr_t)W & 15) == 0;
        if (vec) {
            dim3 grid((unsigned)((rows + 127) / 128), (unsigned)((O + 63) / 64));
            gemm_xwt_f32v_kernel<<<grid, 256, 0, s>>>((const float *)X, ldx, (const float *)W, ldw, (float *)Y, ldy, rows,
                                                       O, K, acc);
            return check_launch("gemm");
        }
    }
    switch (contract_tn(O, sizeof(T) == 8 ? 12 : 8)) {
        case 1: launch_gemm_tn<T, 1>(X, ldx, W, ldw, Y, ldy, rows, O, K, acc, s); break;
        case 2: launch_gemm_tn<T, 2>(X, ldx, W, ldw, Y, ldy, rows, O, K, acc, s); break;
        case 3: launch_gemm_tn<T, 3>(X, ldx, W, ldw, Y, ldy, rows, O, K, acc, s); break;
        case 4: launch_gemm_tn<T, 4>(X, ldx, W, ldw, Y, ldy, rows, O, K, acc, s); break;
        case 5: launch_gemm_tn<T, 5>(X, ldx, W, ldw, Y, ldy, rows, O, K, acc, s); break;
        case 6: launch_gemm_tn<T, 6>(X, ldx, W, ldw, Y, ldy, rows, O, K, acc, s); break;
        case 7: launch_gemm_tn<T, 7>(X, ldx, W, ldw, Y, ldy, rows, O, K, acc, s); break;
        case 8: launch_gemm_tn<T, 8>(X, ldx, W, ldw, Y, ldy, rows, O, K, acc, s); break;
        case 9: launch_gemm_tn<T, 9>(X, ldx, W, ldw, Y, ldy, rows, O, K, acc, s); break;
        case 10: launch_gemm_tn<T, 10>(X, ldx, W, ldw, Y, ldy, rows, O, K, acc, s); break;
        case 11: launch_gemm_tn<T, 11>(X, ldx, W, ldw, Y, ldy, rows, O, K, acc, s); break;
        default: launch_gemm_tn<T, 12>(X, ldx, W, ldw, Y, ldy, rows, O, K, acc, s); break;
    }
    return check_launch("gemm");
}

// ----------------------------------------------------------------------------------------------
// B2 on CUDA cores: for a tile of (target, rhs) rows of one octant, accumulate over the transfer
// vectors of that octant phit[row] += C_t qt[source(row, t)] (Sec. 3.2 steps 3-5 fused: sources
// are gathered on the fly, nothing is materialised per transfer vector). The tile's list holds
// only the transfer vectors that reach a source from one of its targets.
// A CTA computes 64 rows x 16 TN columns, a thread 4 rows x TN columns; TN is picked per rank so
// the column blocks cover k_pad with little padding (every padded column costs as much as a real
// one on the FP64 units, which bound this kernel).
template <class T, int TN>
__global__ void __launch_bounds__(256) contract_simt_kernel(const LevelView *__restrict__ levels,
                                                            const ContractTile *__restrict__ tiles,
                                                            const int *__restrict__ tvl,
                                                            const T *__restrict__ qt, const T *__restrict__ C, int kp,
                                                            int kcp, long long zero_row, T *__restrict__ phit) {
    constexpr int BM = 64, BN = 16 * TN, BK = 16;
    __shared__ T Xs[BK][BM + 4];
    __shared__ T Ws[BK][BN + 4];
    __shared__ long long src_row[BM];
    __shared__ int tgt_b[BM], tgt_r[BM];
    __shared__ uint32_t tgt_xyz[BM];
    const ContractTile tile = tiles[blockIdx.x];
    const LevelView &L = levels[tile.lev];
    const int R = L.R;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int col0 = blockIdx.y * BN;
    if (tid < BM) {
        if (tid < tile.rows) {
            long long j = (long long)tile.j0 + tid;
            int b = L.perm[L.oct_start[tile.oct] + j / R];
            tgt_b[tid] = b;
            tgt_r[tid] = (int)(j % R);
            tgt_xyz[tid] = L.xyz[b];
        } else {
            tgt_b[tid] = -1;
            tgt_r[tid] = 0;
            tgt_xyz[tid] = 0;
        }
    }
    T a[4][TN];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) a[i][j] = T(0);
    const int N = L.N;
    for (int v = 0; v < tile.ntv; ++v) {
        const int pk = tvl[tile.tv0 + v];
        const int dx = (pk & 15) - 3, dy = ((pk >> 4) & 15) - 3, dz = ((pk >> 8) & 15) - 3;
        const int ti = pk >> 12;
        __syncthreads();  // previous src_row fully consumed
        if (tid < BM) {
            long long sr = zero_row;
            if (tgt_b[tid] >= 0) {
                uint32_t p = tgt_xyz[tid];
                int x = (int)(p & 1023) + dx, y = (int)((p >> 10) & 1023) + dy, z = (int)((p >> 20) & 1023) + dz;
                if (x >= 0 && y >= 0 && z >= 0 && x < N && y < N && z < N) {
                    int s = L.slot[((long long)z * N + y) * N + x];
                    if (s >= 0) sr = L.row0 + (long long)s * R + tgt_r[tid];
                }
            }
            src_row[tid] = sr;
        }
        __syncthreads();
        // a warp holds 8 rows; when none of them has a source for this transfer vector (targets
        // at the domain boundary, empty boxes) it skips the products and only helps with loads
        bool mine = false;
#pragma unroll
        for (int i = 0; i < 4; ++i) mine |= src_row[ty * 4 + i] != zero_row;
        const bool live = __any_sync(0xffffffffu, mine);
        const T *Ct = C + (long long)ti * kcp * kp;  // [kcp][kp]
        for (int k0 = 0; k0 < kp; k0 += BK) {
            for (int e = tid; e < BM * BK; e += 256) {
                const int r = e / BK, kk = e % BK;
                Xs[kk][r] = qt[src_row[r] * kp + k0 + kk];
            }
            for (int e = tid; e < BN * BK; e += 256) {
                const int c = e / BK, kk = e % BK, gc = col0 + c;
                Ws[kk][c] = gc < kcp ? Ct[(long long)gc * kp + k0 + kk] : T(0);
            }
            __syncthreads();
            if (live) {
#pragma unroll
                for (int kk = 0; kk < BK; ++kk) {
                    T xa[4], wb[TN];
#pragma unroll
                    for (int i = 0; i < 4; ++i) xa[i] = Xs[kk][ty * 4 + i];
#pragma unroll
                    for (int j = 0; j < TN; ++j) wb[j] = Ws[kk][tx * TN + j];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < TN; ++j) a[i][j] = fma(xa[i], wb[j], a[i][j]);
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int r = ty * 4 + i;
        if (r >= tile.rows) continue;
        long long orow = L.row0 + (long long)tgt_b[r] * R + tgt_r[r];
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int c = col0 + tx * TN + j;
            if (c < kcp) phit[orow * kcp + c] = a[i][j];
        }
    }
}

// B2 with the directional factors of Eq. 15. Per transfer vector t the tile's gathered sources X
// (BM rows x k) go through the two products of Sec. 3.2 step 4: xi = X Vbar'_t (BM x k_t) and
// phit += xi Ubar_t^T, so a pair costs 4 k k_t flops instead of 2 k^2. Stage 1 streams X and
// Vbar'_t^T through shared memory in chunks of 16 along k (as the plain kernel streams C_t). The
// k_t columns of xi (up to 64 per pass) are cut into 8 contiguous groups of floor or ceil(k_t / 8)
// columns, one per warp, and a lane holds BM / 32 consecutive rows of its warp's group: the column
// count is exact (no rounding of k_t up to a multiple of 8), a warp's trip count is uniform and
// its column loads are broadcasts. xi then waits in shared memory for stage 2, which gives a
// thread BM / 16 rows x TN columns and takes Ubar_t in chunks of 16 along k_t. Stage 1 is skipped
// when no row of the tile has a source for t, stage 2 per warp of BM / 8 rows. In FP64, tiles of
// 32 rows (1,176 on the 1M-point workload against 592 of 64) leave a shorter tail of idle SMs
// after the last wave; two CTAs share an SM.
// One 16-deep chunk of stage 1 with exactly NM columns per lane: guarding an unrolled loop with a
// runtime count would leave predicated-off FMAs that still occupy the FP64 pipe.
template <class T, int NM, int RPL, int XP>
__device__ __forceinline__ void dir_stage1_chunk(const T *Xs, const T *Vs, int c0, int lane, T (&y)[8][RPL]) {
    constexpr int VP = 66;
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
        T x[RPL];
        if constexpr (RPL == 2) {
            using T2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
            const T2 x2 = *reinterpret_cast<const T2 *>(Xs + kk * XP + 2 * lane);  // rows 2 l, 2 l + 1
            x[0] = x2.x;
            x[1] = x2.y;
        } else {
            x[0] = Xs[kk * XP + lane];
        }
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const T w = Vs[kk * VP + c0 + m];
#pragma unroll
            for (int r = 0; r < RPL; ++r) y[m][r] = fma(x[r], w, y[m][r]);
        }
    }
}

// FP32 asks for three resident CTAs per SM (80 registers, no spills): its FMAs are cheap, and
// shared-load latency needs more warps to hide. FP64 is bound by its FP64 units at two.
template <class T, int TN, int BM>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) contract_simt_dir_kernel(const LevelView *__restrict__ levels,
                                                                const ContractTile *__restrict__ tiles,
                                                                const int *__restrict__ tvl, const T *__restrict__ qt,
                                                                const T *__restrict__ Ub, const T *__restrict__ Vt,
                                                                const int4 *__restrict__ meta, int k, int kp, int kcp, int kt8max,
                                                                long long zero_row, T *__restrict__ phit) {
    static_assert(BM == 32 || BM == 64, "tile heights of 32 or 64 rows");
    constexpr int BN = 16 * TN, BK = 16, XP = BM + 2, YC = 64, RPL = BM / 32, RPT = BM / 16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Ys = reinterpret_cast<T *>(smem_raw);  // [kt8max][XP]: xi transposed
    T *Xs = Ys + (size_t)kt8max * XP;         // [BK][XP]: a chunk of X transposed
    T *Vs = Xs + (size_t)BK * XP;             // [BK][YC + 2]: a chunk of Vbar'_t
    T *Us = Vs + (size_t)BK * (YC + 2);       // [BK][BN + 4]: a chunk of Ubar_t
    __shared__ long long src_row[BM];
    __shared__ int tgt_b[BM], tgt_r[BM];
    __shared__ uint32_t tgt_xyz[BM];
    const ContractTile tile = tiles[blockIdx.x];
    const LevelView &L = levels[tile.lev];
    const int R = L.R;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, lane = tid & 31, warp = tid >> 5;
    const int col0 = blockIdx.y * BN;
    if (tid < BM) {
        if (tid < tile.rows) {
            long long j = (long long)tile.j0 + tid;
            int b = L.perm[L.oct_start[tile.oct] + j / R];
            tgt_b[tid] = b;
            tgt_r[tid] = (int)(j % R);
            tgt_xyz[tid] = L.xyz[b];
        } else {
            tgt_b[tid] = -1;
            tgt_r[tid] = 0;
            tgt_xyz[tid] = 0;
        }
    }
    T a[RPT][TN];
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) a[i][j] = T(0);
    const int N = L.N;
    for (int v = 0; v < tile.ntv; ++v) {
        const int pk = tvl[tile.tv0 + v];
        const int dx = (pk & 15) - 3, dy = ((pk >> 4) & 15) - 3, dz = ((pk >> 8) & 15) - 3;
        const int4 md = meta[pk >> 12];  // Ubar_t offset, Vbar'_t^T offset, k_t, k_t rounded up to 8
        __syncthreads();                 // previous transfer vector's shared memory fully consumed
        if (tid < BM) {
            long long sr = zero_row;
            if (tgt_b[tid] >= 0) {
                uint32_t p = tgt_xyz[tid];
                int x = (int)(p & 1023) + dx, y = (int)((p >> 10) & 1023) + dy, z = (int)((p >> 20) & 1023) + dz;
                if (x >= 0 && y >= 0 && z >= 0 && x < N && y < N && z < N) {
                    int s = L.slot[((long long)z * N + y) * N + x];
                    if (s >= 0) sr = L.row0 + (long long)s * R + tgt_r[tid];
                }
            }
            src_row[tid] = sr;
        }
        __syncthreads();
        bool mine = false, mine1 = false;
#pragma unroll
        for (int i = 0; i < RPT; ++i) mine |= src_row[ty * RPT + i] != zero_row;
#pragma unroll
        for (int r = 0; r < RPL; ++r) mine1 |= src_row[RPL * lane + r] != zero_row;
        const bool live = __any_sync(0xffffffffu, mine);
        const bool live1 = __any_sync(0xffffffffu, mine1);
        // stage 1: xi = X Vbar'_t, up to 64 columns of xi per pass
        for (int jp0 = 0; jp0 < md.z; jp0 += YC) {
            const int ncol = min(YC, md.z - jp0), q = ncol >> 3, rm = ncol & 7;
            const int nm = q + (warp < rm ? 1 : 0), c0 = warp * q + min(warp, rm);
            T y[8][RPL];
#pragma unroll
            for (int m = 0; m < 8; ++m)
#pragma unroll
                for (int r = 0; r < RPL; ++r) y[m][r] = T(0);
            const T *V = Vt + md.y + (size_t)jp0 * kp;
            for (int k0 = 0; k0 < k; k0 += BK) {
                if (k0) __syncthreads();  // previous chunk consumed
                for (int e = tid; e < BM * BK; e += 256) {
                    const int r = e / BK, kk = e % BK;
                    Xs[kk * XP + r] = k0 + kk < kp ? qt[src_row[r] * kp + k0 + kk] : T(0);
                }
                for (int e = tid; e < ncol * BK; e += 256) {
                    const int j = e / BK, kk = e % BK;
                    Vs[kk * (YC + 2) + j] = k0 + kk < kp ? V[(size_t)j * kp + k0 + kk] : T(0);
                }
                __syncthreads();
                if (live1) {
                    switch (nm) {
                        case 0: break;
                        case 1: dir_stage1_chunk<T, 1, RPL, XP>(Xs, Vs, c0, lane, y); break;
                        case 2: dir_stage1_chunk<T, 2, RPL, XP>(Xs, Vs, c0, lane, y); break;
                        case 3: dir_stage1_chunk<T, 3, RPL, XP>(Xs, Vs, c0, lane, y); break;
                        case 4: dir_stage1_chunk<T, 4, RPL, XP>(Xs, Vs, c0, lane, y); break;
                        case 5: dir_stage1_chunk<T, 5, RPL, XP>(Xs, Vs, c0, lane, y); break;
                        case 6: dir_stage1_chunk<T, 6, RPL, XP>(Xs, Vs, c0, lane, y); break;
                        case 7: dir_stage1_chunk<T, 7, RPL, XP>(Xs, Vs, c0, lane, y); break;
                        default: dir_stage1_chunk<T, 8, RPL, XP>(Xs, Vs, c0, lane, y); break;
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                if (m < nm) {
#pragma unroll
                    for (int r = 0; r < RPL; ++r) Ys[(size_t)(jp0 + c0 + m) * XP + RPL * lane + r] = y[m][r];
                }
            }
            __syncthreads();  // the next pass reuses Xs and Vs; stage 2 reads Ys
        }
        // stage 2: phit += xi Ubar_t^T over the k_t columns of xi
        const T *Ut = Ub + md.x;  // [kcp][k_t8]
        for (int j0 = 0; j0 < md.z; j0 += BK) {
            if (j0) __syncthreads();  // previous chunk of Ubar_t consumed
            for (int e = tid; e < BN * BK; e += 256) {
                const int c = e / BK, kk = e % BK, gc = col0 + c;
                Us[(size_t)kk * (BN + 4) + c] = (gc < kcp && j0 + kk < md.w) ? Ut[(size_t)gc * md.w + j0 + kk] : T(0);
            }
            __syncthreads();
            if (live) {
                const int jn = min(BK, md.z - j0);
                // a full chunk unrolled; the last, partial one with an exact trip count
                auto step = [&](int kk) {
                    T xa[RPT], wb[TN];
#pragma unroll
                    for (int i = 0; i < RPT; ++i) xa[i] = Ys[(size_t)(j0 + kk) * XP + ty * RPT + i];
#pragma unroll
                    for (int j = 0; j < TN; ++j) wb[j] = Us[(size_t)kk * (BN + 4) + tx * TN + j];
#pragma unroll
                    for (int i = 0; i < RPT; ++i)
#pragma unroll
                        for (int j = 0; j < TN; ++j) a[i][j] = fma(xa[i], wb[j], a[i][j]);
                };
                if (jn == BK) {
#pragma unroll
                    for (int kk = 0; kk < BK; ++kk) step(kk);
                } else {
#pragma unroll 1
                    for (int kk = 0; kk < jn; ++kk) step(kk);
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        int r = ty * RPT + i;
        if (r >= tile.rows) continue;
        long long orow = L.row0 + (long long)tgt_b[r] * R + tgt_r[r];
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int c = col0 + tx * TN + j;
            if (c < kcp) phit[orow * kcp + c] = a[i][j];
        }
    }
}


template <class T, int TN>
static void launch_contract_tn(const LevelView *levels, const ContractTile *tiles, long long ntiles, const int *tvl,
                               const T *qt, const T *C, int kp, int kcp, long long zero_row, T *phit, cudaStream_t s) {
    dim3 grid((unsigned)ntiles, (unsigned)((kcp + 16 * TN - 1) / (16 * TN)));
    contract_simt_kernel<T, TN><<<grid, 256, 0, s>>>(levels, tiles, tvl, qt, C, kp, kcp, zero_row, phit);
}

template <class T>
int launch_contract_simt(const LevelView *levels, const ContractTile *tiles, long long ntiles, const int *tvl,
                         const T *qt, const T *C, int kp, int kcp, long long zero_row, T *phit, cudaStream_t s) {
    if (ntiles <= 0) return M2L_OK;
    // FP64: one block of up to 192 columns keeps the FP64 units fed from registers; FP32 keeps
    // more warps resident with narrower blocks
    const int tn = contract_tn(kcp, sizeof(T) == 8 ? 12 : 8);
    switch (tn) {
#define M2L_TN(n) \
    case n: launch_contract_tn<T, n>(levels, tiles, ntiles, tvl, qt, C, kp, kcp, zero_row, phit, s); break;
        M2L_TN(1) M2L_TN(2) M2L_TN(3) M2L_TN(4) M2L_TN(5) M2L_TN(6)
        M2L_TN(7) M2L_TN(8) M2L_TN(9) M2L_TN(10) M2L_TN(11) M2L_TN(12)
#undef M2L_TN
        default:
            set_error("contraction: no column tiling for k_pad = %d", kp);
            return M2L_EINVAL;
    }
    return check_launch("contract");
}

template <class T, int TN>
static int launch_contract_dir_tn(const LevelView *levels, const ContractTile *tiles, long long ntiles, const int *tvl,
                                  const T *qt, const T *Ub, const T *Vt, const int *meta, int k, int kp, int kcp,
                                  int kt8max, long long zero_row, T *phit, cudaStream_t s) {
    constexpr int BN = 16 * TN, BM = kDirTileRows<T>, XP = BM + 2;
    const size_t smem = sizeof(T) * ((size_t)kt8max * XP + (size_t)16 * XP + (size_t)16 * 66 + (size_t)16 * (BN + 4));
    if (smem > 200 * 1024) return M2L_EUNSUPPORTED;
    if (cudaFuncSetAttribute(contract_simt_dir_kernel<T, TN, BM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return M2L_EUNSUPPORTED;
    }
    dim3 grid((unsigned)ntiles, (unsigned)((kcp + BN - 1) / BN));
    contract_simt_dir_kernel<T, TN, BM><<<grid, 256, smem, s>>>(levels, tiles, tvl, qt, Ub, Vt,
                                                             reinterpret_cast<const int4 *>(meta), k, kp, kcp, kt8max,
                                                             zero_row, phit);
    return check_launch("contract_dir");
}

// Returns M2L_EUNSUPPORTED (nothing launched) when the shared-memory tiles do not fit; the caller
// then applies C_t unfactored.
template <class T>
int launch_contract_simt_dir(const LevelView *levels, const ContractTile *tiles, long long ntiles, const int *tvl,
                             const T *qt, const T *Ub, const T *Vt, const int *meta, int k, int kp, int kcp,
                             int kt8max, long long zero_row, T *phit, cudaStream_t s) {
    if (ntiles <= 0) return M2L_OK;
    const int tn = contract_tn(kcp, 12);  // one column block where possible: stage 1 is per block
    switch (tn) {
#define M2L_TN(n) \
    case n:                                                                                                    \
        return launch_contract_dir_tn<T, n>(levels, tiles, ntiles, tvl, qt, Ub, Vt, meta, k, kp, kcp, kt8max, zero_row, \
                                            phit, s);
        M2L_TN(1) M2L_TN(2) M2L_TN(3) M2L_TN(4) M2L_TN(5) M2L_TN(6)
        M2L_TN(7) M2L_TN(8) M2L_TN(9) M2L_TN(10) M2L_TN(11) M2L_TN(12)
#undef M2L_TN
        default:
            return M2L_EUNSUPPORTED;
    }
}

// ----------------------------------------------------------------------------------------------
// FFT form. Lattice entries are packed a << 16 | b << 8 | c. Spectra are stored per
// (cluster, rhs) as [8][F] complex: sibling-major, frequencies contiguous, so the lanes of a warp
// that take consecutive frequencies of one sibling read whole 128-byte lines (App. A.1 interleaves
// the siblings by frequency instead, which suits one CPU core walking all siblings of a frequency;
// on the GPU it made every 16-byte load touch four times the lines it used). A launch covers R
// right-hand sides; rows of the densities and check potentials are b * L.R + L.row0 + r, so a
// launch can take a chunk of the instance's right-hand sides, and spectra of cluster c sit at
// (L.cbase + c) * R + r.

__device__ inline uint32_t parent_linear(uint32_t xyz, int Np) {
    int x = (xyz & 1023) >> 1, y = ((xyz >> 10) & 1023) >> 1, z = ((xyz >> 20) & 1023) >> 1;
    return ((uint32_t)z * Np + y) * Np + x;
}
__device__ inline int octant_of(uint32_t xyz) {
    return (xyz & 1) | (((xyz >> 10) & 1) << 1) | (((xyz >> 20) & 1) << 2);
}

// Embed the n densities of one (box, rhs) on the g^3 grid (lattice points [0, p)^3) and take the
// real 3D DFT, pruned to the nonzero input cube: along z (real -> kz in [0, g/2]), then y, then x.
template <class T>
__global__ void __launch_bounds__(128) fft_forward_kernel(LevelView L, int R, int p, int n, int g,
                                                          const int *__restrict__ lattice,
                                                          const T *__restrict__ tw,
                                                          const T *__restrict__ q, T *__restrict__ qhat) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int H = g / 2 + 1, F = g * g * H;
    T *tws = reinterpret_cast<T *>(smem_raw);     // 2g
    T *xs = tws + 2 * g;                          // p^3
    T *Y1 = xs + p * p * p;                       // p*p*H complex
    T *Y2 = Y1 + 2 * p * p * H;                   // p*g*H complex
    const long long row = blockIdx.x + (long long)blockIdx.y * gridDim.x;
    if (row >= L.nboxes * R) return;
    const long long b = row / R;
    const int r = (int)(row % R);
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < 2 * g; i += nt) tws[i] = tw[i];
    for (int i = tid; i < p * p * p; i += nt) xs[i] = T(0);
    __syncthreads();
    const T *qrow = q + (b * L.R + L.row0 + r) * (long long)n;  // L.R: rhs stride, L.row0: first rhs
    for (int i = tid; i < n; i += nt) {
        int lat = lattice[i];
        int a = lat >> 16, bb = (lat >> 8) & 255, c = lat & 255;
        xs[(a * p + bb) * p + c] = qrow[i];
    }
    __syncthreads();
    for (int e = tid; e < p * p * H; e += nt) {
        int ab = e / H, kz = e % H;
        T re = 0, im = 0;
        int m = 0;
        for (int c = 0; c < p; ++c) {
            T v = xs[ab * p + c];
            re = fma(v, tws[2 * m], re);
            im = fma(v, tws[2 * m + 1], im);
            m += kz;
            if (m >= g) m -= g;
        }
        Y1[2 * e] = re;
        Y1[2 * e + 1] = im;
    }
    __syncthreads();
    for (int e = tid; e < p * g * H; e += nt) {
        int a = e / (g * H), ky = (e / H) % g, kz = e % H;
        T re = 0, im = 0;
        int m = 0;
        for (int bb = 0; bb < p; ++bb) {
            int o = ((a * p + bb) * H + kz) * 2;
            T xr = Y1[o], xi = Y1[o + 1], wr = tws[2 * m], wi = tws[2 * m + 1];
            re = fma(xr, wr, fma(-xi, wi, re));
            im = fma(xr, wi, fma(xi, wr, im));
            m += ky;
            if (m >= g) m -= g;
        }
        Y2[2 * e] = re;
        Y2[2 * e + 1] = im;
    }
    __syncthreads();
    const uint32_t xyz = L.xyz[b];
    const int oct = octant_of(xyz);
    const int cl = L.cslot[parent_linear(xyz, L.N / 2)];
    T *out = qhat + (((L.cbase + cl) * R + r) * 8 + oct) * (long long)F * 2;
    for (int f = tid; f < F; f += nt) {
        int kx = f / (g * H), ky = (f / H) % g, kz = f % H;
        T re = 0, im = 0;
        int m = 0;
        for (int a = 0; a < p; ++a) {
            int o = ((a * g + ky) * H + kz) * 2;
            T xr = Y2[o], xi = Y2[o + 1], wr = tws[2 * m], wi = tws[2 * m + 1];
            re = fma(xr, wr, fma(-xi, wi, re));
            im = fma(xr, wi, fma(xi, wr, im));
            m += kx;
            if (m >= g) m -= g;
        }
        out[2 * f] = re;
        out[2 * f + 1] = im;
    }
}

// The FP32 transforms specialised on (P, G): each thread owns whole lines of the pruned
// separable DFT and keeps them in registers; twiddles are read from c_twf at indices fixed at
// compile time (no index arithmetic or table lookups in the sums). One CTA of round_up(G H, 32)
// threads per (box, rhs).
template <int G>
__device__ __forceinline__ float2 twf(int m) {
    return c_twf[twiddle_offset(G) + m % G];
}
template <int P, int G>
constexpr int fft_pg_threads() {
    return ((G * (G / 2 + 1)) + 31) / 32 * 32;
}

// Forward: embed, then z (real -> kz in [0, H)), y, x; the x stage writes the spectrum.
template <int P, int G>
__global__ void __launch_bounds__(fft_pg_threads<P, G>()) fft_forward_pg_kernel(LevelView L, int R, int n,
                                                                                 const int *__restrict__ lattice,
                                                                                 const float *__restrict__ q,
                                                                                 float *__restrict__ qhat, int sib) {
    constexpr int H = G / 2 + 1, GH = G * H, F = G * GH;
    __shared__ float xs[P * P * P];
    __shared__ float2 Y1[P * P * H];  // [a][b][kz]
    __shared__ float2 Y2[P * GH];     // [a][ky][kz]
    const long long row = blockIdx.x + (long long)blockIdx.y * gridDim.x;
    if (row >= L.nboxes * R) return;
    const long long b = row / R;
    const int r = (int)(row % R), tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < P * P * P; i += nt) xs[i] = 0.f;
    __syncthreads();
    const float *qrow = q + (b * L.R + L.row0 + r) * (long long)n;
    for (int i = tid; i < n; i += nt) {
        const int lat = lattice[i];
        xs[((lat >> 16) * P + ((lat >> 8) & 255)) * P + (lat & 255)] = qrow[i];
    }
    __syncthreads();
    for (int e = tid; e < P * P; e += nt) {  // line (a, b) along z
        float x[P];
#pragma unroll
        for (int c = 0; c < P; ++c) x[c] = xs[e * P + c];
#pragma unroll
        for (int kz = 0; kz < H; ++kz) {
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int c = 0; c < P; ++c) {
                const float2 w = twf<G>(c * kz);
                re = fmaf(x[c], w.x, re);
                im = fmaf(x[c], w.y, im);
            }
            Y1[e * H + kz] = make_float2(re, im);
        }
    }
    __syncthreads();
    for (int e = tid; e < P * H; e += nt) {  // line (a, kz) along y
        const int a = e / H, kz = e % H;
        float2 y[P];
#pragma unroll
        for (int bb = 0; bb < P; ++bb) y[bb] = Y1[(a * P + bb) * H + kz];
#pragma unroll
        for (int ky = 0; ky < G; ++ky) {
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int bb = 0; bb < P; ++bb) {
                const float2 w = twf<G>(bb * ky);
                re = fmaf(y[bb].x, w.x, fmaf(-y[bb].y, w.y, re));
                im = fmaf(y[bb].x, w.y, fmaf(y[bb].y, w.x, im));
            }
            Y2[(a * G + ky) * H + kz] = make_float2(re, im);
        }
    }
    __syncthreads();
    const uint32_t xyz = L.xyz[b];
    const int cl = L.cslot[parent_linear(xyz, L.N / 2)];
    // spectrum row of the cluster: [8][F] (sibling-major), or [F][8] (sibling-minor, sib != 0)
    const int oct = octant_of(xyz);
    float2 *out = reinterpret_cast<float2 *>(qhat) + ((L.cbase + cl) * R + r) * 8 * (long long)F +
                  (sib ? (long long)oct : (long long)oct * F);
    const int fstride = sib ? 8 : 1;
    if (tid < GH) {  // line (ky, kz) along x, written for every kx
        float2 y[P];
#pragma unroll
        for (int a = 0; a < P; ++a) y[a] = Y2[a * GH + tid];
#pragma unroll
        for (int kx = 0; kx < G; ++kx) {
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int a = 0; a < P; ++a) {
                const float2 w = twf<G>(a * kx);
                re = fmaf(y[a].x, w.x, fmaf(-y[a].y, w.y, re));
                im = fmaf(y[a].x, w.y, fmaf(y[a].y, w.x, im));
            }
            out[(long long)(kx * GH + tid) * fstride] = make_float2(re, im);
        }
    }
}

// Inverse: x (read straight from the spectrum, one column per thread), y, then z at the lattice
// cube, scaled by 1 / G^3, and the surface points gathered from the cube.
template <int P, int G>
__global__ void __launch_bounds__(fft_pg_threads<P, G>()) fft_inverse_pg_kernel(LevelView L, int R, int n,
                                                                                 const int *__restrict__ lattice,
                                                                                 const float *__restrict__ phihat,
                                                                                 float *__restrict__ phi, long long ldphi,
                                                                                 int acc, int sib) {
    constexpr int H = G / 2 + 1, GH = G * H, F = G * GH;
    __shared__ float2 Z1[P * GH];     // [a][ky][kz]
    __shared__ float2 Z2[P * P * H];  // [a][b][kz]
    __shared__ float cube[P * P * P];
    const long long row = blockIdx.x + (long long)blockIdx.y * gridDim.x;
    if (row >= L.nboxes * R) return;
    const long long b = row / R;
    const int r = (int)(row % R), tid = threadIdx.x, nt = blockDim.x;
    const uint32_t xyz = L.xyz[b];
    const int cl = L.cslot[parent_linear(xyz, L.N / 2)];
    const int oct = octant_of(xyz), fstride = sib ? 8 : 1;
    const float2 *in = reinterpret_cast<const float2 *>(phihat) + ((L.cbase + cl) * R + r) * 8 * (long long)F +
                       (sib ? (long long)oct : (long long)oct * F);
    if (tid < GH) {  // column (ky, kz) along x, for a < P
        float2 x[G];
#pragma unroll
        for (int kx = 0; kx < G; ++kx) x[kx] = in[(long long)(kx * GH + tid) * fstride];
#pragma unroll
        for (int a = 0; a < P; ++a) {
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int kx = 0; kx < G; ++kx) {
                const float2 w = twf<G>(a * kx);  // times conj(w)
                re = fmaf(x[kx].x, w.x, fmaf(x[kx].y, w.y, re));
                im = fmaf(x[kx].y, w.x, fmaf(-x[kx].x, w.y, im));
            }
            Z1[a * GH + tid] = make_float2(re, im);
        }
    }
    __syncthreads();
    for (int e = tid; e < P * H; e += nt) {  // line (a, kz) along y, for b < P
        const int a = e / H, kz = e % H;
        float2 y[G];
#pragma unroll
        for (int ky = 0; ky < G; ++ky) y[ky] = Z1[(a * G + ky) * H + kz];
#pragma unroll
        for (int bb = 0; bb < P; ++bb) {
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int ky = 0; ky < G; ++ky) {
                const float2 w = twf<G>(bb * ky);
                re = fmaf(y[ky].x, w.x, fmaf(y[ky].y, w.y, re));
                im = fmaf(y[ky].y, w.x, fmaf(-y[ky].x, w.y, im));
            }
            Z2[(a * P + bb) * H + kz] = make_float2(re, im);
        }
    }
    __syncthreads();
    // along z, Hermitian: v(c) = Re Z2[0] + sum_{kz >= 1} wgt Re(Z2[kz] e^{+2 pi i c kz / G})
    constexpr float scale = 1.f / (float)(G * G * G);
    for (int e = tid; e < P * P; e += nt) {
        float2 z[H];
#pragma unroll
        for (int kz = 0; kz < H; ++kz) z[kz] = Z2[e * H + kz];
#pragma unroll
        for (int c = 0; c < P; ++c) {
            float v = z[0].x;
#pragma unroll
            for (int kz = 1; kz < H; ++kz) {
                const float wgt = (G % 2 == 0 && kz == H - 1) ? 1.f : 2.f;
                const float2 w = twf<G>(c * kz);
                v = fmaf(wgt, fmaf(z[kz].x, w.x, z[kz].y * w.y), v);
            }
            cube[e * P + c] = v * scale;
        }
    }
    __syncthreads();
    float *outrow = phi + (b * L.R + L.row0 + r) * ldphi;
    for (int i = tid; i < n; i += nt) {
        const int lat = lattice[i];
        float v = cube[((lat >> 16) * P + ((lat >> 8) & 255)) * P + (lat & 255)];
        if (acc) v += outrow[i];
        outrow[i] = v;
    }
}

// Launch the (P, G) specialisation for the FP32 transforms, if there is one; false otherwise.
template <int P, int G>
static void launch_pg(bool forward, const LevelView &L, int R, int n, const int *lattice, const float *in, float *out,
                      long long ldphi, int acc, int sib, dim3 grid, cudaStream_t s) {
    if (forward)
        fft_forward_pg_kernel<P, G><<<grid, fft_pg_threads<P, G>(), 0, s>>>(L, R, n, lattice, in, out, sib);
    else
        fft_inverse_pg_kernel<P, G><<<grid, fft_pg_threads<P, G>(), 0, s>>>(L, R, n, lattice, in, out, ldphi, acc, sib);
}
bool fft_pg_available(int p, int g) {
    switch (p * 100 + g) {
        case 407: case 408: case 611: case 612: case 815: case 816: case 1019: case 1020: return true;
        default: return false;
    }
}
static bool launch_fft_pg(bool forward, const LevelView &L, int R, int p, int n, int g, const int *lattice,
                          const float *in, float *out, long long ldphi, int acc, int sib, dim3 grid, cudaStream_t s) {
    switch (p * 100 + g) {
        case 407: launch_pg<4, 7>(forward, L, R, n, lattice, in, out, ldphi, acc, sib, grid, s); return true;
        case 408: launch_pg<4, 8>(forward, L, R, n, lattice, in, out, ldphi, acc, sib, grid, s); return true;
        case 611: launch_pg<6, 11>(forward, L, R, n, lattice, in, out, ldphi, acc, sib, grid, s); return true;
        case 612: launch_pg<6, 12>(forward, L, R, n, lattice, in, out, ldphi, acc, sib, grid, s); return true;
        case 815: launch_pg<8, 15>(forward, L, R, n, lattice, in, out, ldphi, acc, sib, grid, s); return true;
        case 816: launch_pg<8, 16>(forward, L, R, n, lattice, in, out, ldphi, acc, sib, grid, s); return true;
        case 1019: launch_pg<10, 19>(forward, L, R, n, lattice, in, out, ldphi, acc, sib, grid, s); return true;
        case 1020: launch_pg<10, 20>(forward, L, R, n, lattice, in, out, ldphi, acc, sib, grid, s); return true;
        default: return false;
    }
}

template <class T>
static size_t fft_forward_smem(int p, int g) {
    int H = g / 2 + 1;
    return sizeof(T) * (size_t)(2 * g + p * p * p + 2 * p * p * H + 2 * p * g * H);
}
template <class T>
static size_t fft_inverse_smem(int p, int g) {
    int H = g / 2 + 1;
    size_t F = (size_t)g * g * H;
    return sizeof(T) * (2 * g + 2 * F + 2 * (size_t)p * g * H);
}

template <class T>
int launch_fft_forward(const LevelView &L, int R, int p, int n, int g, const int *lattice, const T *tw,
                       const T *q, T *qhat, cudaStream_t s, bool sib_minor) {
    long long rows = L.nboxes * R;
    if (rows <= 0) return M2L_OK;
    unsigned gx = (unsigned)(rows < 65535 ? rows : 65535);
    unsigned gy = (unsigned)((rows + gx - 1) / gx);
    if constexpr (sizeof(T) == 4) {
        if (launch_fft_pg(true, L, R, p, n, g, lattice, (const float *)q, (float *)qhat, 0, 0, sib_minor ? 1 : 0,
                          dim3(gx, gy), s))
            return check_launch("fft_forward");
    }
    if (sib_minor) {
        set_error("sibling-minor spectra need the FP32 transforms specialised on (p, g) = (%d, %d)", p, g);
        return M2L_EUNSUPPORTED;
    }
    size_t smem = fft_forward_smem<T>(p, g);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(fft_forward_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    fft_forward_kernel<T><<<dim3(gx, gy), 128, smem, s>>>(L, R, p, n, g, lattice, tw, q, qhat);
    return check_launch("fft_forward");
}

// F3: for each target cluster, rhs and frequency, sum over the 26 source clusters the 8 x 8
// complex products phihat[i] += Khat_{t(d,i,j)} qhat[j] (App. A.1, Hadamard component), skipping
// adjacent pairs. The kernel spectra of a block of FB frequencies sit in shared memory; FB complex
// values make one 128-byte line, so the FB lanes that share an item read one line per sibling.
// The frequency block is blockIdx.y: the CTAs resident at one time work on one or two frequency
// blocks.
template <class T>
struct Complex2;
template <>
struct Complex2<float> {
    using type = float2;
};
template <>
struct Complex2<double> {
    using type = double2;
};

// A thread owns one frequency of IB consecutive items (target cluster, rhs): each kernel value it
// reads from shared memory serves IB products, and the IB source loads of a direction are in
// flight together.
template <class T, int FB, int IB>
__global__ void __launch_bounds__(256) hadamard_kernel(LevelView L, int R, int F, const T *__restrict__ Khat,
                                                       const T *__restrict__ qhat, T *__restrict__ phihat) {
    using C2 = typename Complex2<T>::type;
    __shared__ C2 Ks[kNumTransfer * FB];
    const int f0 = blockIdx.y * FB;
    for (int e = threadIdx.x; e < kNumTransfer * FB; e += blockDim.x) {
        const int ti = e / FB, f = f0 + e % FB;
        C2 k;
        k.x = f < F ? Khat[((long long)ti * F + f) * 2] : T(0);
        k.y = f < F ? Khat[((long long)ti * F + f) * 2 + 1] : T(0);
        Ks[e] = k;
    }
    __syncthreads();
    constexpr int TC = 256 / FB;
    const int fl = threadIdx.x % FB, tcl = threadIdx.x / FB;
    const int f = f0 + fl;
    if (f >= F) return;
    const int Np = L.N / 2;
    const long long items = L.nclusters * R;
    const C2 *q2 = reinterpret_cast<const C2 *>(qhat);
    C2 *o2 = reinterpret_cast<C2 *>(phihat);
    for (long long it0 = ((long long)blockIdx.x * TC + tcl) * IB; it0 < items; it0 += (long long)gridDim.x * TC * IB) {
        long long row[IB];  // (cluster, rhs) block of the item, -1 past the end
        int px[IB], py[IB], pz[IB], rr[IB];
#pragma unroll
        for (int b = 0; b < IB; ++b) {
            const long long it = it0 + b;
            row[b] = -1;
            px[b] = py[b] = pz[b] = rr[b] = 0;
            if (it < items) {
                const long long tc = L.cperm[it / R];
                rr[b] = (int)(it % R);
                row[b] = (L.cbase + tc) * R + rr[b];
                const uint32_t pc = L.cxyz[tc];
                px[b] = pc & 1023;
                py[b] = (pc >> 10) & 1023;
                pz[b] = (pc >> 20) & 1023;
            }
        }
        T ar[IB][8], ai[IB][8];
#pragma unroll
        for (int b = 0; b < IB; ++b)
#pragma unroll
            for (int i = 0; i < 8; ++i) ar[b][i] = ai[b][i] = T(0);
        for (int d = 0; d < kDirections; ++d) {
            C2 q[IB][8];
            bool any = false;
#pragma unroll
            for (int b = 0; b < IB; ++b) {
                const int sx = px[b] + c_dir[d][0], sy = py[b] + c_dir[d][1], sz = pz[b] + c_dir[d][2];
                int sc = -1;
                if (row[b] >= 0 && sx >= 0 && sy >= 0 && sz >= 0 && sx < Np && sy < Np && sz < Np)
                    sc = L.cslot[((long long)sz * Np + sy) * Np + sx];
                const C2 *qs = q2 + ((L.cbase + (sc < 0 ? 0 : sc)) * R + rr[b]) * (long long)F * 8 + f;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (sc >= 0) {
                        q[b][j] = qs[(long long)j * F];
                    } else {
                        q[b][j].x = T(0);
                        q[b][j].y = T(0);
                    }
                }
                any |= sc >= 0;
            }
            if (!any) continue;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int ti = c_clu[d][8 * i + j];
                    if (ti >= 0) {
                        const C2 k = Ks[ti * FB + fl];
#pragma unroll
                        for (int b = 0; b < IB; ++b) {
                            ar[b][i] = fma(k.x, q[b][j].x, fma(-k.y, q[b][j].y, ar[b][i]));
                            ai[b][i] = fma(k.x, q[b][j].y, fma(k.y, q[b][j].x, ai[b][i]));
                        }
                    }
                }
        }
#pragma unroll
        for (int b = 0; b < IB; ++b) {
            if (row[b] < 0) continue;
            C2 *out = o2 + row[b] * (long long)F * 8 + f;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                C2 v;
                v.x = ar[b][i];
                v.y = ai[b][i];
                out[(long long)i * F] = v;
            }
        }
    }
}

// F3 in FP32 on dense levels. The kernel spectra of a block of 16 frequencies sit in shared
// memory on the 7 x 7 x 7 grid of transfer vectors t in [-3,3]^3, with zeros at the 27 adjacent
// offsets |t| <= 1. The transfer vector of target sibling i and source sibling j in direction d is
// t = 2 d + j - i (App. A.1), so its grid index is a per-direction base plus an offset fixed by
// (i, j): with i and j unrolled, every kernel value is one shared load at an immediate offset,
// with no table lookup, index arithmetic or branch. The 152 adjacent products of the 26 x 64
// (App. A.2's "~10%") are multiplied by those zeros rather than skipped. The source sibling j is
// the outer loop, so each loaded source value feeds 8 targets, and each kernel value serves the
// IB items (target cluster, rhs) of the thread.
template <int IB>
__global__ void __launch_bounds__(256, 2) hadamard_grid_kernel(LevelView L, int R, int F, const float *__restrict__ Khat,
                                                               const float *__restrict__ qhat, float *__restrict__ phihat) {
    constexpr int FB = 16, TC = 256 / FB, NI = TC * IB;
    __shared__ float2 Ks[343 * FB];
    __shared__ int s_src[NI][kDirections];  // source row (cluster * R + rhs) of each item and direction, -1: none
    __shared__ int s_dst[NI];                // target row of each item, -1: past the end
    __shared__ int s_mask[NI];               // directions with a source, one bit each
    const int f0 = blockIdx.y * FB;
    for (int e = threadIdx.x; e < 343 * FB; e += blockDim.x) {
        const int g3 = e / FB, f = f0 + e % FB;
        const int ti = c_tidx[g3 / 49][(g3 / 7) % 7][g3 % 7];
        float2 k = make_float2(0.f, 0.f);
        if (ti >= 0 && f < F) {
            k.x = Khat[((long long)ti * F + f) * 2];
            k.y = Khat[((long long)ti * F + f) * 2 + 1];
        }
        Ks[e] = k;
    }
    const int fl = threadIdx.x % FB, tcl = threadIdx.x / FB;
    const int f = f0 + fl;
    const bool fvalid = f < F;  // threads past F still take part in the block's barriers
    const int Np = L.N / 2;
    const long long items = L.nclusters * R;
    const long long F8 = (long long)F * 8;
    const float2 *q2 = reinterpret_cast<const float2 *>(qhat) + (fvalid ? f : 0);
    float2 *o2 = reinterpret_cast<float2 *>(phihat) + f;
    const float2 *kf = Ks + fl;
    for (long long base = (long long)blockIdx.x * NI; base < items; base += (long long)gridDim.x * NI) {
        __syncthreads();  // the spectra block is in place, and the previous group's tables are consumed
        for (int e = threadIdx.x; e < NI * kDirections; e += blockDim.x) {
            const int li = e / kDirections, d = e % kDirections;
            const long long it = base + li;
            int src = -1;
            if (it < items) {
                const long long tc = L.cperm[it / R];
                const int r = (int)(it % R);
                const uint32_t pc = L.cxyz[tc];
                const int sx = (int)(pc & 1023) + c_dir[d][0], sy = (int)((pc >> 10) & 1023) + c_dir[d][1],
                          sz = (int)((pc >> 20) & 1023) + c_dir[d][2];
                if (sx >= 0 && sy >= 0 && sz >= 0 && sx < Np && sy < Np && sz < Np) {
                    const int sc = L.cslot[((long long)sz * Np + sy) * Np + sx];
                    if (sc >= 0) src = (int)((L.cbase + sc) * R + r);
                }
                if (d == 0) s_dst[li] = (int)((L.cbase + tc) * R + r);
            } else if (d == 0) {
                s_dst[li] = -1;
            }
            s_src[li][d] = src;
        }
        __syncthreads();
        if (threadIdx.x < NI) {
            int m = 0;
            for (int d = 0; d < kDirections; ++d) m |= (s_src[threadIdx.x][d] >= 0) << d;
            s_mask[threadIdx.x] = m;
        }
        __syncthreads();
        int mask = 0;
#pragma unroll
        for (int b = 0; b < IB; ++b) mask |= s_mask[tcl * IB + b];
        float ar[IB][8], ai[IB][8];
#pragma unroll
        for (int b = 0; b < IB; ++b)
#pragma unroll
            for (int i = 0; i < 8; ++i) ar[b][i] = ai[b][i] = 0.f;
        int srow[IB];
        float2 qn[IB];
        if (mask) {
            const int d0 = __ffs(mask) - 1;
#pragma unroll
            for (int b = 0; b < IB; ++b) {
                srow[b] = s_src[tcl * IB + b][d0];
                qn[b] = srow[b] >= 0 ? q2[srow[b] * F8] : make_float2(0.f, 0.f);
            }
        }
        while (mask) {
            const int d = __ffs(mask) - 1;
            mask &= mask - 1;
            const int dn = mask ? __ffs(mask) - 1 : -1;  // the next direction with a source
            int snext[IB];
#pragma unroll
            for (int b = 0; b < IB; ++b) snext[b] = dn >= 0 ? s_src[tcl * IB + b][dn] : -1;
            const int dx = c_dir[d][0], dy = c_dir[d][1], dz = c_dir[d][2];
            // grid index of t = 2 d + j - i: base of j = 0, i = 0, plus (j offset) - (i offset)
            const float2 *kd = kf + ((2 * dx + 3) * 49 + (2 * dy + 3) * 7 + (2 * dz + 3)) * FB;
#pragma unroll 1
            for (int j = 0; j < 8; ++j) {
                float2 q[IB];
#pragma unroll
                for (int b = 0; b < IB; ++b) q[b] = qn[b];
                // the values of the next sibling, or of the next direction's first, are in flight
                // while these are used
#pragma unroll
                for (int b = 0; b < IB; ++b) {
                    const int sr = j < 7 ? srow[b] : snext[b];
                    const long long off = j < 7 ? (long long)(j + 1) * F : 0;
                    qn[b] = sr >= 0 ? q2[sr * F8 + off] : make_float2(0.f, 0.f);
                }
                const float2 *kj = kd + ((j & 1) * 49 + ((j >> 1) & 1) * 7 + ((j >> 2) & 1)) * FB;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float2 k = kj[-((i & 1) * 49 + ((i >> 1) & 1) * 7 + ((i >> 2) & 1)) * FB];
#pragma unroll
                    for (int b = 0; b < IB; ++b) {
                        ar[b][i] = fmaf(k.x, q[b].x, fmaf(-k.y, q[b].y, ar[b][i]));
                        ai[b][i] = fmaf(k.x, q[b].y, fmaf(k.y, q[b].x, ai[b][i]));
                    }
                }
            }
#pragma unroll
            for (int b = 0; b < IB; ++b) srow[b] = snext[b];
        }
        if (fvalid) {
#pragma unroll
            for (int b = 0; b < IB; ++b) {
                const int dst = s_dst[tcl * IB + b];
                if (dst < 0) continue;
                float2 *out = o2 + dst * F8;
#pragma unroll
                for (int i = 0; i < 8; ++i) out[(long long)i * F] = make_float2(ar[b][i], ai[b][i]);
            }
        }
    }
}

// F3 with one warp per (target cluster, block of RB right-hand sides) and one lane per frequency
// of a block of 32. Directions, source clusters and child masks are the same across the warp, so
// the missing children of sparse sets (about half of them on a surface) are skipped without
// divergence, the eight sibling spectra of a source load as one coalesced 2 KB row per warp, and
// each kernel spectrum value read from shared memory serves RB right-hand sides.
template <class T, int RB>
__global__ void __launch_bounds__(256) hadamard_warp_kernel(LevelView L, int R, int F, const T *__restrict__ Khat,
                                                            const T *__restrict__ qhat, T *__restrict__ phihat) {
    constexpr int FB = 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Ks = reinterpret_cast<T *>(smem_raw);  // [316][FB] complex
    const int f0 = blockIdx.y * FB;
    for (int e = threadIdx.x; e < kNumTransfer * FB; e += blockDim.x) {
        const int ti = e / FB, f = f0 + e % FB;
        T re = 0, im = 0;
        if (f < F) {
            re = Khat[((long long)ti * F + f) * 2];
            im = Khat[((long long)ti * F + f) * 2 + 1];
        }
        Ks[2 * e] = re;
        Ks[2 * e + 1] = im;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int f = f0 + lane;
    const bool fvalid = f < F;
    const int Np = L.N / 2;
    const int nrb = (R + RB - 1) / RB;
    const long long items = L.nclusters * nrb;
    for (long long item = (long long)blockIdx.x * 8 + warp; item < items; item += (long long)gridDim.x * 8) {
        const long long tc = item / nrb;
        const int r0 = (int)(item % nrb) * RB;
        const uint32_t pc = L.cxyz[tc];
        const int px = pc & 1023, py = (pc >> 10) & 1023, pz = (pc >> 20) & 1023;
        int tmask = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) tmask |= (L.cchild[tc * 8 + i] >= 0) << i;
        T ar[RB][8], ai[RB][8];
#pragma unroll
        for (int rr = 0; rr < RB; ++rr)
#pragma unroll
            for (int i = 0; i < 8; ++i) ar[rr][i] = ai[rr][i] = T(0);
        for (int d = 0; d < kDirections; ++d) {
            const int sx = px + c_dir[d][0], sy = py + c_dir[d][1], sz = pz + c_dir[d][2];
            if (sx < 0 || sy < 0 || sz < 0 || sx >= Np || sy >= Np || sz >= Np) continue;
            const int sc = L.cslot[((long long)sz * Np + sy) * Np + sx];
            if (sc < 0) continue;
            int smask = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) smask |= (L.cchild[(long long)sc * 8 + j] >= 0) << j;
            T qr[RB][8], qi[RB][8];
#pragma unroll
            for (int rr = 0; rr < RB; ++rr) {
                const bool ok = fvalid && r0 + rr < R;
                const T *qs = qhat + ((L.cbase + sc) * R + r0 + rr) * (long long)F * 16 + 2 * f;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    qr[rr][j] = ok ? qs[(long long)j * F * 2] : T(0);
                    qi[rr][j] = ok ? qs[(long long)j * F * 2 + 1] : T(0);
                }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (!((tmask >> i) & 1)) continue;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (!((smask >> j) & 1)) continue;
                    const int ti = c_clu[d][8 * i + j];
                    if (ti < 0) continue;
                    const T kr = Ks[(ti * FB + lane) * 2], ki = Ks[(ti * FB + lane) * 2 + 1];
#pragma unroll
                    for (int rr = 0; rr < RB; ++rr) {
                        ar[rr][i] = fma(kr, qr[rr][j], fma(-ki, qi[rr][j], ar[rr][i]));
                        ai[rr][i] = fma(kr, qi[rr][j], fma(ki, qr[rr][j], ai[rr][i]));
                    }
                }
            }
        }
        if (fvalid) {
#pragma unroll
            for (int rr = 0; rr < RB; ++rr) {
                if (r0 + rr >= R) continue;
                T *out = phihat + ((L.cbase + tc) * R + r0 + rr) * (long long)F * 16 + 2 * f;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    out[(long long)i * F * 2] = ar[rr][i];
                    out[(long long)i * F * 2 + 1] = ai[rr][i];
                }
            }
        }
    }
}

template <class T, int RB>
static int launch_hadamard_warp(const LevelView &L, int R, int F, const T *Khat, const T *qhat, T *phihat,
                                cudaStream_t s) {
    constexpr int FB = 32;
    const long long items = L.nclusters * ((R + RB - 1) / RB);
    const size_t smem = sizeof(T) * 2 * (size_t)kNumTransfer * FB;
    cudaFuncSetAttribute(hadamard_warp_kernel<T, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const unsigned gy = (unsigned)((F + FB - 1) / FB);
    // up to 8 items per warp, fewer when a level is too small to fill four waves of CTAs
    const long long ipw = std::max(1LL, std::min(8LL, items * (long long)gy / (4LL * sm_count() * 8)));
    long long gx = (items + 8 * ipw - 1) / (8 * ipw);
    if (gx < 1) gx = 1;
    if (gx > (1LL << 30)) gx = 1LL << 30;
    hadamard_warp_kernel<T, RB><<<dim3((unsigned)gx, gy), 256, smem, s>>>(L, R, F, Khat, qhat, phihat);
    return check_launch("hadamard");
}

// Resident CTAs of hadamard_kernel on the device (occupancy query, cached on first use).
template <class T>
static int hadamard_resident() {
    constexpr int FB = 128 / (2 * (int)sizeof(T)), IB = sizeof(T) == 4 ? 2 : 1;
    static int resident = 0;
    if (!resident) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hadamard_kernel<T, FB, IB>, 256, 0) != cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        resident = per_sm * sm_count();
    }
    return resident;
}

constexpr int kGridIB = 4;  // items per thread of hadamard_grid_kernel

static int hadamard_grid_resident() {
    static int resident = 0;
    if (!resident) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hadamard_grid_kernel<kGridIB>, 256, 0) != cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        resident = per_sm * sm_count();
    }
    return resident;
}

static void cache_launch_shapes() {
    hadamard_resident<float>();
    hadamard_resident<double>();
    hadamard_grid_resident();
}

// Item groups per thread for a launch of `groups` item groups over gy frequency blocks: every CTA
// does ipt iterations, so the launch takes about ceil(CTAs / resident) x ipt iteration times; the
// ipt in 1..16 that makes this smallest (a partial last wave costs as much as a full one), the
// larger on ties (fewer CTAs load the spectra block).
static long long items_per_thread(long long groups, long long gy, int resident) {
    long long ipt = 1, best = -1;
    for (long long c = 1; c <= 16; ++c) {
        const long long ctas = (groups + c - 1) / c * gy;
        const long long cost = (ctas + resident - 1) / resident * c;
        if (best < 0 || cost <= best) {
            best = cost;
            ipt = c;
        }
    }
    return ipt;
}

static int launch_hadamard_grid(const LevelView &L, int R, int F, const float *Khat, const float *qhat, float *phihat,
                                cudaStream_t s) {
    constexpr int FB = 16, TC = 256 / FB;
    const long long items = L.nclusters * R;
    const unsigned gy = (unsigned)((F + FB - 1) / FB);
    const long long groups = (items + TC * kGridIB - 1) / (TC * kGridIB);
    const long long ipt = items_per_thread(groups, gy, hadamard_grid_resident());
    long long gx = (groups + ipt - 1) / ipt;
    if (gx < 1) gx = 1;
    if (gx > (1LL << 30)) gx = 1LL << 30;
    hadamard_grid_kernel<kGridIB><<<dim3((unsigned)gx, gy), 256, 0, s>>>(L, R, F, Khat, qhat, phihat);
    return check_launch("hadamard");
}

template <class T>
int launch_hadamard(const LevelView &L, int R, int F, const T *Khat, const T *qhat, T *phihat, cudaStream_t s) {
    constexpr int FB = 128 / (2 * (int)sizeof(T)), TC = 256 / FB;  // one 128-byte line of complex values
    long long items = L.nclusters * R;
    if (items <= 0) return M2L_OK;
    // The warp-per-cluster kernel skips missing children and reuses each kernel value for two
    // right-hand sides; on full levels with one right-hand side it has nothing to skip and its
    // larger spectra block halves the resident warps (measured 4.4 ms against 7.8 ms on the
    // 1M-point workload, 52 ms against 98 ms on the sphere surface with 32 right-hand sides).
    const bool sparse = L.nboxes * 4 < L.nclusters * 8 * 3;  // fewer than 6 of 8 children on average
    if constexpr (sizeof(T) == 4) {
        // FP32 on dense levels: spectra on the transfer-vector grid, four items per thread (the
        // consecutive right-hand sides of a cluster when R > 1)
        if (!sparse) return launch_hadamard_grid(L, R, F, Khat, qhat, phihat, s);
    }
    if (R >= 2) return launch_hadamard_warp<T, 2>(L, R, F, Khat, qhat, phihat, s);
    if (sparse) return launch_hadamard_warp<T, 1>(L, R, F, Khat, qhat, phihat, s);
    // FP32 takes two items per thread (its shared-memory loads, not its FMAs, were the limit);
    // FP64 is bound by the FP64 units and keeps one
    constexpr int IB = sizeof(T) == 4 ? 2 : 1;
    const unsigned gy = (unsigned)((F + FB - 1) / FB);
    // Item groups per thread (ipt): the CTAs of a launch all do ipt iterations, so the launch takes
    // about ceil(CTAs / resident CTAs) x ipt iteration times; take the ipt in 1..16 that makes
    // this smallest (a partial last wave costs as much as a full one), the larger ipt on ties
    // (fewer CTAs load the spectra block).
    const int resident = hadamard_resident<T>();
    long long ipt = 1, best = -1;
    for (long long c = 1; c <= 16; ++c) {
        const long long ctas = (items + TC * IB * c - 1) / (TC * IB * c) * (long long)gy;
        const long long cost = (ctas + resident - 1) / resident * c;
        if (best < 0 || cost <= best) {
            best = cost;
            ipt = c;
        }
    }
    long long gx = (items + TC * IB * ipt - 1) / (TC * IB * ipt);
    if (gx < 1) gx = 1;
    if (gx > (1LL << 30)) gx = 1LL << 30;
    hadamard_kernel<T, FB, IB><<<dim3((unsigned)gx, gy), 256, 0, s>>>(L, R, F, Khat, qhat, phihat);
    return check_launch("hadamard");
}

// F4 + F5: inverse DFT of one (box, rhs) spectrum, evaluated only at the surface points of the
// lattice cube [0, p)^3 (along x, then y, then the Hermitian half along z), scaled by 1/g^3.
template <class T>
__global__ void __launch_bounds__(128) fft_inverse_kernel(LevelView L, int R, int p, int n, int g,
                                                          const int *__restrict__ lattice,
                                                          const T *__restrict__ tw,
                                                          const T *__restrict__ phihat, T *__restrict__ phi,
                                                          long long ldphi, int acc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int H = g / 2 + 1, F = g * g * H;
    T *tws = reinterpret_cast<T *>(smem_raw);  // 2g
    T *X = tws + 2 * g;                        // F complex; reused for Z2 (p*p*H complex)
    T *Z1 = X + 2 * F;                         // p*g*H complex
    const long long row = blockIdx.x + (long long)blockIdx.y * gridDim.x;
    if (row >= L.nboxes * R) return;
    const long long b = row / R;
    const int r = (int)(row % R);
    const int tid = threadIdx.x, nt = blockDim.x;
    const uint32_t xyz = L.xyz[b];
    const int oct = octant_of(xyz);
    const int cl = L.cslot[parent_linear(xyz, L.N / 2)];
    const T *in = phihat + (((L.cbase + cl) * R + r) * 8 + oct) * (long long)F * 2;
    for (int i = tid; i < 2 * g; i += nt) tws[i] = tw[i];
    for (int f = tid; f < F; f += nt) {
        X[2 * f] = in[2 * f];
        X[2 * f + 1] = in[2 * f + 1];
    }
    __syncthreads();
    // along x: Z1[a][ky][kz] = sum_kx X[kx][ky][kz] conj(w^(a kx)), a < p
    for (int e = tid; e < p * g * H; e += nt) {
        int a = e / (g * H), kykz = e % (g * H);
        T re = 0, im = 0;
        int m = 0;
        for (int kx = 0; kx < g; ++kx) {
            int o = (kx * g * H + kykz) * 2;
            T xr = X[o], xi = X[o + 1], wr = tws[2 * m], wi = -tws[2 * m + 1];
            re = fma(xr, wr, fma(-xi, wi, re));
            im = fma(xr, wi, fma(xi, wr, im));
            m += a;
            if (m >= g) m -= g;
        }
        Z1[2 * e] = re;
        Z1[2 * e + 1] = im;
    }
    __syncthreads();
    // along y: Z2[a][b][kz] = sum_ky Z1[a][ky][kz] conj(w^(b ky)), b < p  (stored over X)
    T *Z2 = X;
    for (int e = tid; e < p * p * H; e += nt) {
        int a = e / (p * H), bb = (e / H) % p, kz = e % H;
        T re = 0, im = 0;
        int m = 0;
        for (int ky = 0; ky < g; ++ky) {
            int o = ((a * g + ky) * H + kz) * 2;
            T xr = Z1[o], xi = Z1[o + 1], wr = tws[2 * m], wi = -tws[2 * m + 1];
            re = fma(xr, wr, fma(-xi, wi, re));
            im = fma(xr, wi, fma(xi, wr, im));
            m += bb;
            if (m >= g) m -= g;
        }
        Z2[2 * e] = re;
        Z2[2 * e + 1] = im;
    }
    __syncthreads();
    // along z (Hermitian): out = Re Z2[0] + sum_{kz>=1} w_kz Re(Z2[kz] conj(w^(c kz))), at surface points
    const T scale = T(1) / (T)((long long)g * g * g);
    const bool even = (g % 2) == 0;
    T *outrow = phi + (b * L.R + L.row0 + r) * ldphi;
    for (int i = tid; i < n; i += nt) {
        int lat = lattice[i];
        int a = lat >> 16, bb = (lat >> 8) & 255, c = lat & 255;
        const T *z = Z2 + ((a * p + bb) * H) * 2;
        T v = z[0];
        int m = c;
        for (int kz = 1; kz < H; ++kz) {
            T wgt = (even && kz == H - 1) ? T(1) : T(2);
            // Re(Z2[kz] e^{+2 pi i c kz / g}); tws holds e^{-2 pi i m / g}
            v = fma(wgt, fma(z[2 * kz], tws[2 * m], z[2 * kz + 1] * tws[2 * m + 1]), v);
            m += c;
            if (m >= g) m -= g;
        }
        v *= scale;
        if (acc) v += outrow[i];
        outrow[i] = v;
    }
}

template <class T>
int launch_fft_inverse(const LevelView &L, int R, int p, int n, int g, const int *lattice, const T *tw,
                       const T *phihat, T *phi, long long ldphi, int acc, cudaStream_t s, bool sib_minor) {
    long long rows = L.nboxes * R;
    if (rows <= 0) return M2L_OK;
    unsigned gx = (unsigned)(rows < 65535 ? rows : 65535);
    unsigned gy = (unsigned)((rows + gx - 1) / gx);
    if constexpr (sizeof(T) == 4) {
        if (launch_fft_pg(false, L, R, p, n, g, lattice, (const float *)phihat, (float *)phi, ldphi, acc,
                          sib_minor ? 1 : 0, dim3(gx, gy), s))
            return check_launch("fft_inverse");
    }
    if (sib_minor) {
        set_error("sibling-minor spectra need the FP32 transforms specialised on (p, g) = (%d, %d)", p, g);
        return M2L_EUNSUPPORTED;
    }
    size_t smem = fft_inverse_smem<T>(p, g);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(fft_inverse_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    fft_inverse_kernel<T><<<dim3(gx, gy), 128, smem, s>>>(L, R, p, n, g, lattice, tw, phihat, phi, ldphi, acc);
    return check_launch("fft_inverse");
}

size_t fft_smem_bytes(int p, int g, int elt) {
    size_t a = elt == 8 ? fft_forward_smem<double>(p, g) : fft_forward_smem<float>(p, g);
    size_t b = elt == 8 ? fft_inverse_smem<double>(p, g) : fft_inverse_smem<float>(p, g);
    return a > b ? a : b;
}

#define M2L_INSTANTIATE(T)                                                                              \
    template int launch_gemm_xwt<T>(const T *, long long, const T *, long long, T *, long long, long long, \
                                    int, int, int, cudaStream_t);                                       \
    template int launch_contract_simt_dir<T>(const LevelView *, const ContractTile *, long long, const int *,   \
                                             const T *, const T *, const T *, const int *, int, int, int, int,  \
                                             long long, T *, cudaStream_t);                                  \
    template int launch_contract_simt<T>(const LevelView *, const ContractTile *, long long, const int *,       \
                                         const T *, const T *, int, int, long long, T *, cudaStream_t); \
    template int launch_fft_forward<T>(const LevelView &, int, int, int, int, const int *, const T *,   \
                                       const T *, T *, cudaStream_t, bool);                             \
    template int launch_hadamard<T>(const LevelView &, int, int, const T *, const T *, T *, cudaStream_t); \
    template int launch_fft_inverse<T>(const LevelView &, int, int, int, int, const int *, const T *,   \
                                       const T *, T *, long long, int, cudaStream_t, bool);
M2L_INSTANTIATE(double)
M2L_INSTANTIATE(float)

}  // namespace m2l
