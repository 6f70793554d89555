// F6, the pseudo-inverse's two factors (Eq. 9, stored apart as the footnote of Sec. 2.1.1
// recommends), on the tensor cores, exactly: Z = Ut_eps phi, then locals = V_eps Z (+ locals).
//
// The V_eps product must be carried beyond FP32: the locals are measured through the check
// potential they reproduce, which FP32 accumulation error over the r terms roughly doubles (the
// CUDA-core path uses a float-float sum). Here both operands are cut into integer slices, so
// every tensor-core product and every partial sum is an exact integer in FP32 (the error-free
// splitting of Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59, 2012):
//   a row x of X (K values) is scaled by 2^-e_x (e_x: the exponent of its largest entry, so
//   |x| 2^-e_x < 1) and written as sum_s q_s 2^-beta(s+1), s = 0..3, with integers |q_0| <= 2^beta
//   and |q_s| <= 2^(beta-1) after it (round to nearest, each slice the rounded residual of the
//   previous); a row w of W likewise with 2^e_w and integers p_t.
// Then x.w = 2^(e_x + e_w) sum_{s,t} 2^-beta(s+t+2) (q_s . p_t). Every q_s . p_t is an integer of
// magnitude at most 2^(2 beta) K, exact in the FP32 accumulator whatever its rounding while that
// is at most 2^24 (beta = 8: K <= 256, the V_eps product over the rank r; beta = 7: K <= 1024,
// the Ut_eps product over the n check points); the products on the same diagonal s + t share an
// accumulator (exactness matters on the leading diagonal, which holds one pair). Slices are BF16
// (integers of up to 9 bits exactly); the 10 pairs with s + t <= 3 are kept, which reproduces the
// float-float V_eps product's result to rounding (host emulation over p = 6, 8, 10: the locals'
// check-norm error equal to three digits).
//
// Tiles of 128 rows x 64 outputs, K in stages of 64 (128-byte swizzled rows, TMA); per stage the
// 4 K steps x 10 slice pairs are 40 MMAs (M = 128, N = 64, K = 16, BF16) into 4 diagonal
// accumulators, double-buffered in tensor memory across tiles. Warps: 0-3 epilogue (the four
// diagonals added in FP32 from the smallest, scaled by the row and column exponents), 4 TMA, 5 MMA
// issue (warp-uniform, elected lane). Every wait is bounded; an expired wait records where in the
// plan's device status word and the CTA winds down.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "kernels.cuh"
#include "tcgen05.cuh"

namespace m2l {

namespace {

using namespace tc;

constexpr int kSl = 4;                          // slices per operand
constexpr int kRowsP = 128;                     // M
constexpr int kNP = 64;                         // outputs per tile (N)
constexpr int kKS = 64;                         // K per stage: one 128-byte row of BF16
constexpr int kStagesP = 2;
constexpr int kThreadsP = 192;
constexpr uint32_t kASlice = kRowsP * 128;      // 16 KB: one slice of a stage's A
constexpr uint32_t kBSlice = kNP * 128;         // 8 KB
constexpr uint32_t kStageP = kSl * (kASlice + kBSlice);
constexpr uint32_t kSmemP = kStagesP * kStageP;
constexpr int kDiag = 4;                        // accumulators: s + t = 0..3
constexpr uint32_t kBufCols = kDiag * kNP;      // 256 columns per tile; two tiles in flight

struct PtcParams {
    const int *zexp;         // [rows_pad] exponents of the X rows
    const float *vscale;     // [O_pad] 2^e_w of the W rows
    float *out;              // [rows][ldo]
    long long rows, ldo;
    int O, nk;               // outputs; K stages (K_pad / 64)
    long long mtiles, ntiles;
    int acc;
    int *status;
    uint32_t idesc;
    float d1, d2, d3;        // 2^-beta, 2^-2 beta, 2^-3 beta: the diagonals' weights
    int eshift;              // 2 beta
};

// One BF16 slice pair (s, t) of the 10 with s + t <= 3, diagonal-major.
__host__ __device__ constexpr int pair_s(int j) { return j == 0 ? 0 : j < 3 ? j - 1 : j < 6 ? j - 3 : j - 6; }
__host__ __device__ constexpr int pair_d(int j) { return j == 0 ? 0 : j < 3 ? 1 : j < 6 ? 2 : 3; }

// Shared-memory descriptor of a K-major operand in the 128-byte swizzle (8-row groups 1024 B apart).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// X rows -> 4 BF16 integer slices of beta bits [4][rows_pad][K_pad] and exponents (one warp per
// row; rows past `rows` and columns past K are zeros).
__global__ void slice_rows_kernel(const float *__restrict__ Z, long long ldz, long long rows, long long rows_pad, int K,
                                  int Kp, int beta, __nv_bfloat16 *__restrict__ Zs, int *__restrict__ zexp) {
    const float sc = (float)(1 << beta);
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long row = wid; row < rows_pad; row += nw) {
        const bool live = row < rows;
        float mx = 0.f;
        if (live)
            for (int k = lane; k < K; k += 32) mx = fmaxf(mx, fabsf(Z[row * ldz + k]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        int e = 0;
        if (mx > 0.f) frexpf(mx, &e);  // mx < 2^e
        if (lane == 0) zexp[row] = e;
        for (int k = lane; k < Kp; k += 32) {
            float R = (live && k < K) ? ldexpf(Z[row * ldz + k], -e) : 0.f;  // |R| < 1
#pragma unroll
            for (int s = 0; s < kSl; ++s) {
                const float t = R * sc;     // exact
                const float q = rintf(t);
                R = t - q;                  // exact, |R| <= 1/2
                Zs[((long long)s * rows_pad + row) * Kp + k] = __float2bfloat16_rn(q);  // |q| <= 2^beta: exact
            }
        }
    }
}

__global__ void __launch_bounds__(kThreadsP, 1)
    pinv_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const PtcParams P,
                   long long rows_pad, int opad) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kStagesP], empty_bar[kStagesP], accf_bar[2], acce_bar[2], drain_bar;
    __shared__ uint32_t tmem_base_s;
    __shared__ volatile int abort_flag;
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t s0 = smem_u32(smem);
    auto sA = [&](int st, int s) { return s0 + (uint32_t)st * kStageP + (uint32_t)s * kASlice; };
    auto sB = [&](int st, int t) { return s0 + (uint32_t)st * kStageP + kSl * kASlice + (uint32_t)t * kBSlice; };
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long total = P.mtiles * P.ntiles;
    if (tid == 0) {
        for (int i = 0; i < kStagesP; ++i) {
            mbar_init(smem_u32(&full_bar[i]), 1);
            mbar_init(smem_u32(&empty_bar[i]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&accf_bar[b]), 1);
            mbar_init(smem_u32(&acce_bar[b]), 128);
        }
        mbar_init(smem_u32(&drain_bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(2 * kBufCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_s;

    if (warp == 4) {
        // ---------------- TMA: the 4 Z slices and 4 V slices of each K stage ----------------
        if (lane == 0) {
            long long it = 0;
            for (long long tile = blockIdx.x; tile < total && !abort_flag; tile += gridDim.x) {
                const long long mt = tile / P.ntiles, nt = tile % P.ntiles;
                for (int kc = 0; kc < P.nk; ++kc, ++it) {
                    const int st = (int)(it % kStagesP);
                    if (it >= kStagesP && !mbar_wait(smem_u32(&empty_bar[st]), (uint32_t)(((it / kStagesP) - 1) & 1),
                                                     &abort_flag, P.status, M2L_WAIT_TMA))
                        goto tma_done;
                    const uint32_t bar = smem_u32(&full_bar[st]);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kStageP) : "memory");
                    for (int s = 0; s < kSl; ++s) {
                        const int x = kc * kKS, y = (int)(s * rows_pad + mt * kRowsP);
                        asm volatile(
                            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                                sA(st, s)),
                            "l"(&tmA), "r"(x), "r"(y), "r"(bar)
                            : "memory");
                    }
                    for (int t = 0; t < kSl; ++t) {
                        const int x = kc * kKS, y = (int)(t * opad + nt * kNP);
                        asm volatile(
                            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                                sB(st, t)),
                            "l"(&tmB), "r"(x), "r"(y), "r"(bar)
                            : "memory");
                    }
                }
            }
        tma_done:
            if (abort_flag) {
                // let loads already issued land before the CTA leaves
                for (int st = 0; st < kStagesP && st < it; ++st) {
                    const long long last = it - 1 - (((it - 1 - st) % kStagesP) + kStagesP) % kStagesP;
                    const uint32_t parity = (uint32_t)((last / kStagesP) & 1);
                    for (long long w = 0; w < kWaitLimit && !mbar_try(smem_u32(&full_bar[st]), parity); ++w) {
                    }
                }
            }
        }
    } else if (warp == 5) {
        // ---------------- MMA issue: warp-uniform, one elected lane ----------------
        long long it = 0, u = 0;
        bool pending = false;
        for (long long tile = blockIdx.x; tile < total && !abort_flag; tile += gridDim.x, ++u) {
            const int buf = (int)(u & 1);
            if (u >= 2 && !mbar_wait(smem_u32(&acce_bar[buf]), (uint32_t)(((u >> 1) - 1) & 1), &abort_flag, P.status,
                                     M2L_WAIT_ACC_FREE))
                goto mma_done;
            const uint32_t d0 = tmem + (uint32_t)buf * kBufCols;
            for (int kc = 0; kc < P.nk; ++kc, ++it) {
                const int st = (int)(it % kStagesP);
                if (!mbar_wait(smem_u32(&full_bar[st]), (uint32_t)((it / kStagesP) & 1), &abort_flag, P.status,
                               M2L_WAIT_OPERANDS))
                    goto mma_done;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (elect_one()) {
#pragma unroll
                    for (int k = 0; k < kKS / 16; ++k)
#pragma unroll
                        for (int j = 0; j < 10; ++j) {
                            const int s = pair_s(j), dg = pair_d(j), t = dg - s;
                            const bool first = kc == 0 && k == 0 && (j == 0 || j == 1 || j == 3 || j == 6);
                            mma<1>(d0 + (uint32_t)(dg * kNP), desc_sw128(sA(st, s) + 32 * k), desc_sw128(sB(st, t) + 32 * k),
                                   P.idesc, first ? 0u : 1u);
                        }
                    mma_commit(smem_u32(&empty_bar[st]));
                }
                __syncwarp();
            }
            if (elect_one()) mma_commit(smem_u32(&accf_bar[buf]));
            __syncwarp();
            pending = true;
        }
    mma_done:
        __syncwarp();
        if (abort_flag && pending) {
            // no MMA may still write tensor memory when it is released
            if (elect_one()) mma_commit(smem_u32(&drain_bar));
            __syncwarp();
            for (long long w = 0; w < kWaitLimit && !mbar_try(smem_u32(&drain_bar), 0); ++w) {
            }
        }
    } else {
        // ---------------- epilogue: out = 2^(e_x + e_w - 2 beta) sum_d D_d 2^-beta d ----------------
        const int quarter = warp & 3;
        const int rl = quarter * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        long long u = 0;
        for (long long tile = blockIdx.x; tile < total && !abort_flag; tile += gridDim.x, ++u) {
            const long long mt = tile / P.ntiles, nt = tile % P.ntiles;
            const int buf = (int)(u & 1);
            if (!mbar_wait(smem_u32(&accf_bar[buf]), (uint32_t)((u >> 1) & 1), &abort_flag, P.status, M2L_WAIT_ACC_READY))
                goto epi_done;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const long long r = mt * kRowsP + rl;
            const bool live = r < P.rows;
            const int ez = live ? P.zexp[r] : 0;
            float *orow = P.out + r * P.ldo;
            for (int cg = 0; cg < kNP / 16; ++cg) {
                uint32_t v[kDiag][16];
#pragma unroll
                for (int dg = 0; dg < kDiag; ++dg)
                    tmem_ld16(tmem + lane_off + (uint32_t)buf * kBufCols + (uint32_t)(dg * kNP + cg * 16), v[dg]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (!live) continue;
                const int c0 = (int)nt * kNP + cg * 16;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = c0 + 4 * q;
                    if (c >= P.O) break;
                    float y[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int j = 4 * q + i;
                        // the diagonals from the smallest; every D is an exact integer
                        float a = fmaf(__uint_as_float(v[3][j]), P.d3, __uint_as_float(v[2][j]) * P.d2);
                        a = fmaf(__uint_as_float(v[1][j]), P.d1, a);
                        a = __fadd_rn(__uint_as_float(v[0][j]), a);
                        y[i] = ldexpf(a, ez - P.eshift) * P.vscale[c + i];
                    }
                    float4 *o = reinterpret_cast<float4 *>(orow + c);
                    if (P.acc) {
                        const float4 old = *o;
                        y[0] += old.x;
                        y[1] += old.y;
                        y[2] += old.z;
                        y[3] += old.w;
                    }
                    *o = make_float4(y[0], y[1], y[2], y[3]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(smem_u32(&acce_bar[buf]));
        }
    epi_done:;
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 5) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kBufCols));
    }
}

}  // namespace


// Largest K_pad for which the leading diagonal's sums (at most 2^(2 beta) K) stay exact in FP32.
static int max_kp(int beta) { return 1 << (24 - 2 * beta); }

// W (FP64, O x K, row-major) as 4 BF16 integer slices of beta bits [4][O_pad][K_pad] with its row
// scales 2^e_w, and the TMA map of the slices (box 64 x 64, 128-byte swizzle). op.kp stays 0 when
// K_pad is past max_kp(beta).
int build_sliced_operand(const std::vector<double> &W, int O, int K, int beta, SlicedOp &op) {
    if (op.sl) return M2L_OK;
    const int Kp = (K + kKS - 1) / kKS * kKS;
    if (K < 1 || Kp > max_kp(beta)) return M2L_OK;
    const int opad = (O + kNP - 1) / kNP * kNP;
    const double sc = std::ldexp(1.0, beta);
    std::vector<uint16_t> sl((size_t)kSl * opad * Kp, 0);
    std::vector<float> scale(opad, 1.f);
    for (int o = 0; o < O; ++o) {
        double mx = 0;
        for (int k = 0; k < K; ++k) mx = std::max(mx, std::fabs(W[(size_t)o * K + k]));
        int e = 0;
        if (mx > 0) std::frexp(mx, &e);  // mx < 2^e
        scale[o] = std::ldexp(1.0f, e);
        for (int k = 0; k < K; ++k) {
            double R = std::ldexp(W[(size_t)o * K + k], -e);
            for (int s = 0; s < kSl; ++s) {
                const double t = R * sc;
                const double q = std::nearbyint(t);
                R = t - q;
                sl[((size_t)s * opad + o) * Kp + k] = bf16_round((float)q);  // an integer of at most beta + 1 bits
            }
        }
    }
    if (cudaMalloc(&op.sl, sl.size() * 2) != cudaSuccess || cudaMalloc(&op.scale, scale.size() * 4) != cudaSuccess) {
        cudaGetLastError();
        set_error("allocating a sliced operand failed");
        return M2L_ENOMEM;
    }
    cudaMemcpy(op.sl, sl.data(), sl.size() * 2, cudaMemcpyHostToDevice);
    cudaMemcpy(op.scale, scale.data(), scale.size() * 4, cudaMemcpyHostToDevice);
    EncodeTiledFn enc = encode_fn();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return M2L_ECUDA;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)kSl * opad};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kKS, (cuuint32_t)kNP};
    const cuuint32_t estr[2] = {1, 1};
    CUresult rc = enc(reinterpret_cast<CUtensorMap *>(op.map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, op.sl, dims, strides, box,
                      estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (rc != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)rc);
        return M2L_ECUDA;
    }
    op.kp = Kp;
    op.K = K;
    op.O = O;
    op.opad = opad;
    op.beta = beta;
    return M2L_OK;
}

// F6's two factors for the TF32x3 FFT form: Ut_eps (r x n) in slices of 7 bits (K = n up to 1024),
// V_eps (n x r) in slices of 8 bits (K = r up to 256); the product with a factor is taken on the
// tensor cores when its slices exist.
int build_pinv_tc_operand(m2l_plan_t *pl, DevOps &D) {
    // Ut_eps padded with zero rows to r_pad: the product writes every column of Z's rows (the
    // CUDA-core V_eps product, where that one is taken, reads them all)
    std::vector<double> ut((size_t)pl->rp * pl->n, 0.0);
    std::copy(pl->pinv->Uteps32.begin(), pl->pinv->Uteps32.begin() + (size_t)pl->r32 * pl->n, ut.begin());
    int rc = build_sliced_operand(ut, pl->rp, pl->n, 7, D.Us);
    if (rc) return rc;
    return build_sliced_operand(pl->pinv->Veps32, pl->n, pl->r32, 8, D.Vs);
}

// B1 and B3 of the split BLAS forms as sliced products: S^T (k_pad x n, zero rows past k) and
// U (n_c x k_c) in 7-bit slices, A = Ut_eps U (padded to r_pad rows) in 7-bit slices, V_eps as
// for the FFT form. Each product is taken on the tensor cores when its slices exist.
int build_blas_sliced_operands(m2l_plan_t *pl, DevOps &D) {
    const BlasOps &B = *pl->blas;
    const int n = pl->n, k = pl->k, kp = pl->kp, kc = pl->kc, nc = pl->nc;
    std::vector<double> st((size_t)kp * n, 0.0);
    for (int c = 0; c < k; ++c)
        for (int i = 0; i < n; ++i) st[(size_t)c * n + i] = B.S[(size_t)i * k + c];
    int rc = build_sliced_operand(st, kp, n, 7, D.Ss);
    if (rc) return rc;
    if ((rc = build_sliced_operand(B.U, nc, kc, 7, D.Ucs))) return rc;
    std::vector<double> a((size_t)pl->rp * kc, 0.0);
    std::copy(B.Aop32.begin(), B.Aop32.begin() + (size_t)pl->r32 * kc, a.begin());
    if ((rc = build_sliced_operand(a, pl->rp, kc, 7, D.As))) return rc;
    return build_sliced_operand(pl->pinv->Veps32, pl->n, pl->r32, 8, D.Vs);
}

// Largest K_pad any sliced product of a plan takes (workspace sizing).
int sliced_kmax(const m2l_plan_t *pl) {
    auto up = [](int v) { return (v + kKS - 1) / kKS * kKS; };
    return std::max(std::max(up(pl->n), up(pl->kc)), up(pl->r32));
}

// Workspace of launch_sliced for `rows` rows of K_pad: the X slices, then the row exponents.
size_t sliced_workspace(long long rows, int Kp) {
    const long long rows_pad = (rows + kRowsP - 1) / kRowsP * kRowsP;
    return (((size_t)kSl * rows_pad * Kp * 2 + 255) / 256) * 256 + (size_t)rows_pad * 4;
}

bool sliced_usable(const SlicedOp &W, long long ldo, int O, const float *out) {
    return W.sl && W.kp > 0 && O <= W.opad && ldo % 4 == 0 && O % 4 == 0 && ((uintptr_t)out & 15) == 0;
}

int launch_sliced(const m2l_plan_t *pl, const SlicedOp &W, const float *X, long long ldx, long long rows, float *out,
                  long long ldo, int O, int acc, void *ws, cudaStream_t s) {
    if (rows <= 0) return M2L_OK;
    if (!sliced_usable(W, ldo, O, out)) {
        set_error("sliced tensor-core product: operand or output layout not supported");
        return M2L_EUNSUPPORTED;
    }
    const int Kp = W.kp, beta = W.beta;
    const long long rows_pad = (rows + kRowsP - 1) / kRowsP * kRowsP;
    __nv_bfloat16 *Xs = (__nv_bfloat16 *)ws;
    int *xexp = (int *)((char *)ws + (((size_t)kSl * rows_pad * Kp * 2 + 255) / 256) * 256);
    {
        long long blocks = (rows_pad + 7) / 8;  // 8 warps per block, a warp per row
        if (blocks > 65535) blocks = 65535;
        slice_rows_kernel<<<(unsigned)blocks, 256, 0, s>>>(X, ldx, rows, rows_pad, W.K, Kp, beta, Xs, xexp);
    }
    EncodeTiledFn enc = encode_fn();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return M2L_ECUDA;
    }
    alignas(64) CUtensorMap tmA;
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)(kSl * rows_pad)};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kKS, (cuuint32_t)kRowsP};
    const cuuint32_t estr[2] = {1, 1};
    CUresult rc = enc(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Xs, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (rc != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)rc);
        return M2L_ECUDA;
    }
    PtcParams P;
    P.zexp = xexp;
    P.vscale = (const float *)W.scale;
    P.out = out;
    P.rows = rows;
    P.ldo = ldo;
    P.O = O;
    P.nk = Kp / kKS;
    P.mtiles = rows_pad / kRowsP;
    P.ntiles = (O + kNP - 1) / kNP;
    P.acc = acc;
    P.status = pl->dev_status;
    P.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kNP >> 3) << 17) | ((uint32_t)(kRowsP >> 4) << 24);
    P.d1 = std::ldexp(1.0f, -beta);
    P.d2 = std::ldexp(1.0f, -2 * beta);
    P.d3 = std::ldexp(1.0f, -3 * beta);
    P.eshift = 2 * beta;
    const long long total = P.mtiles * P.ntiles;
    const int grid = (int)(total < pl->num_sms ? total : pl->num_sms);
    const size_t smem = kSmemP + 1024;
    cudaFuncSetAttribute(pinv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    pinv_tc_kernel<<<grid, kThreadsP, smem, s>>>(tmA, *reinterpret_cast<const CUtensorMap *>(W.map), P, rows_pad, W.opad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("sliced tensor-core product launch failed: %s", cudaGetErrorString(e));
        return M2L_ECUDA;
    }
    return M2L_OK;
}

}  // namespace m2l
