// F3 (App. A.1 step 4, the Hadamard products of the FFT form) on the 5th-generation tensor cores,
// as split BF16 products accurate to FP32 rounding, for full levels (the FFT form's TF32x3
// precision class: FP32 data, tensor-core products of FP32 accuracy).
//
// At one frequency f the products of a target cluster are
//   phihat_i = sum over the 26 source-cluster directions d of sum_j Khat_{t(d,i,j)}(f) qhat_j(d),
// t = 2 d + j - i (target sibling i, source sibling j; App. A.1). In real arithmetic each direction
// is a 16 x 16 matrix B_d(f) (rows: Re/Im of the 8 targets, columns: Re/Im of the 8 sources)
// applied to a 16-vector, and the same matrix serves every target cluster of the level
// (translation invariance). With 128 target clusters as the rows of one MMA (M = 128), the source
// rows of direction d are those clusters' neighbours in direction d.
//
// A tile is 8 x 16 target clusters of one z plane. Its sources lie in a 10 x 18 halo of each of
// the planes z - 1, z, z + 1. A halo plane sits in shared memory as K-major core matrices whose
// 8 rows are 8 consecutive x and whose 8-row groups are the 18 y lines; the 128 source rows of
// direction (dx, dy, dz) are then the window of plane z + dz shifted by (dx, dy): one operand
// descriptor (start offset, LBO, SBO), with no copy. Each halo plane is loaded once and serves
// the 8 or 9 directions of each of the three tiles (z - 1, z, z + 1) that read it: a CTA sweeps
// the planes of a (frequency, rhs, x block, y block) column in z through a ring of 7 planes.
// Halo clusters outside the domain are zeros.
//
// Split products: q = q_hi + q_mid + q_lo and B = B_hi + B_mid + B_lo, BF16 pieces each the
// nearest to what the previous ones leave (three cover an FP32 significand exactly); the six
// products with piece orders summing to at most 2 are kept (the dropped ones lie 2^-24 and
// further below), with FP32 accumulation in tensor memory. A direction (K = 16, one BF16 MMA
// step) takes three MMAs: q_hi x [B_hi; B_mid; B_lo] (N = 48), q_mid x [B_hi; B_mid] (N = 32) into
// columns 16-47, q_lo x B_hi (N = 16) into columns 32-47, so columns 0-15 hold the leading
// products and 16-31, 32-47 those 2^-8 and 2^-16 below. The tensor cores accumulate by
// truncation, so an error of up to an ulp of the running sum enters at every MMA into it; the 26
// directions are therefore split into chains (default 4, each led by an in-plane direction,
// present in every tile) with accumulators of their own, and the epilogue adds the chains'
// leading parts, then their small parts, with round-to-nearest.
//
// Warps: 0-3 load halo planes (16-byte cp.async of (cluster, frequency, sibling pair) from
// sibling-minor spectra into a staging slot) and split them into the ring's BF16 pieces; 4 loads
// the 26 kernel matrices of a frequency (one 39 KB bulk copy) when the column's frequency
// changes; 5 owns tensor memory and issues the MMAs (accumulators double-buffered across tiles);
// 6-9 read the accumulators and write phihat. Every wait is bounded; a wait that runs out records
// where in the plan's device status word, and the CTA winds down.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cstring>
#include <utility>
#include <vector>

#include "internal.h"
#include "kernels.cuh"
#include "tcgen05.cuh"

namespace m2l {

namespace {

using namespace tc;

constexpr int kThreadsH = 320;
constexpr int kTX = 8, kTY = 16;              // tile: 8 x 16 target clusters of one plane (M = 128)
constexpr int kHX = kTX + 2, kHY = kTY + 2;   // halo of one plane: 10 x 18 clusters
constexpr int kHRows = kHX * kHY;             // 180
constexpr int kPieces = 4 * kHRows;           // 16-byte pieces of a loaded plane (4 per halo row)
constexpr uint32_t kSBO = kHX * 16;           // 160: between y lines (8-row groups)
constexpr uint32_t kLBO = kHY * kSBO;         // 2880: between 16-byte K chunks
constexpr uint32_t kPieceB = 2 * kLBO;        // 5760: one plane, one BF16 piece (16 values a row)
constexpr uint32_t kPlaneB = 3 * kPieceB;     // hi, mid, lo
constexpr uint32_t kStageRow = 64;            // a halo row as loaded: 8 complex FP32 values
constexpr uint32_t kStageB = kHRows * kStageRow;
constexpr int kStageSlots = 3;                // loaded planes awaiting their split
constexpr int kRing = 7;                      // halo planes in shared memory
constexpr int kBBuf = 1;                      // kernel-matrix buffers (one frequency each)
constexpr uint32_t kBDir = 1536;              // one direction: [2 K chunks][6 row groups][8 rows][16 B]
constexpr uint32_t kBLBO = 768, kBSBO = 128;
constexpr uint32_t kBFreq = 26 * kBDir;       // the 26 matrices of one frequency
constexpr uint32_t kSmemH = kRing * kPlaneB + kStageSlots * kStageB + kBBuf * kBFreq;
constexpr int kMaxChains = 4;                 // two buffers x 4 chains x 64 columns = 512

struct HtcParams {
    const float *qhat;       // [(cluster R + rhs)][F][8] complex, sibling-minor
    float *phihat;           // same layout
    const unsigned char *B;  // [F][26][kBDir]: the shared-memory image of each frequency's matrices
    int Np, R, F, XB, YB;
    long long ncols;         // F R XB YB columns, frequency slowest
    int *status;
    uint32_t idesc48, idesc32, idesc16;
};

// The 26 source-cluster directions d in [-1,1]^3 \ {0} are indexed x slowest (di = 0..25). NCH
// chains of directions: chain c holds the in-plane (dz = 0) directions j = c, c + NCH, ... of the
// 8, then the others j = c, c + NCH, ... of the 18, so that every chain starts with a direction
// whose source plane is the tile's own (present in every tile).
__host__ __device__ constexpr int nth_dir(bool in_plane, int j) {
    int cnt = 0;
    for (int di = 0; di < 26; ++di) {
        const int id = di + (di >= 13 ? 1 : 0);
        if ((id % 3 == 1) == in_plane) {
            if (cnt == j) return di;
            ++cnt;
        }
    }
    return -1;
}
struct Slot {
    int di, chain, first;
};
template <int NCH>
__host__ __device__ constexpr Slot slot_of(int k) {
    int idx = 0;
    for (int c = 0; c < NCH; ++c) {
        int pos = 0;
        for (int j = c; j < 8; j += NCH, ++pos, ++idx)
            if (idx == k) return Slot{nth_dir(true, j), c, pos == 0};
        for (int j = c; j < 18; j += NCH, ++pos, ++idx)
            if (idx == k) return Slot{nth_dir(false, j), c, pos == 0};
    }
    return Slot{-1, 0, 0};
}

__device__ __forceinline__ void column_of(const HtcParams &P, long long c, int &f, int &r, int &xb, int &yb) {
    xb = (int)(c % P.XB);
    c /= P.XB;
    yb = (int)(c % P.YB);
    c /= P.YB;
    r = (int)(c % P.R);
    f = (int)(c / P.R);
}

// Cluster of grid point (x, y, z) of a full level: clusters are numbered in Morton order of their
// keys (x in the lowest bit of each triple), and a full level holds all of them.
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
    v &= 0x3FF;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__device__ __forceinline__ long long morton3(int x, int y, int z) {
    return (long long)(spread3((uint32_t)x) | spread3((uint32_t)y) << 1 | spread3((uint32_t)z) << 2);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo_half, float hi_half) {
    const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(lo_half));
    const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(hi_half));
    return a | b << 16;
}

// The plane loaded into staging slot `stage` -> ring slot `plane` as three BF16 pieces
// q = q_hi + q_mid + q_lo (each the nearest BF16 of the remainder; exact: 8 + 8 + 8 bits cover
// an FP32 significand), for the 16-byte pieces this thread loaded (its own cp.async have landed).
__device__ __forceinline__ void split_plane(uint32_t stage, uint32_t plane, int tid) {
    for (int e = tid; e < kPieces; e += 128) {
        const int row = e >> 2, kq = e & 3;
        const int hy = row / kHX, hx = row - hy * kHX;
        float v[4];
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                     : "r"(stage + (uint32_t)row * kStageRow + (uint32_t)kq * 16)
                     : "memory");
        float h[4], m[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            h[i] = __bfloat162float(__float2bfloat16_rn(v[i]));
            const float r1 = v[i] - h[i];
            m[i] = __bfloat162float(__float2bfloat16_rn(r1));
            l[i] = r1 - m[i];
        }
        // values 4 kq .. 4 kq + 3 of the row: half of 16-byte K chunk kq / 2
        const uint32_t a = plane + (uint32_t)(kq >> 1) * kLBO + (uint32_t)hy * kSBO + (uint32_t)hx * 16 + (uint32_t)(kq & 1) * 8;
        asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a), "r"(pack_bf16(h[0], h[1])), "r"(pack_bf16(h[2], h[3]))
                     : "memory");
        asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a + kPieceB), "r"(pack_bf16(m[0], m[1])), "r"(pack_bf16(m[2], m[3]))
                     : "memory");
        asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a + 2 * kPieceB), "r"(pack_bf16(l[0], l[1])),
                     "r"(pack_bf16(l[2], l[3]))
                     : "memory");
    }
}

// The three MMAs of slot K of a tile (one direction, chain order; K = 16, the whole direction),
// all operands warp-uniform: q_hi x [B_hi; B_mid; B_lo] (N = 48), q_mid x [B_hi; B_mid] (N = 32)
// into columns 16-47, q_lo x B_hi (N = 16) into columns 32-47 of the chain: columns 0-15 gather
// the leading products, 16-31 those 2^-8 below, 32-47 those 2^-16 below.
// pdm, pd0, pdp: descriptors of the planes z - 1, z, z + 1 (0 outside the domain).
template <int NCH, int K>
__device__ __forceinline__ void issue_slot(uint32_t dtile, uint64_t pdm, uint64_t pd0, uint64_t pdp, uint64_t bdesc,
                                           uint32_t idesc48, uint32_t idesc32, uint32_t idesc16) {
    constexpr Slot sl = slot_of<NCH>(K);
    static_assert(sl.di >= 0, "direction slot");
    constexpr int id = sl.di + (sl.di >= 13 ? 1 : 0);
    constexpr int dx = id / 9 - 1, dy = (id / 3) % 3 - 1, dz = id % 3 - 1;
    constexpr uint32_t aoff = (uint32_t)((dy + 1) * (int)(kSBO / 16) + (dx + 1));  // 16-byte units
    constexpr uint32_t boff = (uint32_t)sl.di * (kBDir / 16);
    constexpr uint32_t kP = kPieceB / 16;  // next piece
    const uint64_t base = dz < 0 ? pdm : (dz == 0 ? pd0 : pdp);
    if (dz != 0 && base == 0) return;  // the source plane lies outside the domain
    const uint64_t a = base + aoff, b = bdesc + boff;
    const uint32_t d = dtile + 64u * (uint32_t)sl.chain;
    mma<1>(d, a, b, idesc48, sl.first ? 0u : 1u);
    mma<1>(d + 16, a + kP, b, idesc32, 1);
    mma<1>(d + 32, a + 2 * kP, b, idesc16, 1);
}
template <int NCH, int... K>
__device__ __forceinline__ void issue_tile(std::integer_sequence<int, K...>, uint32_t dtile, uint64_t pdm, uint64_t pd0,
                                           uint64_t pdp, uint64_t bdesc, uint32_t idesc48, uint32_t idesc32,
                                           uint32_t idesc16) {
    (issue_slot<NCH, K>(dtile, pdm, pd0, pdp, bdesc, idesc48, idesc32, idesc16), ...);
}

template <int NCH>
__global__ void __launch_bounds__(kThreadsH, 1) hadamard_tc_kernel(const HtcParams P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kRing], empty_bar[kRing], accf_bar[2], acce_bar[2], bfull_bar[kBBuf], bempty_bar[kBBuf],
        drain_bar;
    __shared__ uint32_t tmem_base_s;
    __shared__ volatile int abort_flag;

    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    const uint32_t s_planes = smem_u32(smem);
    const uint32_t s_stage = s_planes + kRing * kPlaneB;
    const uint32_t s_B = s_stage + kStageSlots * kStageB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Np = P.Np;
    constexpr uint32_t bufcols = 64u * NCH;                  // one tile's accumulators (48 used per chain)
    constexpr uint32_t tmem_cols = 2 * bufcols;              // two tiles' (a power of two)
    // columns dealt round-robin: the CTAs resident at one time work on consecutive columns, i.e.
    // the same few frequencies of neighbouring tiles, so halo rows shared by neighbouring tiles
    // meet in L2 and the spectra rows read at one time lie close together in memory
    const long long c0 = blockIdx.x, cstep = gridDim.x;
    if (tid == 0) {
        for (int i = 0; i < kRing; ++i) {
            mbar_init(smem_u32(&full_bar[i]), 128);
            mbar_init(smem_u32(&empty_bar[i]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&accf_bar[b]), 1);
            mbar_init(smem_u32(&acce_bar[b]), 128);
        }
        for (int b = 0; b < kBBuf; ++b) {
            mbar_init(smem_u32(&bfull_bar[b]), 1);
            mbar_init(smem_u32(&bempty_bar[b]), 1);
        }
        mbar_init(smem_u32(&drain_bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_s;

    if (warp < 4) {
        // ---------------- halo planes: load plane ps into staging, then split plane ps - 2 ----------
        // into its ring slot (the MMAs that free that slot, of plane ps - 2 - kRing, need planes up to
        // ps - kRing only, all split before)
        long long ps = 0;
        // split loaded plane q (its copies landed) into ring slot q mod kRing, once that slot is free
        auto finish = [&](long long q) -> bool {
            const int slot = (int)(q % kRing);
            if (q >= kRing && !mbar_wait(smem_u32(&empty_bar[slot]), (uint32_t)(((q / kRing) - 1) & 1), &abort_flag,
                                         P.status, M2L_WAIT_GATHER))
                return false;
            split_plane(s_stage + (uint32_t)(q % kStageSlots) * kStageB, s_planes + (uint32_t)slot * kPlaneB, tid);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(smem_u32(&full_bar[slot]));
            return true;
        };
        for (long long c = c0; c < P.ncols && !abort_flag; c += cstep) {
            int f, r, xb, yb;
            column_of(P, c, f, r, xb, yb);
            const int x0 = xb * kTX - 1, y0 = yb * kTY - 1;
            for (int z = 0; z < Np; ++z, ++ps) {
                const uint32_t stage = s_stage + (uint32_t)(ps % kStageSlots) * kStageB;
                for (int e = tid; e < kPieces; e += 128) {
                    const int row = e >> 2, kq = e & 3;
                    const int hy = row / kHX, hx = row - hy * kHX;
                    const int x = x0 + hx, y = y0 + hy;
                    const uint32_t dst = stage + (uint32_t)row * kStageRow + (uint32_t)kq * 16;
                    if (x >= 0 && y >= 0 && x < Np && y < Np) {
                        const long long cl = morton3(x, y, z);
                        const float *src = P.qhat + (((long long)cl * P.R + r) * P.F + f) * 16 + kq * 4;
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
                    } else {
                        asm volatile("st.shared.v4.b32 [%0], {%1, %1, %1, %1};" ::"r"(dst), "r"(0u) : "memory");
                    }
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
                if (ps >= 2) {
                    // every copy but the two newest groups (planes ps, ps - 1) has landed
                    asm volatile("cp.async.wait_group 2;" ::: "memory");
                    if (!finish(ps - 2)) goto producer_done;
                }
            }
        }
        if (!abort_flag) {
            if (ps >= 2) {
                asm volatile("cp.async.wait_group 1;" ::: "memory");
                if (!finish(ps - 2)) goto producer_done;
            }
            if (ps >= 1) {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
                finish(ps - 1);
            }
        }
    producer_done:
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp == 4) {
        // ---------------- kernel matrices of the column's frequency ----------------
        if (lane == 0) {
            // load j (the j-th distinct frequency of this CTA's columns) goes to buffer j mod kBBuf
            int nb = 0, fprev = -1;
            for (long long c = c0; c < P.ncols && !abort_flag; c += cstep) {
                int f, r, xb, yb;
                column_of(P, c, f, r, xb, yb);
                if (f == fprev) continue;
                const int b = nb % kBBuf;
                if (nb >= kBBuf && !mbar_wait(smem_u32(&bempty_bar[b]), (uint32_t)(((nb / kBBuf) - 1) & 1), &abort_flag,
                                              P.status, M2L_WAIT_TMA))
                    break;
                const uint32_t bar = smem_u32(&bfull_bar[b]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kBFreq) : "memory");
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                 s_B + (uint32_t)b * kBFreq),
                             "l"(P.B + (size_t)f * kBFreq), "r"(kBFreq), "r"(bar)
                             : "memory");
                ++nb;
                fprev = f;
            }
            if (abort_flag) {
                // the copies issued land before the CTA leaves
                for (int j = nb - kBBuf < 0 ? 0 : nb - kBBuf; j < nb; ++j)
                    for (long long w = 0;
                         w < kWaitLimit && !mbar_try(smem_u32(&bfull_bar[j % kBBuf]), (uint32_t)((j / kBBuf) & 1)); ++w) {
                    }
            }
        }
    } else if (warp == 5) {
        // ---------------- MMA issuer: NCH accumulators per tile ----------------
        // The whole warp runs the bookkeeping, so descriptors and counters are warp-uniform (uniform
        // registers); one elected lane issues a tile's MMAs (straight-line, offsets known at
        // compile time) and the commits.
        {
            long long u = 0, ps_col = 0;
            int nb = 0, fprev = -1;  // B loads seen; the current frequency's is nb - 1
            bool pending = false;
            for (long long c = c0; c < P.ncols && !abort_flag; c += cstep, ps_col += Np) {
                int f, r, xb, yb;
                column_of(P, c, f, r, xb, yb);
                if (f != fprev) {
                    if (!mbar_wait(smem_u32(&bfull_bar[nb % kBBuf]), (uint32_t)((nb / kBBuf) & 1), &abort_flag, P.status,
                                   M2L_WAIT_OPERANDS))
                        goto mma_done;
                    ++nb;
                    fprev = f;
                }
                const int bbuf = (nb - 1) % kBBuf;
                const uint64_t bdesc = desc_noswz(s_B + (uint32_t)bbuf * kBFreq, kBLBO, kBSBO);
                bool last_of_f = true;
                if (c + cstep < P.ncols) {
                    int f2, r2, xb2, yb2;
                    column_of(P, c + cstep, f2, r2, xb2, yb2);
                    last_of_f = f2 != f;
                }
                for (int z = 0; z < Np; ++z, ++u) {
                    const int buf = (int)(u & 1);
                    if (u >= 2 && !mbar_wait(smem_u32(&acce_bar[buf]), (uint32_t)(((u >> 1) - 1) & 1), &abort_flag, P.status,
                                             M2L_WAIT_ACC_FREE))
                        goto mma_done;
                    uint64_t pd[3];
                    for (int dz = -1; dz <= 1; ++dz) {
                        const int zs = z + dz;
                        pd[dz + 1] = 0;
                        if (zs < 0 || zs >= Np) continue;
                        const long long q = ps_col + zs;
                        if (!mbar_wait(smem_u32(&full_bar[q % kRing]), (uint32_t)((q / kRing) & 1), &abort_flag, P.status,
                                       M2L_WAIT_OPERANDS))
                            goto mma_done;
                        pd[dz + 1] = desc_noswz(s_planes + (uint32_t)(q % kRing) * kPlaneB, kLBO, kSBO);
                    }
                    const uint64_t pd0 = pd[0], pd1 = pd[1], pd2 = pd[2];
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    // chain ch accumulates columns [32 ch, 32 ch + 32) of this tile's buffer: q_hi B_hi
                    // in the first 16, q_hi B_lo and q_lo B_hi (small) in the last 16; its first
                    // direction is in-plane, so always present, and its first MMA clears the 32 columns
                    if (elect_one())
                        issue_tile<NCH>(std::make_integer_sequence<int, 26>{}, tmem + buf * bufcols, pd0, pd1, pd2, bdesc,
                                        P.idesc48, P.idesc32, P.idesc16);
                    __syncwarp();
                    if (elect_one()) {
                        mma_commit(smem_u32(&accf_bar[buf]));
                        // plane z - 1 has served its last tile; at the column's end so has plane z
                        if (z >= 1) mma_commit(smem_u32(&empty_bar[(ps_col + z - 1) % kRing]));
                        if (z == Np - 1) {
                            mma_commit(smem_u32(&empty_bar[(ps_col + z) % kRing]));
                            if (last_of_f) mma_commit(smem_u32(&bempty_bar[bbuf]));
                        }
                    }
                    __syncwarp();
                    pending = true;
                }
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
        }
    } else {
        // ---------------- epilogue: phihat rows of the tile ----------------
        const int quarter = warp & 3;
        const int m = quarter * 32 + lane;  // MMA row: x = m mod 8, y = m / 8 inside the tile
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        long long u = 0;
        for (long long c = c0; c < P.ncols && !abort_flag; c += cstep) {
            int f, r, xb, yb;
            column_of(P, c, f, r, xb, yb);
            const int x = xb * kTX + (m & 7), y = yb * kTY + (m >> 3);
            for (int z = 0; z < Np; ++z, ++u) {
                const int buf = (int)(u & 1);
                if (!mbar_wait(smem_u32(&accf_bar[buf]), (uint32_t)((u >> 1) & 1), &abort_flag, P.status, M2L_WAIT_ACC_READY))
                    goto epi_done;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // the chains' leading products, then the parts 2^-8 and 2^-16 below, added with
                // round-to-nearest
                float g0[16], g1[16], g2[16];
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) {
                    uint32_t v0[16], v1[16], v2[16];
                    const uint32_t t = tmem + lane_off + buf * bufcols + 64u * (uint32_t)ch;
                    tmem_ld16(t, v0);
                    tmem_ld16(t + 16, v1);
                    tmem_ld16(t + 32, v2);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        g0[j] = ch ? __fadd_rn(g0[j], __uint_as_float(v0[j])) : __uint_as_float(v0[j]);
                        g1[j] = ch ? __fadd_rn(g1[j], __uint_as_float(v1[j])) : __uint_as_float(v1[j]);
                        g2[j] = ch ? __fadd_rn(g2[j], __uint_as_float(v2[j])) : __uint_as_float(v2[j]);
                    }
                }
                float hi[16], lo[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    hi[j] = g0[j];
                    lo[j] = __fadd_rn(g1[j], g2[j]);
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(smem_u32(&acce_bar[buf]));
                {
                    const long long cl = morton3(x, y, z);
                    float4 *o = reinterpret_cast<float4 *>(P.phihat + (((long long)cl * P.R + r) * P.F + f) * 16);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        o[j] = make_float4(__fadd_rn(hi[4 * j], lo[4 * j]), __fadd_rn(hi[4 * j + 1], lo[4 * j + 1]),
                                           __fadd_rn(hi[4 * j + 2], lo[4 * j + 2]), __fadd_rn(hi[4 * j + 3], lo[4 * j + 3]));
                }
            }
        }
    epi_done:;
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 5) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
    }
}

uint32_t idesc_bf16(int N) {
    uint32_t d = 1u << 4;                 // FP32 accumulator
    d |= 1u << 7;                         // A: BF16
    d |= 1u << 10;                        // B: BF16
    d |= (uint32_t)(N >> 3) << 17;        // N
    d |= (uint32_t)(128 >> 4) << 24;      // M = 128
    return d;
}

}  // namespace

bool hadamard_tc_eligible(const LevelView &L) {
    const long long Np = L.N / 2;
    return Np >= 16 && Np % 16 == 0 && L.nclusters == Np * Np * Np && L.nboxes == 8 * L.nclusters;
}

// The kernel matrices B_d(f) of every frequency as the kernel's shared memory holds them: for each
// f and direction d (dx slowest, then dy, dz; the origin left out), 48 rows n x 16 columns k of
// BF16, rows 0-15 the hi piece, 16-31 the mid piece and 32-47 the lo piece of
//   B[2i + a][2j + b] = (Re K, -Im K; Im K, Re K)[a][b],  K = Khat_{t}(f),  t = 2 d + j - i,
// zero where the two boxes are adjacent; K-major core matrices (8 rows x 8 values), row groups
// 128 bytes apart, 16-byte K chunks 768 bytes apart. Built from the FP64 spectra.
int build_hadamard_tc_operand(m2l_plan_t *pl, DevOps &D) {
    if (D.Bhad) return M2L_OK;
    const FftOps &Fo = *pl->fft;
    const int F = Fo.F;
    const size_t per = kBFreq / 2;  // BF16 values per frequency
    std::vector<uint16_t> img((size_t)F * per, 0);
    int tix[26][8][8];
    {
        int dd = 0;
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dz = -1; dz <= 1; ++dz) {
                    if (!dx && !dy && !dz) continue;
                    for (int i = 0; i < 8; ++i)
                        for (int j = 0; j < 8; ++j)
                            tix[dd][i][j] = transfer_index(2 * dx + (j & 1) - (i & 1), 2 * dy + ((j >> 1) & 1) - ((i >> 1) & 1),
                                                           2 * dz + ((j >> 2) & 1) - ((i >> 2) & 1));
                    ++dd;
                }
    }
#pragma omp parallel for schedule(static)
    for (int f = 0; f < F; ++f)
        for (int dd = 0; dd < 26; ++dd) {
            uint16_t *blk = &img[(size_t)f * per + (size_t)dd * (kBDir / 2)];
            for (int n = 0; n < 16; ++n)
                for (int k = 0; k < 16; ++k) {
                    const int i = n >> 1, a = n & 1, j = k >> 1, b = k & 1;
                    const int ti = tix[dd][i][j];
                    double v = 0.0;
                    if (ti >= 0) {
                        const double kr = Fo.Khat[((size_t)ti * F + f) * 2], ki = Fo.Khat[((size_t)ti * F + f) * 2 + 1];
                        v = a == 0 ? (b == 0 ? kr : -ki) : (b == 0 ? ki : kr);
                    }
                    // three BF16 pieces, each the nearest to what the previous ones leave
                    const uint16_t h = bf16_round((float)v);
                    const double r1 = v - (double)bf16_value(h);
                    const uint16_t m = bf16_round((float)r1);
                    const uint16_t l = bf16_round((float)(r1 - (double)bf16_value(m)));
                    const uint16_t pc[3] = {h, m, l};
                    for (int pi = 0; pi < 3; ++pi) {
                        const int nr = pi * 16 + n;  // row of the N = 48 operand
                        blk[(k >> 3) * (kBLBO / 2) + (nr >> 3) * 64 + (nr & 7) * 8 + (k & 7)] = pc[pi];
                    }
                }
        }
    if (cudaMalloc(&D.Bhad, img.size() * sizeof(uint16_t)) != cudaSuccess) {
        cudaGetLastError();
        D.Bhad = nullptr;
        set_error("allocating the tensor-core Hadamard operand failed");
        return M2L_ENOMEM;
    }
    if (cudaMemcpy(D.Bhad, img.data(), img.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        set_error("uploading the tensor-core Hadamard operand failed");
        return M2L_ECUDA;
    }
    return M2L_OK;
}

int launch_hadamard_tc(const LevelView &L, int R, int F, const void *B, const float *qhat, float *phihat, int chains,
                       int num_sms, int *status, cudaStream_t s) {
    if (chains == 0) chains = 4;
    if (chains != 1 && chains != 2 && chains != kMaxChains) {
        set_error("tensor-core Hadamard product: %d partial sums per tile (1, 2 or 4)", chains);
        return M2L_EINVAL;
    }
    if (!hadamard_tc_eligible(L) || !B || R < 1 || F < 1) {
        set_error("tensor-core Hadamard product: level or operand not eligible");
        return M2L_EUNSUPPORTED;
    }
    HtcParams P;
    P.qhat = qhat;
    P.phihat = phihat;
    P.B = (const unsigned char *)B;
    P.Np = L.N / 2;
    P.R = R;
    P.F = F;
    P.XB = P.Np / kTX;
    P.YB = P.Np / kTY;
    P.ncols = (long long)F * R * P.XB * P.YB;
    P.status = status;
    P.idesc48 = idesc_bf16(48);
    P.idesc32 = idesc_bf16(32);
    P.idesc16 = idesc_bf16(16);
    const int grid = (int)(P.ncols < num_sms ? P.ncols : num_sms);
    const size_t smem = kSmemH + 128;
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<grid, kThreadsH, smem, s>>>(P);
    };
    if (chains == 1) go(hadamard_tc_kernel<1>);
    else if (chains == 2) go(hadamard_tc_kernel<2>);
    else go(hadamard_tc_kernel<4>);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("tensor-core Hadamard launch failed: %s", cudaGetErrorString(e));
        return M2L_ECUDA;
    }
    return M2L_OK;
}

}  // namespace m2l
