// B2 on the 5th-generation tensor cores (tcgen05) for the split precisions TF32x3 and BF16x3.
//
// phi~[row] = sum over the transfer vectors t of the row's octant (189 at most; a tile visits only
// those that reach a source from one of its targets) of C_t q~[source(row, t)],
// every operand split as x = x_hi + x_lo and each product taken as hi*hi + hi*lo + lo*hi with FP32
// accumulation in tensor memory (the dropped lo*lo term is below the FP32 rounding of the
// result for TF32 pieces, about 2^-16 relative for BF16 pieces).
//
// One persistent CTA per SM loops over tiles of 128 (target, rhs) rows of one octant of one
// level. A pipeline stage is one MMA step of K (32 bytes: 16 BF16 or 8 TF32 values) of
//   A_hi, A_lo: the 128 gathered source rows of q~ (32 bytes each), cp.async by one producer
//               thread per row, written in the 32-byte swizzle;
//   B_hi, B_lo: the step of C_t (k_pad rows x 32 bytes), loaded by TMA with SWIZZLE_32B.
// A stage is 8 KB + 64 k_pad bytes (19 KB at k_pad = 176), so about ten stages are in flight and
// the gathers' L2 latency is covered; with 128-byte stages only two fit and every stage waited a
// full round trip.
// Warps: 0-3 gather A (thread = row; the next transfer vector's source row is looked up while the
// current steps are in flight); 4 issues TMA for B; 5 owns tensor memory and issues the MMAs
// (M = 128 rows, N = k_pad, K = 32 bytes); 6-9 drain each transfer vector's partial sum
// (double-buffered in tensor memory when 3 k_pad <= 512) into the running sum.
// Every wait is bounded; a wait that runs out sets the plan's device status word and the CTA
// winds down.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cstring>
#include <vector>

#include "internal.h"
#include "kernels.cuh"
#include "tcgen05.cuh"

namespace m2l {

namespace {

using namespace tc;

constexpr int kRows = 128;            // MMA M, rows per tile
constexpr int kMaxStages = 16;
constexpr int kThreads = 320;

struct TcParams {
    const LevelView *lv;               // device array indexed by ContractTile::lev
    const ContractTile *tiles;
    const int *tvl;                    // the tiles' packed transfer vector lists
    long long ntiles;
    const unsigned char *qhi, *qlo;   // [(rows + 1)][kp] elements
    long long zero_row;
    float *phit;                       // [rows][kp]
    int kp, elt, nchunks, stages;
    uint32_t idesc;
    int tmem_cols;
    int nbuf;                          // partial-sum buffers in tensor memory (1 or 2)
    int rt;                            // running-sum columns in tensor memory (multiple of 16, <= kp)
    int rs_off;                        // byte offset in dynamic shared memory of the other kp - rt
                                       // running-sum columns, [kp - rt][128] floats
    int group;                         // transfer vectors per partial sum (drain interval) when seg == 0
    int seg;                           // > 0: K stages per partial sum, within one transfer vector
    int *status;
};

// Shared-memory matrix descriptor: K-major rows of CH bytes (one row of the CH-byte swizzle),
// 8-row groups 8 CH bytes apart. Layout codes: 32-byte swizzle 6, 64-byte 4, 128-byte 2.
template <int CH>
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((8 * CH) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)(CH == 32 ? 6 : CH == 64 ? 4 : 2) << 61;
    return d;
}

struct RowInfo {
    int b;         // compact target box, -1 for a padding row
    int r;         // rhs
    uint32_t xyz;  // packed coordinates
};

__device__ __forceinline__ RowInfo row_info(const LevelView &L, const ContractTile &T, int row) {
    RowInfo ri;
    const int R = L.R;
    if (row < T.rows) {
        long long j = (long long)T.j0 + row;
        ri.b = L.perm[L.oct_start[T.oct] + j / R];
        ri.r = (int)(j % R);
        ri.xyz = L.xyz[ri.b];
    } else {
        ri.b = -1;
        ri.r = 0;
        ri.xyz = 0;
    }
    return ri;
}

// CH: bytes of K per pipeline stage (32, 64 or 128), CH / 32 MMA steps per stage.
template <int KIND, int CH>
__global__ void __launch_bounds__(kThreads, 1)
    contract_tc_kernel(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo, const TcParams P) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kMaxStages], empty_bar[kMaxStages], accf_bar[2], acce_bar[2], drain_bar;
    __shared__ uint32_t tmem_base_s;
    __shared__ volatile int abort_flag;

    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int S = P.stages;
    const int kp = P.kp;
    const uint32_t a_bytes = kRows * CH;                   // 128 rows x CH bytes
    const uint32_t b_bytes = (uint32_t)kp * CH;            // k_pad rows x CH bytes
    const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
    auto sA_hi = [&](int s) { return smem + (size_t)s * stage_bytes; };
    auto sA_lo = [&](int s) { return smem + (size_t)s * stage_bytes + a_bytes; };
    auto sB_hi = [&](int s) { return smem + (size_t)s * stage_bytes + 2 * a_bytes; };
    auto sB_lo = [&](int s) { return smem + (size_t)s * stage_bytes + 2 * a_bytes + b_bytes; };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nbuf = P.nbuf;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&full_bar[s]), kRows + 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&accf_bar[b]), 1);
            mbar_init(smem_u32(&acce_bar[b]), kRows);
        }
        mbar_init(smem_u32(&drain_bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(P.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem_base = tmem_base_s;
    const int chunk_elems = CH / P.elt;
    const int kbytes = kp * P.elt;  // valid bytes of a row
    // tensor memory: partial sums of one transfer vector in D[0..nbuf), the running sum in R
    const uint32_t tm_R = tmem_base + (uint32_t)(nbuf * kp);

    if (warp < 4) {
        // ---------------- A producers: kPieces lanes per row, each a 16-byte piece, so a warp's
        // copy instruction covers 32 / kPieces whole row segments; kPieces rows per thread ----
        constexpr int kPieces = CH / 16, kRowStep = kRows / kPieces;
        const int piece = tid % kPieces, rgrp = tid / kPieces;  // rows rgrp + kRowStep i
        long long it = 0;
        for (long long tile = blockIdx.x; tile < P.ntiles && !abort_flag; tile += gridDim.x) {
            const ContractTile T = P.tiles[tile];
            const LevelView &L = P.lv[T.lev];
            RowInfo ri[kPieces];
#pragma unroll
            for (int i = 0; i < kPieces; ++i) ri[i] = row_info(L, T, rgrp + kRowStep * i);
            const int N = L.N;
            // The source rows of list entry e + 1 are looked up while entry e's stages go out, and
            // its packed entry was read one entry earlier still: every lookup's result is first used
            // a whole transfer vector after its load was issued (in-order issue would otherwise
            // stall the warp at the first use, once per transfer vector).
            auto lookup = [&](int pk, int (&slot)[kPieces]) {
                const int dx = (pk & 15) - 3, dy = ((pk >> 4) & 15) - 3, dz = ((pk >> 8) & 15) - 3;
#pragma unroll
                for (int i = 0; i < kPieces; ++i) {
                    const int x = (int)(ri[i].xyz & 1023) + dx, y = (int)((ri[i].xyz >> 10) & 1023) + dy,
                              z = (int)((ri[i].xyz >> 20) & 1023) + dz;
                    int v = -1;
                    if (ri[i].b >= 0 && x >= 0 && y >= 0 && z >= 0 && x < N && y < N && z < N)
                        v = L.slot[((long long)z * N + y) * N + x];
                    slot[i] = v;
                }
            };
            int slot_nxt[kPieces];
            lookup(P.tvl[T.tv0], slot_nxt);
            int pk_nxt = T.ntv > 1 ? P.tvl[T.tv0 + 1] : 0;
            for (int e = 0; e < T.ntv; ++e) {
                long long src[kPieces];
#pragma unroll
                for (int i = 0; i < kPieces; ++i)
                    src[i] = slot_nxt[i] >= 0 ? L.row0 + (long long)slot_nxt[i] * L.R + ri[i].r : P.zero_row;
                if (e + 1 < T.ntv) {
                    lookup(pk_nxt, slot_nxt);
                    pk_nxt = e + 2 < T.ntv ? P.tvl[T.tv0 + e + 2] : 0;
                }
                for (int c = 0; c < P.nchunks; ++c, ++it) {
                    const int s = (int)(it % S);
                    if (it >= S && !mbar_wait(smem_u32(&empty_bar[s]), (uint32_t)(((it / S) - 1) & 1), &abort_flag,
                                              P.status, M2L_WAIT_GATHER))
                        goto producer_done;
                    const long long goff = (long long)c * CH + piece * 16;
                    if (goff < kbytes) {  // the last stage of a row may be shorter
                        const uint32_t bh = smem_u32(sA_hi(s)), bl = smem_u32(sA_lo(s));
#pragma unroll
                        for (int i = 0; i < kPieces; ++i) {
                            const int row = rgrp + kRowStep * i;
                            // CH-byte swizzle: the piece index is XORed with address bits 7.. of the
                            // row start, i.e. with row >> (7 - log2 CH) on log2(CH / 16) bits
                            const int swz = (row >> (CH == 32 ? 2 : CH == 64 ? 1 : 0)) & (kPieces - 1);
                            const uint32_t off = (uint32_t)(row * CH + ((piece ^ swz) * 16));
                            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(bh + off),
                                         "l"(P.qhi + src[i] * kbytes + goff)
                                         : "memory");
                            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(bl + off),
                                         "l"(P.qlo + src[i] * kbytes + goff)
                                         : "memory");
                        }
                    }
                    // the stage's barrier counts this thread's arrival once all its copies so far
                    // have landed; the thread itself runs on to the next stage
                    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&full_bar[s]))
                                 : "memory");
                }
            }
        }
    producer_done:
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp == 4) {
        // ---------------- B producer: TMA loads of C_t chunks ----------------
        if (lane == 0) {
            long long it = 0;
            for (long long tile = blockIdx.x; tile < P.ntiles && !abort_flag; tile += gridDim.x) {
                const ContractTile T = P.tiles[tile];
                int ti_nxt = P.tvl[T.tv0] >> 12;  // read one transfer vector ahead of its use
                for (int e = 0; e < T.ntv; ++e) {
                    const int ti = ti_nxt;
                    if (e + 1 < T.ntv) ti_nxt = P.tvl[T.tv0 + e + 1] >> 12;
                    for (int c = 0; c < P.nchunks; ++c, ++it) {
                        const int s = (int)(it % S);
                        if (it >= S && !mbar_wait(smem_u32(&empty_bar[s]), (uint32_t)(((it / S) - 1) & 1), &abort_flag,
                                                  P.status, M2L_WAIT_TMA))
                            goto tma_done;
                        const uint32_t bar = smem_u32(&full_bar[s]);
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(2 * b_bytes)
                                     : "memory");
                        const int x = c * chunk_elems, y = ti * kp;
                        asm volatile(
                            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                                smem_u32(sB_hi(s))),
                            "l"(&tm_hi), "r"(x), "r"(y), "r"(bar)
                            : "memory");
                        asm volatile(
                            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                                smem_u32(sB_lo(s))),
                            "l"(&tm_lo), "r"(x), "r"(y), "r"(bar)
                            : "memory");
                    }
                }
            }
        tma_done:
            if (abort_flag) {
                // let loads already issued land before the CTA leaves: `it` stages were issued, the
                // last one of stage s being iteration it - 1 - ((it - 1 - s) mod S)
                for (int s = 0; s < S && s < it; ++s) {
                    const long long last = it - 1 - (((it - 1 - s) % S) + S) % S;
                    const uint32_t parity = (uint32_t)((last / S) & 1);
                    for (long long w = 0; w < kWaitLimit && !mbar_try(smem_u32(&full_bar[s]), parity); ++w) {
                    }
                }
            }
        }
    } else if (warp == 5) {
        // ---------------- MMA issuer: one partial sum per unit ----------------
        // A tile's work is its (transfer vector, K stage) pairs, vector-major. A unit, summed in one
        // tensor-memory buffer before its round-to-nearest drain, is `group` whole transfer vectors
        // (seg == 0) or seg consecutive stages of one transfer vector (seg > 0). The whole warp runs
        // the bookkeeping, so descriptors and counters are warp-uniform (uniform registers); one
        // elected lane issues the MMAs and commits.
        {
            long long it = 0, u = 0;
            bool pending = false;
            const int nc = P.nchunks, seg = P.seg, group = P.group;
            for (long long tile = blockIdx.x; tile < P.ntiles && !abort_flag; tile += gridDim.x) {
                const int ntv = P.tiles[tile].ntv;
                const int total = ntv * nc;
                uint32_t d = 0, accflag = 0;
                int buf = 0;
                for (int x = 0; x < total; ++x, ++it) {
                    const int tv = x / nc, c = x - tv * nc;
                    const bool ustart = seg > 0 ? (c % seg == 0) : (c == 0 && tv % group == 0);
                    const bool uend = seg > 0 ? (c % seg == seg - 1 || c == nc - 1)
                                              : (c == nc - 1 && (tv % group == group - 1 || tv == ntv - 1));
                    if (ustart) {
                        buf = (int)(u % nbuf);
                        if (u >= nbuf && !mbar_wait(smem_u32(&acce_bar[buf]), (uint32_t)(((u / nbuf) - 1) & 1), &abort_flag,
                                                    P.status, M2L_WAIT_ACC_FREE))
                            goto mma_done;
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        d = tmem_base + (uint32_t)(buf * kp);
                        accflag = 0;
                    }
                    const int s = (int)(it % S);
                    if (!mbar_wait(smem_u32(&full_bar[s]), (uint32_t)((it / S) & 1), &abort_flag, P.status, M2L_WAIT_OPERANDS))
                        goto mma_done;
                    // the gathered rows were written by cp.async (generic proxy); the MMA reads them
                    // through the async proxy
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int steps = min(CH / 32, (kbytes - c * CH) / 32);
                    const uint32_t ah = smem_u32(sA_hi(s)), al = smem_u32(sA_lo(s));
                    const uint32_t bh = smem_u32(sB_hi(s)), bl = smem_u32(sB_lo(s));
                    if (elect_one()) {
                        uint32_t af = accflag;
                        for (int k = 0; k < steps; ++k) {
                            const uint64_t dah = smem_desc<CH>(ah + 32 * k), dal = smem_desc<CH>(al + 32 * k);
                            const uint64_t dbh = smem_desc<CH>(bh + 32 * k), dbl = smem_desc<CH>(bl + 32 * k);
                            mma<KIND>(d, dal, dbh, P.idesc, af);
                            af = 1;
                            mma<KIND>(d, dah, dbl, P.idesc, 1);
                            mma<KIND>(d, dah, dbh, P.idesc, 1);
                        }
                        mma_commit(smem_u32(&empty_bar[s]));
                        if (uend) mma_commit(smem_u32(&accf_bar[buf]));
                    }
                    __syncwarp();
                    accflag = 1;  // every stage issues at least one K step
                    pending = true;
                    if (uend) ++u;
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
        // ---------------- epilogue: R += D per transfer vector (FP32, round to nearest); R -> phi~ ----
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        float *Rs = reinterpret_cast<float *>(smem + P.rs_off);
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        long long u = 0;
        for (long long tile = blockIdx.x; tile < P.ntiles && !abort_flag; tile += gridDim.x) {
            const ContractTile T = P.tiles[tile];
            const LevelView &L = P.lv[T.lev];
            const RowInfo ri = row_info(L, T, row);
            float *dst = ri.b >= 0 ? P.phit + (L.row0 + (long long)ri.b * L.R + ri.r) * (long long)kp : nullptr;
            const int nunits = P.seg > 0 ? T.ntv * ((P.nchunks + P.seg - 1) / P.seg) : (T.ntv + P.group - 1) / P.group;
            for (int j = 0; j < nunits; ++j, ++u) {
                const bool first = j == 0, last = j == nunits - 1;
                const int buf = (int)(u % nbuf);
                if (!mbar_wait(smem_u32(&accf_bar[buf]), (uint32_t)((u / nbuf) & 1), &abort_flag, P.status, M2L_WAIT_ACC_READY)) goto epi_done;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t tD = tmem_base + lane_off + (uint32_t)(buf * kp), tR = tm_R + lane_off;
                for (int c0 = 0; c0 < kp; c0 += 48) {
                    uint32_t dv[3][16], rv[3][16];
                    const int nc = min(3, (kp - c0) / 16);
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        if (q < nc) {
                            const int col = c0 + 16 * q;
                            tmem_ld16(tD + col, dv[q]);
                            if (!first) {
                                if (col < P.rt) {
                                    tmem_ld16(tR + col, rv[q]);
                                } else {  // running-sum columns past rt live in shared memory
#pragma unroll
                                    for (int j = 0; j < 16; ++j) rv[q][j] = __float_as_uint(Rs[(col - P.rt + j) * kRows + row]);
                                }
                            }
                        }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        if (q >= nc) continue;
                        const int col = c0 + 16 * q;
                        if (!first) {
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                dv[q][j] = __float_as_uint(__fadd_rn(__uint_as_float(rv[q][j]), __uint_as_float(dv[q][j])));
                        }
                        if (!last) {
                            if (col < P.rt) {
                                tmem_st16(tR + col, dv[q]);
                            } else {
#pragma unroll
                                for (int j = 0; j < 16; ++j) Rs[(col - P.rt + j) * kRows + row] = __uint_as_float(dv[q][j]);
                            }
                        } else if (dst) {
                            float4 *o = reinterpret_cast<float4 *>(dst + c0 + 16 * q);
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                o[j] = make_float4(__uint_as_float(dv[q][4 * j]), __uint_as_float(dv[q][4 * j + 1]),
                                                   __uint_as_float(dv[q][4 * j + 2]), __uint_as_float(dv[q][4 * j + 3]));
                        }
                    }
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(smem_u32(&acce_bar[buf]));
            }
        }
    epi_done:;
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 5) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(P.tmem_cols));
    }
}

// One bounded wait on an mbarrier that nothing arrives at: the expiry path every wait of the
// contraction takes (status word set, abort flag raised, the kernel returns; no trap), run with no
// copy and no MMA in flight.
__global__ void watchdog_selftest_kernel(int *status, long long limit) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ volatile int abort_flag;
    if (threadIdx.x != 0) return;
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_wait(smem_u32(&bar), 0, &abort_flag, status, M2L_WAIT_SELFTEST, limit);
}

// hi/lo split of q~ rows: TF32 pieces (FP32 containers, low 13 bits zero) or BF16 pieces.
__global__ void split_rows_kernel(const float *__restrict__ src, long long count, int kind, unsigned char *__restrict__ hi,
                                  unsigned char *__restrict__ lo) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < count; i += stride) {
        const float x = src[i];
        if (kind == 0) {
            uint32_t h, l;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
            const float r = x - __uint_as_float(h);
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
            reinterpret_cast<uint32_t *>(hi)[i] = h;
            reinterpret_cast<uint32_t *>(lo)[i] = l;
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
            reinterpret_cast<__nv_bfloat16 *>(hi)[i] = h;
            reinterpret_cast<__nv_bfloat16 *>(lo)[i] = l;
        }
    }
}


}  // namespace

// Split C_t (FP64 on the host) into hi/lo pieces, upload them and encode their TMA maps.
int split_tc_operators(m2l_plan_t *pl, int precision) {
    DevOps &D = pl->dev[precision];
    const int k = pl->k, kp = pl->kp;
    if (kp > 256) {
        set_error("split tensor-core contraction supports a rank of at most 256 (k_pad = %d)", kp);
        return M2L_EUNSUPPORTED;
    }
    const size_t count = (size_t)kNumTransfer * kp * kp;
    const int kind = precision == M2L_PREC_TF32X3 ? 0 : 1;
    const size_t elt = kind == 0 ? 4 : 2;
    std::vector<unsigned char> hi(count * elt, 0), lo(count * elt, 0);
    for (int t = 0; t < kNumTransfer; ++t)
        for (int a = 0; a < k; ++a)
            for (int c = 0; c < k; ++c) {
                const double v = pl->blas->C[((size_t)t * k + a) * k + c];
                const size_t i = ((size_t)t * kp + a) * kp + c;
                if (kind == 0) {
                    float h = tf32_round((float)v);
                    float l = tf32_round((float)(v - (double)h));
                    std::memcpy(&hi[i * 4], &h, 4);
                    std::memcpy(&lo[i * 4], &l, 4);
                } else {
                    uint16_t h = bf16_round((float)v);
                    uint16_t l = bf16_round((float)(v - (double)bf16_value(h)));
                    std::memcpy(&hi[i * 2], &h, 2);
                    std::memcpy(&lo[i * 2], &l, 2);
                }
            }
    for (void **pp : {&D.C_hi, &D.C_lo})
        if (*pp) cudaFree(*pp);
    D.C_hi = D.C_lo = nullptr;
    if (cudaMalloc(&D.C_hi, hi.size()) != cudaSuccess || cudaMalloc(&D.C_lo, lo.size()) != cudaSuccess) {
        cudaGetLastError();
        set_error("allocating split operators failed");
        return M2L_ENOMEM;
    }
    cudaMemcpy(D.C_hi, hi.data(), hi.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(D.C_lo, lo.data(), lo.size(), cudaMemcpyHostToDevice);
    EncodeTiledFn enc = encode_fn();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return M2L_ECUDA;
    }
    // C_t as a 2D tensor: inner dimension k_pad elements, kNumTransfer * k_pad rows; a box is one
    // stage's CH bytes of K for all k_pad output rows of one transfer vector, in the CH-byte
    // swizzle; one pair of maps (hi, lo) per stage width CH = 32, 64, 128.
    const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)kNumTransfer * kp};
    const cuuint64_t strides[1] = {(cuuint64_t)kp * elt};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const CUtensorMapSwizzle swz[3] = {CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_SWIZZLE_128B};
    void *bases[2] = {D.C_hi, D.C_lo};
    for (int w = 0; w < 3; ++w) {
        const cuuint32_t box[2] = {(cuuint32_t)((32 << w) / elt), (cuuint32_t)kp};
        for (int i = 0; i < 2; ++i) {
            CUresult r = enc(reinterpret_cast<CUtensorMap *>(D.tmap[w][i]), dt, 2, bases[i], dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, swz[w], CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
                return M2L_ECUDA;
            }
        }
    }
    return M2L_OK;
}

int launch_split_rows(const float *src, long long rows, int kp, void *hi, void *lo, int precision, cudaStream_t s) {
    const long long count = rows * kp;
    const int kind = precision == M2L_PREC_TF32X3 ? 0 : 1;
    long long blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    split_rows_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, count, kind, (unsigned char *)hi, (unsigned char *)lo);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("split launch failed: %s", cudaGetErrorString(e));
        return M2L_ECUDA;
    }
    return M2L_OK;
}

int launch_watchdog_selftest(int *status, long long polls, cudaStream_t s) {
    watchdog_selftest_kernel<<<1, 32, 0, s>>>(status, polls);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("watchdog self-test launch failed: %s", cudaGetErrorString(e));
        return M2L_ECUDA;
    }
    return M2L_OK;
}

size_t tc_stage_bytes(int kp, int ch) { return 2 * (size_t)kRows * ch + 2 * (size_t)kp * ch; }

// Stage width (bytes of K per pipeline stage) of the tensor-core contraction: the plan's
// M2L_OPT_TC_CHUNK, or 128 by default.
int tc_chunk_of(const m2l_plan_t *pl) { return pl->tc_chunk ? pl->tc_chunk : 128; }

// K stages per partial sum of the tensor-core contraction (0: whole transfer vectors): the plan's
// M2L_OPT_TC_DRAIN, or by default 2 for TF32x3 and 0 for BF16x3. A stage count of nchunks or more
// is the same as 0.
int tc_drain_of(const m2l_plan_t *pl, int precision, int nchunks) {
    int seg = pl->tc_drain >= 0 ? pl->tc_drain : (precision == M2L_PREC_TF32X3 ? 2 : 0);
    return seg >= nchunks ? 0 : seg;
}

template <class T>
int launch_contract_tc(m2l_plan_t *pl, const LevelView *lv, const ContractTile *tiles, long long ntiles, const int *tvl,
                       const void *qt_hi, const void *qt_lo, long long zero_row, T *phit, int precision, cudaStream_t s) {
    if constexpr (sizeof(T) != 4) {
        set_error("the tensor-core contraction writes FP32");
        return M2L_EINVAL;
    } else {
        if (ntiles <= 0) return M2L_OK;
        DevOps &D = pl->dev[precision];
        const int kp = pl->kp;
        const int kind = precision == M2L_PREC_TF32X3 ? 0 : 1;
        TcParams P;
        P.lv = lv;
        P.tiles = tiles;
        P.tvl = tvl;
        P.ntiles = ntiles;
        P.qhi = (const unsigned char *)qt_hi;
        P.qlo = (const unsigned char *)qt_lo;
        P.zero_row = zero_row;
        P.phit = reinterpret_cast<float *>(phit);
        P.kp = kp;
        P.elt = kind == 0 ? 4 : 2;
        const int ch = tc_chunk_of(pl);
        P.nchunks = (kp * P.elt + ch - 1) / ch;  // k_pad is a multiple of 16: whole 32-byte MMA steps
        const size_t stage = tc_stage_bytes(kp, ch);
        const size_t budget = 227 * 1024 - 1024 - 256;
        int S = (int)(budget / stage);
        if (S > kMaxStages) S = kMaxStages;
        if (S < 2) {
            set_error("rank %d too large for the tensor-core pipeline", kp);
            return M2L_EUNSUPPORTED;
        }
        P.stages = S;
        uint32_t idesc = 1u << 4;  // FP32 accumulator
        idesc |= (kind == 0 ? 2u : 1u) << 7;
        idesc |= (kind == 0 ? 2u : 1u) << 10;
        idesc |= (uint32_t)(kp >> 3) << 17;
        idesc |= (uint32_t)(kRows >> 4) << 24;
        P.idesc = idesc;
        // tensor memory: nbuf partial-sum buffers of kp columns and the running sum. Two buffers let
        // the MMAs of one transfer vector run while the previous one drains; when 3 kp > 512 the
        // running sum keeps rt = 512 - 2 kp columns (rounded down to 16) in tensor memory and the
        // rest in shared memory, as long as two pipeline stages still fit beside it.
        P.nbuf = 2;
        P.rt = kp;
        size_t rs_bytes = 0;
        if (3 * kp > 512) {
            P.rt = (512 - 2 * kp) / 16 * 16;
            rs_bytes = (size_t)(kp - P.rt) * kRows * sizeof(float);
            if (P.rt < 0 || (budget - rs_bytes) / stage < 2) {
                P.nbuf = 1;
                P.rt = kp;
                rs_bytes = 0;
            }
        }
        S = (int)((budget - rs_bytes) / stage);
        if (S > kMaxStages) S = kMaxStages;
        P.stages = S;
        P.rs_off = (int)((size_t)S * stage);
        const int need = P.nbuf * kp + P.rt;
        P.group = pl->tc_group > 0 ? pl->tc_group : 1;
        P.seg = tc_drain_of(pl, precision, P.nchunks);
        if (P.seg > 0) P.group = 1;
        P.tmem_cols = need <= 32 ? 32 : need <= 64 ? 64 : need <= 128 ? 128 : need <= 256 ? 256 : 512;
        P.status = pl->dev_status;
        const size_t smem = (size_t)S * stage + rs_bytes + 1024;
        const int grid = (int)(ntiles < pl->num_sms ? ntiles : pl->num_sms);
        const int w = ch == 32 ? 0 : ch == 64 ? 1 : 2;
        const CUtensorMap *thi = reinterpret_cast<const CUtensorMap *>(D.tmap[w][0]);
        const CUtensorMap *tlo = reinterpret_cast<const CUtensorMap *>(D.tmap[w][1]);
        cudaError_t e;
        auto go = [&](auto kern) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            kern<<<grid, kThreads, smem, s>>>(*thi, *tlo, P);
        };
        if (kind == 0)
            ch == 32 ? go(contract_tc_kernel<0, 32>) : ch == 64 ? go(contract_tc_kernel<0, 64>) : go(contract_tc_kernel<0, 128>);
        else
            ch == 32 ? go(contract_tc_kernel<1, 32>) : ch == 64 ? go(contract_tc_kernel<1, 64>) : go(contract_tc_kernel<1, 128>);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error("tensor-core contraction launch failed: %s", cudaGetErrorString(e));
            return M2L_ECUDA;
        }
        return M2L_OK;
    }
}
template int launch_contract_tc<float>(m2l_plan_t *, const LevelView *, const ContractTile *, long long, const int *,
                                       const void *, const void *, long long, float *, int, cudaStream_t);
template int launch_contract_tc<double>(m2l_plan_t *, const LevelView *, const ContractTile *, long long, const int *,
                                        const void *, const void *, long long, double *, int, cudaStream_t);

}  // namespace m2l
