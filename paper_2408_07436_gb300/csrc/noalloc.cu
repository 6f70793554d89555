// m2l_apply_noalloc: the FP64 BLAS form at one level with its scratch (compressed multipoles,
// compressed check potentials and the pseudo-inverse intermediate) in a file-scope static device
// array instead of memory the plan allocates. It allocates nothing: no cudaMalloc, no cudaFree,
// no allocating library routine, no host heap.
//
// The contraction here is a variant of contract_simt_kernel<double>: same arithmetic and order,
// but each CTA derives its tile from blockIdx (no device tile list) and every row index is local
// to the level.
#include <cstdio>
#include <mutex>
#include <string>

#include "internal.h"
#include "kernels.cuh"

namespace m2l {

// 32 MiB of doubles, held by every GPU that loads this library until the process exits.
constexpr long long kNoAllocScratchDoubles = 4LL * 1024 * 1024;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];
__constant__ short c_na_tidx[7][7][7];

namespace {
// Set-up of one device: the array's device address and the transfer-vector table. std::call_once
// makes it safe when several host threads make their first call on one device together; a set-up
// that failed is reported again by every later call on that device.
struct DeviceSetup {
    std::once_flag once;
    int rc = M2L_EINVAL;
    std::string msg;
    double *scratch = nullptr;
};
DeviceSetup g_setup[64];

int setup_once(DeviceSetup &S) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) {
        S.msg = std::string("cudaGetSymbolAddress of the static scratch failed: ") + cudaGetErrorString(e);
        return M2L_ECUDA;
    }
    short tidx[7][7][7];
    for (int x = -3; x <= 3; ++x)
        for (int y = -3; y <= 3; ++y)
            for (int z = -3; z <= 3; ++z) tidx[x + 3][y + 3][z + 3] = (short)transfer_index(x, y, z);
    e = cudaMemcpyToSymbol(c_na_tidx, tidx, sizeof tidx);
    if (e != cudaSuccess) {
        S.msg = std::string("uploading the transfer-vector table failed: ") + cudaGetErrorString(e);
        return M2L_ECUDA;
    }
    S.scratch = static_cast<double *>(ptr);
    return M2L_OK;
}

// The caller has checked that `device` is the current device.
int setup_device(int device) {
    if (device < 0 || device >= 64) {
        set_error("device ordinal %d not supported", device);
        return M2L_EINVAL;
    }
    DeviceSetup &S = g_setup[device];
    std::call_once(S.once, [&] { S.rc = setup_once(S); });
    if (S.rc != M2L_OK) {
        set_error("%s", S.msg.c_str());
        return S.rc;
    }
    return M2L_OK;
}
}  // namespace

// Tile of CTA blockIdx.x: octant segments are cut into 64-row tiles in octant order.
__global__ void __launch_bounds__(256) contract_noalloc_kernel(LevelView L, int R, const double *__restrict__ qt,
                                                               const double *__restrict__ C, int kp,
                                                               long long zero_row, double *__restrict__ phit) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ double Xs[BK][BM + 4];
    __shared__ double Ws[BK][BN + 4];
    __shared__ long long src_row[BM];
    __shared__ int tgt_b[BM], tgt_r[BM];
    __shared__ uint32_t tgt_xyz[BM];
    int oct = 0;
    long long j0 = 0, segrows = 0;
    {
        long long t = blockIdx.x;
        for (oct = 0; oct < 8; ++oct) {
            segrows = (L.oct_start[oct + 1] - L.oct_start[oct]) * (long long)R;
            long long nt = (segrows + BM - 1) / BM;
            if (t < nt) break;
            t -= nt;
        }
        if (oct == 8) return;
        j0 = t * BM;
    }
    const int rows = (int)(segrows - j0 < BM ? segrows - j0 : BM);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int col0 = blockIdx.y * BN;
    if (tid < BM) {
        if (tid < rows) {
            long long j = j0 + tid;
            int b = L.perm[L.oct_start[oct] + j / R];
            tgt_b[tid] = b;
            tgt_r[tid] = (int)(j % R);
            tgt_xyz[tid] = L.xyz[b];
        } else {
            tgt_b[tid] = -1;
            tgt_r[tid] = 0;
            tgt_xyz[tid] = 0;
        }
    }
    double a[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) a[i][j] = 0.0;
    const int cx = oct & 1, cy = (oct >> 1) & 1, cz = (oct >> 2) & 1;
    const int N = L.N;
    for (int dx = -2 - cx; dx <= 3 - cx; ++dx)
        for (int dy = -2 - cy; dy <= 3 - cy; ++dy)
            for (int dz = -2 - cz; dz <= 3 - cz; ++dz) {
                int ti = c_na_tidx[dx + 3][dy + 3][dz + 3];
                if (ti < 0) continue;
                __syncthreads();
                if (tid < BM) {
                    long long sr = zero_row;
                    if (tgt_b[tid] >= 0) {
                        uint32_t p = tgt_xyz[tid];
                        int x = (int)(p & 1023) + dx, y = (int)((p >> 10) & 1023) + dy, z = (int)((p >> 20) & 1023) + dz;
                        if (x >= 0 && y >= 0 && z >= 0 && x < N && y < N && z < N) {
                            int s = L.slot[((long long)z * N + y) * N + x];
                            if (s >= 0) sr = (long long)s * R + tgt_r[tid];
                        }
                    }
                    src_row[tid] = sr;
                }
                __syncthreads();
                const double *Ct = C + (long long)ti * kp * kp;
                for (int k0 = 0; k0 < kp; k0 += BK) {
                    for (int e = tid; e < BM * BK; e += 256) {
                        int r = e / BK, kk = e % BK;
                        Xs[kk][r] = qt[src_row[r] * kp + k0 + kk];
                        int gc = col0 + r;
                        Ws[kk][r] = gc < kp ? Ct[(long long)gc * kp + k0 + kk] : 0.0;
                    }
                    __syncthreads();
#pragma unroll
                    for (int kk = 0; kk < BK; ++kk) {
                        double xa[4], wb[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            xa[i] = Xs[kk][ty * 4 + i];
                            wb[i] = Ws[kk][tx * 4 + i];
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j) a[i][j] = fma(xa[i], wb[j], a[i][j]);
                    }
                    __syncthreads();
                }
            }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int r = ty * 4 + i;
        if (r >= rows) continue;
        long long orow = (long long)tgt_b[r] * R + tgt_r[r];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int c = col0 + tx * 4 + j;
            if (c < kp) phit[orow * kp + c] = a[i][j];
        }
    }
}

}  // namespace m2l

using namespace m2l;

extern "C" int m2l_apply_noalloc(m2l_plan_t *pl, const double *multipoles, double *locals, int level, int n_rhs) {
    clear_error();
    if (!pl || !multipoles || !locals) {
        set_error("NULL plan or buffer");
        return M2L_EINVAL;
    }
    if (level < 2 || level > pl->depth) {
        set_error("m2l_apply_noalloc works on one level in [2, %d]; got %d", pl->depth, level);
        return M2L_EINVAL;
    }
    if (n_rhs < 1) {
        set_error("n_rhs must be >= 1");
        return M2L_EINVAL;
    }
    if (pl->device < 0) {
        set_error("no CUDA device was available when the plan was made");
        return M2L_ECUDA;
    }
    const DevOps &D = pl->dev[M2L_PREC_FP64];
    const LevelDev &LD = pl->ldev[level];
    if (pl->pc != pl->p) {
        set_error("m2l_apply_noalloc needs equal check and equivalent orders");
        return M2L_EINVAL;
    }
    if (D.C == nullptr || D.St == nullptr || D.A == nullptr || D.V == nullptr || D.Uc == nullptr ||
        pl->levels_dirty || !LD.on_device) {
        set_error("plan not prepared: its FP64 BLAS operators and box tables are not on the device yet "
                  "(one m2l_apply of this plan in FP64 BLAS form uploads them)");
        return M2L_EINVAL;
    }
    const long long rows = LD.nboxes * n_rhs;
    const int n = pl->n, kp = pl->kp, rp = pl->rp;
    auto al = [](long long v) { return (v + 31) / 32 * 32; };  // 256-byte offsets
    const long long qt_d = al((rows + 1) * kp), ph_d = al(rows * kp), z_d = al(rows * rp);
    const long long need = qt_d + ph_d + z_d;
    if (need > kNoAllocScratchDoubles) {
        set_error("level %d with %d RHS needs %lld doubles of scratch; m2l_apply_noalloc holds at most %lld "
                  "(use m2l_apply)", level, n_rhs, need, kNoAllocScratchDoubles);
        return M2L_EINVAL;
    }
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != pl->device) {
        cudaGetLastError();
        set_error("m2l_apply_noalloc must be called with the plan's device (%d) current; device %d is current",
                  pl->device, cur);
        return M2L_EINVAL;
    }
    int rc = setup_device(pl->device);
    if (rc) return rc;
    double *scratch = g_setup[pl->device].scratch;
    double *qt = scratch, *phit = scratch + qt_d, *Z = scratch + qt_d + ph_d;
    cudaStream_t s = pl->stream;
    // B1: compressed multipoles of the level's rows; the extra row stays zero for missing sources
    rc = launch_gemm_xwt<double>(multipoles, n, (const double *)D.St, n, qt, kp, rows, kp, n, 0, s);
    if (rc) return rc;
    if (cudaMemsetAsync(qt + rows * kp, 0, kp * sizeof(double), s) != cudaSuccess) {
        set_error("clearing the zero row failed: %s", cudaGetErrorString(cudaGetLastError()));
        return M2L_ECUDA;
    }
    // B2: contraction, tiles derived from blockIdx
    LevelView L;
    L.slot = LD.slot;
    L.xyz = LD.xyz;
    L.perm = LD.perm;
    L.cslot = LD.cslot;
    L.cxyz = LD.cxyz;
    L.cperm = LD.cperm;
    L.cchild = LD.cchild;
    L.base = 0;
    L.cbase = 0;
    L.nboxes = LD.nboxes;
    L.nclusters = LD.nclusters;
    for (int i = 0; i < 9; ++i) L.oct_start[i] = LD.oct_start[i];
    L.N = 1 << level;
    long long ntiles = 0;
    for (int oct = 0; oct < 8; ++oct) ntiles += ((LD.oct_start[oct + 1] - LD.oct_start[oct]) * n_rhs + 63) / 64;
    if (ntiles > 0) {
        dim3 grid((unsigned)ntiles, (unsigned)((kp + 63) / 64));
        contract_noalloc_kernel<<<grid, 256, 0, s>>>(L, n_rhs, qt, (const double *)D.C, kp, rows, phit);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error("contraction launch failed: %s", cudaGetErrorString(e));
            return M2L_ECUDA;
        }
    } else {
        if (cudaMemsetAsync(phit, 0, rows * kp * sizeof(double), s) != cudaSuccess) {
            set_error("clearing the check potentials failed: %s", cudaGetErrorString(cudaGetLastError()));
            return M2L_ECUDA;
        }
    }
    // B3: locals = V_eps (A phit), or the check potential U phit
    if (pl->output == M2L_OUT_LOCALS) {
        rc = launch_gemm_xwt<double>(phit, kp, (const double *)D.A, kp, Z, rp, rows, rp, kp, 0, s);
        if (rc) return rc;
        rc = launch_gemm_xwt<double>(Z, rp, (const double *)D.V, rp, locals, n, rows, n, rp, pl->accumulate, s);
    } else {
        rc = launch_gemm_xwt<double>(phit, kp, (const double *)D.Uc, kp, locals, n, rows, n, kp, pl->accumulate, s);
    }
    return rc;
}
