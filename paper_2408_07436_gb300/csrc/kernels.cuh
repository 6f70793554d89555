// Device-side declarations shared by the kernel translation units and the launcher.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace m2l {

constexpr int kMaxLevels = 7;  // levels 2..8

// Per-level box tables as seen by the kernels.
struct LevelView {
    const int *slot;        // [N^3] grid (x + N(y + N z)) -> compact box or -1
    const uint32_t *xyz;    // [nboxes] packed x | y << 10 | z << 20
    const int *perm;        // [nboxes] boxes grouped by octant
    const int *cslot;       // [(N/2)^3] parent grid -> cluster or -1
    const uint32_t *cxyz;   // [nclusters] packed parent coordinates
    const int *cchild;      // [nclusters][8] compact child box or -1
    const int *cperm;       // [nclusters] clusters grouped by domain-boundary class
    long long base;         // first global box row of the level
    long long cbase;        // first global cluster of the level
    long long nboxes, nclusters;
    long long oct_start[9];
    int N;                  // boxes per axis, 2^level
    long long row0;         // contraction rows of this level: row0 + b * R + r (box b, rhs r)
    int R;                  // right-hand sides of the instance
};

// One CTA of the contraction: rows [j0, j0 + rows) of the octant segment `oct` of level view
// `lev` (index into a device array of LevelView), where segment row j is
// (target perm[oct_start + j / R], rhs j % R). The tile visits the ntv transfer vectors
// tvl[tv0 .. tv0 + ntv) of a device list: those of the octant (189 at most, Sec. 3.1) that reach
// an existing source from at least one of its targets, each packed as
// (dx + 3) | (dy + 3) << 4 | (dz + 3) << 8 | (index in [-3,3]^3 \ [-1,1]^3, x slowest) << 12.
// A tile with no source at all keeps one entry, so its rows are still written (as zeros).
struct ContractTile {
    int lev;
    int oct;
    int j0;
    int rows;
    long long tv0;
    int ntv;
    int pad_;
};

// Y[r][o] (+)= sum_i X[r][i] W[o][i]; X rows x K (row stride ldx), W O x K (stride ldw).
template <class T>
int launch_gemm_xwt(const T *X, long long ldx, const T *W, long long ldw, T *Y, long long ldy,
                    long long rows, int O, int K, int acc, cudaStream_t s);

// Y[r][o] (+)= sum_i X[r][i] (Wh[o][i] + Wl[o][i]) with a compensated (float-float) sum, FP32 in
// and out.
int launch_gemm_xwt_ff(const float *X, long long ldx, const float *Wh, const float *Wl, long long ldw, float *Y,
                       long long ldy, long long rows, int O, int K, int acc, cudaStream_t s);

// B2 on CUDA cores: phit[row0 + b R + r][:] = sum_t C_t qt[row0 + src R + r][:] over the tiles,
// qt rows of kp values, C_t [kcp][kp], phit rows of kcp values (kcp = kp unless the check order
// exceeds the equivalent order),
// `levels` a device array of LevelView indexed by ContractTile::lev, `tvl` the tiles' transfer
// vector lists.
template <class T>
int launch_contract_simt(const LevelView *levels, const ContractTile *tiles, long long ntiles, const int *tvl,
                         const T *qt, const T *C, int kp, int kcp, long long zero_row, T *phit, cudaStream_t s);

// B2 with the directional factors (Eq. 15): Ub = Ubar_t [kc_pad][k_t8], Vt = Vbar'_t^T [k_t8][k_pad]
// concatenated over t, meta = [316] int4 (Ub offset, Vt offset, k_t, k_t8). Its tiles hold at most
// kDirTileRows<T> rows: 32 in FP64, where the kernel is bound by the FP64 units and finer tiles
// shorten the tail after the last wave of CTAs; 64 in FP32, where the taller register tile's reuse
// of each shared-memory load matters more. M2L_EUNSUPPORTED (nothing launched) when its
// shared-memory tiles do not fit.
template <class T>
constexpr int kDirTileRows = sizeof(T) == 8 ? 32 : 64;
template <class T>
int launch_contract_simt_dir(const LevelView *levels, const ContractTile *tiles, long long ntiles, const int *tvl,
                             const T *qt, const T *Ub, const T *Vt, const int *meta, int k, int kp, int kcp,
                             int kt8max, long long zero_row, T *phit, cudaStream_t s);

// FFT form, one level at a time. Spectra rows (cluster * R + rhs) hold the 8 siblings' half
// spectra as [8][F] complex values, or as [F][8] with sib_minor (the FP32 transforms specialised
// on (p, g) only, fft_pg_available): the layout of the tensor-core Hadamard product.
template <class T>
int launch_fft_forward(const LevelView &L, int R, int p, int n, int g, const int *lattice,
                       const T *tw, const T *q, T *qhat, cudaStream_t s, bool sib_minor = false);
template <class T>
int launch_hadamard(const LevelView &L, int R, int F, const T *Khat, const T *qhat, T *phihat,
                    cudaStream_t s);
template <class T>
int launch_fft_inverse(const LevelView &L, int R, int p, int n, int g, const int *lattice,
                       const T *tw, const T *phihat, T *phi, long long ldphi, int acc, cudaStream_t s,
                       bool sib_minor = false);
bool fft_pg_available(int p, int g);

// F3 on the tensor cores in TF32x3 for a full level (every cluster of the (N/2)^3 grid present,
// N/2 a multiple of 16) with sibling-minor spectra; B: the per-frequency kernel matrices of
// build_hadamard_tc_operand. Returns M2L_EUNSUPPORTED, launching nothing, for other levels.
bool hadamard_tc_eligible(const LevelView &L);
int launch_hadamard_tc(const LevelView &L, int R, int F, const void *B, const float *qhat, float *phihat,
                       int chains, int num_sms, int *status, cudaStream_t s);

// Constant tables (transfer index lookup and the cluster-pair table); once per device.
int ensure_constants(int device);

}  // namespace m2l
