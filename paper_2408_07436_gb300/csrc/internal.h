// Internal structures of the M2L library: the plan (host FP64 operators, device tables and
// workspace) and the helpers shared by the host code and the launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/m2l.h"

namespace m2l {

constexpr int kNumTransfer = 316;   // |T| = 7^3 - 3^3 (Sec. 3.1)
constexpr int kPerOctant = 189;     // far pairs per target octant, 6^3 - 3^3 (Sec. 3.1)
constexpr int kDirections = 26;     // source clusters around a target cluster (App. A.1)
constexpr double kAlphaInner = 1.05;  // upward-equivalent / downward-check radius (box half-widths)
constexpr double kAlphaOuter = 2.95;  // downward-equivalent / upward-check radius
constexpr int kMaxDepth = 8;

void set_error(const char *fmt, ...);
void clear_error();

// Index of transfer vector (x, y, z) in [-3,3]^3 \ [-1,1]^3, enumerated x slowest then y, z.
int transfer_index(int x, int y, int z);
void transfer_vector(int idx, int &x, int &y, int &z);

// Host operators (FP64). They depend on the kernel, the orders and the thresholds, never on the
// tree, so plans alive at the same time with the same parameters (the instances of a batch, the
// autotuner's proxy plans) share one read-only build (see plan.cpp).
struct PinvOps {                              // Eqs. 7-10, two-factor storage
    int r = 0, r32 = 0;                       // kept singular values: alpha = 0 and alpha = 1e-9
    std::vector<double> Veps, Uteps;          // [n][r], [r][nc]
    std::vector<double> Veps32, Uteps32;      // the factors used by single-precision paths
};
struct BlasOps {                              // Sec. 3.1-3.2 compression
    int k = 0, kc = 0;                        // ranks of the equivalent (S) and check (U) sides
    std::vector<double> U, S, C, s_fat, s_thin;  // U: nc x kc, S: n x k (row-major); C: 316 x kc x k
    std::vector<double> Aop, Aop32;           // [r][kc] = Uteps * U (and with the alpha = 1e-9 factor)
};
struct DirOps {                               // Eq. 15 factors, packed as on the device
    std::vector<int> kt;                      // [316] k_t
    std::vector<double> ub, vt;
    std::vector<int> meta;                    // [316][4]
    int kt8_max = 0;
};
struct FftOps {                               // App. A.1 kernel spectra
    int g = 0, F = 0;
    std::vector<double> Khat;                 // [316][F][2]
    std::vector<double> twiddle;              // [g][2]
};

struct LevelSet {
    bool dense = true;
    std::vector<uint64_t> keys;  // sorted Morton keys when sparse
    long long nboxes = 0;
};

// Device copy of the operators in one arithmetic precision.
// A matrix W (O x K) as 4 BF16 integer slices of `beta` bits under a power-of-two scale per row,
// for the exact sliced tensor-core products (pinv_tc.cu).
struct SlicedOp {
    void *sl = nullptr;          // [4][O_pad][K_pad] BF16
    void *scale = nullptr;       // [O_pad] float, 2^e_w
    int K = 0, kp = 0, O = 0, opad = 0, beta = 8;  // kp = 0: not built
    alignas(64) unsigned char map[128] = {};        // TMA map (CUtensorMap) of the slices
};

struct DevOps {
    bool ready = false;
    int elt = 8;                 // bytes per real (8: double, 4: float)
    // BLAS form (row-major, inner dimension padded to kp / rp)
    void *St = nullptr;          // [kp][np_]   S^T
    void *C = nullptr;           // [316][kp][kp] C_t
    void *A = nullptr;           // [rp][kp]    Ut_eps * U
    void *V = nullptr;           // [n][rp]     V_eps
    void *Vlo = nullptr;         // [n][rp]     V_eps - fl32(V_eps) (single-precision plans)
    void *Uc = nullptr;          // [n][kp]     U (check-potential output)
    void *C_hi = nullptr, *C_lo = nullptr;  // split C_t for the tensor-core forms
    void *Ub = nullptr, *Vt = nullptr;      // directional factors (Eq. 15): Ubar_t [k_pad][k_t8],
                                            // Vbar'_t^T [k_t8][k_pad], concatenated over t
    void *dir_meta = nullptr;               // [316] int4: Ub offset, Vt offset, k_t, k_t8
    alignas(64) unsigned char tmap[3][2][128] = {};  // TMA maps (CUtensorMap) of C_hi and C_lo per stage
                                                     // width of the tensor-core contraction (32, 64, 128 B)
    // FFT form
    void *Khat = nullptr;        // [316+1][F] complex kernel spectra (last row zero)
    void *Ut = nullptr;          // [rp][np_]   Ut_eps
    void *tw = nullptr;          // [g] complex twiddles exp(-2 pi i m / g)
    void *Bhad = nullptr;        // TF32x3 FFT form: [F][26] kernel matrices of the tensor-core Hadamard
    SlicedOp Us, Vs;             // TF32x3 FFT form: Ut_eps and V_eps as BF16 integer slices
    SlicedOp Ss, As, Ucs;        // split BLAS forms: S^T, Ut_eps U and U as BF16 integer slices
};

struct LevelDev {
    int level = 0;
    long long nboxes = 0, base = 0;     // compact boxes and their first global row
    long long nclusters = 0, cbase = 0; // non-empty parents (FFT clusters) and first global cluster
    int *slot = nullptr;                // [8^l] grid (x + N(y + N z)) -> compact box or -1
    uint32_t *xyz = nullptr;            // [nboxes] packed x | y << 10 | z << 20
    int *perm = nullptr;                // [nboxes] compact boxes sorted by (octant, Morton)
    long long oct_start[9] = {0};       // segment of each octant in perm
    int *cslot = nullptr;               // [8^(l-1)] parent grid -> cluster or -1
    uint32_t *cxyz = nullptr;           // [nclusters] packed parent coordinates
    int *cchild = nullptr;              // [nclusters][8] compact child box or -1
    int *cperm = nullptr;               // [nclusters] clusters by domain-boundary class, Morton inside
    long long pairs = 0;                // M2L (target, source) pairs
    // host copies (built without a GPU; uploaded on first use)
    std::vector<int> h_slot, h_perm, h_cslot, h_cchild, h_cperm;
    std::vector<uint32_t> h_xyz, h_cxyz;
    bool on_device = false;
};

struct Workspace {
    void *buf = nullptr;
    size_t bytes = 0;
};

// Device level views and contraction tiles of the last group of instances run with this plan
// as owner, with the key they were built for.
struct ExecCache {
    std::vector<long long> key;
    void *levels = nullptr;
    void *tiles = nullptr;
    void *tvl = nullptr;               // transfer vector lists of the tiles
    long long ntiles = 0;
    long long nvectors = 0;            // (tile, transfer vector) products the contraction runs
};

// The CUDA graph of the last batch pass led by this plan and the arguments it was captured for.
struct BatchGraph {
    std::vector<long long> sig;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture_stream = nullptr;
    long long launches = 0;
};

}  // namespace m2l

struct m2l_plan_s {
    int depth = 0, p = 0, n = 0, kernel = 0;
    double rank_tol = 0.0;
    // options
    int form = M2L_FORM_BLAS, precision = M2L_PREC_FP64, accumulate = 0, output = M2L_OUT_LOCALS;
    double target_tol = 1e-6;
    int fft_grid_opt = 0;
    int tc_group = 1;                           // transfer vectors per tensor-memory partial sum
    int tc_chunk = 0;                           // bytes of K per tensor-core pipeline stage (0: default)
    int tc_drain = -1;                          // K stages per tensor-core partial sum (-1: default)
    int had_chains = 0;                         // partial sums of the tensor-core Hadamard (0: default)
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 148;
    // geometry
    std::vector<int> lattice;                 // n x 3: equivalent surfaces, order p
    int pc = 0, nc = 0;                       // check surface order (M2L_OPT_CHECK_ORDER) and points
    std::vector<int> lattice_c;               // nc x 3: the downward check surface
    int *lattice_dev = nullptr;               // packed a << 16 | b << 8 | c
    m2l::LevelSet levels[m2l::kMaxDepth + 1];
    // host operators (FP64), shared read-only with other plans of the same parameters; null until
    // built, reset by the options that change them
    std::shared_ptr<const m2l::PinvOps> pinv;
    std::shared_ptr<const m2l::BlasOps> blas;
    std::shared_ptr<const m2l::DirOps> dirop;
    std::shared_ptr<const m2l::FftOps> fft;
    int k = 0, kp = 0, r = 0, rp = 0, np_ = 0;    // k: rank of the equivalent side (S), padded kp
    int kc = 0, kcp = 0;                          // rank of the check side (U), padded; k unless pc > p
    int r32 = 0;                                  // singular values kept with Eq. 10's alpha = 1e-9
    double dir_tol = 0.0;                         // directional recompression threshold (0: off)
    int dir_kt8_max = 0;
    int g = 0, F = 0;
    // device
    m2l::DevOps dev[4];                           // by precision (FP64, FP32, TF32X3, BF16X3 share FP32 data)
    bool levels_dirty = true;
    m2l::LevelDev ldev[m2l::kMaxDepth + 1];
    long long total_rows = 0, total_clusters = 0;
    m2l::Workspace ws, spec, stage_in, stage_out;   // spec: FFT spectra (one level, a chunk of rhs)
    m2l::Workspace batch_ws;                        // workspace shared by the groups of a batch it leads
    size_t mem_budget = 0;                          // bytes one workspace may take (1/4 of the GPU)
    m2l::ExecCache exec;
    m2l::BatchGraph batch_graph;
    long long levels_version = 0;                  // bumped whenever a box set changes
    int capturing = 0;                             // inside a batch capture: no timing events
    struct Tuned { int R; double tol; int form_opt, prec_opt; long long levels_version; int form, precision; double rank; };
    int rank_auto = 0;                             // M2L_OPT_RANK_AUTO
    int svd_mode = 0;                              // M2L_OPT_SVD: 0 exact, 1 one-shot randomised
    std::shared_ptr<const void> svd_hold;          // the SVD bases the rank tuner read (kept while the plan
                                                   // lives, so plans of one order share one SVD)
    double rank_auto_tol = -1.0;                   // target the rank was last chosen for (explicit form)
    std::vector<Tuned> tuned;                      // autotuner decisions
    long long launches = 0;
    int *dev_status = nullptr;                     // device status word written by bounded waits
    // stage timing (M2L_OPT_TIMING)
    int timing = 0;
    struct StageEvent { int stage; cudaEvent_t a, b; long long launches; };
    std::vector<StageEvent> events;   // recorded by the last apply
    std::vector<cudaEvent_t> event_pool;
    size_t events_used = 0;
};

namespace m2l {
// plan.cpp
int build_pinv(m2l_plan_t *pl);
int build_blas_host(m2l_plan_t *pl);
int build_directional(m2l_plan_t *pl);
// Host estimate of the relative check-potential error that truncation at (rank_tol, dir_tol) adds
// (plan.cpp): one target with its 189 transfer vectors, four seeded density draws, the largest.
double truncation_estimate(m2l_plan_t *pl, double rank_tol, double dir_tol);
void release_operators(m2l_plan_t *pl);
// Pseudo-inverse factors of Eq. 10 from the SVD of an m x n (m >= n) matrix, U, V column-major:
// Veps [n][r], Uteps [r][m] with the singular values above (alpha + max(m, n) eps) s_0.
void pinv_truncation(int m, int n, const std::vector<double> &U, const std::vector<double> &s,
                     const std::vector<double> &V, double alpha, int &r, std::vector<double> &Veps,
                     std::vector<double> &Uteps);
int contract_flops(m2l_plan_t *pl, int level, double *out);
int build_fft_host(m2l_plan_t *pl);
int build_level_tables(m2l_plan_t *pl);     // host tables and pair counts
int upload_level_tables(m2l_plan_t *pl);    // device copies
int upload_ops(m2l_plan_t *pl, int precision, int form);
void free_device(m2l_plan_t *pl);
// autotune.cpp
int resolve_form(const m2l_plan_t *pl, int R, int *form, int *precision);
double stated_bound(int form, int precision, int p);
void set_rank(m2l_plan_t *pl, double rank_tol);
// apply.cu
int prepare_plan(m2l_plan_t *pl, int form, int precision);
size_t workspace_estimate(const m2l_plan_t *pl, int form, int precision, int R);
int apply_batch(m2l_plan_t *const *plans, int n_inst, const void *const *q, void *const *L, const int *R);
void free_exec(m2l_plan_t *pl);
void stage_begin(m2l_plan_t *pl, int stage);
void stage_end(m2l_plan_t *pl, long long launches);
int apply_device(m2l_plan_t *pl, const void *q, void *L, int level, int nrhs);
// pinv_tc.cu: exact sliced products on the tensor cores (4 BF16 integer slices per operand, 10
// slice pairs): out[row][0..O) (+)= W X[row] for `rows` rows of X (row stride ldx, W.K values),
// output row stride ldo, O a multiple of 4 and at most W's padded rows; `ws` holds
// sliced_workspace(rows, W.kp) bytes. Used for both factors of F6 in the TF32x3 FFT form.
int build_sliced_operand(const std::vector<double> &W, int O, int K, int beta, SlicedOp &op);
int build_blas_sliced_operands(m2l_plan_t *pl, DevOps &D);
int sliced_kmax(const m2l_plan_t *pl);
size_t sliced_workspace(long long rows, int Kp);
bool sliced_usable(const SlicedOp &W, long long ldo, int O, const float *out);
int launch_sliced(const m2l_plan_t *pl, const SlicedOp &W, const float *X, long long ldx, long long rows, float *out,
                  long long ldo, int O, int acc, void *ws, cudaStream_t s);
}  // namespace m2l
