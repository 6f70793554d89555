/*
 * m2l.h - C ABI of the GB300 (sm_103a) multipole-to-local (M2L) library for the 3D Laplace
 * kernel-independent FMM on a uniform octree (arxiv 2408.07436).
 *
 * What one call computes (Sec. 2.2, Eq. 11): for every target box tau at a level and every
 * right-hand side r,
 *        q_tau = (K_tau)^+  sum_{sigma in I_tau}  K_{sigma,tau} q_sigma
 * where q_sigma are the upward-equivalent densities of the source boxes (the multipoles),
 * K_{sigma,tau} is the 3D Laplace kernel 1/(4 pi |x - y|) (Eq. 2) between the downward-check
 * points of tau and the upward-equivalent points of sigma, (K_tau)^+ is the regularised
 * pseudo-inverse of the downward check -> downward equivalent kernel matrix (Eqs. 7-10,
 * alpha = 0), and q_tau are the downward-equivalent densities (the locals).
 * I_tau holds the children of the parent's neighbours that are not adjacent to tau
 * (|I_tau| <= 189; Sec. 2). Two forms are provided:
 *   BLAS-M2L (Sec. 3.1-3.2): SVD-compressed operators C_t = U^T K_t S over the 316
 *            transfer vectors, applied as dense contractions on the GPU.
 *   FFT-M2L  (App. A.1): kernel spectra on the 2p convolution grid, Hadamard products of
 *            the transformed densities, inverse transform.
 *
 * Geometry (stated once, used by every call):
 *   - n = 6(p-1)^2 + 2 surface points per box (App. A.3), the boundary points of a p^3
 *     lattice, lexicographic (x slowest). Upward-equivalent and downward-check surfaces sit
 *     at 1.05 box half-widths, downward-equivalent (and upward-check) at 2.95.
 *   - Boxes at level l are indexed by Morton key (x in the lowest bit of each triple).
 *   - The map is scale free (Laplace homogeneity, Sec. 3.1): K_t scales as 1/w and (K_tau)^+
 *     as w, so no box width is passed and one set of operators serves every level.
 *
 * Data layout of multipoles / locals for one level: [B_l boxes][n_rhs][n], row major,
 * boxes in ascending Morton order (every box of the level unless m2l_set_boxes gave a
 * sparse set). For level = -1 the buffer is levels 2..depth concatenated in ascending order.
 * Element type: double for M2L_PREC_FP64, float for every other precision.
 *
 * Pointers: multipoles and locals may be device pointers (the normal case) or host
 * pointers (pinned or pageable); host buffers are staged through the plan's device
 * workspace with copies on the plan's stream, and the call then returns after the result
 * has been copied back. Device buffers are owned by the caller; the plan owns its operator
 * tables and workspace (device memory allocated by the plan) until m2l_destroy.
 * Device-pointer calls are asynchronous on the plan's stream.
 *
 * Errors: every function that returns int returns M2L_OK (0) or a negative M2L_E* code;
 * functions returning pointers return NULL on error. m2l_last_error() gives a message for
 * the calling thread. Invalid arguments are rejected before any launch. CUDA failures map to
 * M2L_ECUDA. No call aborts, traps or exits the process.
 */
#ifndef M2L_GB300_H
#define M2L_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct m2l_plan_s m2l_plan_t;

enum m2l_kernel_e { M2L_LAPLACE3D = 0 };

enum m2l_status_e {
    M2L_OK = 0,
    M2L_EINVAL = -1,        /* invalid argument or call order */
    M2L_ENOMEM = -2,        /* host or device allocation failed */
    M2L_ECUDA = -3,         /* a CUDA runtime or launch error */
    M2L_ETIMEOUT = -4,      /* a device-side bounded wait ran out */
    M2L_EUNSUPPORTED = -5   /* valid request this build does not implement */
};

enum m2l_option_e {
    M2L_OPT_FORM = 1,        /* M2L_FORM_*; default M2L_FORM_BLAS */
    M2L_OPT_PRECISION = 2,   /* M2L_PREC_*; default M2L_PREC_FP64 */
    M2L_OPT_ACCUMULATE = 3,  /* 0: locals are overwritten (default); 1: locals += M2L result */
    M2L_OPT_OUTPUT = 4,      /* M2L_OUT_*; default M2L_OUT_LOCALS */
    M2L_OPT_TARGET_TOL = 5,  /* accuracy asked of AUTO form / precision: the bits of a double (default
                                1e-6). AUTO keeps the (form, precision) candidates whose stated bound
                                (relative error of the check potential) and rank truncation are within
                                it, times them on the plan's boxes and keeps the fastest, per n_rhs. */
    M2L_OPT_FFT_GRID = 6,    /* convolution grid side: 0 = 2p (default), else 2p-1 <= g <= 2p */
    M2L_OPT_TIMING = 7,      /* 1: record CUDA events around every stage (see m2l_stage_times) */
    M2L_OPT_TC_GROUP = 8,    /* split tensor-core forms: transfer vectors summed in tensor memory before
                                each round-to-nearest FP32 drain, 1..189 (default 1). Larger is faster;
                                the tensor cores' truncating accumulation grows with it */
    M2L_OPT_DIR_TOL = 9,     /* directional recompression of the BLAS operators (Sec. 3.1, Eq. 15):
                                the bits of a double dir_tol >= 0; 0 (default) = off. With
                                dir_tol > 0 each C_t is factored as Ubar_t Vbar'_t^T keeping its
                                singular values >= dir_tol s_0(C_t), and the CUDA-core contraction
                                (FP64, FP32) applies the two factors; the tensor-core forms keep C_t */
    M2L_OPT_TC_CHUNK = 11,   /* split tensor-core forms: bytes of K per pipeline stage of the contraction,
                                32, 64 or 128 (0: 128, the default). Smaller stages fit more of them in
                                shared memory (deeper prefetch of the gathered rows) at more barrier
                                round trips per MMA; the result does not depend on it */
    M2L_OPT_TC_DRAIN = 12,   /* split tensor-core forms: pipeline stages (M2L_OPT_TC_CHUNK bytes of K each)
                                summed in tensor memory before each round-to-nearest FP32 drain into the
                                running sum, within one transfer vector; 0 = whole transfer vectors (see
                                M2L_OPT_TC_GROUP), -1 = the default (2 for TF32x3, 0 for BF16x3). Fewer
                                stages per drain shorten the truncating tensor-core accumulation chains
                                (more accurate) at more drain work */
    M2L_OPT_RANK_AUTO = 13,  /* 1: the library picks the SVD rank threshold of the BLAS form for the target
                                (M2L_OPT_TARGET_TOL), replacing m2l_plan's rank_tol: the coarsest of 1e-3,
                                3e-4, ..., 1e-9 (else full rank) whose truncation error, estimated on the
                                host for one target with all 189 transfer vectors and four density draws
                                (of both signs and of one sign) and taken 1.5 times, plus ten times the
                                directional threshold, fits in the target beside the precision's stated bound
                                (m2l_stated_bound). With M2L_OPT_DIR_TOL set, the directional threshold
                                follows at a tenth of it. Resolved, and the plan's operators rebuilt, at
                                the first apply or M2L_Q_FORM / M2L_Q_PRECISION query per target; read the
                                result with M2L_Q_RANK_TOL. 0 (default): rank_tol as given */
    M2L_OPT_SVD = 14,        /* SVD of the stacked operators K_fat, K_thin (Eqs. 12-13) for a truncated rank:
                                0 exact (default: tall-skinny QR, then one-sided Jacobi), 1 one-shot
                                randomised (Sec. 3.1: Gaussian sketch with ten oversamples, no power
                                iterations, its width grown from 0.6 n + 10 until the sketch's smallest
                                singular value falls below rank_tol times the largest). Setup only; the
                                rank tuner (M2L_OPT_RANK_AUTO) estimates with the exact bases */
    M2L_OPT_HADAMARD_CHAINS = 15, /* FFT form in TF32x3: partial sums per tile of the tensor-core Hadamard
                                products, 1, 2 or 4 (0: 4, the default). Each sums the products of a
                                fixed subset of the 26 source-cluster directions in tensor memory (every
                                subset holds an in-plane direction); the epilogue adds them in FP32 with
                                round-to-nearest. More partial sums shorten the truncating tensor-core
                                accumulation chains (more accurate); the result is otherwise the same */
    M2L_OPT_CHECK_ORDER = 10 /* order p_c of the downward check surface, p <= p_c <= 16 (0: p, the
                                default). p_c > p gives n_c = 6(p_c-1)^2+2 check points for the n
                                equivalent points (the BLAS tables' P_c > P_e): K_t and the
                                pseudo-inverse become n_c x n, U is n_c x k_c, C_t is k_c x k.
                                BLAS form in FP64 or FP32 only (the FFT form needs one grid, the
                                tensor-core contraction a square C_t); check potentials written
                                with M2L_OUT_CHECK_POTENTIAL then have n_c values per row */
};

/* Stages of one application, as indexed by m2l_stage_times. */
enum m2l_stage_e {
    M2L_STAGE_COMPRESS = 0,    /* B1: q~ = S^T q                           (Sec. 3.2 step 2) */
    M2L_STAGE_CONTRACT = 1,    /* B2: phi~ = sum_t C_t q~, gathered        (Sec. 3.2 steps 3-5) */
    M2L_STAGE_EXPAND = 2,      /* B3: locals = V_eps Ut_eps U phi~          (Sec. 3.2 step 5, Eq. 9) */
    M2L_STAGE_FFT_FORWARD = 3, /* F1+F2: embed and transform               (App. A.1 step 2) */
    M2L_STAGE_HADAMARD = 4,    /* F3: Hadamard products over I_tau          (App. A.1 step 4) */
    M2L_STAGE_FFT_INVERSE = 5, /* F4+F5: inverse transform, check surface   (App. A.1 step 6) */
    M2L_STAGE_PINV = 6,        /* F6: locals = V_eps Ut_eps phi             (Eq. 9) */
    M2L_NUM_STAGES = 7
};

enum m2l_form_e { M2L_FORM_AUTO = 0, M2L_FORM_BLAS = 1, M2L_FORM_FFT = 2 };

enum m2l_precision_e {
    M2L_PREC_AUTO = -1,   /* chosen per (p, n_rhs, M2L_OPT_TARGET_TOL) by the library */
    M2L_PREC_FP64 = 0,    /* FP64 data and arithmetic */
    M2L_PREC_FP32 = 1,    /* FP32 data and arithmetic (CUDA cores) */
    M2L_PREC_TF32X3 = 2,  /* FP32 data; BLAS contractions as three TF32 tensor-core products. FFT form:
                             FP32 transforms; the Hadamard products of full levels ((N/2)^3 clusters,
                             N/2 a multiple of 16) on the tensor cores as split products accurate to
                             FP32 rounding (three BF16 pieces per operand, six products), and both
                             factors of the pseudo-inverse on the tensor cores exactly (BF16 integer
                             slices; the second one when the rank is at most 256) */
    M2L_PREC_BF16X3 = 3   /* FP32 data; BLAS contractions as three BF16 tensor-core products */
};

enum m2l_output_e {
    M2L_OUT_LOCALS = 0,          /* downward-equivalent densities q_tau (Eq. 11) */
    M2L_OUT_CHECK_POTENTIAL = 1  /* the check potential sum_{sigma} K_{sigma,tau} q_sigma before
                                    the pseudo-inverse, in units of a box of width 1 */
};

enum m2l_query_e {
    M2L_Q_N = 1,          /* surface points per box, n */
    M2L_Q_RANK = 2,       /* SVD rank k of the BLAS form (n at full rank) */
    M2L_Q_BOXES = 3,      /* boxes at `level` (after m2l_set_boxes) */
    M2L_Q_PAIRS = 4,      /* (target, source) M2L pairs at `level`; level -1: all levels */
    M2L_Q_GRID = 5,       /* convolution grid side g of the FFT form */
    M2L_Q_FREQS = 6,      /* complex half-spectrum length g*g*(g/2+1) */
    M2L_Q_PINV_RANK = 7,  /* singular values kept by the pseudo-inverse */
    M2L_Q_ROWS = 8,       /* boxes summed over levels 2..depth */
    M2L_Q_FORM = 9,       /* form the next apply with n_rhs = `level` (>= 1) will run; resolves AUTO */
    M2L_Q_PRECISION = 10, /* precision of that apply (so the caller knows the element type) */
    M2L_Q_LAUNCHES = 11,  /* kernels launched by the last apply */
    M2L_Q_DEVICE_STATUS = 12, /* waits for the plan's stream, reads the device status word into *out
                                (0, or the m2l_wait_e code of the first bounded wait that ran out
                                since the last query) and clears it; returns M2L_ETIMEOUT when it
                                was nonzero: results written since the last query are invalid */
    M2L_Q_CONTRACT_FLOPS = 13, /* algorithmic flops of the BLAS contraction for one right-hand side at
                                  `level` (-1: all levels): 2 k^2 per pair, or 4 k k_t with
                                  M2L_OPT_DIR_TOL in a precision that applies the factors (FP64,
                                  FP32, AUTO), rounded to an integer */
    M2L_Q_DIR_RANK_SUM = 14,   /* sum of k_t over the 316 transfer vectors (0 when M2L_OPT_DIR_TOL is 0) */
    M2L_Q_NC = 15,             /* check points per box, n_c (n unless M2L_OPT_CHECK_ORDER > p) */
    M2L_Q_RANK_CHECK = 16,     /* rank k_c of the check-side basis U (k unless M2L_OPT_CHECK_ORDER > p) */
    M2L_Q_RANK_TOL = 17        /* the plan's current rank threshold, as the bits of a double (the one
                                  m2l_plan was given, or the one M2L_OPT_RANK_AUTO chose) */
};

/* Where a bounded device wait ran out (the value of M2L_Q_DEVICE_STATUS). Every wait of a kernel
 * that waits on other warps (the tensor-core contraction) polls at most a fixed number of times,
 * then records its code, raises the CTA's abort flag, lets the copies and MMAs it issued finish
 * and returns: no trap, no hang, and the CUDA context stays usable. */
enum m2l_wait_e {
    M2L_WAIT_GATHER = 1,     /* source-row producers waiting for a free pipeline stage */
    M2L_WAIT_TMA = 2,        /* operator (TMA) producer waiting for a free pipeline stage */
    M2L_WAIT_ACC_FREE = 3,   /* MMA issuer waiting for a drained tensor-memory accumulator */
    M2L_WAIT_OPERANDS = 4,   /* MMA issuer waiting for a filled pipeline stage */
    M2L_WAIT_ACC_READY = 5,  /* drain warps waiting for a finished partial sum */
    M2L_WAIT_SELFTEST = 6    /* m2l_selftest_watchdog */
};

/* Build a plan (host, FP64; arxiv 2408.07436 Sec. 3.1 for the BLAS operators and App. A.1
 * step 1 for the kernel spectra). depth in [2, 8]; p in [2, 16]; kernel = M2L_LAPLACE3D.
 * rank_tol <= 0: full rank (k = n, exact). rank_tol > 0: keep the singular values of the
 * stacked operators K_fat and K_thin (Eqs. 12-13) with s_i / s_0 >= rank_tol.
 * Operator tables are built lazily on the first apply that needs them.
 * Returns NULL on error (see m2l_last_error). Uses the current CUDA device. */
m2l_plan_t *m2l_plan(int depth, int p, int kernel, double rank_tol);

/* Apply M2L (Eq. 11) at `level` in [2, depth], or at every level 2..depth when level == -1.
 * multipoles: [rows][n_rhs][n] (see the layout above), read only.
 * locals:     same shape; overwritten, or accumulated when M2L_OPT_ACCUMULATE is 1; with
 *             M2L_OPT_OUTPUT = M2L_OUT_CHECK_POTENTIAL it receives the check potentials.
 * n_rhs >= 1. The two buffers must not overlap.
 * Returns M2L_OK, M2L_EINVAL (bad level / n_rhs / NULL / overlapping buffers),
 * M2L_EUNSUPPORTED (precision not offered by the chosen form), M2L_ENOMEM or M2L_ECUDA. */
int m2l_apply(m2l_plan_t *plan, const void *multipoles, void *locals, int level, int n_rhs);

/* Release the plan and its device memory. NULL-safe. Synchronises the plan's stream. */
void m2l_destroy(m2l_plan_t *plan);

/* Message for the last error on the calling thread ("" if none). Valid until the next call. */
const char *m2l_last_error(void);

/* Set an option (enum m2l_option_e). Takes effect at the next apply. M2L_EINVAL on an unknown
 * key or value. */
int m2l_set_option(m2l_plan_t *plan, int key, long long value);

/* Stream the plan launches on (a cudaStream_t; NULL = legacy default stream). */
int m2l_set_stream(m2l_plan_t *plan, void *stream);

/* Restrict `level` to the non-empty boxes listed by `keys` (n strictly ascending Morton keys
 * < 8^level, host memory, copied). Empty boxes are neither sources nor targets (the pruning of
 * empty branches, Sec. 2.1). n == 8^level with keys == NULL restores the full level. */
int m2l_set_boxes(m2l_plan_t *plan, int level, const uint64_t *keys, long long n);

/* Apply several independent plans (uneven FMM instances) with DEVICE buffers, every level of
 * each (level = -1 semantics), in one pass on the first plan's stream. Instances whose plans
 * resolve to the same (p, form, precision, rank) form one group: the BLAS contraction of a group
 * is ONE launch over the tiles of all its instances (the compress/expand GEMMs and the FFT stages
 * are launched per instance). The whole pass is captured once in a CUDA graph (on a stream the
 * first plan owns) and replayed on later calls with the same plans, buffers, n_rhs, options and
 * box sets; anything else re-captures. Plans may not repeat; all belong to one device.
 * plans[i], multipoles[i], locals[i], n_rhs[i] as for m2l_apply (M2L_OPT_TIMING is ignored).
 * Returns M2L_OK, M2L_EINVAL, M2L_EUNSUPPORTED, M2L_ENOMEM or M2L_ECUDA. */
int m2l_apply_batch(m2l_plan_t *const *plans, int n_inst, const void *const *multipoles,
                    void *const *locals, const int *n_rhs);

/* The relative error bound the library states for a (form, precision) at order p, the one
 * M2L_FORM_AUTO / M2L_PREC_AUTO compare with M2L_OPT_TARGET_TOL: Eq. 16 on the check potential
 * (and on the locals through the check potential they reproduce) against the FP64 definition,
 * before any rank truncation. Measured per p = 4..10 over uniform, signed, Gaussian and physical
 * (P2M + M2M) multipoles with a margin of at least 1.8. form: M2L_FORM_BLAS or M2L_FORM_FFT;
 * precision: M2L_PREC_FP64..M2L_PREC_BF16X3 (the FFT form offers FP64, FP32 and TF32x3).
 * Returns M2L_OK, or M2L_EINVAL for a NULL out, a bad form, precision or p outside [2, 16]. */
int m2l_stated_bound(int form, int precision, int p, double *bound);

/* Integer facts about a plan (enum m2l_query_e). `level` is used by M2L_Q_BOXES/PAIRS. */
int m2l_query(const m2l_plan_t *plan, int what, int level, long long *out);

/* Device time in milliseconds of every stage of the last application made with
 * M2L_OPT_TIMING = 1, measured with CUDA events on the plan's stream (waits for them).
 * ms must hold M2L_NUM_STAGES doubles; stages that did not run read 0. Also reports the
 * number of kernel launches of each stage in `launches` (may be NULL). */
int m2l_stage_times(m2l_plan_t *plan, double *ms, long long *launches);

/* m2l_apply without allocation. The paper has no counterpart; this entry point is for callers
 * that cannot allocate device memory at the time they apply M2L: applications that hand all
 * device memory to their own pool or caching allocator up front (a cudaMalloc would then fail or
 * fragment it), and latency-bounded loops in which the implicit device synchronisation of
 * cudaMalloc / cudaFree is not acceptable.
 *
 * It computes what m2l_apply computes for the BLAS form in FP64 at ONE level (honouring
 * M2L_OPT_OUTPUT and M2L_OPT_ACCUMULATE) and calls no cudaMalloc, no cudaFree and no allocating
 * library routine. Its scratch (compressed multipoles, compressed check potentials and the
 * pseudo-inverse intermediate) is one static device array of 4,194,304 doubles (32 MiB) that
 * every GPU which loads this library holds until the process exits. A request needs
 * (B_l n_rhs + 1) k_pad + B_l n_rhs (k_pad + r_pad) doubles (each part rounded up to 32);
 * larger requests return M2L_EINVAL with the size in the message (use m2l_apply instead).
 *
 * multipoles, locals: DEVICE pointers, FP64, layout [B_l][n_rhs][n] of `level`.
 * Preconditions: the plan's FP64 BLAS operators and box tables are already on the device (one
 * earlier m2l_apply of this plan with M2L_FORM_BLAS and M2L_PREC_FP64, after the last
 * m2l_set_boxes, uploads them); otherwise M2L_EINVAL.
 * Device: the plan's device must be the current device (otherwise M2L_EINVAL, nothing runs).
 * Set-up: the first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and uploads a small constant table, once per device even when several host threads make that
 * first call together; make that first call before any stream capture.
 * Sharing: every call uses the same array and leaves the last call's contents in it (the one
 * part that must start at zero is cleared on every call). Calls that overlap on the GPU (other
 * streams, other plans, other host threads) race on the array and give wrong results.
 * Asynchronous on the plan's stream. Returns M2L_OK, M2L_EINVAL or M2L_ECUDA. */
int m2l_apply_noalloc(m2l_plan_t *plan, const double *multipoles, double *locals, int level, int n_rhs);

/* Exercise the device watchdog: one thread waits, with the same bounded-wait code the
 * contraction uses, on a barrier that nothing completes, for at most `polls` polls (1 <= polls <=
 * 2^24, the limit of the contraction's own waits), then
 * records M2L_WAIT_SELFTEST in the plan's status word and returns. No copy or MMA is in flight,
 * so nothing else is affected. Asynchronous on the plan's stream; read the outcome with
 * m2l_query(M2L_Q_DEVICE_STATUS), which then returns M2L_ETIMEOUT. The paper has no counterpart.
 * Returns M2L_OK, M2L_EINVAL (no GPU plan, polls out of range) or M2L_ECUDA. */
int m2l_selftest_watchdog(m2l_plan_t *plan, long long polls);

/* ---------------------------------------------------------------------------------------------
 * A whole FMM around the M2L plan: the other stages of the kiFMM (Sec. 2.1-2.2, Fig. 2), namely
 * P2M, M2M, L2L, L2P and the near-field P2P, on the GPU, with M2L through an m2l plan on the
 * occupied boxes of every level. It turns M2L into potentials that can be compared with direct
 * summation (Eq. 16). FP64, one charge vector; check and equivalent orders equal. The upward and
 * downward operators use the surfaces and the pseudo-inverse rule of M2L; like M2L they are
 * scale free (Laplace kernel of degree -1) and built once at unit width.
 */
typedef struct m2l_fmm_s m2l_fmm_t;

/* points: HOST pointer, n_points x 3 (x, y, z) inside [origin, origin + width)^3 (origin: 3
 * doubles, NULL for 0). depth in [2, 8] (leaves are the boxes of that level), p in [2, 16],
 * rank_tol as for m2l_plan. Sorts the points into leaves and builds the box lists, neighbour
 * lists, operators and the inner M2L plan. NULL on error (m2l_last_error). */
m2l_fmm_t *m2l_fmm_plan(const double *points, long long n_points, int depth, int p, double rank_tol,
                        const double *origin, double width);

/* Set an option of the inner M2L plan (M2L_OPT_FORM, M2L_OPT_DIR_TOL, M2L_OPT_TC_GROUP ...).
 * M2L_OPT_PRECISION other than FP64 and M2L_OPT_CHECK_ORDER are refused (M2L_EINVAL). */
int m2l_fmm_set_m2l_option(m2l_fmm_t *fmm, int key, long long value);

/* potentials[i] = sum over j != i of charges[j] / (4 pi |x_i - x_j|), by the FMM: P2M at the
 * leaves, M2M up to level 2, M2L at levels 2..depth, L2L down, L2P and P2P at the leaves.
 * charges, potentials: n_points doubles each, HOST or DEVICE pointers, in the order the points
 * were given. Synchronous. Returns M2L_OK, M2L_EINVAL, M2L_ENOMEM or M2L_ECUDA. */
int m2l_fmm_evaluate(m2l_fmm_t *fmm, const double *charges, double *potentials);

/* The inner M2L plan (owned by the FMM; valid until m2l_fmm_destroy), for queries. */
m2l_plan_t *m2l_fmm_m2l_plan(m2l_fmm_t *fmm);

void m2l_fmm_destroy(m2l_fmm_t *fmm); /* NULL-safe */

/* Copy a plan operator to host memory (FP64), for tests and inspection:
 * which = 0: U (n_c x k_c), 1: S (n x k), 2: C_t (316 x k_c x k), 3: singular values of K_fat
 *         (n_c), 4: pseudo-inverse factor V_eps (n x r), 5: Ut_eps = Sigma_eps^-1 U_eps^T (r x n_c),
 *         6: the directional products Ubar_t Vbar'_t^T (316 x k_c x k; needs M2L_OPT_DIR_TOL > 0).
 * (n_c = n and k_c = k unless M2L_OPT_CHECK_ORDER > p.)
 * *count receives the number of doubles; dst may be NULL to query the size. */
int m2l_get_operator(m2l_plan_t *plan, int which, double *dst, long long *count);

#ifdef __cplusplus
}
#endif

#endif /* M2L_GB300_H */
