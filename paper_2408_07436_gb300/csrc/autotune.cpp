// Choice of form and precision for M2L_FORM_AUTO / M2L_PREC_AUTO, per (p, n_rhs, target tolerance).
//
// A (form, precision) candidate is eligible when its stated relative error bound for the plan's
// order (Eq. 16 on the check potential, measured per p = 4..10, see stated_bound and the GPU
// parity tests) and the truncation of the plan's rank are both at most the target. Eligible
// candidates are timed with the library's scratch data (the arithmetic does not depend on the
// values) on a proxy plan with the same order, rank and options and full levels up to depth
// min(depth, 4): both forms cost a fixed amount per (target, source) pair, so their ratio carries
// over to deeper trees. FP64 candidates are timed only when no reduced-precision candidate is
// eligible: on this GPU the FP64 units run at about one sixtieth of the FP32 rate. Decisions are
// cached per plan and process-wide per (device, p, n_rhs, rank_tol, target, requested form and
// precision), so many instances of one kind tune once.
#include <cuda_runtime.h>

#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"

namespace m2l {

int prepare_plan(m2l_plan_t *pl, int form, int precision);

// Stated bounds: relative L2 error (Eq. 16) of the check potential, and of the locals measured
// through the check potential they reproduce, against the FP64 definition. Largest values
// measured on depth-3 trees over densities uniform in [0,1), uniform in [-1,1], Gaussian, and
// physical multipoles (P2M + M2M of a seeded 40,000-point cloud), per order (in brackets: p = 4,
// 6, 8, 10; the tensor-core forms at p >= 8 with rank 1e-7, against the compressed form), with
// at least a factor 1.8 of margin.
double stated_bound(int form, int precision, int p) {
    if (precision == M2L_PREC_FP64) {
        // check potentials agree to rounding (1.4e-14). Locals are defined only up to the backward
        // error of the pseudo-inverse solve, n eps ||K_tau|| ||q|| / ||K_tau q||: two correct
        // solvers differ by up to 3.6e-12 in the check norm at p = 10 (4e-12 at p = 8 for signed
        // densities), 1.7e-13 at p = 6
        return p >= 8 ? 1e-11 : 1e-12;
    }
    if (form == M2L_FORM_FFT) return 1e-6;   // FP32 FFT (3.9e-7, 3.9e-7, 5.1e-7, 5.3e-7); TF32x3 FFT, whose
                                             // tensor-core levels measured 1.6e-7, 2.2e-7, 2.6e-7 (p = 4..8)
    if (precision == M2L_PREC_TF32X3)          // FP32 accumulation of 22-bit pieces
        return p <= 4 ? 1e-6 : 3e-6;           // (5.2e-7, 1.4e-6, 1.1e-6, 1.3e-6)
    if (precision == M2L_PREC_FP32)            // FP32 CUDA-core contraction
        return p <= 4 ? 3e-6 : 6e-6;           // (1.5e-6, 3.1e-6, 2.4e-6, 1.9e-6)
    return 1.2e-5;                             // BF16x3 (5.5e-6, 5.3e-6, 5.0e-6, 5.9e-6)
}

// Set a plan's rank threshold (and, when it uses directional factors, their threshold at a tenth
// of it), dropping every operator built for the old one.
void set_rank(m2l_plan_t *pl, double rank_tol) {
    if (rank_tol == pl->rank_tol) return;
    pl->rank_tol = rank_tol;
    if (pl->dir_tol > 0) pl->dir_tol = rank_tol > 0 ? rank_tol / 10 : 0.0;
    pl->blas.reset();
    pl->dirop.reset();
    release_operators(pl);
}

// Rank thresholds the tuner tries, coarsest first; full rank (0) after the last.
static const double kRankLadder[] = {1e-3, 3e-4, 1e-4, 3e-5, 1e-5, 3e-6, 1e-6, 3e-7, 1e-7, 3e-8, 1e-8, 3e-9, 1e-9};

// With M2L_OPT_RANK_AUTO: the coarsest rank threshold whose truncation, estimated on the host
// (truncation_estimate, times 1.5 for the spread across boxes and levels), fits in the target
// beside the precision's stated bound; -1 when none does.
static double choose_rank(m2l_plan_t *pl, int prec) {
    const double budget = pl->target_tol - stated_bound(M2L_FORM_BLAS, prec, pl->p);
    if (budget <= 0) return -1.0;
    const bool dir = pl->dir_tol > 0 && (prec == M2L_PREC_FP64 || prec == M2L_PREC_FP32);
    for (double r : kRankLadder) {
        if (1.5 * truncation_estimate(pl, r, dir ? r / 10 : 0.0) <= budget) return r;
    }
    return 0.0;
}

static bool eligible(const m2l_plan_t *pl, int form, int prec) {
    if (form == M2L_FORM_FFT && prec == M2L_PREC_BF16X3) return false;
    // a check order above p: BLAS form on CUDA cores only
    if (pl->pc != pl->p && (form == M2L_FORM_FFT || prec == M2L_PREC_TF32X3 || prec == M2L_PREC_BF16X3)) return false;
    double bound = stated_bound(form, prec, pl->p);
    if (form == M2L_FORM_BLAS && pl->rank_tol > 0 && !pl->rank_auto) bound = std::max(bound, pl->rank_tol);
    if (bound > pl->target_tol) return false;
    if (form == M2L_FORM_BLAS && (prec == M2L_PREC_TF32X3 || prec == M2L_PREC_BF16X3)) {
        // the tensor-core contraction holds k_pad <= 256 columns
        if ((pl->blas ? pl->kp : 0) > 256) return false;
    }
    return true;
}

static int time_candidate(m2l_plan_t *pl, int form, int prec, int R, float *ms) {
    int rc = prepare_plan(pl, form, prec);
    if (rc) return rc;
    if (form == M2L_FORM_BLAS && (prec == M2L_PREC_TF32X3 || prec == M2L_PREC_BF16X3) && pl->kp > 256)
        return M2L_EUNSUPPORTED;
    const size_t elt = prec == M2L_PREC_FP64 ? 8 : 4;
    long long rows = 0;
    for (int l = 2; l <= pl->depth; ++l) rows += pl->ldev[l].nboxes;
    const size_t bytes = (size_t)rows * R * pl->n * elt;
    void *q = nullptr, *L = nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess || cudaMalloc(&L, bytes) != cudaSuccess) {
        cudaGetLastError();
        if (q) cudaFree(q);
        set_error("autotuner scratch allocation failed");
        return M2L_ENOMEM;
    }
    cudaMemsetAsync(q, 0, bytes, pl->stream);
    const int keep_form = pl->form, keep_prec = pl->precision, keep_timing = pl->timing, keep_acc = pl->accumulate;
    pl->form = form;
    pl->precision = prec;
    pl->timing = 0;
    pl->accumulate = 0;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    rc = apply_device(pl, q, L, -1, R);  // warm
    if (!rc) {
        cudaEventRecord(a, pl->stream);
        rc = apply_device(pl, q, L, -1, R);
        cudaEventRecord(b, pl->stream);
        if (!rc && cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(ms, a, b);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    pl->form = keep_form;
    pl->precision = keep_prec;
    pl->timing = keep_timing;
    pl->accumulate = keep_acc;
    cudaStreamSynchronize(pl->stream);
    cudaFree(q);
    cudaFree(L);
    return rc;
}

using TuneKey = std::tuple<int, int, int, double, double, int, int, int, int, double, int>;
struct Decision {
    int form, prec;
    double rank;
};
static std::map<TuneKey, Decision> g_decisions;
static std::mutex g_decisions_mu;

// The real plan decides which candidates fit its memory budget; the proxy times them.
struct Candidate {
    int form, prec;
    double rank;  // rank threshold the candidate runs at (the plan's own unless M2L_OPT_RANK_AUTO)
};

static int tune_on(m2l_plan_t *pl, const m2l_plan_t *real, int R, int *form, int *prec, double *rank) {
    std::vector<Candidate> fast, slow;
    const int forms[2] = {M2L_FORM_BLAS, M2L_FORM_FFT};
    const int precs[4] = {M2L_PREC_BF16X3, M2L_PREC_TF32X3, M2L_PREC_FP32, M2L_PREC_FP64};
    const double own = pl->rank_tol;
    if (pl->rank_tol > 0 || pl->form == M2L_FORM_BLAS) build_blas_host(pl);
    for (int f : forms) {
        if (pl->form != M2L_FORM_AUTO && pl->form != f) continue;
        for (int pr : precs) {
            if (pl->precision != M2L_PREC_AUTO && pl->precision != pr) continue;
            if (!eligible(pl, f, pr)) continue;
            if (f == M2L_FORM_BLAS && pl->rank_auto && stated_bound(f, pr, pl->p) >= pl->target_tol) continue;
            const size_t need = workspace_estimate(real, f, pr, R);
            if (real->mem_budget && need > 2 * real->mem_budget) continue;
            (pr == M2L_PREC_FP64 ? slow : fast).push_back({f, pr, own});
        }
    }
    std::vector<Candidate> &cands = fast.empty() ? slow : fast;
    // ranks only for the candidates that will be timed, estimated with the real plan (it keeps the
    // SVD bases for the next tuning of the same order)
    for (auto &c : cands)
        if (c.form == M2L_FORM_BLAS && pl->rank_auto) c.rank = choose_rank(const_cast<m2l_plan_t *>(real), c.prec);
    if (cands.empty()) {
        set_error("no form/precision reaches the target tolerance %.3g with this plan", pl->target_tol);
        return M2L_EUNSUPPORTED;
    }
    float best = 1e30f;
    Candidate win = cands[0];
    for (auto &c : cands) {
        float ms = 1e30f;
        if (c.form == M2L_FORM_BLAS) set_rank(pl, c.rank);
        int rc = time_candidate(pl, c.form, c.prec, R, &ms);
        if (rc == M2L_EUNSUPPORTED) continue;
        if (rc) return rc;
        if (ms < best) {
            best = ms;
            win = c;
        }
    }
    *form = win.form;
    *prec = win.prec;
    *rank = win.form == M2L_FORM_BLAS ? win.rank : own;
    return M2L_OK;
}

static int tune(m2l_plan_t *pl, int R, int *form, int *prec, double *rank) {
    // box counts enter through the memory check, so the decision is shared per tree size too
    const TuneKey key{pl->device, pl->p * 1000 + pl->depth, R, pl->rank_tol, pl->target_tol, pl->form, pl->precision,
                      pl->fft_grid_opt, pl->pc, pl->dir_tol, pl->rank_auto};
    {
        std::lock_guard<std::mutex> g(g_decisions_mu);
        auto it = g_decisions.find(key);
        if (it != g_decisions.end()) {
            *form = it->second.form;
            *prec = it->second.prec;
            *rank = it->second.rank;
            return M2L_OK;
        }
    }
    m2l_plan_t *proxy = m2l_plan(std::min(pl->depth, 4), pl->p, pl->kernel, pl->rank_tol);
    if (!proxy) return M2L_ENOMEM;
    proxy->form = pl->form;
    proxy->precision = pl->precision;
    proxy->target_tol = pl->target_tol;
    proxy->fft_grid_opt = pl->fft_grid_opt;
    proxy->tc_group = pl->tc_group;
    proxy->tc_chunk = pl->tc_chunk;
    proxy->tc_drain = pl->tc_drain;
    proxy->rank_auto = pl->rank_auto;
    proxy->dir_tol = pl->dir_tol;
    if (pl->pc != pl->p) m2l_set_option(proxy, M2L_OPT_CHECK_ORDER, pl->pc);
    proxy->stream = pl->stream;
    if (build_level_tables(pl) || build_pinv(pl)) return M2L_ECUDA;
    if (pl->rank_tol > 0 || pl->form != M2L_FORM_FFT) build_blas_host(pl);
    if (pl->form != M2L_FORM_BLAS) build_fft_host(pl);
    int rc = tune_on(proxy, pl, R, form, prec, rank);
    cudaStreamSynchronize(proxy->stream);
    m2l_destroy(proxy);
    if (rc) return rc;
    std::lock_guard<std::mutex> g(g_decisions_mu);
    g_decisions[key] = {*form, *prec, *rank};
    return M2L_OK;
}

int resolve_form(const m2l_plan_t *cpl, int R, int *form, int *precision) {
    m2l_plan_t *pl = const_cast<m2l_plan_t *>(cpl);
    if (pl->form != M2L_FORM_AUTO && pl->precision != M2L_PREC_AUTO) {
        // explicit form and precision: with M2L_OPT_RANK_AUTO the BLAS form still takes the coarsest
        // rank that fits the target (no timing needed)
        if (pl->rank_auto && pl->form == M2L_FORM_BLAS && pl->rank_auto_tol != pl->target_tol) {
            const double r = choose_rank(pl, pl->precision);
            if (r < 0) {
                set_error("the stated bound of this precision (%.3g) leaves no room for truncation within the target "
                          "%.3g", stated_bound(M2L_FORM_BLAS, pl->precision, pl->p), pl->target_tol);
                return M2L_EUNSUPPORTED;
            }
            set_rank(pl, r);
            pl->rank_auto_tol = pl->target_tol;
        }
        *form = pl->form;
        *precision = pl->precision;
        return M2L_OK;
    }
    for (const auto &d : pl->tuned)
        if (d.R == R && d.tol == pl->target_tol && d.form_opt == pl->form && d.prec_opt == pl->precision &&
            d.levels_version == pl->levels_version) {
            if (pl->rank_auto && d.form == M2L_FORM_BLAS) set_rank(pl, d.rank);
            *form = d.form;
            *precision = d.precision;
            return M2L_OK;
        }
    if (pl->device < 0) {
        set_error("choosing a form needs the GPU the plan was made on");
        return M2L_ECUDA;
    }
    int f, p;
    double r = pl->rank_tol;
    int rc = tune(pl, R, &f, &p, &r);
    if (rc) return rc;
    if (pl->rank_auto && f == M2L_FORM_BLAS) set_rank(pl, r);
    m2l_plan_s::Tuned d;
    d.R = R;
    d.tol = pl->target_tol;
    d.form_opt = pl->form;
    d.prec_opt = pl->precision;
    d.levels_version = pl->levels_version;
    d.form = f;
    d.precision = p;
    d.rank = pl->rank_tol;
    pl->tuned.push_back(d);
    *form = f;
    *precision = p;
    return M2L_OK;
}

}  // namespace m2l
