// extern "C" entry points of include/m2l.h: argument checks, host/device pointer handling,
// and dispatch to the plan builders and launchers.
#include <cmath>
#include <cstring>
#include <algorithm>

#include "internal.h"

namespace m2l {
const char *last_error();
int launch_watchdog_selftest(int *status, long long polls, cudaStream_t s);  // kernels_tc.cu
}

using namespace m2l;

static bool is_device_pointer(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static long long rows_of(m2l_plan_t *pl, int level) {
    long long rows = 0;
    int l0 = level < 0 ? 2 : level, l1 = level < 0 ? pl->depth : level;
    for (int l = l0; l <= l1; ++l) {
        const LevelSet &S = pl->levels[l];
        rows += S.dense ? (1LL << (3 * l)) : (long long)S.keys.size();
    }
    return rows;
}

extern "C" {

const char *m2l_last_error(void) { return m2l::last_error(); }

m2l_plan_t *m2l_plan(int depth, int p, int kernel, double rank_tol) {
    clear_error();
    if (depth < 2 || depth > kMaxDepth) {
        set_error("depth %d outside [2, %d]", depth, kMaxDepth);
        return nullptr;
    }
    if (p < 2 || p > 16) {
        set_error("expansion order p = %d outside [2, 16]", p);
        return nullptr;
    }
    if (kernel != M2L_LAPLACE3D) {
        set_error("unknown kernel %d (only M2L_LAPLACE3D)", kernel);
        return nullptr;
    }
    if (!std::isfinite(rank_tol) || rank_tol >= 1.0) {
        set_error("rank_tol must be finite and < 1 (<= 0 selects full rank)");
        return nullptr;
    }
    m2l_plan_t *pl = new (std::nothrow) m2l_plan_t;
    if (!pl) {
        set_error("out of host memory");
        return nullptr;
    }
    pl->depth = depth;
    pl->p = p;
    pl->kernel = kernel;
    pl->rank_tol = rank_tol;
    for (int a = 0; a < p; ++a)
        for (int b = 0; b < p; ++b)
            for (int c = 0; c < p; ++c)
                if (a == 0 || a == p - 1 || b == 0 || b == p - 1 || c == 0 || c == p - 1) {
                    pl->lattice.push_back(a);
                    pl->lattice.push_back(b);
                    pl->lattice.push_back(c);
                }
    pl->n = (int)pl->lattice.size() / 3;
    pl->np_ = pl->n;
    pl->pc = p;
    pl->nc = pl->n;
    pl->lattice_c = pl->lattice;
    for (int l = 2; l <= depth; ++l) {
        pl->levels[l].dense = true;
        pl->levels[l].nboxes = 1LL << (3 * l);
    }
    // A plan can be built and queried without a GPU (host operators, box tables); applying it
    // needs the device that was current when the plan was made.
    if (cudaGetDevice(&pl->device) != cudaSuccess) {
        cudaGetLastError();
        pl->device = -1;
    } else {
        cudaDeviceGetAttribute(&pl->num_sms, cudaDevAttrMultiProcessorCount, pl->device);
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) pl->mem_budget = total_b / 4;
        else cudaGetLastError();
    }
    return pl;
}

void m2l_destroy(m2l_plan_t *pl) {
    if (!pl) return;
    if (pl->device >= 0) cudaStreamSynchronize(pl->stream);
    free_device(pl);
    delete pl;
}

int m2l_set_option(m2l_plan_t *pl, int key, long long value) {
    clear_error();
    if (!pl) {
        set_error("NULL plan");
        return M2L_EINVAL;
    }
    switch (key) {
        case M2L_OPT_FORM:
            if (value < M2L_FORM_AUTO || value > M2L_FORM_FFT) break;
            pl->form = (int)value;
            return M2L_OK;
        case M2L_OPT_PRECISION:
            if (value < M2L_PREC_AUTO || value > M2L_PREC_BF16X3) break;
            pl->precision = (int)value;
            return M2L_OK;
        case M2L_OPT_ACCUMULATE:
            if (value != 0 && value != 1) break;
            pl->accumulate = (int)value;
            return M2L_OK;
        case M2L_OPT_OUTPUT:
            if (value != M2L_OUT_LOCALS && value != M2L_OUT_CHECK_POTENTIAL) break;
            pl->output = (int)value;
            return M2L_OK;
        case M2L_OPT_TARGET_TOL: {
            double d;
            std::memcpy(&d, &value, sizeof d);
            if (!(d > 0.0) || !std::isfinite(d)) break;
            pl->target_tol = d;
            return M2L_OK;
        }
        case M2L_OPT_TIMING:
            if (value != 0 && value != 1) break;
            pl->timing = (int)value;
            return M2L_OK;
        case M2L_OPT_TC_GROUP:
            if (value < 1 || value > kPerOctant) break;
            pl->tc_group = (int)value;
            return M2L_OK;
        case M2L_OPT_SVD:
            if (value != 0 && value != 1) break;
            if ((int)value != pl->svd_mode) {
                pl->svd_mode = (int)value;
                pl->blas.reset();
                pl->dirop.reset();
                pl->tuned.clear();
                release_operators(pl);
            }
            return M2L_OK;
        case M2L_OPT_RANK_AUTO:
            if (value != 0 && value != 1) break;
            if ((int)value != pl->rank_auto) {
                pl->rank_auto = (int)value;
                pl->rank_auto_tol = -1.0;
                pl->tuned.clear();
            }
            return M2L_OK;
        case M2L_OPT_TC_DRAIN:
            if (value < -1 || value > 64) break;
            pl->tc_drain = (int)value;
            return M2L_OK;
        case M2L_OPT_HADAMARD_CHAINS:
            if (value != 0 && value != 1 && value != 2 && value != 4) break;
            pl->had_chains = (int)value;
            return M2L_OK;
        case M2L_OPT_TC_CHUNK:
            if (value != 0 && value != 32 && value != 64 && value != 128) break;
            pl->tc_chunk = (int)value;
            return M2L_OK;
        case M2L_OPT_FFT_GRID:
            if (value != 0 && (value < 2 * pl->p - 1 || value > 2 * pl->p)) break;
            if ((int)value != pl->fft_grid_opt) {
                pl->fft_grid_opt = (int)value;
                pl->fft.reset();
                for (auto &D : pl->dev) {
                    if (D.Khat) cudaFree(D.Khat);
                    if (D.tw) cudaFree(D.tw);
                    D.Khat = nullptr;
                    D.tw = nullptr;
                }
            }
            return M2L_OK;
        case M2L_OPT_CHECK_ORDER: {
            const int pc = value == 0 ? pl->p : (int)value;
            if (pc < pl->p || pc > 16) break;
            if (pc != pl->pc) {
                pl->pc = pc;
                pl->lattice_c.clear();
                for (int a = 0; a < pc; ++a)
                    for (int b = 0; b < pc; ++b)
                        for (int c = 0; c < pc; ++c)
                            if (a == 0 || a == pc - 1 || b == 0 || b == pc - 1 || c == 0 || c == pc - 1) {
                                pl->lattice_c.push_back(a);
                                pl->lattice_c.push_back(b);
                                pl->lattice_c.push_back(c);
                            }
                pl->nc = (int)pl->lattice_c.size() / 3;
                // every operator that touches the check surface is rebuilt on next use
                pl->pinv.reset();
                pl->blas.reset();
                pl->dirop.reset();
                pl->tuned.clear();
                release_operators(pl);
            }
            return M2L_OK;
        }
        case M2L_OPT_DIR_TOL: {
            double d;
            std::memcpy(&d, &value, sizeof d);
            if (!(d >= 0.0) || !std::isfinite(d) || d >= 1.0) break;
            if (d != pl->dir_tol) {
                pl->dir_tol = d;
                pl->dirop.reset();
                for (auto &D : pl->dev) {
                    for (void **pp : {&D.Ub, &D.Vt, &D.dir_meta}) {
                        if (*pp) cudaFree(*pp);
                        *pp = nullptr;
                    }
                }
            }
            return M2L_OK;
        }
        default:
            set_error("unknown option key %d", key);
            return M2L_EINVAL;
    }
    set_error("invalid value %lld for option %d", value, key);
    return M2L_EINVAL;
}

int m2l_set_stream(m2l_plan_t *pl, void *stream) {
    clear_error();
    if (!pl) {
        set_error("NULL plan");
        return M2L_EINVAL;
    }
    pl->stream = (cudaStream_t)stream;
    return M2L_OK;
}

int m2l_set_boxes(m2l_plan_t *pl, int level, const uint64_t *keys, long long n) {
    clear_error();
    if (!pl) {
        set_error("NULL plan");
        return M2L_EINVAL;
    }
    if (level < 2 || level > pl->depth) {
        set_error("level %d outside [2, %d]", level, pl->depth);
        return M2L_EINVAL;
    }
    const unsigned long long full = 1ULL << (3 * level);
    if (keys == nullptr) {
        if ((unsigned long long)n != full) {
            set_error("keys == NULL restores the full level and needs n == 8^level");
            return M2L_EINVAL;
        }
        pl->levels[level].dense = true;
        pl->levels[level].keys.clear();
        pl->levels[level].nboxes = (long long)full;
        pl->levels_dirty = true;
        return M2L_OK;
    }
    if (n < 1 || (unsigned long long)n > full) {
        set_error("box count %lld outside [1, 8^level]", n);
        return M2L_EINVAL;
    }
    for (long long i = 0; i < n; ++i) {
        if (keys[i] >= full || (i > 0 && keys[i] <= keys[i - 1])) {
            set_error("keys must be strictly ascending Morton keys below 8^level (index %lld)", i);
            return M2L_EINVAL;
        }
    }
    LevelSet &S = pl->levels[level];
    S.dense = (unsigned long long)n == full;
    S.keys.assign(keys, keys + (S.dense ? 0 : n));
    S.nboxes = n;
    pl->levels_dirty = true;
    return M2L_OK;
}


int m2l_apply(m2l_plan_t *pl, const void *q, void *L, int level, int n_rhs) {
    clear_error();
    if (!pl || !q || !L) {
        set_error("NULL plan or buffer");
        return M2L_EINVAL;
    }
    if (!(level == -1 || (level >= 2 && level <= pl->depth))) {
        set_error("level %d: use -1 or a level in [2, %d]", level, pl->depth);
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
    int form, prec;
    int rc = m2l::resolve_form(pl, n_rhs, &form, &prec);
    if (rc) return rc;
    size_t elt = prec == M2L_PREC_FP64 ? 8 : 4;
    size_t bytes = (size_t)rows_of(pl, level) * n_rhs * pl->n * elt;  // multipoles; locals alike
    const size_t out_bytes = pl->output == M2L_OUT_CHECK_POTENTIAL && form == M2L_FORM_BLAS
                                 ? (size_t)rows_of(pl, level) * n_rhs * pl->nc * elt  // check potentials: nc per row
                                 : bytes;
    const char *qa = (const char *)q, *la = (const char *)L;
    if (qa < la + out_bytes && la < qa + bytes) {
        set_error("multipoles and locals overlap");
        return M2L_EINVAL;
    }
    bool qdev = is_device_pointer(q), ldev = is_device_pointer(L);
    if (qdev && ldev) {
        rc = apply_device(pl, q, L, level, n_rhs);
    } else {
        // host buffers: stage through device memory on the plan's stream
        const void *dq = q;
        void *dl = L;
        if (!qdev) {
            if (!pl->stage_in.buf || pl->stage_in.bytes < bytes) {
                if (pl->stage_in.buf) cudaFree(pl->stage_in.buf);
                pl->stage_in = {};
                if (cudaMalloc(&pl->stage_in.buf, bytes) != cudaSuccess) {
                    cudaGetLastError();
                    set_error("staging allocation failed");
                    return M2L_ENOMEM;
                }
                pl->stage_in.bytes = bytes;
            }
            cudaMemcpyAsync(pl->stage_in.buf, q, bytes, cudaMemcpyHostToDevice, pl->stream);
            dq = pl->stage_in.buf;
        }
        if (!ldev) {
            if (!pl->stage_out.buf || pl->stage_out.bytes < out_bytes) {
                if (pl->stage_out.buf) cudaFree(pl->stage_out.buf);
                pl->stage_out = {};
                if (cudaMalloc(&pl->stage_out.buf, out_bytes) != cudaSuccess) {
                    cudaGetLastError();
                    set_error("staging allocation failed");
                    return M2L_ENOMEM;
                }
                pl->stage_out.bytes = out_bytes;
            }
            if (pl->accumulate) cudaMemcpyAsync(pl->stage_out.buf, L, out_bytes, cudaMemcpyHostToDevice, pl->stream);
            dl = pl->stage_out.buf;
        }
        rc = apply_device(pl, dq, dl, level, n_rhs);
        if (rc == M2L_OK && !ldev) cudaMemcpyAsync(L, dl, out_bytes, cudaMemcpyDeviceToHost, pl->stream);
        if (rc == M2L_OK && cudaStreamSynchronize(pl->stream) != cudaSuccess) {
            set_error("stream synchronisation failed: %s", cudaGetErrorString(cudaGetLastError()));
            rc = M2L_ECUDA;
        }
    }
    return rc;
}

int m2l_apply_batch(m2l_plan_t *const *plans, int n_inst, const void *const *multipoles, void *const *locals,
                    const int *n_rhs) {
    clear_error();
    if (!plans || n_inst < 1 || !multipoles || !locals || !n_rhs) {
        set_error("invalid batch arguments");
        return M2L_EINVAL;
    }
    for (int i = 0; i < n_inst; ++i) {
        if (!plans[i] || !multipoles[i] || !locals[i] || n_rhs[i] < 1) {
            set_error("invalid plan, buffer or n_rhs at index %d", i);
            return M2L_EINVAL;
        }
        if (plans[i]->device < 0 || plans[i]->device != plans[0]->device) {
            set_error("every plan of a batch must belong to the device of the first");
            return M2L_EINVAL;
        }
        if (!is_device_pointer(multipoles[i]) || !is_device_pointer(locals[i])) {
            set_error("m2l_apply_batch takes device buffers (index %d)", i);
            return M2L_EINVAL;
        }
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) {
                set_error("plan at index %d appears twice in the batch", i);
                return M2L_EINVAL;
            }
    }
    return apply_batch(plans, n_inst, multipoles, locals, n_rhs);
}

int m2l_query(const m2l_plan_t *cpl, int what, int level, long long *out) {
    clear_error();
    m2l_plan_t *pl = const_cast<m2l_plan_t *>(cpl);
    if (!pl || !out) {
        set_error("NULL plan or output");
        return M2L_EINVAL;
    }
    int rc;
    switch (what) {
        case M2L_Q_N:
            *out = pl->n;
            return M2L_OK;
        case M2L_Q_RANK:
            if ((rc = build_blas_host(pl))) return rc;
            *out = pl->k;
            return M2L_OK;
        case M2L_Q_BOXES:
            if (level < 2 || level > pl->depth) break;
            *out = pl->levels[level].dense ? (1LL << (3 * level)) : (long long)pl->levels[level].keys.size();
            return M2L_OK;
        case M2L_Q_PAIRS:
        case M2L_Q_ROWS: {
            if (!(level == -1 || (level >= 2 && level <= pl->depth))) break;
            if ((rc = build_level_tables(pl))) return rc;
            long long s = 0;
            int l0 = level < 0 ? 2 : level, l1 = level < 0 ? pl->depth : level;
            for (int l = l0; l <= l1; ++l) s += what == M2L_Q_PAIRS ? pl->ldev[l].pairs : pl->ldev[l].nboxes;
            *out = s;
            return M2L_OK;
        }
        case M2L_Q_CONTRACT_FLOPS: {
            if (!(level == -1 || (level >= 2 && level <= pl->depth))) break;
            double f = 0.0;
            if ((rc = contract_flops(pl, level, &f))) return rc;
            *out = (long long)(f + 0.5);
            return M2L_OK;
        }
        case M2L_Q_NC:
            *out = pl->nc;
            return M2L_OK;
        case M2L_Q_RANK_CHECK:
            if ((rc = build_blas_host(pl))) return rc;
            *out = pl->kc;
            return M2L_OK;
        case M2L_Q_RANK_TOL: {
            const double r = pl->rank_tol;
            std::memcpy(out, &r, sizeof r);
            return M2L_OK;
        }
        case M2L_Q_DIR_RANK_SUM: {
            *out = 0;
            if (pl->dir_tol <= 0) return M2L_OK;
            if ((rc = build_directional(pl))) return rc;
            for (int v : pl->dirop->kt) *out += v;
            return M2L_OK;
        }
        case M2L_Q_GRID:
        case M2L_Q_FREQS:
            if ((rc = build_fft_host(pl))) return rc;
            *out = what == M2L_Q_GRID ? pl->g : pl->F;
            return M2L_OK;
        case M2L_Q_PINV_RANK:
            if ((rc = build_pinv(pl))) return rc;
            *out = pl->r;
            return M2L_OK;
        case M2L_Q_FORM:
        case M2L_Q_PRECISION: {
            int f, p;
            if ((rc = resolve_form(pl, level > 0 ? level : 1, &f, &p))) return rc;
            *out = what == M2L_Q_FORM ? f : p;
            return M2L_OK;
        }
        case M2L_Q_LAUNCHES:
            *out = pl->launches;
            return M2L_OK;
        case M2L_Q_DEVICE_STATUS: {
            *out = 0;
            if (pl->device < 0 || !pl->dev_status) return M2L_OK;
            int v = 0;
            if (cudaStreamSynchronize(pl->stream) != cudaSuccess ||
                cudaMemcpy(&v, pl->dev_status, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) {
                set_error("reading the device status failed: %s", cudaGetErrorString(cudaGetLastError()));
                return M2L_ECUDA;
            }
            *out = v;
            if (v) {
                cudaMemset(pl->dev_status, 0, sizeof(int));
                set_error("a bounded device wait ran out (site %d); results since the last status query are invalid", v);
                return M2L_ETIMEOUT;
            }
            return M2L_OK;
        }
        default:
            set_error("unknown query %d", what);
            return M2L_EINVAL;
    }
    set_error("invalid level %d for query %d", level, what);
    return M2L_EINVAL;
}

int m2l_stage_times(m2l_plan_t *pl, double *ms, long long *launches) {
    clear_error();
    if (!pl || !ms) {
        set_error("NULL plan or output");
        return M2L_EINVAL;
    }
    for (int i = 0; i < M2L_NUM_STAGES; ++i) {
        ms[i] = 0.0;
        if (launches) launches[i] = 0;
    }
    for (auto &ev : pl->events) {
        float t = 0.f;
        if (cudaEventSynchronize(ev.b) != cudaSuccess || cudaEventElapsedTime(&t, ev.a, ev.b) != cudaSuccess) {
            set_error("stage timing events failed: %s", cudaGetErrorString(cudaGetLastError()));
            return M2L_ECUDA;
        }
        ms[ev.stage] += t;
        if (launches) launches[ev.stage] += ev.launches;
    }
    return M2L_OK;
}

int m2l_get_operator(m2l_plan_t *pl, int which, double *dst, long long *count) {
    clear_error();
    if (!pl || !count) {
        set_error("NULL plan or count");
        return M2L_EINVAL;
    }
    int rc = which <= 3 ? build_blas_host(pl) : which == 6 ? build_directional(pl) : build_pinv(pl);
    if (rc) return rc;
    const std::vector<double> *src = nullptr;
    std::vector<double> prod;
    switch (which) {
        case 6: {
            if (pl->dir_tol <= 0) {
                set_error("operator 6 (directional products) needs M2L_OPT_DIR_TOL > 0");
                return M2L_EINVAL;
            }
            // Ubar_t Vbar'_t^T (kc x k) from the packed factors, for every t
            const DirOps &d = *pl->dirop;
            const int k = pl->k, kc = pl->kc, kp = pl->kp;
            prod.assign((size_t)kNumTransfer * kc * k, 0.0);
            for (int t = 0; t < kNumTransfer; ++t) {
                const double *ub = &d.ub[d.meta[4 * t]], *vt = &d.vt[d.meta[4 * t + 1]];
                const int kt = d.meta[4 * t + 2], kt8 = d.meta[4 * t + 3];
                double *P = &prod[(size_t)t * kc * k];
                for (int a = 0; a < kc; ++a)
                    for (int j = 0; j < kt; ++j) {
                        const double u = ub[(size_t)a * kt8 + j];
                        for (int c = 0; c < k; ++c) P[(size_t)a * k + c] += u * vt[(size_t)j * kp + c];
                    }
            }
            src = &prod;
            break;
        }
        case 0: src = &pl->blas->U; break;
        case 1: src = &pl->blas->S; break;
        case 2: src = &pl->blas->C; break;
        case 3: src = &pl->blas->s_fat; break;
        case 4: src = &pl->pinv->Veps; break;
        case 5: src = &pl->pinv->Uteps; break;
        default:
            set_error("unknown operator %d", which);
            return M2L_EINVAL;
    }
    *count = (long long)src->size();
    if (dst && !src->empty()) std::memcpy(dst, src->data(), src->size() * sizeof(double));
    return M2L_OK;
}

int m2l_stated_bound(int form, int precision, int p, double *bound) {
    clear_error();
    if (!bound || (form != M2L_FORM_BLAS && form != M2L_FORM_FFT) || precision < M2L_PREC_FP64 ||
        precision > M2L_PREC_BF16X3 || p < 2 || p > 16 ||
        (form == M2L_FORM_FFT && precision == M2L_PREC_BF16X3)) {
        set_error("m2l_stated_bound: bad form %d, precision %d or order %d", form, precision, p);
        return M2L_EINVAL;
    }
    *bound = stated_bound(form, precision, p);
    return M2L_OK;
}

int m2l_selftest_watchdog(m2l_plan_t *pl, long long polls) {
    clear_error();
    if (!pl || pl->device < 0) {
        set_error("the watchdog self-test needs a plan made on a GPU");
        return M2L_EINVAL;
    }
    if (polls < 1 || polls > (1LL << 24)) {
        set_error("polls must be in [1, 2^24] (the bound of the contraction's own waits); got %lld", polls);
        return M2L_EINVAL;
    }
    if (!pl->dev_status) {
        if (cudaMalloc((void **)&pl->dev_status, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            set_error("status word allocation failed");
            return M2L_ENOMEM;
        }
        cudaMemset(pl->dev_status, 0, sizeof(int));
    }
    return launch_watchdog_selftest(pl->dev_status, polls, pl->stream);
}

}  // extern "C"
