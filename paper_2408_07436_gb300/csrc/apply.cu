// Orchestration of one M2L application: workspace, tile lists and the stage sequence of
// each form (BLAS: B1 compress, B2 contract, B3 uncompress + pseudo-inverse; FFT: F1+F2
// forward transform, F3 Hadamard, F4+F5 inverse transform, F6 pseudo-inverse).
#include <algorithm>
#include <vector>

#include "internal.h"
#include "kernels.cuh"

namespace m2l {

size_t fft_smem_bytes(int p, int g, int elt);  // kernels_simt.cu
template <class T>
int launch_contract_tc(m2l_plan_t *pl, const LevelsArg &lv, const ContractTile *tiles, long long ntiles, int R,
                       const void *qt_hi, const void *qt_lo, long long zero_row, T *phit, int precision,
                       cudaStream_t s);                                         // kernels_tc.cu
int launch_split_rows(const float *src, long long rows, int kp, void *hi, void *lo, int precision,
                      cudaStream_t s);                                          // kernels_tc.cu

static cudaEvent_t pool_event(m2l_plan_t *pl) {
    if (pl->events_used == pl->event_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        pl->event_pool.push_back(e);
    }
    return pl->event_pool[pl->events_used++];
}

void stage_begin(m2l_plan_t *pl, int stage) {
    if (!pl->timing) return;
    m2l_plan_s::StageEvent ev;
    ev.stage = stage;
    ev.a = pool_event(pl);
    ev.b = pool_event(pl);
    ev.launches = 0;
    cudaEventRecord(ev.a, pl->stream);
    pl->events.push_back(ev);
}

void stage_end(m2l_plan_t *pl, long long launches) {
    pl->launches += launches;
    if (!pl->timing || pl->events.empty()) return;
    pl->events.back().launches = launches;
    cudaEventRecord(pl->events.back().b, pl->stream);
}

static int ensure_buffer(Workspace &w, size_t bytes) {
    if (w.bytes >= bytes && w.buf) return M2L_OK;
    if (w.buf) cudaFree(w.buf);
    w.buf = nullptr;
    w.bytes = 0;
    if (cudaMalloc(&w.buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("workspace allocation of %zu bytes failed", bytes);
        return M2L_ENOMEM;
    }
    w.bytes = bytes;
    return M2L_OK;
}

static LevelView view_of(const LevelDev &D) {
    LevelView v;
    v.slot = D.slot;
    v.xyz = D.xyz;
    v.perm = D.perm;
    v.cslot = D.cslot;
    v.cxyz = D.cxyz;
    v.cchild = D.cchild;
    v.base = D.base;
    v.cbase = D.cbase;
    v.nboxes = D.nboxes;
    v.nclusters = D.nclusters;
    for (int i = 0; i < 9; ++i) v.oct_start[i] = D.oct_start[i];
    v.N = 1 << D.level;
    return v;
}

static int ensure_tiles(m2l_plan_t *pl, int l0, int l1, int R, int rows_per_tile) {
    int key = l0 == l1 ? l0 : -1;
    if (pl->tiles && pl->tiles_rhs == R && pl->tiles_level == key && pl->tiles_rows == rows_per_tile) return M2L_OK;
    std::vector<ContractTile> t;
    for (int l = l0; l <= l1; ++l) {
        const LevelDev &D = pl->ldev[l];
        for (int oct = 0; oct < 8; ++oct) {
            long long segrows = (D.oct_start[oct + 1] - D.oct_start[oct]) * (long long)R;
            for (long long j0 = 0; j0 < segrows; j0 += rows_per_tile) {
                ContractTile c;
                c.lev = l - l0;
                c.oct = oct;
                c.j0 = (int)j0;
                c.rows = (int)std::min<long long>(rows_per_tile, segrows - j0);
                t.push_back(c);
            }
        }
    }
    if (pl->tiles) cudaFree(pl->tiles);
    pl->tiles = nullptr;
    size_t bytes = std::max<size_t>(1, t.size()) * sizeof(ContractTile);
    if (cudaMalloc(&pl->tiles, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("tile list allocation failed");
        return M2L_ENOMEM;
    }
    if (!t.empty() && cudaMemcpy(pl->tiles, t.data(), t.size() * sizeof(ContractTile), cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("tile list upload failed");
        return M2L_ECUDA;
    }
    pl->ntiles = (long long)t.size();
    pl->tiles_rhs = R;
    pl->tiles_level = key;
    pl->tiles_rows = rows_per_tile;
    return M2L_OK;
}

static int ensure_lattice(m2l_plan_t *pl) {
    if (pl->lattice_dev) return M2L_OK;
    std::vector<int> packed(pl->n);
    for (int i = 0; i < pl->n; ++i)
        packed[i] = (pl->lattice[3 * i] << 16) | (pl->lattice[3 * i + 1] << 8) | pl->lattice[3 * i + 2];
    if (cudaMalloc((void **)&pl->lattice_dev, packed.size() * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        set_error("lattice allocation failed");
        return M2L_ENOMEM;
    }
    cudaMemcpy(pl->lattice_dev, packed.data(), packed.size() * sizeof(int), cudaMemcpyHostToDevice);
    return M2L_OK;
}

#define M2L_TRY(x)              \
    do {                        \
        int _rc = (x);          \
        if (_rc) return _rc;    \
    } while (0)

template <class T>
static int apply_blas(m2l_plan_t *pl, const T *q, T *out, int l0, int l1, int R, int precision) {
    const DevOps &D = pl->dev[precision];
    const int n = pl->n, kp = pl->kp, rp = pl->rp;
    const long long base0 = pl->ldev[l0].base;
    long long rows_in = 0;
    for (int l = l0; l <= l1; ++l) rows_in += pl->ldev[l].nboxes * R;
    const long long allrows = pl->total_rows * R;
    const bool tc = precision == M2L_PREC_TF32X3 || precision == M2L_PREC_BF16X3;
    // workspace: qt [(allrows + 1) x kp], phit [allrows x kp], Z [allrows x rp], and for the
    // tensor-core forms the split qt_hi / qt_lo [(allrows + 1) x kp] (4 or 2 bytes each)
    size_t e = sizeof(T);
    size_t qt_b = (size_t)(allrows + 1) * kp * e, ph_b = (size_t)allrows * kp * e, z_b = (size_t)allrows * rp * e;
    size_t split_b = tc ? (size_t)(allrows + 1) * kp * (precision == M2L_PREC_TF32X3 ? 4 : 2) : 0;
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    M2L_TRY(ensure_buffer(pl->ws, al(qt_b) + al(ph_b) + al(z_b) + 2 * al(split_b)));
    char *w = (char *)pl->ws.buf;
    T *qt = (T *)w;
    T *phit = (T *)(w + al(qt_b));
    T *Z = (T *)(w + al(qt_b) + al(ph_b));
    char *hi = w + al(qt_b) + al(ph_b) + al(z_b);
    char *lo = hi + al(split_b);
    cudaStream_t s = pl->stream;
    // B1: compressed multipoles qt = q S (rows of the requested levels), zero source row at the end
    stage_begin(pl, M2L_STAGE_COMPRESS);
    M2L_TRY(launch_gemm_xwt<T>(q, n, (const T *)D.St, n, qt + base0 * R * kp, kp, rows_in, kp, n, 0, s));
    cudaMemsetAsync(qt + allrows * kp, 0, kp * e, s);
    stage_end(pl, 1);
    // B2: gathered contraction over the transfer vectors of each target octant
    M2L_TRY(ensure_tiles(pl, l0, l1, R, tc ? 128 : 64));
    LevelsArg lv;
    lv.count = l1 - l0 + 1;
    for (int l = l0; l <= l1; ++l) lv.L[l - l0] = view_of(pl->ldev[l]);
    if (!tc) {
        stage_begin(pl, M2L_STAGE_CONTRACT);
        M2L_TRY(launch_contract_simt<T>(lv, (const ContractTile *)pl->tiles, pl->ntiles, R, qt, (const T *)D.C, kp,
                                        allrows, phit, s));
        stage_end(pl, 1);
    } else {
        if constexpr (sizeof(T) == 4) {
            const long long split_rows = allrows + 1;
            stage_begin(pl, M2L_STAGE_COMPRESS);
            M2L_TRY(launch_split_rows((const float *)qt, split_rows, kp, hi, lo, precision, s));
            stage_end(pl, 1);
            stage_begin(pl, M2L_STAGE_CONTRACT);
            M2L_TRY(launch_contract_tc<T>(pl, lv, (const ContractTile *)pl->tiles, pl->ntiles, R, hi, lo, allrows,
                                          phit, precision, s));
            stage_end(pl, 1);
        } else {
            set_error("split tensor-core precisions operate on FP32 data");
            return M2L_EINVAL;
        }
    }
    // B3: locals = V_eps (A phit) with A = Ut_eps U, or the check potential U phit
    const T *ph = phit + base0 * R * kp;
    stage_begin(pl, M2L_STAGE_EXPAND);
    if (pl->output == M2L_OUT_LOCALS) {
        M2L_TRY(launch_gemm_xwt<T>(ph, kp, (const T *)D.A, kp, Z, rp, rows_in, rp, kp, 0, s));
        M2L_TRY(launch_gemm_xwt<T>(Z, rp, (const T *)D.V, rp, out, n, rows_in, n, rp, pl->accumulate, s));
        stage_end(pl, 2);
    } else {
        M2L_TRY(launch_gemm_xwt<T>(ph, kp, (const T *)D.Uc, kp, out, n, rows_in, n, kp, pl->accumulate, s));
        stage_end(pl, 1);
    }
    return M2L_OK;
}

template <class T>
static int apply_fft(m2l_plan_t *pl, const T *q, T *out, int l0, int l1, int R, int precision) {
    const DevOps &D = pl->dev[precision];
    const int n = pl->n, rp = pl->rp, g = pl->g, F = pl->F, p = pl->p;
    if (fft_smem_bytes(p, g, (int)sizeof(T)) > 227 * 1024) {
        set_error("FFT form: grid %d does not fit shared memory in this precision", g);
        return M2L_EUNSUPPORTED;
    }
    M2L_TRY(ensure_lattice(pl));
    const long long base0 = pl->ldev[l0].base;
    long long rows_in = 0;
    for (int l = l0; l <= l1; ++l) rows_in += pl->ldev[l].nboxes * R;
    const long long allrows = pl->total_rows * R;
    size_t e = sizeof(T);
    size_t spec_b = (size_t)pl->total_clusters * R * F * 16 * e;
    size_t phi_b = (size_t)allrows * n * e, z_b = (size_t)allrows * rp * e;
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    M2L_TRY(ensure_buffer(pl->ws, 2 * al(spec_b) + al(phi_b) + al(z_b)));
    char *w = (char *)pl->ws.buf;
    T *qhat = (T *)w;
    T *phihat = (T *)(w + al(spec_b));
    T *Phi = (T *)(w + 2 * al(spec_b));
    T *Z = (T *)(w + 2 * al(spec_b) + al(phi_b));
    cudaStream_t s = pl->stream;
    const bool check_out = pl->output == M2L_OUT_CHECK_POTENTIAL;
    // clusters with missing children keep zero spectra for them
    stage_begin(pl, M2L_STAGE_FFT_FORWARD);
    cudaMemsetAsync(qhat, 0, spec_b, s);
    stage_end(pl, 0);
    for (int l = l0; l <= l1; ++l) {
        LevelView L = view_of(pl->ldev[l]);
        const T *ql = q + (L.base - base0) * R * n;
        stage_begin(pl, M2L_STAGE_FFT_FORWARD);
        M2L_TRY(launch_fft_forward<T>(L, R, p, n, g, pl->lattice_dev, (const T *)D.tw, ql, qhat, s));
        stage_end(pl, 1);
        stage_begin(pl, M2L_STAGE_HADAMARD);
        M2L_TRY(launch_hadamard<T>(L, R, F, (const T *)D.Khat, qhat, phihat, s));
        stage_end(pl, 1);
        T *dst = check_out ? out + (L.base - base0) * R * n : Phi + L.base * R * n;
        stage_begin(pl, M2L_STAGE_FFT_INVERSE);
        M2L_TRY(launch_fft_inverse<T>(L, R, p, n, g, pl->lattice_dev, (const T *)D.tw, phihat, dst, n,
                                      check_out ? pl->accumulate : 0, s));
        stage_end(pl, 1);
    }
    if (!check_out) {
        // F6: locals = V_eps (Ut_eps Phi)
        stage_begin(pl, M2L_STAGE_PINV);
        M2L_TRY(launch_gemm_xwt<T>(Phi + base0 * R * n, n, (const T *)D.Ut, n, Z, rp, rows_in, rp, n, 0, s));
        M2L_TRY(launch_gemm_xwt<T>(Z, rp, (const T *)D.V, rp, out, n, rows_in, n, rp, pl->accumulate, s));
        stage_end(pl, 2);
    }
    return M2L_OK;
}

int resolve_form(const m2l_plan_t *pl, int R, int *form, int *precision);  // autotune.cpp

int apply_device(m2l_plan_t *pl, const void *q, void *L, int level, int R) {
    int l0 = level < 0 ? 2 : level, l1 = level < 0 ? pl->depth : level;
    M2L_TRY(ensure_constants(pl->device));
    M2L_TRY(upload_level_tables(pl));
    int form, precision;
    M2L_TRY(resolve_form(pl, R, &form, &precision));
    if (form == M2L_FORM_FFT && (precision == M2L_PREC_TF32X3 || precision == M2L_PREC_BF16X3)) {
        set_error("the FFT form runs in FP64 or FP32; split tensor-core precisions apply to the BLAS form");
        return M2L_EUNSUPPORTED;
    }
    M2L_TRY(upload_ops(pl, precision, form));
    if (!pl->dev_status) {
        if (cudaMalloc((void **)&pl->dev_status, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            set_error("status word allocation failed");
            return M2L_ENOMEM;
        }
        cudaMemset(pl->dev_status, 0, sizeof(int));
    }
    pl->launches = 0;
    pl->events.clear();
    pl->events_used = 0;
    int rc;
    if (precision == M2L_PREC_FP64) {
        rc = form == M2L_FORM_BLAS ? apply_blas<double>(pl, (const double *)q, (double *)L, l0, l1, R, precision)
                                   : apply_fft<double>(pl, (const double *)q, (double *)L, l0, l1, R, precision);
    } else {
        rc = form == M2L_FORM_BLAS ? apply_blas<float>(pl, (const float *)q, (float *)L, l0, l1, R, precision)
                                   : apply_fft<float>(pl, (const float *)q, (float *)L, l0, l1, R, precision);
    }
    return rc;
}

}  // namespace m2l
