// Orchestration of M2L applications: preparation (device tables, operators, workspace), the
// stage sequence of each form (BLAS: B1 compress, B2 contract, B3 uncompress + pseudo-inverse;
// FFT: F1+F2 forward transform, F3 Hadamard, F4+F5 inverse transform, F6 pseudo-inverse), and
// batches of independent instances: instances that share (p, form, precision, rank) share one
// contraction launch over all their tiles, and a whole batch pass is replayed from a CUDA graph.
#include <algorithm>
#include <vector>

#include "internal.h"
#include "kernels.cuh"

namespace m2l {

size_t fft_smem_bytes(int p, int g, int elt);  // kernels_simt.cu
template <class T>
int launch_contract_tc(m2l_plan_t *pl, const LevelView *lv, const ContractTile *tiles, long long ntiles, const int *tvl,
                       const void *qt_hi, const void *qt_lo, long long zero_row, T *phit, int precision, cudaStream_t s);
int launch_split_rows(const float *src, long long rows, int kp, void *hi, void *lo, int precision, cudaStream_t s);

#define M2L_TRY(x)           \
    do {                     \
        int _rc = (x);       \
        if (_rc) return _rc; \
    } while (0)

// ---------------------------------------------------------------------------------------------
// Stage timing (M2L_OPT_TIMING): event pairs recorded on the plan's stream.

static cudaEvent_t pool_event(m2l_plan_t *pl) {
    if (pl->events_used == pl->event_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        pl->event_pool.push_back(e);
    }
    return pl->event_pool[pl->events_used++];
}

void stage_begin(m2l_plan_t *pl, int stage) {
    if (!pl->timing || pl->capturing) return;
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
    if (!pl->timing || pl->capturing || pl->events.empty()) return;
    pl->events.back().launches = launches;
    cudaEventRecord(pl->events.back().b, pl->stream);
}

static void reset_stage_log(m2l_plan_t *pl) {
    pl->launches = 0;
    pl->events.clear();
    pl->events_used = 0;
}

// ---------------------------------------------------------------------------------------------
// Preparation: everything that allocates or copies synchronously happens here, never inside a
// stream capture.

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

int prepare_plan(m2l_plan_t *pl, int form, int precision) {
    M2L_TRY(ensure_constants(pl->device));
    M2L_TRY(upload_level_tables(pl));
    if (form == M2L_FORM_FFT && precision == M2L_PREC_BF16X3) {
        set_error("the FFT form runs in FP64, FP32 or TF32x3 (Hadamard products on the tensor cores)");
        return M2L_EUNSUPPORTED;
    }
    if (pl->pc != pl->p && form == M2L_FORM_FFT) {
        // the convolution needs the check and equivalent surfaces on one grid (Sec. 3.3)
        set_error("the FFT form needs equal check and equivalent orders (check order %d, order %d)", pl->pc, pl->p);
        return M2L_EUNSUPPORTED;
    }
    if (pl->pc != pl->p && (precision == M2L_PREC_TF32X3 || precision == M2L_PREC_BF16X3)) {
        set_error("the tensor-core contraction needs equal check and equivalent orders; use FP64 or FP32");
        return M2L_EUNSUPPORTED;
    }
    M2L_TRY(upload_ops(pl, precision, form));
    if (form == M2L_FORM_FFT) M2L_TRY(ensure_lattice(pl));
    if (!pl->dev_status) {
        if (cudaMalloc((void **)&pl->dev_status, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            set_error("status word allocation failed");
            return M2L_ENOMEM;
        }
        cudaMemset(pl->dev_status, 0, sizeof(int));
    }
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
    v.cperm = D.cperm;
    v.base = D.base;
    v.cbase = D.cbase;
    v.nboxes = D.nboxes;
    v.nclusters = D.nclusters;
    for (int i = 0; i < 9; ++i) v.oct_start[i] = D.oct_start[i];
    v.N = 1 << D.level;
    v.row0 = 0;
    v.R = 1;
    return v;
}

// One instance inside a group: its buffers, right-hand sides and levels, and the first row it
// owns in the group's contraction row space.
struct Run {
    m2l_plan_t *pl;
    const void *q;
    void *L;
    int R, l0, l1;
    long long rows, row_off;
};

static long long rows_of(const m2l_plan_t *pl, int l0, int l1, int R) {
    long long r = 0;
    for (int l = l0; l <= l1; ++l) r += pl->ldev[l].nboxes * R;
    return r;
}

// Transfer vectors of target octant o in the order the contraction visits them (dx slowest),
// packed as the kernels read them (see ContractTile).
static int octant_table(int o, int *tab) {
    const int cx = o & 1, cy = (o >> 1) & 1, cz = (o >> 2) & 1;
    int e = 0;
    for (int dx = -2 - cx; dx <= 3 - cx; ++dx)
        for (int dy = -2 - cy; dy <= 3 - cy; ++dy)
            for (int dz = -2 - cz; dz <= 3 - cz; ++dz) {
                const int ti = transfer_index(dx, dy, dz);
                if (ti >= 0) tab[e++] = (dx + 3) | ((dy + 3) << 4) | ((dz + 3) << 8) | (ti << 12);
            }
    return e;
}

// The entries of `tab` that reach an existing box from at least one target of the tile (the
// targets perm[oct_start + j / R] for its rows j); at least one entry, so the tile's rows are
// always written.
static int tile_vectors(const LevelDev &D, int R, const ContractTile &c, const int *tab, int *out) {
    const int N = 1 << D.level;
    const long long j0 = c.j0 / R, j1 = (c.j0 + c.rows - 1) / R;
    int cnt = 0;
    for (int e = 0; e < kPerOctant; ++e) {
        const int pk = tab[e];
        const int dx = (pk & 15) - 3, dy = ((pk >> 4) & 15) - 3, dz = ((pk >> 8) & 15) - 3;
        for (long long j = j0; j <= j1; ++j) {
            const uint32_t p = D.h_xyz[D.h_perm[D.oct_start[c.oct] + j]];
            const int x = (int)(p & 1023) + dx, y = (int)((p >> 10) & 1023) + dy, z = (int)((p >> 20) & 1023) + dz;
            if (x < 0 || y < 0 || z < 0 || x >= N || y >= N || z >= N) continue;
            if (D.h_slot[((size_t)z * N + y) * N + x] >= 0) {
                out[cnt++] = pk;
                break;
            }
        }
    }
    if (cnt == 0) out[cnt++] = tab[0];
    return cnt;
}

// Device level views, contraction tiles and the tiles' transfer vector lists of a group, cached on
// the group's owner plan.
static int ensure_exec(m2l_plan_t *owner, std::vector<Run> &runs, int rows_per_tile, long long *ntiles_out,
                       long long *total_rows_out) {
    std::vector<long long> key;
    key.push_back(rows_per_tile);
    for (const Run &r : runs) {
        key.push_back((long long)(uintptr_t)r.pl);
        key.push_back(r.R);
        key.push_back(r.l0);
        key.push_back(r.l1);
        key.push_back(r.pl->levels_version);
    }
    long long off = 0;
    for (Run &r : runs) {
        r.rows = rows_of(r.pl, r.l0, r.l1, r.R);
        r.row_off = off;
        off += r.rows;
    }
    *total_rows_out = off;
    ExecCache &E = owner->exec;
    if (E.levels && E.key == key) {
        *ntiles_out = E.ntiles;
        return M2L_OK;
    }
    std::vector<LevelView> views;
    std::vector<ContractTile> tiles;
    std::vector<const LevelDev *> tile_level;
    std::vector<int> tile_R;
    for (const Run &r : runs) {
        for (int l = r.l0; l <= r.l1; ++l) {
            const LevelDev &D = r.pl->ldev[l];
            LevelView v = view_of(D);
            v.R = r.R;
            v.row0 = r.row_off + (D.base - r.pl->ldev[r.l0].base) * r.R;
            const int lev = (int)views.size();
            views.push_back(v);
            for (int oct = 0; oct < 8; ++oct) {
                long long segrows = (D.oct_start[oct + 1] - D.oct_start[oct]) * (long long)r.R;
                for (long long j0 = 0; j0 < segrows; j0 += rows_per_tile) {
                    ContractTile c{};
                    c.lev = lev;
                    c.oct = oct;
                    c.j0 = (int)j0;
                    c.rows = (int)std::min<long long>(rows_per_tile, segrows - j0);
                    tiles.push_back(c);
                    tile_level.push_back(&D);
                    tile_R.push_back(r.R);
                }
            }
        }
    }
    // transfer vector lists, built per tile in parallel, then packed
    int tab[8][kPerOctant];
    for (int o = 0; o < 8; ++o) octant_table(o, tab[o]);
    const long long nt = (long long)tiles.size();
    std::vector<int> lists((size_t)nt * kPerOctant);
#pragma omp parallel for schedule(dynamic, 64)
    for (long long i = 0; i < nt; ++i)
        tiles[i].ntv = tile_vectors(*tile_level[i], tile_R[i], tiles[i], tab[tiles[i].oct], &lists[(size_t)i * kPerOctant]);
    // longest lists first, so the last wave of CTAs holds the shortest tiles
    std::vector<long long> order(nt);
    for (long long i = 0; i < nt; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](long long x, long long y) { return tiles[x].ntv > tiles[y].ntv; });
    std::vector<ContractTile> sorted(nt);
    std::vector<int> packed;
    packed.reserve(lists.size());
    for (long long i = 0; i < nt; ++i) {
        ContractTile c = tiles[order[i]];
        c.tv0 = (long long)packed.size();
        const int *src = &lists[(size_t)order[i] * kPerOctant];
        packed.insert(packed.end(), src, src + c.ntv);
        sorted[i] = c;
    }
    tiles.swap(sorted);
    lists.swap(packed);
    const long long nv = (long long)lists.size();
    if (E.levels) cudaFree(E.levels);
    if (E.tiles) cudaFree(E.tiles);
    if (E.tvl) cudaFree(E.tvl);
    E.levels = E.tiles = E.tvl = nullptr;
    E.key.clear();
    if (cudaMalloc(&E.levels, std::max<size_t>(1, views.size()) * sizeof(LevelView)) != cudaSuccess ||
        cudaMalloc(&E.tiles, std::max<size_t>(1, tiles.size()) * sizeof(ContractTile)) != cudaSuccess ||
        cudaMalloc(&E.tvl, std::max<size_t>(1, (size_t)nv) * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        set_error("tile list allocation failed");
        return M2L_ENOMEM;
    }
    cudaMemcpy(E.levels, views.data(), views.size() * sizeof(LevelView), cudaMemcpyHostToDevice);
    if (!tiles.empty()) cudaMemcpy(E.tiles, tiles.data(), tiles.size() * sizeof(ContractTile), cudaMemcpyHostToDevice);
    if (nv) cudaMemcpy(E.tvl, lists.data(), (size_t)nv * sizeof(int), cudaMemcpyHostToDevice);
    E.ntiles = nt;
    E.nvectors = nv;
    E.key = key;
    *ntiles_out = E.ntiles;
    return M2L_OK;
}

static size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

struct BlasLayout {
    size_t qt_b, ph_b, z_b, split_b, sl_b;
    size_t total() const { return al256(qt_b) + al256(ph_b) + al256(z_b) + 2 * al256(split_b) + al256(sl_b); }
};

static BlasLayout blas_layout(const m2l_plan_t *pl, long long total_rows, int precision) {
    const bool tc = precision == M2L_PREC_TF32X3 || precision == M2L_PREC_BF16X3;
    const size_t e = precision == M2L_PREC_FP64 ? 8 : 4;
    BlasLayout b;
    b.qt_b = (size_t)(total_rows + 1) * pl->kp * e;
    b.ph_b = (size_t)total_rows * pl->kcp * e;
    b.z_b = (size_t)total_rows * pl->rp * e;
    b.split_b = tc ? (size_t)(total_rows + 1) * pl->kp * (precision == M2L_PREC_TF32X3 ? 4 : 2) : 0;
    b.sl_b = tc ? sliced_workspace(total_rows, sliced_kmax(pl)) : 0;  // B1 and B3 as sliced products
    return b;
}

// FFT workspace: check potentials and the pseudo-inverse intermediate for every row, in ws; the
// spectra of one level and a chunk of right-hand sides, in a separate buffer.
static long long max_clusters(const m2l_plan_t *pl) {
    long long m = 0;
    for (int l = 2; l <= pl->depth; ++l) m = std::max(m, pl->ldev[l].nclusters);
    return m;
}

// Phi [rows][n], Z [rows][rp], and for TF32x3 the slices of the tensor-core V_eps product.
static size_t fft_rows_bytes(const m2l_plan_t *pl, int R, int precision) {
    const size_t e = precision == M2L_PREC_FP64 ? 8 : 4;
    const long long allrows = pl->total_rows * R;
    size_t b = al256((size_t)allrows * pl->n * e) + al256((size_t)allrows * pl->rp * e);
    if (precision == M2L_PREC_TF32X3) {
        const int ku = (pl->n + 63) / 64 * 64, kv = (pl->r32 + 63) / 64 * 64;
        b += al256(sliced_workspace(allrows, std::max(ku, kv)));
    }
    return b;
}

static size_t fft_spec_bytes_per_rhs(const m2l_plan_t *pl, int precision) {
    const size_t e = precision == M2L_PREC_FP64 ? 8 : 4;
    return 2 * (size_t)max_clusters(pl) * pl->F * 16 * e;
}

// Right-hand sides the spectra buffer holds at once: as many as fit the plan's budget.
static int fft_rhs_chunk(const m2l_plan_t *pl, int R, int precision) {
    const size_t per = fft_spec_bytes_per_rhs(pl, precision);
    if (per == 0) return R;
    const size_t budget = pl->mem_budget ? pl->mem_budget : (size_t)8 << 30;
    long long c = (long long)(budget / per);
    if (c < 1) return 0;
    return (int)std::min<long long>(R, c);
}

size_t workspace_estimate(const m2l_plan_t *pl, int form, int precision, int R) {
    if (form == M2L_FORM_BLAS) {
        const bool tc = precision == M2L_PREC_TF32X3 || precision == M2L_PREC_BF16X3;
        const size_t e = precision == M2L_PREC_FP64 ? 8 : 4;
        const size_t rows = (size_t)pl->total_rows * R + 1;
        size_t b = rows * ((size_t)pl->kp + pl->kcp + pl->rp) * e;
        if (tc) b += 2 * rows * pl->kp * (precision == M2L_PREC_TF32X3 ? 4 : 2);
        return b;
    }
    const int rc = fft_rhs_chunk(pl, R, precision);
    if (rc < 1) return (size_t)-1;
    return fft_rows_bytes(pl, R, precision) + (size_t)rc * fft_spec_bytes_per_rhs(pl, precision);
}

// ---------------------------------------------------------------------------------------------
// BLAS form over a group of instances with the same operators; owner = runs[0].pl.

// Second factor of the pseudo-inverse, out = V_eps Z (+ out). Its sum cancels by up to the
// inverse of the pseudo-inverse threshold, and plain FP32 accumulation leaves up to about 8e-7
// of the check potential in the locals. `compensated` (FP32 only) takes the float-float product
// with V_eps carried as hi + lo, which removes that term: the FFT form in FP32 uses it, as its
// other stages stay below 5.2e-7; the BLAS forms' contraction error is larger than the term.
template <class T>
static int apply_veps(const m2l_plan_t *pl, const DevOps &D, const T *Z, T *out, long long rows, int acc, bool compensated,
                      cudaStream_t s) {
    const int n = pl->n, rp = pl->rp;
    if constexpr (sizeof(T) == 4) {
        if (compensated)
            return launch_gemm_xwt_ff(Z, rp, (const float *)D.V, (const float *)D.Vlo, rp, out, n, rows, n, rp, acc, s);
    }
    return launch_gemm_xwt<T>(Z, rp, (const T *)D.V, rp, out, n, rows, n, rp, acc, s);
}

// Rows per contraction tile: 128 for the tensor-core kernel (one MMA tile), kDirTileRows for the
// directional CUDA-core kernel, 64 for the plain one (which also runs on shorter tiles).
static int contract_tile_rows(const m2l_plan_t *own, int precision) {
    if (precision == M2L_PREC_TF32X3 || precision == M2L_PREC_BF16X3) return 128;
    if (own->dir_tol > 0) return precision == M2L_PREC_FP64 ? kDirTileRows<double> : kDirTileRows<float>;
    return 64;
}

template <class T>
static int blas_group(std::vector<Run> &runs, int precision, Workspace &ws, cudaStream_t s) {
    m2l_plan_t *own = runs[0].pl;
    const DevOps &D = own->dev[precision];
    const int n = own->n, nc = own->nc, kp = own->kp, kcp = own->kcp, rp = own->rp;
    const bool tc = precision == M2L_PREC_TF32X3 || precision == M2L_PREC_BF16X3;
    long long ntiles = 0, total = 0;
    M2L_TRY(ensure_exec(own, runs, contract_tile_rows(own, precision), &ntiles, &total));
    const BlasLayout lay = blas_layout(own, total, precision);
    M2L_TRY(ensure_buffer(ws, lay.total()));
    char *w = (char *)ws.buf;
    T *qt = (T *)w;
    T *phit = (T *)(w + al256(lay.qt_b));
    T *Z = (T *)(w + al256(lay.qt_b) + al256(lay.ph_b));
    char *hi = w + al256(lay.qt_b) + al256(lay.ph_b) + al256(lay.z_b);
    char *lo = hi + al256(lay.split_b);
    void *sl = lo + al256(lay.split_b);  // slices of the sliced products (split forms)
    // B1: compressed multipoles of every instance, one zero row after the last; the split forms
    // take it on the tensor cores, exactly
    stage_begin(own, M2L_STAGE_COMPRESS);
    long long nl1 = 0;
    for (const Run &r : runs) {
        T *dst = qt + r.row_off * kp;
        if constexpr (sizeof(T) == 4) {
            if (tc && sliced_usable(D.Ss, kp, kp, (const float *)dst)) {
                M2L_TRY(launch_sliced(own, D.Ss, (const float *)r.q, n, r.rows, (float *)dst, kp, kp, 0, sl, s));
                nl1 += 2;
                continue;
            }
        }
        M2L_TRY(launch_gemm_xwt<T>((const T *)r.q, n, (const T *)D.St, n, dst, kp, r.rows, kp, n, 0, s));
        nl1 += 1;
    }
    cudaMemsetAsync(qt + total * kp, 0, kp * sizeof(T), s);
    stage_end(own, nl1);
    // B2: one contraction launch over the tiles of every instance
    const LevelView *lv = (const LevelView *)own->exec.levels;
    const ContractTile *tl = (const ContractTile *)own->exec.tiles;
    const int *tvl = (const int *)own->exec.tvl;
    if (!tc) {
        stage_begin(own, M2L_STAGE_CONTRACT);
        int rc = M2L_EUNSUPPORTED;
        if (own->dir_tol > 0 && D.Ub)
            rc = launch_contract_simt_dir<T>(lv, tl, ntiles, tvl, qt, (const T *)D.Ub, (const T *)D.Vt,
                                             (const int *)D.dir_meta, own->k, kp, kcp, own->dir_kt8_max, total, phit, s);
        if (rc == M2L_EUNSUPPORTED)
            rc = launch_contract_simt<T>(lv, tl, ntiles, tvl, qt, (const T *)D.C, kp, kcp, total, phit, s);
        M2L_TRY(rc);
        stage_end(own, 1);
    } else {
        if constexpr (sizeof(T) == 4) {
            stage_begin(own, M2L_STAGE_COMPRESS);
            M2L_TRY(launch_split_rows((const float *)qt, total + 1, kp, hi, lo, precision, s));
            stage_end(own, 1);
            stage_begin(own, M2L_STAGE_CONTRACT);
            M2L_TRY(launch_contract_tc<T>(own, lv, tl, ntiles, tvl, hi, lo, total, phit, precision, s));
            stage_end(own, 1);
        } else {
            set_error("split tensor-core precisions operate on FP32 data");
            return M2L_EINVAL;
        }
    }
    // B3: locals = V_eps (A phit) with A = Ut_eps U, or the check potential U phit
    stage_begin(own, M2L_STAGE_EXPAND);
    long long nl = 0;
    for (const Run &r : runs) {
        const T *ph = phit + r.row_off * kcp;
        T *zr = Z + r.row_off * rp;
        if (r.pl->output == M2L_OUT_LOCALS) {
            bool done_a = false, done_v = false;
            if constexpr (sizeof(T) == 4) {
                if (tc && sliced_usable(D.As, rp, rp, (const float *)zr)) {  // every column of Z (zeros past r)
                    M2L_TRY(launch_sliced(own, D.As, (const float *)ph, kcp, r.rows, (float *)zr, rp, rp, 0, sl, s));
                    done_a = true;
                    nl += 2;
                }
                if (tc && done_a && sliced_usable(D.Vs, n, n, (const float *)r.L)) {
                    M2L_TRY(launch_sliced(own, D.Vs, (const float *)zr, rp, r.rows, (float *)r.L, n, n, r.pl->accumulate, sl,
                                          s));
                    done_v = true;
                    nl += 2;
                }
            }
            if (!done_a) {
                M2L_TRY(launch_gemm_xwt<T>(ph, kcp, (const T *)D.A, kcp, zr, rp, r.rows, rp, kcp, 0, s));
                nl += 1;
            }
            if (!done_v) {
                M2L_TRY(apply_veps<T>(own, D, zr, (T *)r.L, r.rows, r.pl->accumulate, false, s));
                nl += 1;
            }
        } else {
            if constexpr (sizeof(T) == 4) {
                if (tc && sliced_usable(D.Ucs, nc, nc, (const float *)r.L)) {
                    M2L_TRY(launch_sliced(own, D.Ucs, (const float *)ph, kcp, r.rows, (float *)r.L, nc, nc, r.pl->accumulate,
                                          sl, s));
                    nl += 2;
                    continue;
                }
            }
            M2L_TRY(launch_gemm_xwt<T>(ph, kcp, (const T *)D.Uc, kcp, (T *)r.L, nc, r.rows, nc, kcp, r.pl->accumulate, s));
            nl += 1;
        }
    }
    stage_end(own, nl);
    return M2L_OK;
}

// FFT form, one instance; levels one after another and right-hand sides in chunks that fit the
// spectra buffer `spec` (the plan's own, or the one a batch shares).
template <class T>
static int fft_run(const Run &r, int precision, Workspace &ws, Workspace &spec, cudaStream_t s) {
    m2l_plan_t *pl = r.pl;
    const DevOps &D = pl->dev[precision];
    const int n = pl->n, rp = pl->rp, g = pl->g, F = pl->F, p = pl->p, R = r.R;
    if (fft_smem_bytes(p, g, (int)sizeof(T)) > 227 * 1024) {
        set_error("FFT form: grid %d does not fit shared memory in this precision", g);
        return M2L_EUNSUPPORTED;
    }
    const int Rc = fft_rhs_chunk(pl, R, precision);
    if (Rc < 1) {
        set_error("FFT form: the spectra of one right-hand side of the largest level exceed the memory budget");
        return M2L_ENOMEM;
    }
    const long long base0 = pl->ldev[r.l0].base;
    const size_t e = sizeof(T);
    const size_t half = al256((size_t)max_clusters(pl) * Rc * F * 16 * e);
    const size_t phi_b = (size_t)pl->total_rows * R * n * e;
    M2L_TRY(ensure_buffer(ws, fft_rows_bytes(pl, R, precision)));
    M2L_TRY(ensure_buffer(spec, 2 * half));
    T *qhat = (T *)spec.buf;
    T *phihat = (T *)((char *)spec.buf + half);
    T *Phi = (T *)ws.buf;
    T *Z = (T *)((char *)ws.buf + al256(phi_b));
    const T *q = (const T *)r.q;
    T *out = (T *)r.L;
    const bool check_out = pl->output == M2L_OUT_CHECK_POTENTIAL;
    for (int l = r.l0; l <= r.l1; ++l) {
        LevelView L = view_of(pl->ldev[l]);
        L.cbase = 0;       // spectra of this level only
        L.R = R;           // row stride of densities and check potentials
        const T *ql = q + (L.base - base0) * R * n;
        T *dst = check_out ? out + (L.base - base0) * R * n : Phi + L.base * R * n;
        // TF32x3: the Hadamard products of full levels on the tensor cores, with the spectra
        // sibling-minor; other levels (and FP32) on the CUDA cores
        const bool tcl = precision == M2L_PREC_TF32X3 && D.Bhad && hadamard_tc_eligible(L) && fft_pg_available(p, g);
        for (int r0 = 0; r0 < R; r0 += Rc) {
            const int rc = std::min(Rc, R - r0);
            L.row0 = r0;
            stage_begin(pl, M2L_STAGE_FFT_FORWARD);
            // missing children's spectra stay zero; on a full level the transform writes every one
            if (L.nboxes != 8 * L.nclusters) cudaMemsetAsync(qhat, 0, (size_t)L.nclusters * rc * F * 16 * e, s);
            M2L_TRY(launch_fft_forward<T>(L, rc, p, n, g, pl->lattice_dev, (const T *)D.tw, ql, qhat, s, tcl));
            stage_end(pl, 1);
            stage_begin(pl, M2L_STAGE_HADAMARD);
            if constexpr (sizeof(T) == 4) {
                if (tcl)
                    M2L_TRY(launch_hadamard_tc(L, rc, F, D.Bhad, qhat, phihat, pl->had_chains, pl->num_sms, pl->dev_status, s));
                else
                    M2L_TRY(launch_hadamard<T>(L, rc, F, (const T *)D.Khat, qhat, phihat, s));
            } else {
                M2L_TRY(launch_hadamard<T>(L, rc, F, (const T *)D.Khat, qhat, phihat, s));
            }
            stage_end(pl, 1);
            stage_begin(pl, M2L_STAGE_FFT_INVERSE);
            M2L_TRY(launch_fft_inverse<T>(L, rc, p, n, g, pl->lattice_dev, (const T *)D.tw, phihat, dst, n,
                                          check_out ? pl->accumulate : 0, s, tcl));
            stage_end(pl, 1);
        }
    }
    if (!check_out) {
        // F6: locals = V_eps (Ut_eps Phi); in TF32x3 both products on the tensor cores, exact
        stage_begin(pl, M2L_STAGE_PINV);
        long long nl = 0;
        bool done_u = false, done_v = false;
        if constexpr (sizeof(T) == 4) {
            if (precision == M2L_PREC_TF32X3) {
                void *tws = (char *)ws.buf + al256(phi_b) + al256((size_t)pl->total_rows * R * rp * e);
                if (sliced_usable(D.Us, rp, rp, (const float *)Z)) {  // every column of Z (zeros past r)
                    M2L_TRY(launch_sliced(pl, D.Us, (const float *)(Phi + base0 * R * n), n, r.rows, (float *)Z, rp, rp, 0,
                                          tws, s));
                    done_u = true;
                    nl += 2;
                }
                if (sliced_usable(D.Vs, n, n, (const float *)out)) {
                    if (!done_u) {
                        M2L_TRY(launch_gemm_xwt<T>(Phi + base0 * R * n, n, (const T *)D.Ut, n, Z, rp, r.rows, rp, n, 0, s));
                        done_u = true;
                        nl += 1;
                    }
                    M2L_TRY(launch_sliced(pl, D.Vs, (const float *)Z, rp, r.rows, (float *)out, n, n, pl->accumulate, tws, s));
                    done_v = true;
                    nl += 2;
                }
            }
        }
        if (!done_u) {
            M2L_TRY(launch_gemm_xwt<T>(Phi + base0 * R * n, n, (const T *)D.Ut, n, Z, rp, r.rows, rp, n, 0, s));
            nl += 1;
        }
        if (!done_v) {
            M2L_TRY(apply_veps<T>(pl, D, Z, out, r.rows, pl->accumulate, true, s));
            nl += 1;
        }
        stage_end(pl, nl);
    }
    return M2L_OK;
}

// Runs a group on `s`. Workspaces: the plans' own, or (ws, spec) shared by every group of a batch:
// groups of a batch run one after another on one stream, so they can reuse the same memory.
static int run_group(std::vector<Run> &runs, int form, int precision, Workspace *ws, Workspace *spec, cudaStream_t s) {
    if (form == M2L_FORM_BLAS) {
        Workspace &w = ws ? *ws : runs[0].pl->ws;
        return precision == M2L_PREC_FP64 ? blas_group<double>(runs, precision, w, s)
                                          : blas_group<float>(runs, precision, w, s);
    }
    for (Run &r : runs) {
        r.rows = rows_of(r.pl, r.l0, r.l1, r.R);
        Workspace &w = ws ? *ws : r.pl->ws;
        Workspace &sp = spec ? *spec : r.pl->spec;
        int rc = precision == M2L_PREC_FP64 ? fft_run<double>(r, precision, w, sp, s)
                                            : fft_run<float>(r, precision, w, sp, s);
        if (rc) return rc;
    }
    return M2L_OK;
}

int apply_device(m2l_plan_t *pl, const void *q, void *L, int level, int R) {
    int l0 = level < 0 ? 2 : level, l1 = level < 0 ? pl->depth : level;
    int form, precision;
    M2L_TRY(resolve_form(pl, R, &form, &precision));
    M2L_TRY(prepare_plan(pl, form, precision));
    reset_stage_log(pl);
    std::vector<Run> runs(1);
    runs[0] = Run{pl, q, L, R, l0, l1, 0, 0};
    return run_group(runs, form, precision, nullptr, nullptr, pl->stream);
}

// ---------------------------------------------------------------------------------------------
// Batches of independent instances (device buffers, every level of each).

struct GroupKey {
    int p, pc, form, precision, kp, g;
    double rank_tol, dir_tol;
    bool operator==(const GroupKey &o) const {
        return p == o.p && pc == o.pc && form == o.form && precision == o.precision && kp == o.kp && g == o.g &&
               rank_tol == o.rank_tol &&
               dir_tol == o.dir_tol;
    }
};

int apply_batch(m2l_plan_t *const *plans, int n_inst, const void *const *q, void *const *L, const int *R) {
    m2l_plan_t *lead = plans[0];
    // resolve, prepare and group
    std::vector<GroupKey> keys;
    std::vector<std::vector<Run>> groups;
    std::vector<int> forms, precs;
    std::vector<long long> sig;
    for (int i = 0; i < n_inst; ++i) {
        m2l_plan_t *pl = plans[i];
        int form, prec;
        M2L_TRY(resolve_form(pl, R[i], &form, &prec));
        M2L_TRY(prepare_plan(pl, form, prec));
        GroupKey k{pl->p, pl->pc, form, prec, form == M2L_FORM_BLAS ? pl->kp : 0, form == M2L_FORM_FFT ? pl->g : 0,
                   form == M2L_FORM_BLAS ? pl->rank_tol : 0.0, form == M2L_FORM_BLAS ? pl->dir_tol : 0.0};
        size_t gi = 0;
        while (gi < keys.size() && !(keys[gi] == k)) ++gi;
        if (gi == keys.size()) {
            keys.push_back(k);
            groups.emplace_back();
            forms.push_back(form);
            precs.push_back(prec);
        }
        groups[gi].push_back(Run{pl, q[i], L[i], R[i], 2, pl->depth, 0, 0});
        for (long long v : {(long long)(uintptr_t)pl, (long long)(uintptr_t)q[i], (long long)(uintptr_t)L[i], (long long)R[i],
                            (long long)form, (long long)prec, (long long)pl->output, (long long)pl->accumulate,
                            pl->levels_version})
            sig.push_back(v);
    }
    // allocate everything the pass needs before any capture: one batch workspace and one spectra
    // buffer, each sized for the largest group or instance
    size_t ws_need = 0, spec_need = 0;
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        m2l_plan_t *own = groups[gi][0].pl;
        if (forms[gi] == M2L_FORM_BLAS) {
            long long nt = 0, total = 0;
            M2L_TRY(ensure_exec(own, groups[gi], contract_tile_rows(own, precs[gi]), &nt, &total));
            ws_need = std::max(ws_need, blas_layout(own, total, precs[gi]).total());
        } else {
            for (const Run &r : groups[gi]) {
                ws_need = std::max(ws_need, fft_rows_bytes(r.pl, r.R, precs[gi]));
                const int Rc = fft_rhs_chunk(r.pl, r.R, precs[gi]);
                if (Rc < 1) {
                    set_error("FFT form: the spectra of one right-hand side exceed the memory budget");
                    return M2L_ENOMEM;
                }
                const size_t e = precs[gi] == M2L_PREC_FP64 ? 8 : 4;
                spec_need = std::max(spec_need, 2 * al256((size_t)max_clusters(r.pl) * Rc * r.pl->F * 16 * e));
            }
        }
    }
    M2L_TRY(ensure_buffer(lead->batch_ws, ws_need));
    if (spec_need) M2L_TRY(ensure_buffer(lead->spec, spec_need));
    // the graph bakes in every device pointer it was captured with
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        for (const Run &r : groups[gi]) {
            const DevOps &D = r.pl->dev[precs[gi]];
            for (const void *ptr : {lead->batch_ws.buf, lead->spec.buf, r.pl->exec.levels, r.pl->exec.tiles,
                                    r.pl->exec.tvl, D.C, D.C_hi, D.C_lo, D.Ub, D.Vt, D.dir_meta, D.Khat, D.A, D.V, D.Vlo})
                sig.push_back((long long)(uintptr_t)ptr);
            sig.push_back(r.pl->tc_group);
            sig.push_back(r.pl->tc_chunk);
            sig.push_back(r.pl->tc_drain);
            sig.push_back(r.pl->fft_grid_opt);
        }
    }
    for (int i = 0; i < n_inst; ++i) reset_stage_log(plans[i]);
    cudaStream_t user = lead->stream;
    BatchGraph &G = lead->batch_graph;
    if (G.exec && G.sig == sig) {
        if (cudaGraphLaunch(G.exec, user) != cudaSuccess) {
            set_error("graph launch failed: %s", cudaGetErrorString(cudaGetLastError()));
            return M2L_ECUDA;
        }
        lead->launches = G.launches;
        return M2L_OK;
    }
    // capture the pass on a private stream, then run it on the caller's stream
    if (G.exec) cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
    G.sig.clear();
    if (!G.capture_stream && cudaStreamCreateWithFlags(&G.capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
        set_error("creating the capture stream failed");
        return M2L_ECUDA;
    }
    for (int i = 0; i < n_inst; ++i) plans[i]->capturing = 1;
    cudaGraph_t graph = nullptr;
    int rc = M2L_OK;
    if (cudaStreamBeginCapture(G.capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        set_error("stream capture failed to begin: %s", cudaGetErrorString(cudaGetLastError()));
        rc = M2L_ECUDA;
    } else {
        for (size_t gi = 0; gi < groups.size() && !rc; ++gi)
            rc = run_group(groups[gi], forms[gi], precs[gi], &lead->batch_ws, &lead->spec, G.capture_stream);
        cudaError_t e = cudaStreamEndCapture(G.capture_stream, &graph);
        if (!rc && e != cudaSuccess) {
            set_error("stream capture failed: %s", cudaGetErrorString(e));
            rc = M2L_ECUDA;
        }
    }
    long long launches = 0;
    for (int i = 0; i < n_inst; ++i) {
        plans[i]->capturing = 0;
        launches += plans[i]->launches;
    }
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc;
    }
    if (cudaGraphInstantiate(&G.exec, graph, 0) != cudaSuccess) {
        cudaGraphDestroy(graph);
        G.exec = nullptr;
        set_error("graph instantiation failed: %s", cudaGetErrorString(cudaGetLastError()));
        return M2L_ECUDA;
    }
    cudaGraphDestroy(graph);
    G.sig = sig;
    G.launches = launches;
    if (cudaGraphLaunch(G.exec, user) != cudaSuccess) {
        set_error("graph launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        return M2L_ECUDA;
    }
    lead->launches = launches;
    return M2L_OK;
}

void free_exec(m2l_plan_t *pl) {
    if (pl->exec.levels) cudaFree(pl->exec.levels);
    if (pl->exec.tiles) cudaFree(pl->exec.tiles);
    if (pl->exec.tvl) cudaFree(pl->exec.tvl);
    pl->exec = ExecCache();
    if (pl->batch_graph.exec) cudaGraphExecDestroy(pl->batch_graph.exec);
    if (pl->batch_graph.capture_stream) cudaStreamDestroy(pl->batch_graph.capture_stream);
    pl->batch_graph = BatchGraph();
}

}  // namespace m2l
