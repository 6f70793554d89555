// Device-side view of a whole FMM around the M2L plan (the m2l_fmm_* entry points).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace m2l {

// One level of the FMM tree as the kernels see it (device pointers).
struct FmmLevel {
    const uint32_t *xyz = nullptr;  // [nboxes] packed x | y << 10 | z << 20, Morton order
    const int *child = nullptr;     // [nboxes][8] compact child at the next level or -1 (levels < depth)
    const int *parent = nullptr;    // [nboxes] compact parent at the previous level (levels > 2)
    long long base = 0;             // first row of the level in the multipole / local arrays
    double width = 0.0;             // box width of the level
};

struct FmmArgs {
    int depth = 0, n = 0, r_up = 0;
    double origin[3] = {0, 0, 0};
    FmmLevel levels[kMaxDepth + 1];
    const double *pts = nullptr;        // [N][3] sorted by leaf
    const double *q = nullptr;          // [N] charges, sorted order
    double *pot = nullptr;              // [N] potentials, sorted order
    const long long *leaf_start = nullptr;  // [leaves + 1]
    const long long *nbr_start = nullptr;   // [leaves + 1]
    const int *nbr = nullptr;               // neighbour leaves (P2P), itself included
    const double *unit = nullptr;       // [n][3] surface lattice mapped to [-1, 1]^3
    const double *v_up = nullptr;       // [n][r_up] upward pseudo-inverse factors at unit width
    const double *ut_up = nullptr;      // [r_up][n]
    const double *m2m = nullptr;        // [8][n][n] M2M operators by child octant
    const double *l2l = nullptr;        // [8][n][n] L2L operators by child octant
    double *Q = nullptr;                // [rows][n] multipoles, levels 2..depth
    double *L = nullptr;                // [rows][n] locals
};

int fmm_gather(const double *src, const long long *perm, long long n, double *dst, cudaStream_t s);
int fmm_scatter(const double *src, const long long *perm, long long n, double *dst, cudaStream_t s);
int fmm_upward(const FmmArgs &A, const long long *nboxes, cudaStream_t s);
int fmm_downward(const FmmArgs &A, const long long *nboxes, cudaStream_t s);

}  // namespace m2l
