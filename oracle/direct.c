/*
 * Oracle helper (test infrastructure; see oracle/__init__.py): check potentials of the
 * M2L translation by plain direct summation, FP64.
 *
 * For every target box tau in the list and every right-hand side r,
 *     phi[tau][r][i] = sum_{sigma in I_tau} sum_j K(x_i, y_j) q[sigma][r][j]
 * with x_i the downward-check points of tau, y_j the upward-equivalent points of sigma and
 * K(x, y) = 1 / (4 pi |x - y|): the sum inside Eq. 11 of arxiv 2408.07436 (Sec. 2.2), with
 * the kernel of Eq. 2. Each K_{sigma,tau} entry is evaluated from the two boxes' actual
 * coordinates; nothing is cached or reordered. Sources are taken in the order of the list
 * (ascending Morton order) and j ascending.
 *
 * Arguments (row-major, caller-owned host arrays):
 *   n          points per surface
 *   x_off      n x 3  downward-check points relative to the target centre
 *   y_off      n x 3  upward-equivalent points relative to the source centre
 *   n_targets  number of targets
 *   t_centre   n_targets x 3 target centres
 *   offsets    n_targets + 1 CSR offsets into the source arrays
 *   s_centre   S x 3  centre of each listed source
 *   s_row      S      row of each listed source in q
 *   q          rows x R x n equivalent densities
 *   R          right-hand sides
 *   phi        n_targets x R x n output (overwritten)
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

void oracle_check_potential(int nx, int ny, const double *x_off, const double *y_off,
                            long long n_targets, const double *t_centre,
                            const long long *offsets, const double *s_centre,
                            const long long *s_row, const double *q, int R, double *phi)
{
    const double four_pi = 4.0 * 3.14159265358979323846;
#pragma omp parallel for schedule(dynamic, 4)
    for (long long t = 0; t < n_targets; ++t) {
        double *out = phi + (size_t)t * R * nx;
        memset(out, 0, sizeof(double) * (size_t)R * nx);
        for (long long e = offsets[t]; e < offsets[t + 1]; ++e) {
            const double *qs = q + (size_t)s_row[e] * R * ny;
            for (int i = 0; i < nx; ++i) {
                double xi0 = t_centre[3 * t + 0] + x_off[3 * i + 0];
                double xi1 = t_centre[3 * t + 1] + x_off[3 * i + 1];
                double xi2 = t_centre[3 * t + 2] + x_off[3 * i + 2];
                for (int j = 0; j < ny; ++j) {
                    double d0 = xi0 - (s_centre[3 * e + 0] + y_off[3 * j + 0]);
                    double d1 = xi1 - (s_centre[3 * e + 1] + y_off[3 * j + 1]);
                    double d2 = xi2 - (s_centre[3 * e + 2] + y_off[3 * j + 2]);
                    double k = 1.0 / (four_pi * sqrt(d0 * d0 + d1 * d1 + d2 * d2));
                    for (int r = 0; r < R; ++r)
                        out[(size_t)r * nx + i] += k * qs[(size_t)r * ny + j];
                }
            }
        }
    }
}

/* Potential at arbitrary points from a set of point charges: out[i] = sum_j K(x_i, y_j) q_j,
 * skipping coincident points (used by the oracle's direct P2P reference, Eq. 1). */
void oracle_direct_potential(long long m, const double *x, long long nsrc, const double *y,
                             const double *q, double *out)
{
    const double four_pi = 4.0 * 3.14159265358979323846;
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < m; ++i) {
        double acc = 0.0;
        for (long long j = 0; j < nsrc; ++j) {
            double d0 = x[3 * i + 0] - y[3 * j + 0];
            double d1 = x[3 * i + 1] - y[3 * j + 1];
            double d2 = x[3 * i + 2] - y[3 * j + 2];
            double r2 = d0 * d0 + d1 * d1 + d2 * d2;
            if (r2 > 0.0) acc += q[j] / (four_pi * sqrt(r2));
        }
        out[i] = acc;
    }
}
