/*
 * Oracle direct-sum matvec for the collocation system of the first-kind Laplace
 * volume integral equation (Sec. 2.1, Eqs. e:ie, e:k, e:a_2d, e:a_3d).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is part of the plain FP64 CPU oracle.  Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may build or call it; the
 * library under paper_2108_12574_gb300/ never does, and it shares no code with it.
 *
 * For every requested row i it forms, with one sequential double loop over j,
 *
 *     y_i = diag * x_i + sum_{j != i} w * K(p_i - p_j) * x_j,
 *
 * where K(r) = -(1/(2 pi)) log|r| in 2D and 1/(4 pi |r|) in 3D (Eq. e:k), p_j are the grid
 * points p_j = offset + spacing * (j_1, ..., j_d) with the point index row-major (last
 * coordinate fastest), w is the quadrature weight h^d and diag is the self-cell integral
 * (plus any shift), both computed by the Python side of the oracle and passed in.
 *
 * x and y are point-major: entry (j, k) of x, for right-hand side k, is x[j * nrhs + k];
 * y has one row of nrhs values per requested row, in the order of `rows`.
 * Rows are independent, so OpenMP spreads them over the host cores.
 */
#include <math.h>
#include <stdlib.h>

static void point_of(long long j, int dim, int n, double spacing, double offset, double *p)
{
    for (int d = dim - 1; d >= 0; --d) {
        p[d] = offset + spacing * (double)(j % n);
        j /= n;
    }
}

int oracle_matvec_rows(int dim, int n, double spacing, double offset, double weight,
                       double diag, const double *x, int nrhs, const long long *rows,
                       long long nrows, double *y)
{
    if (dim != 2 && dim != 3) return -1;
    if (nrhs < 1) return -1;
    long long N = 1;
    for (int d = 0; d < dim; ++d) N *= n;
    const double pi = 3.14159265358979323846;

    int bad = 0;
#pragma omp parallel for schedule(dynamic, 4)
    for (long long r = 0; r < nrows; ++r) {
        long long i = rows[r];
        if (i < 0 || i >= N) { bad = 1; continue; }
        double *acc = (double *)calloc((size_t)nrhs, sizeof(double));
        if (!acc) { bad = 1; continue; }
        double pi_[3], pj[3];
        point_of(i, dim, n, spacing, offset, pi_);
        for (long long j = 0; j < N; ++j) {
            if (j == i) continue;
            point_of(j, dim, n, spacing, offset, pj);
            double s = 0.0;
            for (int d = 0; d < dim; ++d) {
                double dd = pi_[d] - pj[d];
                s += dd * dd;
            }
            double dist = sqrt(s);
            double kern = (dim == 2) ? -log(dist) / (2.0 * pi) : 1.0 / (4.0 * pi * dist);
            double a = weight * kern;
            for (int k = 0; k < nrhs; ++k) acc[k] += a * x[j * nrhs + k];
        }
        for (int k = 0; k < nrhs; ++k) y[r * nrhs + k] = diag * x[i * nrhs + k] + acc[k];
        free(acc);
    }
    return bad ? -1 : 0;
}
