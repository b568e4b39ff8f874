/*
 * Row-parallel twin of oracle_propagate -- TEST INFRASTRUCTURE ONLY.
 *
 * The paper distributes the work of one state over OpenMP threads by rows
 * of the Hamiltonian (Sec. 3.7: MPI over random states, OpenMP over the
 * matrix-vector products).  This file is that scheme on the host cores, for
 * the all-cores CPU baseline and for parity runs at full size.  It computes
 * exactly what oracle_propagate computes (tbpm_oracle.c), in the same
 * floating-point operations:
 *   - H~ x row by row from a row list built from the bond list in bond
 *     order, so row i adds H_ij x_j in the same order as the bond-list
 *     scatter of oracle_apply_h (the states are bit-identical);
 *   - the same forward modified Chebyshev recurrence (Sec. 2.2, Eq. psi_t);
 *   - C_k = <psi0|phi_k> and <phi_k|phi_k> by compensated sums over fixed
 *     blocks of rows, the blocks combined in order: deterministic for any
 *     thread count, equal to the serial sums to about one rounding.
 * Pinned against oracle_propagate by tests/test_oracle_pins.py.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

#define ORACLE_OK 0
#define ORACLE_E_ARG -1
#define ORACLE_E_RANGE -2
#define ORACLE_E_NOMEM -3

int oracle_bessel(double z, int m_max, double *J);
int oracle_n_terms(double z);

/* Threads the parallel loops use (OMP_NUM_THREADS, else the cores). */
int oracle_threads(void) { return omp_get_max_threads(); }

typedef struct {
    double s, c;
} rsum;

static void rsum_add(rsum *k, double x)
{
    double t = k->s + x;
    if (fabs(k->s) >= fabs(x))
        k->c += (k->s - t) + x;
    else
        k->c += (x - t) + k->s;
    k->s = t;
}

/* Row list of H: row i holds (j, H_ij) for every bond touching i, in bond
 * order (a bond (i, j, t) gives (j, t) to row i and (i, conj t) to row j). */
typedef struct {
    int64_t *ptr;
    int64_t *col;
    double complex *val;
} rows_t;

static int build_rows(int64_t n, int64_t n_hop, const int64_t *hop_i, const int64_t *hop_j,
                      const double *hop_re, const double *hop_im, rows_t *R)
{
    R->ptr = calloc((size_t)n + 1, sizeof(int64_t));
    R->col = malloc((size_t)(2 * n_hop + 1) * sizeof(int64_t));
    R->val = malloc((size_t)(2 * n_hop + 1) * sizeof(double complex));
    int64_t *fill = malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!R->ptr || !R->col || !R->val || !fill) {
        free(fill);
        return ORACLE_E_NOMEM;
    }
    for (int64_t b = 0; b < n_hop; ++b) {
        ++R->ptr[hop_i[b] + 1];
        ++R->ptr[hop_j[b] + 1];
    }
    for (int64_t i = 0; i < n; ++i)
        R->ptr[i + 1] += R->ptr[i];
    memcpy(fill, R->ptr, (size_t)n * sizeof(int64_t));
    for (int64_t b = 0; b < n_hop; ++b) {
        int64_t i = hop_i[b], j = hop_j[b];
        double complex t = hop_re[b] + I * (hop_im ? hop_im[b] : 0.0);
        R->col[fill[i]] = j;
        R->val[fill[i]++] = t;
        R->col[fill[j]] = i;
        R->val[fill[j]++] = conj(t);
    }
    free(fill);
    return ORACLE_OK;
}

/* y = H~ x, each row on its own: eps_i x_i, then the row's entries in order,
 * then / s -- the operations of oracle_apply_h for that row. */
static void apply_rows(int64_t n, const double *onsite, const rows_t *R, double s,
                       const double complex *x, double complex *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double complex v = onsite ? onsite[i] * x[i] : 0.0;
        for (int64_t e = R->ptr[i]; e < R->ptr[i + 1]; ++e)
            v += R->val[e] * x[R->col[e]];
        y[i] = v / s;
    }
}

#define SUM_BLOCK 65536

int oracle_propagate_rows(int64_t n, const double *onsite, int64_t n_hop, const int64_t *hop_i,
                          const int64_t *hop_j, const double *hop_re, const double *hop_im,
                          double s, double z, int n_steps, int n_states,
                          const double complex *psi0, double complex *corr, double *norms,
                          double complex *psi_out)
{
    if (n <= 0 || n_steps < 0 || n_states <= 0 || !(s > 0.0) || !psi0 || !corr)
        return ORACLE_E_ARG;
    int M = oracle_n_terms(z);
    if (M < 2)
        return ORACLE_E_RANGE;
    double J[129];
    oracle_bessel(z, M, J);
    rows_t R = {NULL, NULL, NULL};
    int64_t n_blk = (n + SUM_BLOCK - 1) / SUM_BLOCK;
    double complex *phi = malloc((size_t)n * sizeof(double complex));
    double complex *t0 = malloc((size_t)n * sizeof(double complex));
    double complex *t1 = malloc((size_t)n * sizeof(double complex));
    double complex *t2 = malloc((size_t)n * sizeof(double complex));
    double complex *acc = malloc((size_t)n * sizeof(double complex));
    rsum *blk = malloc((size_t)n_blk * 3 * sizeof(rsum));
    int rc = (phi && t0 && t1 && t2 && acc && blk) ? ORACLE_OK : ORACLE_E_NOMEM;
    if (rc == ORACLE_OK)
        rc = build_rows(n, n_hop, hop_i, hop_j, hop_re, hop_im, &R);
    if (rc != ORACLE_OK) {
        free(phi); free(t0); free(t1); free(t2); free(acc); free(blk);
        free(R.ptr); free(R.col); free(R.val);
        return rc;
    }
    for (int p = 0; p < n_states; ++p) {
        const double complex *a = psi0 + (size_t)p * n;
        memcpy(phi, a, (size_t)n * sizeof(double complex));
        for (int k = 0; k <= n_steps; ++k) {
            if (k > 0) {
                memcpy(t0, phi, (size_t)n * sizeof(double complex));
                apply_rows(n, onsite, &R, s, t0, t1);
#pragma omp parallel for schedule(static)
                for (int64_t i = 0; i < n; ++i) {
                    t1[i] *= -I;
                    acc[i] = J[0] * t0[i] + 2.0 * J[1] * t1[i];
                }
                for (int m = 2; m < M; ++m) {
                    apply_rows(n, onsite, &R, s, t1, t2);
#pragma omp parallel for schedule(static)
                    for (int64_t i = 0; i < n; ++i) {
                        t2[i] = -2.0 * I * t2[i] + t0[i];
                        acc[i] += 2.0 * J[m] * t2[i];
                    }
                    double complex *tmp = t0;
                    t0 = t1;
                    t1 = t2;
                    t2 = tmp;
                }
                memcpy(phi, acc, (size_t)n * sizeof(double complex));
            }
            /* compensated sums per block of rows, then the blocks in order */
#pragma omp parallel for schedule(static)
            for (int64_t q = 0; q < n_blk; ++q) {
                rsum cre = {0, 0}, cim = {0, 0}, nn = {0, 0};
                int64_t hi = (q + 1) * SUM_BLOCK < n ? (q + 1) * SUM_BLOCK : n;
                for (int64_t i = q * SUM_BLOCK; i < hi; ++i) {
                    double complex v = conj(a[i]) * phi[i];
                    rsum_add(&cre, creal(v));
                    rsum_add(&cim, cimag(v));
                    rsum_add(&nn, creal(phi[i]) * creal(phi[i]) + cimag(phi[i]) * cimag(phi[i]));
                }
                blk[3 * q] = cre;
                blk[3 * q + 1] = cim;
                blk[3 * q + 2] = nn;
            }
            rsum cre = {0, 0}, cim = {0, 0}, nn = {0, 0};
            for (int64_t q = 0; q < n_blk; ++q) {
                rsum_add(&cre, blk[3 * q].s);
                rsum_add(&cre, blk[3 * q].c);
                rsum_add(&cim, blk[3 * q + 1].s);
                rsum_add(&cim, blk[3 * q + 1].c);
                rsum_add(&nn, blk[3 * q + 2].s);
                rsum_add(&nn, blk[3 * q + 2].c);
            }
            corr[(size_t)p * (n_steps + 1) + k] = (cre.s + cre.c) + I * (cim.s + cim.c);
            if (norms)
                norms[(size_t)p * (n_steps + 1) + k] = nn.s + nn.c;
        }
        if (psi_out)
            memcpy(psi_out + (size_t)p * n, phi, (size_t)n * sizeof(double complex));
    }
    free(phi); free(t0); free(t1); free(t2); free(acc); free(blk);
    free(R.ptr); free(R.col); free(R.val);
    return ORACLE_OK;
}
