/*
 * cg_oracle.c -- FP64 CPU oracle for the conjugate-gradient companion solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may include, link
 * or call this file; tests, the smoke check and the benchmark's CPU baseline
 * use it to check and time the CUDA path.  It shares no code with the CUDA
 * sources.
 *
 * What it computes (Section 7.5, the conjugate-gradient case study):
 *   - the operator A is the 7-point Dirichlet Laplacian on the nx*ny*nz
 *     interior grid, 6 on the diagonal and -1 towards each interior face
 *     neighbour (the matrix an implicit step of the heat problem of Section 4
 *     gives; symmetric positive definite);
 *   - y = A p either matrix-free or from a CSR matrix (rowptr, col, val) with
 *     the row loop of Algorithm "spmv" (a):  s = 0; s = s + val[k] * p[col[k]]
 *     over the row's entries in storage order;
 *   - textbook unpreconditioned CG in FP64 (the paper runs double precision
 *     with a convergence tolerance of 1e-8 on the relative residual):
 *        r0 = b - A x0, p0 = r0, rho0 = r0.r0
 *        repeat:  q = A p;  alpha = rho / (p.q);  x = x + alpha p;
 *                 r = r - alpha q;  rho' = r.r;
 *                 stop when sqrt(rho') / ||b|| <= rtol;
 *                 beta = rho' / rho;  p = r + beta p;  rho = rho'
 *   - dot products summed sequentially in index order, in FP64.
 *
 * The matrix-free operator adds its terms in the same order as a CSR row with
 * ascending columns (z-1, y-1, x-1, diagonal, x+1, y+1, z+1), each term formed
 * as (coefficient * value), so for the 7-point matrix the two operators agree
 * bit for bit.  Compiled with -ffp-contract=off.  SpMV and the vector updates
 * are point-wise and may run on OpenMP threads without changing any result;
 * the dot products always run on one thread.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OP_STENCIL7 = 0, OP_CSR = 1 };

typedef struct {
    int32_t kind;
    int32_t nx, ny, nz;
    int64_t n;
    const int32_t* rowptr;
    const int32_t* col;
    const double* val;
} oracle_op;

typedef struct {
    int32_t iters;
    double relres_recur;   /* sqrt(r.r)/||b|| from the recurrence at exit */
    double relres_true;    /* ||b - A x|| / ||b|| recomputed at exit      */
    int32_t status;        /* 0 converged, 1 max_iter reached, -1 breakdown */
    double loop_seconds;   /* wall time of the iteration loop alone         */
} oracle_cg_info;

/* y = A p for the matrix-free 7-point Dirichlet Laplacian. */
void oracle_lap7_apply(int32_t nx, int32_t ny, int32_t nz, const double* p, double* y,
                       int32_t nthreads)
{
    const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
#ifdef _OPENMP
#pragma omp parallel for collapse(2) schedule(static) num_threads(nthreads < 1 ? 1 : nthreads)
#endif
    for (int64_t k = 0; k < nz; ++k) {
        for (int64_t j = 0; j < ny; ++j) {
            for (int64_t i = 0; i < nx; ++i) {
                const int64_t row = (k * ny + j) * nx + i;
                double s = 0.0;
                if (k > 0)      s = s + (-1.0) * p[row - sz];
                if (j > 0)      s = s + (-1.0) * p[row - sy];
                if (i > 0)      s = s + (-1.0) * p[row - sx];
                s = s + 6.0 * p[row];
                if (i < nx - 1) s = s + (-1.0) * p[row + sx];
                if (j < ny - 1) s = s + (-1.0) * p[row + sy];
                if (k < nz - 1) s = s + (-1.0) * p[row + sz];
                y[row] = s;
            }
        }
    }
    (void)nthreads;
}

/* y = A p for a CSR matrix, one row at a time (Algorithm "spmv" (a)). */
void oracle_csr_spmv(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                     const double* p, double* y, int32_t nthreads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads < 1 ? 1 : nthreads)
#endif
    for (int64_t r = 0; r < n; ++r) {
        double s = 0.0;
        for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) s = s + val[k] * p[col[k]];
        y[r] = s;
    }
    (void)nthreads;
}

static void apply_op(const oracle_op* A, const double* p, double* y, int32_t nthreads)
{
    if (A->kind == OP_STENCIL7)
        oracle_lap7_apply(A->nx, A->ny, A->nz, p, y, nthreads);
    else
        oracle_csr_spmv(A->n, A->rowptr, A->col, A->val, p, y, nthreads);
}

/* Sequential FP64 dot product in index order. */
double oracle_dot(int64_t n, const double* a, const double* b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s = s + a[i] * b[i];
    return s;
}

/*
 * Solve A x = b.  x holds x0 on entry and the last iterate on exit.
 * Returns 0 on success (info->status tells converged / max_iter / breakdown),
 * -1 on a bad argument, -2 when memory runs out.
 */
int oracle_cg(const oracle_op* A, const double* b, double* x, double rtol, int32_t max_iter,
              int32_t nthreads, oracle_cg_info* info)
{
    if (!A || !b || !x || !info || max_iter < 0 || !(rtol >= 0.0)) return -1;
    if (A->kind != OP_STENCIL7 && A->kind != OP_CSR) return -1;
    if (A->kind == OP_CSR && (!A->rowptr || !A->col || !A->val)) return -1;
    const int64_t n = A->n;
    if (n < 1) return -1;
    double* r = (double*)malloc(sizeof(double) * n);
    double* p = (double*)malloc(sizeof(double) * n);
    double* q = (double*)malloc(sizeof(double) * n);
    if (!r || !p || !q) { free(r); free(p); free(q); return -2; }

    memset(info, 0, sizeof(*info));
    const double bnorm = sqrt(oracle_dot(n, b, b));
    if (bnorm == 0.0) {                       /* A x = 0 has the solution x = 0 */
        memset(x, 0, sizeof(double) * n);
        free(r); free(p); free(q);
        return 0;
    }

    apply_op(A, x, q, nthreads);              /* r0 = b - A x0 */
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    memcpy(p, r, sizeof(double) * n);
    double rho = oracle_dot(n, r, r);
    double relres = sqrt(rho) / bnorm;
    int32_t it = 0;
    int32_t status = 1;
    if (relres <= rtol) status = 0;
    struct timespec t0, t1;
    clock_gettime(CLOCK_MONOTONIC, &t0);
    while (status == 1 && it < max_iter) {
        apply_op(A, p, q, nthreads);
        const double pq = oracle_dot(n, p, q);
        if (!(pq > 0.0)) { status = -1; break; }
        const double alpha = rho / pq;
        for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
        for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
        const double rho_new = oracle_dot(n, r, r);
        ++it;
        relres = sqrt(rho_new) / bnorm;
        if (relres <= rtol) { status = 0; break; }
        const double beta = rho_new / rho;
        for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        rho = rho_new;
    }
    clock_gettime(CLOCK_MONOTONIC, &t1);

    apply_op(A, x, q, nthreads);              /* true residual b - A x */
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    info->iters = it;
    info->relres_recur = relres;
    info->relres_true = sqrt(oracle_dot(n, r, r)) / bnorm;
    info->status = status;
    info->loop_seconds = (double)(t1.tv_sec - t0.tv_sec) + 1e-9 * (double)(t1.tv_nsec - t0.tv_nsec);
    free(r); free(p); free(q);
    return 0;
}
