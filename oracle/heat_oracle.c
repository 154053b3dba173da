/*
 * heat_oracle.c -- FP64 CPU oracle for the explicit 7-point heat update.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may include, link
 * or call this file; it exists so that tests, the smoke check and the CPU
 * baseline of the benchmark can compare the CUDA path against a plain,
 * obviously correct definition.  It shares no code, header or constant with
 * the CUDA sources.
 *
 * What it computes (Section 4, "Mathematical Details"):
 *   - the explicit update of Eq. 4, u^{m+1} = u^m + dt f + dt/(2h^2)(Dx+Dy+Dz),
 *     in its constant-coefficient form (kappa = 1, f = 0): every interior node
 *     becomes  u + r * (sum of its six face neighbours - 6 u)  with r = dt/h^2;
 *   - zero Dirichlet values on every boundary node, never updated
 *     (Section 4, text after Eq. 4; Algorithm heat3d initialises them to 0);
 *   - a double buffer that is swapped after every step, both buffers holding
 *     the same zero boundary (Algorithm "1-GPU Baseline": both u_old and u_new
 *     are initialised and copied, then swapped by pointer);
 *   - an integer step count instead of the paper's floating "while t < T"
 *     loop, so the number of steps is exact.
 *
 * Layout: the interior grid is nx*ny*nz values with x fastest and z slowest
 * (the paper loops k outer, j, i inner -- Algorithm COMPUTE_SINGLE_GPU -- and
 * splits along k, the slowest axis, Section 6.1).  Internally the oracle keeps
 * a padded (nx+2)(ny+2)(nz+2) array whose outer layer is the Dirichlet
 * boundary.
 *
 * Rounding: compiled with -ffp-contract=off (the paper builds its codes
 * without FMA contraction: Section 5, table of compiler flags), so every
 * operation below rounds once, in the written order:
 *     s  = ((u[i-1] + u[i+1]) + (u[j-1] + u[j+1])) + (u[k-1] + u[k+1])
 *     u' = u + r * (s - 6 u)
 * Each output point depends only on the previous time level, so the OpenMP
 * loop gives results identical to one thread.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline size_t pad_index(int64_t i, int64_t j, int64_t k, int64_t nx, int64_t ny)
{
    return (size_t)((k * (ny + 2) + j) * (nx + 2) + i);
}

/* One FTCS step on padded arrays: every interior node of dst from src. */
static void heat_one_step(const double* src, double* dst, int64_t nx, int64_t ny, int64_t nz,
                          double r, int nthreads)
{
    const int64_t sy = nx + 2;
    const int64_t sz = (nx + 2) * (ny + 2);
#ifdef _OPENMP
#pragma omp parallel for collapse(2) schedule(static) num_threads(nthreads)
#endif
    for (int64_t k = 1; k <= nz; ++k) {
        for (int64_t j = 1; j <= ny; ++j) {
            for (int64_t i = 1; i <= nx; ++i) {
                const size_t c = pad_index(i, j, k, nx, ny);
                const double u = src[c];
                const double along_x = src[c - 1] + src[c + 1];
                const double along_y = src[c - sy] + src[c + sy];
                const double along_z = src[c - sz] + src[c + sz];
                const double s = (along_x + along_y) + along_z;
                dst[c] = u + r * (s - 6.0 * u);
            }
        }
    }
    (void)nthreads;
}

/*
 * Run n_steps FTCS steps from the interior field u0 and write the interior of
 * the final field to u_out (both nx*ny*nz, x fastest).  u0 and u_out may
 * alias.  Returns 0, or -1 on a bad argument, -2 when memory runs out.
 */
int oracle_heat_run_timed(int32_t nx, int32_t ny, int32_t nz, double r, int64_t n_steps,
                          const double* u0, double* u_out, int32_t nthreads, double* loop_seconds);

int oracle_heat_run(int32_t nx, int32_t ny, int32_t nz, double r, int64_t n_steps,
                    const double* u0, double* u_out, int32_t nthreads)
{
    return oracle_heat_run_timed(nx, ny, nz, r, n_steps, u0, u_out, nthreads, NULL);
}

static double now_seconds(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* As oracle_heat_run; if loop_seconds is not NULL it receives the wall time
 * of the step loop alone (no allocation or copies), as the paper times only
 * its time-stepping loop (Algorithm "1-GPU Baseline"). */
int oracle_heat_run_timed(int32_t nx, int32_t ny, int32_t nz, double r, int64_t n_steps,
                          const double* u0, double* u_out, int32_t nthreads, double* loop_seconds)
{
    if (nx < 1 || ny < 1 || nz < 1 || n_steps < 0 || !u0 || !u_out) return -1;
    if (nthreads < 1) nthreads = 1;
    const size_t total = (size_t)(nx + 2) * (size_t)(ny + 2) * (size_t)(nz + 2);
    double* a = (double*)calloc(total, sizeof(double));
    double* b = (double*)calloc(total, sizeof(double));
    if (!a || !b) { free(a); free(b); return -2; }

    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j) {
            const double* row = u0 + ((size_t)k * ny + j) * nx;
            memcpy(a + pad_index(1, j + 1, k + 1, nx, ny), row, sizeof(double) * nx);
            memcpy(b + pad_index(1, j + 1, k + 1, nx, ny), row, sizeof(double) * nx);
        }

    const double t0 = now_seconds();
    for (int64_t m = 0; m < n_steps; ++m) {
        heat_one_step(a, b, nx, ny, nz, r, nthreads);
        double* t = a; a = b; b = t;   /* pointer swap, no data movement */
    }
    if (loop_seconds) *loop_seconds = now_seconds() - t0;

    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            memcpy(u_out + ((size_t)k * ny + j) * nx, a + pad_index(1, j + 1, k + 1, nx, ny),
                   sizeof(double) * nx);
    free(a);
    free(b);
    return 0;
}

/* Number of OpenMP threads the oracle would use by default (1 without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * The paper's variable-coefficient problem (Section 4, Eqs. 1-4):
 *     du/dt = div(kappa grad u) + f,
 *     kappa = 0.5 + 0.45 sin(pi x) sin(pi y) sin(pi z)      (Eq. 2)
 *     f     = 1 + cos(pi x) cos(pi y) cos(pi z)               (Eq. 3)
 *     u^{m+1} = u^m + dt f + dt/(2h^2) (Dx + Dy + Dz)          (Eq. 4)
 * with the face-averaged differences (the paper does not print D; this is
 * the reading consistent with beta = dt/(2h^2)):
 *     Dx = (k[i+1] + k[i]) (u[i+1] - u[i]) - (k[i] + k[i-1]) (u[i] - u[i-1])
 * On a grid of nx x ny x nz interior nodes, node i of the padded axis sits at
 * x = i h_x, h_x = 1/(nx+1) (the boundary nodes at x = 0 and 1 carry kappa
 * too).  dt = r h^2 with h = the smallest h_d (the paper's cubic grid has one
 * h and dt = h^2/(12 kappa_max), i.e. r = 1/(12 * 0.95)); each axis gets its
 * own beta_d = dt/(2 h_d^2).  Evaluation order (no FMA):
 *     s  = (bx Dx + by Dy) + bz Dz,   u' = (u + dt f) + s.
 * kappa_const > 0 replaces kappa by that constant, and with_source == 0 drops f
 * (both used to pin this routine).
 */
int oracle_heat_vk_run(int32_t nx, int32_t ny, int32_t nz, double r, int64_t n_steps,
                       const double* u0, double* u_out, int32_t nthreads, double kappa_const,
                       int32_t with_source)
{
    if (nx < 1 || ny < 1 || nz < 1 || n_steps < 0 || !u0 || !u_out) return -1;
    if (nthreads < 1) nthreads = 1;
    const double pi = 3.14159265358979323846;
    const double hx = 1.0 / (nx + 1), hy = 1.0 / (ny + 1), hz = 1.0 / (nz + 1);
    double h = hx;
    if (hy < h) h = hy;
    if (hz < h) h = hz;
    const double dt = r * h * h;
    const double bx = dt / (2.0 * hx * hx), by = dt / (2.0 * hy * hy), bz = dt / (2.0 * hz * hz);
    const size_t total = (size_t)(nx + 2) * (size_t)(ny + 2) * (size_t)(nz + 2);
    double* a = (double*)calloc(total, sizeof(double));
    double* b = (double*)calloc(total, sizeof(double));
    double* kap = (double*)calloc(total, sizeof(double));
    double* fdt = (double*)calloc(total, sizeof(double));
    if (!a || !b || !kap || !fdt) { free(a); free(b); free(kap); free(fdt); return -2; }
#ifdef _OPENMP
#pragma omp parallel for collapse(2) schedule(static) num_threads(nthreads)
#endif
    for (int64_t k = 0; k <= nz + 1; ++k)
        for (int64_t j = 0; j <= ny + 1; ++j)
            for (int64_t i = 0; i <= nx + 1; ++i) {
                const size_t c = pad_index(i, j, k, nx, ny);
                const double x = i * hx, y = j * hy, z = k * hz;
                kap[c] = kappa_const > 0.0 ? kappa_const
                                           : 0.5 + 0.45 * sin(pi * x) * sin(pi * y) * sin(pi * z);
                fdt[c] = with_source ? dt * (1.0 + cos(pi * x) * cos(pi * y) * cos(pi * z)) : 0.0;
            }
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j) {
            const double* row = u0 + ((size_t)k * ny + j) * nx;
            memcpy(a + pad_index(1, j + 1, k + 1, nx, ny), row, sizeof(double) * nx);
        }
    const int64_t sy = nx + 2, sz = (int64_t)(nx + 2) * (ny + 2);
    for (int64_t m = 0; m < n_steps; ++m) {
#ifdef _OPENMP
#pragma omp parallel for collapse(2) schedule(static) num_threads(nthreads)
#endif
        for (int64_t k = 1; k <= nz; ++k)
            for (int64_t j = 1; j <= ny; ++j)
                for (int64_t i = 1; i <= nx; ++i) {
                    const size_t c = pad_index(i, j, k, nx, ny);
                    const double u = a[c], kc = kap[c];
                    const double dx = (kap[c + 1] + kc) * (a[c + 1] - u) - (kc + kap[c - 1]) * (u - a[c - 1]);
                    const double dy = (kap[c + sy] + kc) * (a[c + sy] - u) - (kc + kap[c - sy]) * (u - a[c - sy]);
                    const double dz = (kap[c + sz] + kc) * (a[c + sz] - u) - (kc + kap[c - sz]) * (u - a[c - sz]);
                    const double s = (bx * dx + by * dy) + bz * dz;
                    b[c] = (u + fdt[c]) + s;
                }
        double* t = a; a = b; b = t;
    }
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            memcpy(u_out + ((size_t)k * ny + j) * nx, a + pad_index(1, j + 1, k + 1, nx, ny),
                   sizeof(double) * nx);
    free(a); free(b); free(kap); free(fdt);
    return 0;
}
