/*
 * Plain binary64 CPU loop for Eq. 1-2 (section 1): the CPU throughput figure
 * that the benchmark reports beside the oracle.
 *
 * TEST AND MEASUREMENT INFRASTRUCTURE ONLY, and not the oracle: no
 * compensated summation, the compiler may fuse multiply-adds and vectorise
 * (the j loop is an OpenMP simd reduction), and no parity check uses it.  It is what a straightforward OpenMP program
 * on the host cores achieves for the same sums, so that the GPU's speedup is
 * quoted against a fair CPU number as well as against the slow oracle.  It
 * shares no code with the GPU library.
 *
 * acc_k = -G sum_{j != i} m_j (r_i - r_j) / (|r_i - r_j|^2 + eps^2)^{3/2},
 * pot_k = -G sum_{j != i} m_j / (|r_i - r_j|^2 + eps^2)^{1/2}, for i = rows[k]
 * (all particles in order when rows == NULL).  pos, acc n x 3 row-major.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int plain_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int plain_accel(int64_t n, const double *pos, const double *mass, double eps, double G,
                int64_t nrows, const int64_t *rows, double *acc, double *pot, int nthreads) {
    if (n < 0 || !pos || !mass || !acc) return -1;
    const int64_t m = rows ? nrows : n;
    double *x = malloc(sizeof(double) * (size_t)(4 * n + 1));
    if (!x) return -1;
    double *y = x + n, *z = y + n, *w = z + n;
    for (int64_t j = 0; j < n; j++) {  /* structure of arrays for the vector units */
        x[j] = pos[3 * j];
        y[j] = pos[3 * j + 1];
        z[j] = pos[3 * j + 2];
        w[j] = mass[j];
    }
    const double e2 = eps * eps;
#ifdef _OPENMP
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
#endif
    for (int64_t k = 0; k < m; k++) {
        const int64_t i = rows ? rows[k] : k;
        const double xi = x[i], yi = y[i], zi = z[i];
        double ax = 0, ay = 0, az = 0, p = 0;
        /* j != i in Eq. 1: the two ranges on either side of i */
        for (int half = 0; half < 2; half++) {
            const int64_t j0 = half ? i + 1 : 0, j1 = half ? n : i;
#pragma omp simd reduction(+ : ax, ay, az, p)
            for (int64_t j = j0; j < j1; j++) {
                const double dx = xi - x[j], dy = yi - y[j], dz = zi - z[j];
                const double r2 = dx * dx + dy * dy + dz * dz + e2;
                const double inv = 1.0 / sqrt(r2);
                const double mi = w[j] * inv;
                const double f = mi * inv * inv;
                ax -= f * dx;
                ay -= f * dy;
                az -= f * dz;
                p -= mi;
            }
        }
        acc[3 * k] = G * ax;
        acc[3 * k + 1] = G * ay;
        acc[3 * k + 2] = G * az;
        if (pot) pot[k] = G * p;
    }
    free(x);
    return 0;
}
