/*
 * FP64 CPU oracle for the direct particle-particle (PP) N-body method of
 * Khrapov, Khoperskov & Khoperskov (2018), "New features of parallel
 * implementation of N-body problems on GPU".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * GPU library is checked against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the CUDA library, and it never calls it.
 *
 * What it computes, each function citing the passage it follows:
 *   oracle_accel  -- Eq. 1-2 (section 1): a_i = sum_{j != i} f_ij with
 *                    f_ij = -G m_j (r_i - r_j) / (|r_i - r_j|^2 + delta^2)^{3/2};
 *                    the softened distance is the paper's definition
 *                    |r_i - r_j + delta| = sqrt(dx^2 + dy^2 + dz^2 + delta^2).
 *                    The potential pot_i = -G sum_{j != i} m_j / sqrt(d^2 + delta^2)
 *                    is the per-particle factor of the energy, Eq. 8.
 *   oracle_kdk    -- Eq. 5-7 (section 1): predictor, drift, new force, corrector.
 *   oracle_rk4    -- the fourth-order scheme of the abstract, read as the
 *                    classical Runge-Kutta method on (r, v) (the paper does not
 *                    define its fourth-order scheme).
 *   oracle_fr4    -- the other reading of that scheme: the fourth-order
 *                    symplectic composition of the KDK step of Eq. 5-7
 *                    (Yoshida 1990; Forest and Ruth 1990).
 *   oracle_diag   -- Eq. 8-10 (section 3): E, P, L (full vector; L_z is Eq. 10).
 *                    Eq. 8 prints the potential term with a + sign; a bound
 *                    self-gravitating system has negative potential energy, so
 *                    the term is taken as -1/2 sum_i sum_{j != i} G m_i m_j / |r_ij + delta|.
 *
 * Arithmetic: IEEE binary64, round to nearest, compiled with
 * -ffp-contract=off so that no fused multiply-add changes a rounding.  Every
 * sum over particles uses Neumaier's compensated summation (A. Neumaier, 1974,
 * "Rundungsfehleranalyse einiger Verfahren zur Summation endlicher Summen"),
 * taken in plain index order j = 0..n-1, so a result is accurate to about one
 * rounding of each term.  The self pair j == i is skipped explicitly, so
 * delta = 0 is allowed.  Loops over i may run on several OpenMP threads; the
 * result does not depend on the thread count.
 *
 * Layout: pos, vel, acc are n x 3 row-major (x, y, z of particle i at
 * 3i..3i+2); mass, pot, smag are length n.  All pointers are host memory owned
 * by the caller.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double s, c; } nsum_t;

static void nsum_add(nsum_t *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double nsum_val(const nsum_t *a) { return a->s + a->c; }

static int threads_for(int nthreads) {
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int oracle_max_threads(void) { return threads_for(0); }

/*
 * Eq. 1-2 for one particle i against all j != i.
 * acc_i[3] <- sum_j -G m_j d_ij / w_ij,   w_ij = (|d_ij|^2 + eps^2)^{3/2}
 * *pot_i   <- sum_j -G m_j / sqrt(|d_ij|^2 + eps^2)
 * *smag_i  <- sum_j  G m_j |d_ij| / w_ij  (the sum of term magnitudes; it sets
 *             the scale of rounding error in acc_i)
 */
static void accel_one(int64_t n, const double *pos, const double *mass,
                      double eps, double G, int64_t i,
                      double acc_i[3], double *pot_i, double *smag_i) {
    nsum_t ax = {0, 0}, ay = {0, 0}, az = {0, 0}, p = {0, 0}, s = {0, 0};
    const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
    const double eps2 = eps * eps;
    for (int64_t j = 0; j < n; j++) {
        if (j == i) continue;                       /* j != i in Eq. 1 */
        double dx = xi - pos[3 * j];
        double dy = yi - pos[3 * j + 1];
        double dz = zi - pos[3 * j + 2];
        double d2 = dx * dx + dy * dy + dz * dz;
        double soft2 = d2 + eps2;                   /* |r_i - r_j + delta|^2 */
        double soft = sqrt(soft2);
        double w = soft2 * soft;                    /* |r_i - r_j + delta|^3 */
        double gm = G * mass[j];
        nsum_add(&ax, -gm * dx / w);
        nsum_add(&ay, -gm * dy / w);
        nsum_add(&az, -gm * dz / w);
        nsum_add(&p, -gm / soft);
        nsum_add(&s, gm * sqrt(d2) / w);
    }
    acc_i[0] = nsum_val(&ax);
    acc_i[1] = nsum_val(&ay);
    acc_i[2] = nsum_val(&az);
    *pot_i = nsum_val(&p);
    *smag_i = nsum_val(&s);
}

/*
 * Accelerations and potentials for the particles listed in rows[0..nrows-1]
 * (all n particles, in order, when rows == NULL; then nrows is ignored).
 * Output k refers to particle rows[k]: acc[3k..3k+2], pot[k], smag[k].
 * pot and smag may be NULL.  Returns 0, or -1 on a bad argument.
 */
int oracle_accel(int64_t n, const double *pos, const double *mass,
                 double eps, double G, int64_t nrows, const int64_t *rows,
                 double *acc, double *pot, double *smag, int nthreads) {
    if (n < 0 || !pos || !mass || !acc) return -1;
    int64_t m = rows ? nrows : n;
    for (int64_t k = 0; rows && k < m; k++)
        if (rows[k] < 0 || rows[k] >= n) return -1;
    int nt = threads_for(nthreads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t k = 0; k < m; k++) {
        int64_t i = rows ? rows[k] : k;
        double a[3], p, s;
        accel_one(n, pos, mass, eps, G, i, a, &p, &s);
        acc[3 * k] = a[0];
        acc[3 * k + 1] = a[1];
        acc[3 * k + 2] = a[2];
        if (pot) pot[k] = p;
        if (smag) smag[k] = s;
    }
    return 0;
}

/*
 * KDK leapfrog, Eq. 5-7, nsteps steps of size dt, in place on pos and vel.
 * acc holds a(t) on entry (the caller evaluates it once at the start, since
 * Eq. 5 needs it before the first step) and a(t + nsteps*dt) on exit.
 *   (5) vt = v + dt * a(t)
 *   (6) r  = r + dt/2 * (vt + v)
 *       a  = accel(r)                      (the recomputation after Eq. 6)
 *   (7) v  = (v + vt)/2 + dt/2 * a
 * pot (may be NULL) receives the potential at the final positions.
 */
int oracle_kdk(int64_t n, double *pos, double *vel, const double *mass,
               double eps, double G, double dt, int64_t nsteps,
               double *acc, double *pot, int nthreads) {
    if (n < 1 || !pos || !vel || !mass || !acc || nsteps < 0) return -1;
    double *vt = malloc(sizeof(double) * 3 * n);
    double *pp = malloc(sizeof(double) * n);
    double *ss = malloc(sizeof(double) * n);
    if (!vt || !pp || !ss) { free(vt); free(pp); free(ss); return -1; }
    for (int64_t st = 0; st < nsteps; st++) {
        for (int64_t k = 0; k < 3 * n; k++) {
            vt[k] = vel[k] + dt * acc[k];                   /* Eq. 5 */
            pos[k] = pos[k] + (dt / 2) * (vt[k] + vel[k]);  /* Eq. 6 */
        }
        oracle_accel(n, pos, mass, eps, G, 0, NULL, acc, pp, ss, nthreads);
        for (int64_t k = 0; k < 3 * n; k++)
            vel[k] = (vel[k] + vt[k]) / 2 + (dt / 2) * acc[k];  /* Eq. 7 */
    }
    if (pot) {
        if (nsteps == 0) oracle_accel(n, pos, mass, eps, G, 0, NULL, acc, pp, ss, nthreads);
        memcpy(pot, pp, sizeof(double) * n);
    }
    free(vt); free(pp); free(ss);
    return 0;
}

/*
 * Classical fourth-order Runge-Kutta on y = (r, v), y' = (v, a(r)), nsteps
 * steps of size dt, in place.  Four force evaluations per step:
 *   k1 = (v,            a(r))
 *   k2 = (v + dt/2 a1,  a(r + dt/2 v))
 *   k3 = (v + dt/2 a2,  a(r + dt/2 (v + dt/2 a1)))
 *   k4 = (v + dt a3,    a(r + dt (v + dt/2 a2)))
 *   y += dt/6 (k1 + 2 k2 + 2 k3 + k4)
 * acc receives a at the final positions.
 */
int oracle_rk4(int64_t n, double *pos, double *vel, const double *mass,
               double eps, double G, double dt, int64_t nsteps,
               double *acc, int nthreads) {
    if (n < 1 || !pos || !vel || !mass || !acc || nsteps < 0) return -1;
    size_t b = sizeof(double) * 3 * n;
    double *a1 = malloc(b), *a2 = malloc(b), *a3 = malloc(b), *a4 = malloc(b);
    double *v2 = malloc(b), *v3 = malloc(b), *v4 = malloc(b), *rs = malloc(b);
    if (!a1 || !a2 || !a3 || !a4 || !v2 || !v3 || !v4 || !rs) {
        free(a1); free(a2); free(a3); free(a4); free(v2); free(v3); free(v4); free(rs);
        return -1;
    }
    for (int64_t st = 0; st < nsteps; st++) {
        oracle_accel(n, pos, mass, eps, G, 0, NULL, a1, NULL, NULL, nthreads);
        for (int64_t k = 0; k < 3 * n; k++) {
            v2[k] = vel[k] + (dt / 2) * a1[k];
            rs[k] = pos[k] + (dt / 2) * vel[k];
        }
        oracle_accel(n, rs, mass, eps, G, 0, NULL, a2, NULL, NULL, nthreads);
        for (int64_t k = 0; k < 3 * n; k++) {
            v3[k] = vel[k] + (dt / 2) * a2[k];
            rs[k] = pos[k] + (dt / 2) * v2[k];
        }
        oracle_accel(n, rs, mass, eps, G, 0, NULL, a3, NULL, NULL, nthreads);
        for (int64_t k = 0; k < 3 * n; k++) {
            v4[k] = vel[k] + dt * a3[k];
            rs[k] = pos[k] + dt * v3[k];
        }
        oracle_accel(n, rs, mass, eps, G, 0, NULL, a4, NULL, NULL, nthreads);
        for (int64_t k = 0; k < 3 * n; k++) {
            pos[k] = pos[k] + (dt / 6) * (vel[k] + 2 * v2[k] + 2 * v3[k] + v4[k]);
            vel[k] = vel[k] + (dt / 6) * (a1[k] + 2 * a2[k] + 2 * a3[k] + a4[k]);
        }
    }
    oracle_accel(n, pos, mass, eps, G, 0, NULL, acc, NULL, NULL, nthreads);
    free(a1); free(a2); free(a3); free(a4); free(v2); free(v3); free(v4); free(rs);
    return 0;
}

/*
 * Fourth-order symplectic composition of the KDK step (H. Yoshida, 1990,
 * "Construction of higher order symplectic integrators", Phys. Lett. A 150,
 * 262; E. Forest and R. D. Ruth, 1990, Physica D 43, 105): one step of size
 * dt is three steps of Eq. 5-7 of sizes w1 dt, w0 dt, w1 dt, with
 *   w1 = 1 / (2 - 2^(1/3)),   w0 = -2^(1/3) / (2 - 2^(1/3)),
 * so that 2 w1 + w0 = 1 (consistency) and 2 w1^3 + w0^3 = 0, which cancels
 * the third-order error term of the time-symmetric KDK step.  The middle step
 * runs backwards in time.  Three force evaluations per step: the force at the
 * end of one KDK step is the start of the next.  acc holds a(t0) on entry and
 * a at the final positions on return; pot (may be NULL) the potential there.
 * The weights are the binary64 roundings of the exact values.
 */
#define FR4_W1 0x1.59e8b6eb96338p+0  /* 1.3512071919596576... */
#define FR4_W0 -0x1.b3d16dd72c671p+0 /* -1.7024143839193153... */
int oracle_fr4(int64_t n, double *pos, double *vel, const double *mass,
               double eps, double G, double dt, int64_t nsteps,
               double *acc, double *pot, int nthreads) {
    if (n < 1 || !pos || !vel || !mass || !acc || nsteps < 0) return -1;
    const double w[3] = {FR4_W1, FR4_W0, FR4_W1};
    if (nsteps == 0) return oracle_kdk(n, pos, vel, mass, eps, G, dt, 0, acc, pot, nthreads);
    for (int64_t st = 0; st < nsteps; st++)
        for (int s = 0; s < 3; s++) {
            double *p = (st == nsteps - 1 && s == 2) ? pot : NULL;
            if (oracle_kdk(n, pos, vel, mass, eps, G, w[s] * dt, 1, acc, p, nthreads)) return -1;
        }
    return 0;
}

/*
 * Eq. 8-10.  out[0] = E, out[1] = K = sum m |v|^2 / 2, out[2] = W (potential
 * energy, negative), out[3..5] = P (Eq. 9), out[6..8] = L = sum m r x v
 * (out[8] = L_z is Eq. 10).  W is summed over ordered pairs j != i and halved.
 */
int oracle_diag(int64_t n, const double *pos, const double *vel,
                const double *mass, double eps, double G, double *out,
                int nthreads) {
    if (n < 1 || !pos || !vel || !mass || !out) return -1;
    double *pot = malloc(sizeof(double) * n);
    double *acc = malloc(sizeof(double) * 3 * n);
    if (!pot || !acc) { free(pot); free(acc); return -1; }
    oracle_accel(n, pos, mass, eps, G, 0, NULL, acc, pot, NULL, nthreads);
    nsum_t K = {0, 0}, W = {0, 0}, P[3] = {{0, 0}, {0, 0}, {0, 0}}, L[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int64_t i = 0; i < n; i++) {
        const double *r = pos + 3 * i, *v = vel + 3 * i;
        double m = mass[i];
        nsum_add(&K, m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / 2);
        nsum_add(&W, m * pot[i] / 2);   /* pot_i already carries -G sum_j m_j / |r_ij + delta| */
        for (int c = 0; c < 3; c++) nsum_add(&P[c], m * v[c]);
        nsum_add(&L[0], m * (r[1] * v[2] - r[2] * v[1]));
        nsum_add(&L[1], m * (r[2] * v[0] - r[0] * v[2]));
        nsum_add(&L[2], m * (r[0] * v[1] - r[1] * v[0]));
    }
    out[1] = nsum_val(&K);
    out[2] = nsum_val(&W);
    out[0] = out[1] + out[2];
    for (int c = 0; c < 3; c++) { out[3 + c] = nsum_val(&P[c]); out[6 + c] = nsum_val(&L[c]); }
    free(pot); free(acc);
    return 0;
}
