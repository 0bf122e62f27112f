/*
 * Plain FP64 CPU oracle for the adaptive-force-update gravity path
 * (Grudic 2020, "Accelerating self-gravitating hydrodynamics simulations
 * with adaptive force updates", Section 2 and Section 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no source, header, table or helper with
 * the CUDA library; both sides are written from the paper independently.
 *
 * Everything here is the plain definition, written out:
 *   - force evaluation: O(n_tgt * N) direct summation over all sources j != i
 *     of the softened acceleration, its time derivative (jerk, Eq. 4) and its
 *     position derivative (the tidal tensor of Section 3), each sum
 *     Neumaier-compensated; the tidal timestep of Eq. (tidaltimestep);
 *   - the force-update counter (Eq. 3) and update condition
 *     (Eq. updatecondition) on power-of-two time bins (Section 3);
 *   - compaction of the due set in ascending index order;
 *   - the first-order jerk predictor (Eq. jerkupdate) in closed form, and
 *     the first-order polynomial predictor from logged accelerations
 *     (Section 2.2);
 *   - the adjoint (reverse-mode) sums for a loss on a and on the potential
 *     energy (not in the paper; derived from Eq. 4 and the tidal tensor);
 *   - adaptive softening (Section 3: fully adaptive softening with the
 *     energy-conserving correction terms of Price & Monaghan 2007): supports
 *     h_i from a mass-density constraint by safeguarded Newton iterations,
 *     the correction coefficients zeta_i, and the sums with pair-averaged
 *     kernels plus the correction term.
 *
 * Readings where the paper is silent (all listed with reasons in the design
 * notes of the repository):
 *   - softening: cubic-spline (M4) density kernel of compact support radius
 *     h, W(r,h) = 8/(pi h^3) w(r/h); the force is exactly Newtonian for
 *     r >= h.  f(r) = M(<r)/(m r^3), g(r) = f'(r)/r, phi the potential kernel
 *     (Phi_i = -G sum m_j phi(r_ij)), all derived by integrating W.
 *   - the self term j == i is excluded by index, not by distance;
 *   - T is d a / d x_i (negative semi-definite at a point mass' far field);
 *     stored as xx, yy, zz, xy, xz, yz;
 *   - time is counted in integer ticks of dt_min = dt_max * 2^-k_max;
 *   - every floating-point step of selection and binning is a single
 *     correctly rounded IEEE operation (built with -ffp-contract=off).
 *
 * All functions return 0 on success and a negative value on bad arguments.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* Softened kernel functions (cubic spline of support h).                      */
/* f = M(<r)/(m r^3), g = f'(r)/r, phi: potential kernel, phi = 1/r for r>=h.  */
/* Obtained by integrating W: M(<r)/m = 4 pi int_0^r s^2 W ds and              */
/* phi(r) = int_r^inf s f(s) ds.  The Newtonian limit is f = r^-3, g = -3r^-5. */
/* ------------------------------------------------------------------------- */
void oracle_kernel(double r, double h, double *f, double *g, double *phi)
{
    if (r >= h) {
        double r2 = r * r;
        *f = 1.0 / (r2 * r);
        *g = -3.0 / (r2 * r2 * r);
        *phi = 1.0 / r;
        return;
    }
    double u = r / h;
    double h2 = h * h;
    double h3 = h2 * h;
    double h5 = h3 * h2;
    if (u < 0.5) {
        double u2 = u * u;
        *f = (32.0 / 3.0 + u2 * (-192.0 / 5.0 + 32.0 * u)) / h3;
        *g = (-384.0 / 5.0 + 96.0 * u) / h5;
        *phi = (14.0 / 5.0 + u2 * (-16.0 / 3.0 + u2 * (48.0 / 5.0 - 32.0 / 5.0 * u))) / h;
    } else {
        double u2 = u * u;
        double u3 = u2 * u;
        double u5 = u3 * u2;
        *f = (64.0 / 3.0 + u * (-48.0 + u * (192.0 / 5.0 - 32.0 / 3.0 * u)) - 1.0 / (15.0 * u3)) / h3;
        *g = (-48.0 / u + 384.0 / 5.0 - 32.0 * u + 1.0 / (5.0 * u5)) / h5;
        *phi = (16.0 / 5.0 - 1.0 / (15.0 * u) + u2 * (-32.0 / 3.0 + u * (16.0 + u * (-48.0 / 5.0 + 32.0 / 15.0 * u)))) / h;
    }
}

/* Neumaier-compensated running sum. */
typedef struct { double s, c; } nsum;

static inline void nadd(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static inline double nval(const nsum *a) { return a->s + a->c; }

/* Tidal timestep, Eq. (tidaltimestep): sqrt(eta) * (||T||_F^2 / 6)^(-1/4).
 * ||T||_F^2 summed in the fixed order xx, yy, zz, then the off-diagonals
 * counted twice.  +inf when T vanishes. */
double oracle_tidal_dt(const double *t6, double eta)
{
    double s = t6[0] * t6[0];
    s = s + t6[1] * t6[1];
    s = s + t6[2] * t6[2];
    s = s + 2.0 * (t6[3] * t6[3]);
    s = s + 2.0 * (t6[4] * t6[4]);
    s = s + 2.0 * (t6[5] * t6[5]);
    if (s == 0.0) return INFINITY;
    return sqrt(eta) / sqrt(sqrt(s / 6.0));
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Force evaluation at n_tgt targets (idx[t], or t itself when idx is NULL)
 * against all n_src sources, j != i.  Outputs are per target slot t:
 *   acc[3t..]   a_i   = G sum_j m_j f(r) d
 *   jerk[3t..]  j_i   = G sum_j m_j [ f(r) v_ji + g(r) (d . v_ji) d ]     (Eq. 4)
 *   tidal[6t..] T_i   = -G sum_j m_j [ f(r) I + g(r) d d^T ]    (d a_i / d x_i)
 *   pot[t]      Phi_i = -G sum_j m_j phi(r)                       (nullable)
 *   dt_grav[t]  sqrt(eta) (||T_i||^2/6)^(-1/4)                    (nullable)
 * with d = x_j - x_i, v_ji = v_j - v_i, r = |d|.
 */
void oracle_kernel_w(double r, double h, double *w, double *w_r, double *w_h, double *psi_h);

/* Shared by oracle_eval (one support h for every pair, hs == NULL) and
 * oracle_eval_soft (per-element supports hs[], optional zeta). */
static int eval_core(int64_t n_src, const double *pos, const double *vel, const double *mass,
                     const double *hs, const double *zeta, int64_t n_tgt, const int32_t *idx,
                     double G, double h, double eta, double box, double *acc, double *jerk,
                     double *tidal, double *pot, double *dt_grav, int nthreads)
{
    set_threads(nthreads);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(|: bad)
    for (int64_t t = 0; t < n_tgt; ++t) {
        int64_t i = idx ? (int64_t)idx[t] : t;
        if (i < 0 || i >= n_src) { bad = 1; continue; }
        nsum a[3], jk[3], tt[6], ph;
        memset(a, 0, sizeof a);
        memset(jk, 0, sizeof jk);
        memset(tt, 0, sizeof tt);
        memset(&ph, 0, sizeof ph);
        const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
        const double ui = vel[3 * i], vi = vel[3 * i + 1], wi = vel[3 * i + 2];
        for (int64_t j = 0; j < n_src; ++j) {
            if (j == i) continue;
            double d[3] = {pos[3 * j] - xi, pos[3 * j + 1] - yi, pos[3 * j + 2] - zi};
            if (box > 0.0)
                for (int c = 0; c < 3; ++c) d[c] -= box * nearbyint(d[c] / box);
            double v[3] = {vel[3 * j] - ui, vel[3 * j + 1] - vi, vel[3 * j + 2] - wi};
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double f, g, phi, fc = 0.0;
            if (hs) {
                /* per-element supports: the mean of the two kernels */
                double fi, gi, pi_, fj, gj, pj;
                oracle_kernel(r, hs[i], &fi, &gi, &pi_);
                oracle_kernel(r, hs[j], &fj, &gj, &pj);
                f = 0.5 * (fi + fj);
                g = 0.5 * (gi + gj);
                phi = 0.5 * (pi_ + pj);
                /* correction: -(1/2)[zeta_i W_r(r,h_i) + zeta_j W_r(r,h_j)] / r per unit m d */
                if (zeta && r > 0.0) {
                    double w, wri, wrj, wh, psh;
                    oracle_kernel_w(r, hs[i], &w, &wri, &wh, &psh);
                    oracle_kernel_w(r, hs[j], &w, &wrj, &wh, &psh);
                    fc = -0.5 * (zeta[i] * wri + zeta[j] * wrj) / r;
                }
            } else {
                oracle_kernel(r, h, &f, &g, &phi);
            }
            double m = mass[j];
            double dv = d[0] * v[0] + d[1] * v[1] + d[2] * v[2];
            for (int c = 0; c < 3; ++c) {
                nadd(&a[c], m * f * d[c]);
                if (fc != 0.0) nadd(&a[c], m * fc * d[c]);
                nadd(&jk[c], m * (f * v[c] + g * dv * d[c]));
            }
            /* T_ab = -m (f delta_ab + g d_a d_b) */
            nadd(&tt[0], -m * (f + g * d[0] * d[0]));
            nadd(&tt[1], -m * (f + g * d[1] * d[1]));
            nadd(&tt[2], -m * (f + g * d[2] * d[2]));
            nadd(&tt[3], -m * (g * d[0] * d[1]));
            nadd(&tt[4], -m * (g * d[0] * d[2]));
            nadd(&tt[5], -m * (g * d[1] * d[2]));
            nadd(&ph, -m * phi);
        }
        double t6[6];
        for (int c = 0; c < 3; ++c) {
            acc[3 * t + c] = G * nval(&a[c]);
            jerk[3 * t + c] = G * nval(&jk[c]);
        }
        for (int c = 0; c < 6; ++c) {
            t6[c] = G * nval(&tt[c]);
            tidal[6 * t + c] = t6[c];
        }
        if (pot) pot[t] = G * nval(&ph);
        if (dt_grav) dt_grav[t] = oracle_tidal_dt(t6, eta);
    }
    return bad ? -1 : 0;
}

int oracle_eval(int64_t n_src, const double *pos, const double *vel, const double *mass,
                int64_t n_tgt, const int32_t *idx, double G, double h, double eta, double box,
                double *acc, double *jerk, double *tidal, double *pot, double *dt_grav,
                int nthreads)
{
    /* box > 0: periodic cube of side `box`, every separation taken to its
     * nearest periodic image, d_c -> d_c - box * nearbyint(d_c / box) (the
     * paper's Zeldovich runs used only the nearest image for the jerk). */
    if (n_src < 0 || n_tgt < 0 || !(h > 0.0) || box < 0.0) return -1;
    if (n_tgt > 0 && (!pos || !vel || !mass || !acc || !jerk || !tidal)) return -1;
    return eval_core(n_src, pos, vel, mass, NULL, NULL, n_tgt, idx, G, h, eta, box, acc, jerk,
                     tidal, pot, dt_grav, nthreads);
}

/*
 * Conditioning of the sums of oracle_eval, the scale against which their
 * rounding errors grow (the error metric's kappa_i = sum_j |a_ij| / |a_i|):
 * at the same targets and over the same pairs (j != i, nearest image when
 * box > 0), per target slot t
 *   cond[3t]     = G sum_j m_j |f(r)| r                    (sum_j |a_ij|)
 *   cond[3t + 1] = G sum_j m_j |f v_ji + g (d . v_ji) d|   (sum_j |j_ij|)
 *   cond[3t + 2] = G sum_j m_j ||f I + g d d^T||_F          (sum_j ||T_ij||_F)
 * with ||f I + g d d^T||_F^2 = 2 f^2 + (f + g r^2)^2 (eigenvalues f, f and
 * f + g r^2).  Sums of non-negative terms, added in order.
 */
int oracle_conditioning(int64_t n_src, const double *pos, const double *vel, const double *mass,
                        int64_t n_tgt, const int32_t *idx, double G, double h, double box,
                        double *cond, int nthreads)
{
    if (n_src < 0 || n_tgt < 0 || !(h > 0.0) || box < 0.0) return -1;
    if (n_tgt > 0 && (!pos || !vel || !mass || !cond)) return -1;
    set_threads(nthreads);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(|: bad)
    for (int64_t t = 0; t < n_tgt; ++t) {
        int64_t i = idx ? (int64_t)idx[t] : t;
        if (i < 0 || i >= n_src) { bad = 1; continue; }
        double sa = 0.0, sj = 0.0, st = 0.0;
        for (int64_t j = 0; j < n_src; ++j) {
            if (j == i) continue;
            double d[3], v[3];
            for (int c = 0; c < 3; ++c) {
                d[c] = pos[3 * j + c] - pos[3 * i + c];
                if (box > 0.0) d[c] -= box * nearbyint(d[c] / box);
                v[c] = vel[3 * j + c] - vel[3 * i + c];
            }
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double r = sqrt(r2);
            double f, g, phi;
            oracle_kernel(r, h, &f, &g, &phi);
            double m = mass[j];
            double dv = d[0] * v[0] + d[1] * v[1] + d[2] * v[2];
            double jv[3];
            for (int c = 0; c < 3; ++c) jv[c] = f * v[c] + g * dv * d[c];
            double e3 = f + g * r2;
            sa += m * fabs(f) * r;
            sj += m * sqrt(jv[0] * jv[0] + jv[1] * jv[1] + jv[2] * jv[2]);
            st += m * sqrt(2.0 * f * f + e3 * e3);
        }
        cond[3 * t] = G * sa;
        cond[3 * t + 1] = G * sj;
        cond[3 * t + 2] = G * st;
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------- */
/* Adaptive softening (Section 3: fully adaptive softening with the extra     */
/* force terms of Price & Monaghan 2007 that keep energy conserved).          */
/*                                                                            */
/* Readings (the paper gives no formulas):                                    */
/*  - each element i has its own support h_i, fixed by the mass-density       */
/*    constraint (4 pi / 3) h_i^3 rho_i = n_ngb m_i with                       */
/*    rho_i = sum_j m_j W(r_ij, h_i), the self term j = i included;           */
/*  - the potential energy is U = -(G/2) sum_i sum_{j != i} m_i m_j           */
/*    (psi(r_ij, h_i) + psi(r_ij, h_j)) / 2 (self terms excluded, as in the    */
/*    fixed-h evaluation); the pair force is the average of the two kernels; */
/*  - the acceleration is -grad_i U / m_i with h's dependence on the          */
/*    positions through the constraint, which adds                            */
/*      a_i^zeta = -(G/2) sum_j m_j [zeta_i W_r(r,h_i) + zeta_j W_r(r,h_j)] d/r */
/*    where W_r = dW/dr, zeta_i = (dh_i/drho_i) / Omega_i                     */
/*    * sum_{j != i} m_j dpsi(r_ij, h_i)/dh, dh/drho = -h / (3 rho),           */
/*    Omega_i = 1 + h_i / (3 rho_i) * sum_j m_j dW(r_ij, h_i)/dh;             */
/*  - jerk and tidal tensor are those of the averaged pair force at fixed    */
/*    h_i, h_j (the correction term and the motion of h are not              */
/*    differentiated).                                                        */
/* ------------------------------------------------------------------------- */

/* Density kernel W(r,h) = 8/(pi h^3) w(r/h) and the derivatives the adaptive
 * terms need: dW/dr, dW/dh and dpsi/dh of the potential kernel psi
 * (psi = phi of oracle_kernel, psi(r,h) = p(r/h)/h, dpsi/dh = -(u p)'(u)/h^2). */
void oracle_kernel_w(double r, double h, double *w, double *w_r, double *w_h, double *psi_h)
{
    double u = r / h;
    double c = 8.0 / (ORACLE_PI * h * h * h);
    double wu, dwu, dup;
    if (u < 0.5) {
        wu = 1.0 + u * u * (-6.0 + 6.0 * u);
        dwu = u * (-12.0 + 18.0 * u);
        double u2 = u * u;
        dup = 14.0 / 5.0 + u2 * (-16.0 + u2 * (48.0 - 192.0 / 5.0 * u));
    } else if (u < 1.0) {
        double q = 1.0 - u;
        wu = 2.0 * q * q * q;
        dwu = -6.0 * q * q;
        double u2 = u * u;
        dup = 16.0 / 5.0 + u2 * (-32.0 + u * (64.0 + u * (-48.0 + 64.0 / 5.0 * u)));
    } else {
        wu = 0.0;
        dwu = 0.0;
        dup = 0.0;
    }
    *w = c * wu;
    *w_r = c * dwu / h;
    *w_h = -c * (3.0 * wu + u * dwu) / h;
    *psi_h = -dup / (h * h);
}

/* The sums of element i at support h:
 *   rho   = sum_j m_j W(r_ij, h)               (j = i included)
 *   rho_h = sum_j m_j dW(r_ij, h)/dh           (j = i included)
 *   psi_h = sum_{j != i} m_j dpsi(r_ij, h)/dh
 * (the density of the support constraint, its derivative in h, and the sum
 * that gives the correction coefficient zeta). */
static void soft_sums_at(int64_t n, const double *pos, const double *mass, int64_t i, double h,
                         double *rho, double *rho_h, double *psi_h)
{
    nsum sr, srh, sp;
    memset(&sr, 0, sizeof sr);
    memset(&srh, 0, sizeof srh);
    memset(&sp, 0, sizeof sp);
    for (int64_t j = 0; j < n; ++j) {
        double d[3] = {pos[3 * j] - pos[3 * i], pos[3 * j + 1] - pos[3 * i + 1],
                       pos[3 * j + 2] - pos[3 * i + 2]};
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (r >= h) continue;
        double w, wr, wh, ph;
        oracle_kernel_w(r, h, &w, &wr, &wh, &ph);
        nadd(&sr, mass[j] * w);
        nadd(&srh, mass[j] * wh);
        if (j != i) nadd(&sp, mass[j] * ph);
    }
    *rho = nval(&sr);
    *rho_h = nval(&srh);
    *psi_h = nval(&sp);
}

/* Per element, the sums of soft_sums_at at the given supports h_i. */
int oracle_soft_sums(int64_t n, const double *pos, const double *mass, const double *hs,
                     double *rho, double *rho_h, double *psi_h, int nthreads)
{
    if (n < 0 || (n > 0 && (!pos || !mass || !hs || !rho || !rho_h || !psi_h))) return -1;
    set_threads(nthreads);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(|: bad)
    for (int64_t i = 0; i < n; ++i) {
        double h = hs[i];
        if (!(h > 0.0)) { bad = 1; continue; }
        soft_sums_at(n, pos, mass, i, h, &rho[i], &rho_h[i], &psi_h[i]);
    }
    return bad ? -1 : 0;
}

/* Solves (4 pi / 3) h_i^3 rho_i(h_i) = n_ngb m_i for every element by Newton
 * iterations limited to a factor of 2 in h and kept inside a bracket
 * [lo, hi] (F(h) is non-decreasing in h); a step that leaves the bracket
 * doubles h (no upper end yet) or bisects.
 * h[] holds the starting guesses on entry.  Converged when
 * |F| <= tol * n_ngb * m_i; the sums of the last iteration are those at the
 * returned h, from which zeta follows:
 *   Omega_i = 1 + h_i rho_h_i / (3 rho_i),
 *   zeta_i  = -h_i psi_h_i / (3 rho_i Omega_i).
 * iters[i] (nullable) = iterations used, -1 where max_iter ran out.
 * Returns 0, or 1 when some element did not converge, -1 on bad arguments. */
int oracle_soft_solve(int64_t n, const double *pos, const double *mass, double n_ngb, double tol,
                      int32_t max_iter, double *hs, double *zeta, double *omega, int32_t *iters,
                      int nthreads)
{
    if (n < 0 || !(n_ngb > 32.0 / 3.0) || !(tol > 0.0) || max_iter < 1) return -1;
    if (n > 0 && (!pos || !mass || !hs)) return -1;
    set_threads(nthreads);
    int bad = 0, stuck = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(|: bad, stuck)
    for (int64_t i = 0; i < n; ++i) {
        double h = hs[i];
        if (!(h > 0.0) || !(mass[i] > 0.0)) { bad = 1; continue; }
        const double target = n_ngb * mass[i];
        double lo = 0.0, hi = INFINITY;
        int32_t it = 0;
        int done = 0;
        double rho = 0.0, rho_h = 0.0, psi_h = 0.0;
        for (; it < max_iter; ++it) {
            soft_sums_at(n, pos, mass, i, h, &rho, &rho_h, &psi_h);
            double vol = 4.0 * ORACLE_PI / 3.0 * h * h * h;
            double F = vol * rho - target;
            if (fabs(F) <= tol * target) { done = 1; break; }
            if (F < 0.0) lo = h; else hi = h;
            double dF = 4.0 * ORACLE_PI * h * h * rho + vol * rho_h;
            /* Newton step, limited to a factor of 2 in h (with only the self
             * term inside, F is flat and the plain step would be huge) */
            double hn = (F < 0.0) ? 2.0 * h : 0.5 * h;
            if (dF > 0.0) {
                hn = h - F / dF;
                if (hn > 2.0 * h) hn = 2.0 * h;
                if (hn < 0.5 * h) hn = 0.5 * h;
            }
            if (!(hn > lo && hn < hi)) hn = isinf(hi) ? 2.0 * h : 0.5 * (lo + hi);
            h = hn;
        }
        hs[i] = h;
        double om = 1.0 + h * rho_h / (3.0 * rho);
        if (omega) omega[i] = om;
        if (zeta) zeta[i] = -h * psi_h / (3.0 * rho * om);
        if (iters) iters[i] = done ? it : -1;
        if (!done) stuck = 1;
    }
    if (bad) return -1;
    return stuck ? 1 : 0;
}

/*
 * Force evaluation with per-element supports hs[] (and, when zeta is not
 * NULL, the correction term of the adaptive-softening readings above):
 *   a_i   = G sum_j m_j fbar d + a_i^zeta,  fbar = (f(r,h_i) + f(r,h_j)) / 2
 *   j_i   = G sum_j m_j [fbar v_ji + gbar (d . v_ji) d]
 *   T_i   = -G sum_j m_j [fbar I + gbar d d^T]
 *   Phi_i = -G sum_j m_j (psi(r,h_i) + psi(r,h_j)) / 2
 * Output slots and nullability as in oracle_eval (open boundaries only).
 */
int oracle_eval_soft(int64_t n_src, const double *pos, const double *vel, const double *mass,
                     const double *hs, const double *zeta, int64_t n_tgt, const int32_t *idx,
                     double G, double eta, double *acc, double *jerk, double *tidal, double *pot,
                     double *dt_grav, int nthreads)
{
    if (n_src < 0 || n_tgt < 0) return -1;
    if (n_tgt > 0 && (!pos || !vel || !mass || !hs || !acc || !jerk || !tidal)) return -1;
    for (int64_t j = 0; j < n_src; ++j)
        if (!(hs[j] > 0.0)) return -1;
    return eval_core(n_src, pos, vel, mass, hs, zeta, n_tgt, idx, G, 1.0, eta, 0.0, acc, jerk,
                     tidal, pot, dt_grav, nthreads);
}

/* ------------------------------------------------------------------------- */
/* Time bins, counter and update condition.                                   */
/* ------------------------------------------------------------------------- */

/* An element of bin k (0 <= k <= k_max) takes steps of 2^(k_max-k) ticks and
 * is active at every tick that is a multiple of its step (Section 3: the
 * hierarchical power-of-two block timesteps). */
static int is_active(int64_t tick, int32_t k_max, int32_t k)
{
    int64_t step = (int64_t)1 << (k_max - k);
    return (tick % step) == 0;
}

/*
 * Counter update (Eq. 3) and update condition (Eq. updatecondition).
 * For every element active at `tick`: T_f += its step (in ticks); it is due
 * when T_f * dt_min >= q_f * dt_grav (two correctly rounded products and a
 * compare); a due element's counter is reset to 0, because its force is
 * re-evaluated in this substep.  Inactive elements keep their counter and get
 * active = due = 0.  dt_grav = 0 marks "never evaluated" and is always due.
 */
int oracle_select_due(int64_t n, int64_t tick, int32_t k_max, const int8_t *bin,
                      int64_t *tf_ticks, const double *dt_grav, double q_f, double dt_min,
                      uint8_t *active, uint8_t *due, int64_t *elapsed_ticks)
{
    /* elapsed_ticks (nullable): for due elements, T_f before the reset, i.e. the
     * time since the previous evaluation in ticks; untouched otherwise. */
    if (n < 0 || k_max < 0 || k_max > 62 || tick < 0) return -1;
    for (int64_t i = 0; i < n; ++i) {
        int32_t k = bin[i];
        if (k < 0 || k > k_max) return -1;
        if (!is_active(tick, k_max, k)) {
            active[i] = 0;
            due[i] = 0;
            continue;
        }
        active[i] = 1;
        tf_ticks[i] += (int64_t)1 << (k_max - k);
        double elapsed = (double)tf_ticks[i] * dt_min;
        double need = q_f * dt_grav[i];
        if (elapsed >= need) {
            due[i] = 1;
            if (elapsed_ticks) elapsed_ticks[i] = tf_ticks[i];
            tf_ticks[i] = 0;
        } else {
            due[i] = 0;
        }
    }
    return 0;
}

/* Indices i with flags[i] != 0, ascending; *count = their number. */
int oracle_compact(int64_t n, const uint8_t *flags, int32_t *idx, int32_t *count)
{
    if (n < 0 || n > INT32_MAX) return -1;
    int32_t c = 0;
    for (int64_t i = 0; i < n; ++i)
        if (flags[i]) idx[c++] = (int32_t)i;
    *count = c;
    return 0;
}

/*
 * Jerk predictor (Eq. jerkupdate) in closed form: for active, not-due
 * elements a_out = a_last + j_last * tau with tau = T_f * dt_min the time since
 * the last evaluation (the paper's incremental form summed exactly); active due
 * elements get a_out = a_last (just re-evaluated); inactive ones are untouched.
 */
int oracle_predict(int64_t n, const uint8_t *active, const uint8_t *due, const double *a_last,
                   const double *j_last, const int64_t *tf_ticks, double dt_min, double *a_out)
{
    if (n < 0) return -1;
    for (int64_t i = 0; i < n; ++i) {
        if (!active[i]) continue;
        if (due[i]) {
            for (int c = 0; c < 3; ++c) a_out[3 * i + c] = a_last[3 * i + c];
            continue;
        }
        double tau = (double)tf_ticks[i] * dt_min;
        for (int c = 0; c < 3; ++c) {
            double inc = j_last[3 * i + c] * tau;
            a_out[3 * i + c] = a_last[3 * i + c] + inc;
        }
    }
    return 0;
}

/*
 * History for the polynomial predictor (Section 2.2: log past g_i values and
 * extrapolate).  For every element due now, before its new evaluation
 * overwrites a_last: a_prev = a_last (the acceleration of the evaluation
 * before the new one) and dt_prev = elapsed * dt_min, the gap between the two,
 * where elapsed is T_f at the moment it became due (from the selection).  An
 * element never evaluated before (dt_grav == 0) gets dt_prev = 0: no history.
 */
int oracle_push_history(int64_t n, const uint8_t *due, const int64_t *elapsed_ticks,
                        const double *dt_grav, const double *a_last, double *a_prev,
                        double *dt_prev, double dt_min)
{
    if (n < 0) return -1;
    for (int64_t i = 0; i < n; ++i) {
        if (!due[i]) continue;
        dt_prev[i] = (dt_grav[i] == 0.0) ? 0.0 : (double)elapsed_ticks[i] * dt_min;
        for (int c = 0; c < 3; ++c) a_prev[3 * i + c] = a_last[3 * i + c];
    }
    return 0;
}

/*
 * First-order polynomial predictor through the last two evaluations
 * (Section 2.2): for active, not-due elements with dt_prev > 0
 *     a_out = a_last + (a_last - a_prev) * (tau / dt_prev),  tau = T_f * dt_min,
 * evaluated as tau, the ratio, the difference, the product and the sum, each
 * correctly rounded; with dt_prev = 0 (one evaluation so far) a_out = a_last.
 * Active due elements get a_last; inactive ones are untouched.
 */
int oracle_predict_poly(int64_t n, const uint8_t *active, const uint8_t *due, const double *a_last,
                        const double *a_prev, const double *dt_prev, const int64_t *tf_ticks,
                        double dt_min, double *a_out)
{
    if (n < 0) return -1;
    for (int64_t i = 0; i < n; ++i) {
        if (!active[i]) continue;
        if (due[i] || !(dt_prev[i] > 0.0)) {
            for (int c = 0; c < 3; ++c) a_out[3 * i + c] = a_last[3 * i + c];
            continue;
        }
        double tau = (double)tf_ticks[i] * dt_min;
        double frac = tau / dt_prev[i];
        for (int c = 0; c < 3; ++c) {
            double diff = a_last[3 * i + c] - a_prev[3 * i + c];
            double inc = diff * frac;
            a_out[3 * i + c] = a_last[3 * i + c] + inc;
        }
    }
    return 0;
}

/*
 * Bin assignment for elements active at `tick`: dt_i = min(dt_grav, dt_hydro)
 * (Section 2); the target bin is the smallest k in [0, k_max] whose step
 * dt_max 2^-k does not exceed dt_i (comparisons are exact: only exponents and
 * mantissas are compared); a step may only grow at a tick that is a multiple
 * of the new step, so the bin is raised to the smallest k aligned with `tick`.
 * dt_hydro may be NULL (no limit).  NaN or non-positive dt_i -> k_max.
 */
static int32_t target_bin(double dt_i, double dt_max, int32_t k_max)
{
    if (!(dt_i > 0.0)) return k_max;          /* 0, negative or NaN */
    if (isinf(dt_i)) return 0;
    int ei, em;
    double mi = frexp(dt_i, &ei);
    double mm = frexp(dt_max, &em);
    /* dt_max 2^-k <= dt_i  <=>  mm 2^(em-k) <= mi 2^ei */
    int64_t k = (int64_t)em - (int64_t)ei;
    if (mm > mi) k += 1;
    if (k < 0) k = 0;
    if (k > k_max) k = k_max;
    return (int32_t)k;
}

int oracle_assign_bins(int64_t n, int64_t tick, int32_t k_max, double dt_max,
                       const uint8_t *active, const double *dt_grav, const double *dt_hydro,
                       int8_t *bin)
{
    if (n < 0 || k_max < 0 || k_max > 62 || tick < 0 || !(dt_max > 0.0)) return -1;
    int32_t k_align = 0;
    if (tick != 0) {
        int32_t tz = 0;
        while (((tick >> tz) & 1) == 0) ++tz;
        k_align = k_max - tz;
        if (k_align < 0) k_align = 0;
    }
    for (int64_t i = 0; i < n; ++i) {
        if (!active[i]) continue;
        double dt = dt_grav[i];
        if (dt_hydro && dt_hydro[i] < dt) dt = dt_hydro[i];
        if (dt_hydro && isnan(dt_hydro[i])) dt = dt_hydro[i];
        int32_t k = target_bin(dt, dt_max, k_max);
        if (k < k_align) k = k_align;
        bin[i] = (int8_t)k;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Adjoint of the force evaluation at all n elements.                         */
/* ------------------------------------------------------------------------- */
/*
 * For a loss L(a, W) with a_bar = dL/da (n x 3, nullable = 0) and
 * w_bar = dL/dW, W = 1/2 sum_i m_i Phi_i the potential energy:
 *   pos_bar_k  = T_k a_bar_k + G m_k sum_{i!=k} [ f a_bar_i + g d (d . a_bar_i) ]
 *                - w_bar m_k a_k
 *   mass_bar_k = -G sum_{i!=k} f (d . a_bar_i) + w_bar Phi_k
 * with d = x_i - x_k.  acc, tidal and pot are the forward results at all n
 * elements (pot needed only when w_bar != 0, acc only when w_bar != 0).
 */
int oracle_backward(int64_t n, const double *pos, const double *mass, const double *a_bar,
                    double w_bar, const double *acc, const double *tidal, const double *pot,
                    double G, double h, int64_t n_sel, const int32_t *sel, double *pos_bar,
                    double *mass_bar, int nthreads)
{
    /* sel (nullable): compute only rows k = sel[0..n_sel) (outputs still
     * indexed by k); NULL means every k in [0, n). */
    if (n < 0 || !(h > 0.0)) return -1;
    if (w_bar != 0.0 && (!acc || !pot)) return -1;
    if (a_bar && !tidal) return -1;
    if (!sel) n_sel = n;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < n_sel; ++s) {
        int64_t k = sel ? (int64_t)sel[s] : s;
        if (k < 0 || k >= n) continue;
        nsum xb[3], mb;
        memset(xb, 0, sizeof xb);
        memset(&mb, 0, sizeof mb);
        if (a_bar) {
            const double xk = pos[3 * k], yk = pos[3 * k + 1], zk = pos[3 * k + 2];
            for (int64_t i = 0; i < n; ++i) {
                if (i == k) continue;
                double d[3] = {pos[3 * i] - xk, pos[3 * i + 1] - yk, pos[3 * i + 2] - zk};
                double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                double f, g, phi;
                oracle_kernel(r, h, &f, &g, &phi);
                const double *ab = a_bar + 3 * i;
                double da = d[0] * ab[0] + d[1] * ab[1] + d[2] * ab[2];
                for (int c = 0; c < 3; ++c) nadd(&xb[c], f * ab[c] + g * d[c] * da);
                nadd(&mb, -f * da);
            }
        }
        double px[3] = {0.0, 0.0, 0.0};
        double pm = 0.0;
        if (a_bar) {
            const double *t6 = tidal + 6 * k;
            const double *ak = a_bar + 3 * k;
            /* symmetric T from xx, yy, zz, xy, xz, yz */
            double ta[3];
            ta[0] = t6[0] * ak[0] + t6[3] * ak[1] + t6[4] * ak[2];
            ta[1] = t6[3] * ak[0] + t6[1] * ak[1] + t6[5] * ak[2];
            ta[2] = t6[4] * ak[0] + t6[5] * ak[1] + t6[2] * ak[2];
            for (int c = 0; c < 3; ++c) px[c] = ta[c] + G * mass[k] * nval(&xb[c]);
            pm = G * nval(&mb);
        }
        if (w_bar != 0.0) {
            for (int c = 0; c < 3; ++c) px[c] -= w_bar * mass[k] * acc[3 * k + c];
            pm += w_bar * pot[k];
        }
        for (int c = 0; c < 3; ++c) pos_bar[3 * k + c] = px[c];
        mass_bar[k] = pm;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Approximate solver: the oct-tree code of Section 3 (Barnes & Hut with the  */
/* geometric opening criterion L/r > Theta always splitting a node, Theta =   */
/* 0.5; optionally the relative criterion of the tree-code it supplements).   */
/*                                                                            */
/* Readings (the paper gives the criterion, not the tree):                    */
/*  - the root is the cube of side ext = the largest extent of the elements'  */
/*    bounding box, at its low corner; an element's cell coordinates are      */
/*    q_c = floor((x_c - lo_c) / ext * 2^21), clamped to [0, 2^21 - 1], its   */
/*    key the 63-bit interleave (x, y, z from the highest bit down);          */
/*  - elements are ordered by (key, index); a node at level l holds the run   */
/*    of elements sharing the key's top 3l bits, side L = ext 2^-l; it is a   */
/*    leaf when it holds at most leaf_size elements or l = 21, otherwise its  */
/*    non-empty octants are its children, in octant order;                    */
/*  - node moments are monopoles: mass M, centre of mass and mean velocity,   */
/*    summed in order (a leaf over its elements, a node over its children);   */
/*  - from the root, a node is accepted when L^2 < Theta^2 r^2 (r from the   */
/*    target to the node's centre of mass) and, if alpha > 0 and a_old is    */
/*    given, also G M L^2 <= alpha |a_old,i| r^4; an accepted node acts as a  */
/*    point mass M at its centre of mass moving with its mean velocity (the   */
/*    same softened pair terms as the direct sum, with h); a leaf that is not */
/*    accepted is summed element by element (j != i); any other node is       */
/*    opened, its children visited in octant order.                          */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t first, count;       /* run in the sorted order */
    int64_t child_first;        /* -1 for a leaf */
    int32_t n_child, level;
    double m, com[3], vcom[3];
} tnode;

typedef struct {
    uint64_t key;
    int64_t idx;
} tkey;

static int tkey_cmp(const void *a, const void *b)
{
    const tkey *x = (const tkey *)a, *y = (const tkey *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static uint64_t spread21(uint64_t v)
{
    uint64_t out = 0;
    for (int b = 0; b < 21; ++b) out |= ((v >> b) & 1u) << (3 * b);
    return out;
}

typedef struct {
    int64_t n;
    const double *pos, *vel, *mass;
    int64_t *order;
    uint64_t *keys;
    tnode *nodes;
    int64_t n_nodes, cap;
    double lo[3], ext;
    int32_t leaf_size;
} otree;

/* Children of node k (its run already set), appended contiguously. */
static int tree_split(otree *t, int64_t k)
{
    tnode *nd = &t->nodes[k];
    nd->child_first = -1;
    nd->n_child = 0;
    if (nd->count <= t->leaf_size || nd->level >= 21) return 0;
    int shift = 3 * (20 - nd->level);
    int64_t cnt[8] = {0};
    for (int64_t s = nd->first; s < nd->first + nd->count; ++s) cnt[(t->keys[s] >> shift) & 7u]++;
    int nc = 0;
    for (int o = 0; o < 8; ++o) nc += cnt[o] > 0;
    if (t->n_nodes + nc > t->cap) return -1;
    int64_t base = t->n_nodes, f = nd->first;
    int32_t lvl = nd->level;
    t->n_nodes += nc;
    nd = &t->nodes[k];
    nd->child_first = base;
    nd->n_child = nc;
    int c = 0;
    for (int o = 0; o < 8; ++o) {
        if (!cnt[o]) continue;
        tnode *ch = &t->nodes[base + c++];
        ch->first = f;
        ch->count = cnt[o];
        ch->level = lvl + 1;
        f += cnt[o];
    }
    return nc;
}

static void tree_moments(otree *t, int64_t k)
{
    tnode *nd = &t->nodes[k];
    double m = 0.0, mx[3] = {0, 0, 0}, mv[3] = {0, 0, 0};
    if (nd->child_first < 0) {
        for (int64_t s = nd->first; s < nd->first + nd->count; ++s) {
            int64_t j = t->order[s];
            double mj = t->mass[j];
            m = m + mj;
            for (int c = 0; c < 3; ++c) {
                mx[c] = mx[c] + mj * t->pos[3 * j + c];
                mv[c] = mv[c] + mj * t->vel[3 * j + c];
            }
        }
    } else {
        for (int q = 0; q < nd->n_child; ++q) {
            tnode *ch = &t->nodes[nd->child_first + q];
            m = m + ch->m;
            for (int c = 0; c < 3; ++c) {
                mx[c] = mx[c] + ch->m * ch->com[c];
                mv[c] = mv[c] + ch->m * ch->vcom[c];
            }
        }
    }
    nd->m = m;
    for (int c = 0; c < 3; ++c) {
        nd->com[c] = m > 0.0 ? mx[c] / m : 0.0;
        nd->vcom[c] = m > 0.0 ? mv[c] / m : 0.0;
    }
}

static int tree_build(otree *t)
{
    int64_t n = t->n;
    double hi[3];
    for (int c = 0; c < 3; ++c) {
        t->lo[c] = INFINITY;
        hi[c] = -INFINITY;
    }
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) {
            if (t->pos[3 * i + c] < t->lo[c]) t->lo[c] = t->pos[3 * i + c];
            if (t->pos[3 * i + c] > hi[c]) hi[c] = t->pos[3 * i + c];
        }
    t->ext = 0.0;
    for (int c = 0; c < 3; ++c)
        if (hi[c] - t->lo[c] > t->ext) t->ext = hi[c] - t->lo[c];
    if (!(t->ext > 0.0)) t->ext = 1.0;
    tkey *kv = (tkey *)malloc((size_t)n * sizeof(tkey));
    if (!kv) return -1;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t q[3];
        for (int c = 0; c < 3; ++c) {
            double s = floor((t->pos[3 * i + c] - t->lo[c]) / t->ext * 2097152.0);
            if (s < 0.0) s = 0.0;
            if (s > 2097151.0) s = 2097151.0;
            q[c] = (uint64_t)s;
        }
        kv[i].key = (spread21(q[0]) << 2) | (spread21(q[1]) << 1) | spread21(q[2]);
        kv[i].idx = i;
    }
    qsort(kv, (size_t)n, sizeof(tkey), tkey_cmp);
    for (int64_t s = 0; s < n; ++s) {
        t->order[s] = kv[s].idx;
        t->keys[s] = kv[s].key;
    }
    free(kv);
    t->nodes[0].first = 0;
    t->nodes[0].count = n;
    t->nodes[0].level = 0;
    t->n_nodes = 1;
    for (int64_t k = 0; k < t->n_nodes; ++k)       /* breadth first */
        if (tree_split(t, k) < 0) return -1;
    for (int64_t k = t->n_nodes - 1; k >= 0; --k)   /* children come after parents */
        tree_moments(t, k);
    return 0;
}

typedef struct {
    nsum a[3], jk[3], tt[6], ph;
    int64_t inter;
} tacc;

static void tree_pair(tacc *s, double m, const double d[3], const double v[3], double h)
{
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double f, g, phi;
    oracle_kernel(r, h, &f, &g, &phi);
    double dv = d[0] * v[0] + d[1] * v[1] + d[2] * v[2];
    for (int c = 0; c < 3; ++c) {
        nadd(&s->a[c], m * f * d[c]);
        nadd(&s->jk[c], m * (f * v[c] + g * dv * d[c]));
    }
    nadd(&s->tt[0], -m * (f + g * d[0] * d[0]));
    nadd(&s->tt[1], -m * (f + g * d[1] * d[1]));
    nadd(&s->tt[2], -m * (f + g * d[2] * d[2]));
    nadd(&s->tt[3], -m * (g * d[0] * d[1]));
    nadd(&s->tt[4], -m * (g * d[0] * d[2]));
    nadd(&s->tt[5], -m * (g * d[1] * d[2]));
    nadd(&s->ph, -m * phi);
    s->inter++;
}

static void tree_walk(const otree *t, int64_t k, int64_t i, double G, double h, double theta2,
                      double rel, tacc *s)
{
    const tnode *nd = &t->nodes[k];
    const double *xi = &t->pos[3 * i], *vi = &t->vel[3 * i];
    double d[3] = {nd->com[0] - xi[0], nd->com[1] - xi[1], nd->com[2] - xi[2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double L = ldexp(t->ext, -nd->level);
    double L2 = L * L;
    int accept = L2 < theta2 * r2;
    if (accept && rel > 0.0) accept = (G * nd->m) * L2 <= (rel * r2) * r2;
    if (accept) {
        double v[3] = {nd->vcom[0] - vi[0], nd->vcom[1] - vi[1], nd->vcom[2] - vi[2]};
        tree_pair(s, nd->m, d, v, h);
        return;
    }
    if (nd->child_first < 0) {
        for (int64_t q = nd->first; q < nd->first + nd->count; ++q) {
            int64_t j = t->order[q];
            if (j == i) continue;
            double dj[3] = {t->pos[3 * j] - xi[0], t->pos[3 * j + 1] - xi[1], t->pos[3 * j + 2] - xi[2]};
            double vj[3] = {t->vel[3 * j] - vi[0], t->vel[3 * j + 1] - vi[1], t->vel[3 * j + 2] - vi[2]};
            tree_pair(s, t->mass[j], dj, vj, h);
        }
        return;
    }
    for (int q = 0; q < nd->n_child; ++q) tree_walk(t, nd->child_first + q, i, G, h, theta2, rel, s);
}

/*
 * Tree-code evaluation at n_tgt targets (idx[t], or t when idx is NULL) over
 * all n elements: outputs per target slot as in oracle_eval.  theta >= 0;
 * leaf_size >= 1; alpha > 0 with a_old [n][3] adds the relative criterion.
 * order_out [n] (nullable): the elements in tree order; n_nodes_out and
 * interactions_out (nullable): node count and total interactions (accepted
 * nodes plus leaf pairs).
 */
int oracle_tree_eval(int64_t n, const double *pos, const double *vel, const double *mass,
                     int64_t n_tgt, const int32_t *idx, double G, double h, double eta,
                     double theta, int32_t leaf_size, double alpha, const double *a_old,
                     double *acc, double *jerk, double *tidal, double *pot, double *dt_grav,
                     int64_t *order_out, int64_t *n_nodes_out, int64_t *interactions_out,
                     int nthreads)
{
    if (n < 1 || n_tgt < 0 || !(h > 0.0) || !(theta >= 0.0) || leaf_size < 1 || alpha < 0.0)
        return -1;
    if (!pos || !vel || !mass || (n_tgt > 0 && (!acc || !jerk || !tidal))) return -1;
    otree t;
    memset(&t, 0, sizeof t);
    t.n = n;
    t.pos = pos;
    t.vel = vel;
    t.mass = mass;
    t.leaf_size = leaf_size;
    t.cap = 2 * n + 22 * (n / (leaf_size + 1) + 1) + 64;
    t.order = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    t.keys = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    t.nodes = (tnode *)calloc((size_t)t.cap, sizeof(tnode));
    int rc = (t.order && t.keys && t.nodes) ? tree_build(&t) : -1;
    if (rc == 0) {
        if (order_out) memcpy(order_out, t.order, (size_t)n * sizeof(int64_t));
        if (n_nodes_out) *n_nodes_out = t.n_nodes;
        set_threads(nthreads);
        const double theta2 = theta * theta;
        int bad = 0;
        int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(|: bad) reduction(+: total)
        for (int64_t s = 0; s < n_tgt; ++s) {
            int64_t i = idx ? (int64_t)idx[s] : s;
            if (i < 0 || i >= n) { bad = 1; continue; }
            tacc ac;
            memset(&ac, 0, sizeof ac);
            double rel = 0.0;
            if (alpha > 0.0 && a_old) {
                const double *ao = &a_old[3 * i];
                rel = alpha * sqrt(ao[0] * ao[0] + ao[1] * ao[1] + ao[2] * ao[2]);
            }
            tree_walk(&t, 0, i, G, h, theta2, rel, &ac);
            total += ac.inter;
            double t6[6];
            for (int c = 0; c < 3; ++c) {
                acc[3 * s + c] = G * nval(&ac.a[c]);
                jerk[3 * s + c] = G * nval(&ac.jk[c]);
            }
            for (int c = 0; c < 6; ++c) {
                t6[c] = G * nval(&ac.tt[c]);
                tidal[6 * s + c] = t6[c];
            }
            if (pot) pot[s] = G * nval(&ac.ph);
            if (dt_grav) dt_grav[s] = oracle_tidal_dt(t6, eta);
        }
        if (interactions_out) *interactions_out = total;
        if (bad) rc = -1;
    }
    free(t.order);
    free(t.keys);
    free(t.nodes);
    return rc;
}
