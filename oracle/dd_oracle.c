/*
 * dd_oracle.c -- plain, slow CPU reference of the cumulative damage-diffusion field.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load this code.  The product path never calls it,
 * and it shares no code, header or constant table with the CUDA library.
 *
 * What it computes (Javadi Rad et al., "Fast Simulation of Damage Diffusion
 * Distribution in STEM", Sec. 2):
 *   phi_i(r,t)  single-probe field, Eq. 1 (beam on, t_i <= t <= t_i+tau_i) and
 *               Eq. 2 (beam off, t > t_i+tau_i), with D_s = r_s^2 and
 *               E_1(v) = int_v^inf e^-u/u du (the definition given below Eq. 2);
 *               at the probe's own position (rho = 0) Eq. 3 / Eq. 4.
 *   psi(r,t)    cumulative field, Eq. 5: the sum of phi_i over the probes in
 *               visit order.  A probe that has not started (t <= t_i) adds 0.
 * Everything is in SI units exactly as the paper writes it; no rescaling.
 *
 * E_1(x):  x <= 1: power series  E1 = -gamma - ln x - sum_{n>=1} (-x)^n/(n n!)
 *          (Abramowitz & Stegun 5.1.11);  x > 1: the continued fraction
 *          e^x E1(x) = 1/(x+1- 1/(x+3- 4/(x+5- ...)))  (A&S 5.1.22, even form),
 *          evaluated with the modified Lentz method.
 * E_1(a) - E_1(b):  when the difference of the two FP64 values is well conditioned
 *          ((E1(a)+E1(b)) <= 16 (E1(a)-E1(b))) it is that difference.  Otherwise
 *          it is the definition itself, int_a^b e^-u/u du = int_{ln a}^{ln b}
 *          exp(-e^v) dv, integrated by adaptive Gauss-Legendre quadrature; the
 *          integrand is positive, so nothing cancels.
 * Parity status: every function here is pinned by tests against libraries,
 * closed forms and physical invariants (see the test files named oracle_*).
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define EULER_GAMMA 0.57721566490153286060651209008240243
#define PI_D 3.14159265358979323846264338327950288

/* ---------------------------------------------------------------- E_1(x) */

static double e1_series(double x) {
    /* A&S 5.1.11: E1(x) = -gamma - ln x - sum_{n>=1} (-1)^n x^n / (n n!) */
    double term = 1.0;  /* (-1)^n x^n / n! , built incrementally */
    double sum = 0.0;
    for (int n = 1; n < 200; ++n) {
        term *= -x / n;
        double add = term / n;
        sum += add;
        if (fabs(add) < 1e-18 * fabs(sum)) break;
    }
    return -EULER_GAMMA - log(x) - sum;
}

static double e1_cfrac(double x) {
    /* A&S 5.1.22 (even contraction):  e^x E1(x) = 1/(b0 + a1/(b1 + a2/(b2 + ...)))
       with b_k = x + 2k + 1 and a_k = -k^2.  Modified Lentz evaluation of the
       continued fraction f = b0 + a1/(b1 + a2/(b2 + ...)). */
    const double tiny = 1e-300;
    double f = x + 1.0;
    double C = f, Dn = 0.0;
    for (int k = 1; k < 100000; ++k) {
        double ak = -(double)k * (double)k;
        double bk = x + 2.0 * k + 1.0;
        Dn = bk + ak * Dn;
        if (fabs(Dn) < tiny) Dn = tiny;
        C = bk + ak / C;
        if (fabs(C) < tiny) C = tiny;
        Dn = 1.0 / Dn;
        double delta = C * Dn;
        f *= delta;
        if (fabs(delta - 1.0) < 1e-17) break;
    }
    return exp(-x) / f;
}

double ddo_e1(double x) {
    if (!(x >= 0.0)) return NAN;
    if (x == 0.0) return INFINITY;          /* E1(0) = +inf (definition below Eq. 2) */
    if (x > 745.0) return 0.0;              /* below the smallest FP64 subnormal */
    return x <= 1.0 ? e1_series(x) : e1_cfrac(x);
}

/* ------------------------------------- int_a^b e^-u/u du by quadrature */

#define GL_N 16
static double gl_x[GL_N], gl_w[GL_N];
static int gl_ready = 0;

static void gl_init(void) {
    /* Gauss-Legendre nodes on [-1,1]: roots of P_n by Newton's method,
       weights 2 / ((1-x^2) P_n'(x)^2). */
    const int n = GL_N;
    for (int i = 0; i < n; ++i) {
        double x = cos(PI_D * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) <= 4e-16 * fabs(x)) break;
        }
        /* P_n'(x) at the converged root, for the weight */
        {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
        }
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    gl_ready = 1;
}

/* Integrand of int_a^{a e^ell} e^-u/u du after u = a e^y:  exp(-a e^y). */
static double gl_panel(double a, double lo, double hi) {
    double m = 0.5 * (lo + hi), h = 0.5 * (hi - lo), s = 0.0;
    for (int i = 0; i < GL_N; ++i) s += gl_w[i] * exp(-a * exp(m + h * gl_x[i]));
    return s * h;
}

static double gl_adapt(double a, double lo, double hi, double whole, int depth) {
    /* accept once two refinement levels agree to 1e-14 relative (reachable in FP64) */
    double mid = 0.5 * (lo + hi);
    double L = gl_panel(a, lo, mid), R = gl_panel(a, mid, hi);
    if (depth >= 10 || fabs(L + R - whole) <= 1e-14 * fabs(L + R) + 1e-300) return L + R;
    return gl_adapt(a, lo, mid, L, depth + 1) + gl_adapt(a, mid, hi, R, depth + 1);
}

/* E1(a) - E1(a e^ell) = int_a^{a e^ell} e^-u/u du = int_0^ell exp(-a e^y) dy,
   for a > 0, ell >= 0.  The integrand is positive and varies on the scale
   min(1, 1/(a e^y)) in y, so panels are no wider than that; each panel is then
   refined until two levels agree.  Taking ell (= ln(b/a)) as an input keeps the
   near-equal case b ~ a free of the rounding of b - a. */
double ddo_e1_diff_log(double a, double ell) {
    if (!gl_ready) gl_init();
    if (!(a > 0.0) || !(ell >= 0.0)) return NAN;
    double hi = ell;
    double ycut = log(750.0 / a);       /* exp(-a e^y) is 0 in FP64 beyond */
    if (hi > ycut) hi = ycut;
    if (!(hi > 0.0)) return 0.0;
    double total = 0.0, y = 0.0;
    for (int k = 0; k < 1000000 && y < hi; ++k) {
        double scale = a * exp(y);
        double width = scale > 1.0 ? 1.0 / scale : 1.0;
        double end = y + width < hi ? y + width : hi;
        total += gl_adapt(a, y, end, gl_panel(a, y, end), 0);
        y = end;
    }
    return total;
}

/* E1(a) - E1(b) for 0 < a <= b given as two numbers (used by the tests). */
double ddo_e1_diff_quad(double a, double b) {
    if (!(a > 0.0) || !(b >= a)) return NAN;
    return ddo_e1_diff_log(a, log1p((b - a) / a));
}

/* E1(a) - E1(b) with b = a e^ell: the FP64 difference of the two values where
   that is well conditioned, the quadrature of the definition otherwise. */
static double e1_diff_ab(double a, double b, double ell) {
    if (ell == 0.0 || a == b) return 0.0;
    if (a == 0.0) return INFINITY;
    double ea = ddo_e1(a), eb = ddo_e1(b);
    double d = ea - eb;
    if (ea + eb <= 16.0 * d) return d;
    return ddo_e1_diff_log(a, ell);
}

/* E1(a) - E1(b) for 0 <= a <= b. */
double ddo_e1_diff(double a, double b) {
    if (!(a >= 0.0) || !(b >= a)) return NAN;
    if (a == 0.0) return a == b ? 0.0 : INFINITY;
    return e1_diff_ab(a, b, log1p((b - a) / a));
}

/* ------------------------------------------------- single probe, Eq. 1-4 */

/* phi_i at squared distance rho2 [m^2] and elapsed time dt = t - t_i [s].
   Ds = r_s^2 [m^2], D [m^2/s], Q0 [u/s], tau [s].  Returns u/m^2. */
double ddo_phi(double rho2, double dt, double tau, double Ds, double D, double Q0) {
    if (!(dt > 0.0)) return 0.0;                       /* not started: no deposit yet */
    double pref = Q0 / (4.0 * PI_D * D);
    int on = dt <= tau;                                /* Eq. 1 for t_i <= t <= t_i + tau_i */
    double w1 = 2.0 * Ds + 4.0 * D * dt;               /* 2Ds + 4D(t - t_i) */
    double w0 = on ? 2.0 * Ds                          /* Eq. 1: 2Ds */
                   : 2.0 * Ds + 4.0 * D * (dt - tau);  /* Eq. 2: 2Ds + 4D(t - (t_i + tau_i)) */
    if (rho2 == 0.0) {
        /* Eq. 3 / Eq. 4: ln((Ds + 2D(t-t_i)) / Ds) and
           ln((Ds + 2D(t-t_i)) / (Ds + 2D(t-t_i-tau))), as ln(1 + (num - den)/den)
           with num - den = 2D min(t - t_i, tau_i) taken directly: long after the dwell
           the ratio is 1 + O(tau/(t - t_i)), and rounding it first would cost
           u / (num/den - 1) of relative accuracy */
        double den = on ? Ds : Ds + 2.0 * D * (dt - tau);
        return pref * log1p(2.0 * D * (on ? dt : tau) / den);
    }
    /* ln(b/a) = ln(w1/w0), with w1 - w0 = 4D min(t - t_i, tau_i) taken directly */
    double ell = log1p(4.0 * D * (on ? dt : tau) / w0);
    return pref * e1_diff_ab(rho2 / w1, rho2 / w0, ell);
}

/* --------------------------------------------------- cumulative field, Eq. 5 */

/* Threads of one call: `threads` if positive, else every thread OpenMP offers (the
   request applies to that call only). */
static int oracle_threads(int threads) {
#ifdef _OPENMP
    return threads > 0 ? threads : omp_get_max_threads();
#else
    (void)threads;
    return 1;
#endif
}

/* out[it * n_pts + ip] = sum_{i} phi_i(|p - r_i|^2, t - t_i), summed in visit order.
   Sources: xs, ys [m], ts start times [s], taus dwell [s] (n_src each). */
void ddo_field(int64_t n_src, const double *xs, const double *ys, const double *ts,
               const double *taus, double Ds, double D, double Q0,
               int64_t n_pts, const double *px, const double *py,
               int64_t n_t, const double *times, double *out, int threads) {
    if (!gl_ready) gl_init();
    const int nt = oracle_threads(threads);
    int64_t total = n_t * n_pts;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t k = 0; k < total; ++k) {
        int64_t it = k / n_pts, ip = k % n_pts;
        double t = times[it], acc = 0.0;
        for (int64_t i = 0; i < n_src; ++i) {
            double dx = px[ip] - xs[i], dy = py[ip] - ys[i];
            acc += ddo_phi(dx * dx + dy * dy, t - ts[i], taus[i], Ds, D, Q0);
        }
        out[k] = acc;
    }
}

/* Field at an explicit list of (point, time) pairs: out[k] = psi(p_k, t_k). */
void ddo_field_pairs(int64_t n_src, const double *xs, const double *ys, const double *ts,
                     const double *taus, double Ds, double D, double Q0,
                     int64_t n_pairs, const double *px, const double *py, const double *pt,
                     double *out, int threads) {
    if (!gl_ready) gl_init();
    const int nt = oracle_threads(threads);
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
    for (int64_t k = 0; k < n_pairs; ++k) {
        double acc = 0.0;
        for (int64_t i = 0; i < n_src; ++i) {
            double dx = px[k] - xs[i], dy = py[k] - ys[i];
            acc += ddo_phi(dx * dx + dy * dy, pt[k] - ts[i], taus[i], Ds, D, Q0);
        }
        out[k] = acc;
    }
}

/* Dwell-start dose of visit j: psi_{j-1}(r_j, t_j) = sum_{i<j} phi_i(r_j, t_j).
   Only the n_targets visits listed in `targets` are computed. */
void ddo_dose(int64_t n_src, const double *xs, const double *ys, const double *ts,
              const double *taus, double Ds, double D, double Q0,
              int64_t n_targets, const int64_t *targets, double *out, int threads) {
    if (!gl_ready) gl_init();
    const int nt = oracle_threads(threads);
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
    for (int64_t k = 0; k < n_targets; ++k) {
        int64_t j = targets[k];
        double acc = 0.0;
        if (j < 0 || j >= n_src) { out[k] = NAN; continue; }
        for (int64_t i = 0; i < j; ++i) {
            double dx = xs[j] - xs[i], dy = ys[j] - ys[i];
            acc += ddo_phi(dx * dx + dy * dy, ts[j] - ts[i], taus[i], Ds, D, Q0);
        }
        out[k] = acc;
    }
}

int ddo_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
