/*
 * pitn_oracle.c -- plain, slow, FP64 CPU reference for the parallel-in-time
 * Newton ODE solver of arXiv 2511.01465 ("A parallel-in-time Newton's
 * method-based ODE solver").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header or constant table with the CUDA
 * path: every formula here is written out again from the paper.
 *
 * Everything runs on one host core, in IEEE double, with no blocking, fusion
 * or reordering beyond what the paper's definitions state.  It is compiled
 * with -ffp-contract=off so that no a*b+c is silently fused and results are
 * the same on x86-64 and aarch64 hosts.
 *
 * What each routine follows:
 *   rhs / rhs_jac / rhs_dparam  the ODE right-hand sides, eq. (2.1); the test
 *                               systems of Sec. 4.1 (logistic, van der Pol)
 *                               and Sec. 4.2 (Dahlquist, Robertson) plus the
 *                               Lorenz-63, damped oscillator and Fisher-KPP
 *                               method-of-lines systems used as synthetic
 *                               workloads.
 *   step                        one-step maps: explicit Euler, eq. (2.2), and
 *                               the classical four-stage Runge-Kutta rule,
 *                               eq. (2.3), with their Jacobians by the chain
 *                               rule through the stages; the implicit rules
 *                               of Sec. 3.4 (backward Euler, eq. (2.5), and
 *                               the trapezoidal rule) in the residual and
 *                               Newton step of eqs. (3.15)-(3.19) (Dahlquist
 *                               and Robertson systems of Sec. 4.2).
 *   oracle_sequential           the sequential solver, Sec. 2.1.
 *   oracle_residual             the root-finding residual h(xi), eq. (3.8),
 *                               and its infinity norm, Sec. 4 (stopping rule).
 *   oracle_combine              the associative operator, eq. (3.3).
 *   oracle_affine_scan          the affine recursion, eq. (3.2), with the
 *                               element initialisation of eq. (3.4), run as a
 *                               plain sequential loop (the prefix sums of
 *                               eq. (3.1) evaluated left to right).
 *   oracle_newton               Newton's method, eqs. (3.10)-(3.11), with the
 *                               Newton step taken from the affine recursion
 *                               of eq. (3.13).
 *   oracle_newton_batch         independent IVPs solved one after another.
 *   oracle_adjoint              the reverse (transposed) recursion of the
 *                               same affine structure, for gradients of a
 *                               loss of the trajectory.
 *
 * Rounding variants (test builds only; the default build defines none of
 * these and computes exactly as described above).  Each variant is the same
 * mathematics in another rounding order; the tests build them to measure how
 * far rounding alone moves an iteration count whose decisions compare
 * rounded values (the guard's cut, reading R8):
 *   ORACLE_SUM_REVERSED       the sums of the Newton recursion's matrix-vector
 *                             products run from the last index to the first;
 *   ORACLE_RESID_DIFF_FIRST   the explicit Euler residual is grouped as
 *                             (x_n - x_{n-1}) - h f(x_{n-1}) instead of
 *                             x_n - (x_{n-1} + h f(x_{n-1}));
 *   ORACLE_BLOCK=C            the recursion of eq. (3.13) is bracketed in
 *                             blocks of C elements: block aggregates folded
 *                             with eq. (3.3), carried from block to block,
 *                             each block replayed from its incoming vector
 *                             (the same Newton step in exact arithmetic, by
 *                             the associativity of Lemma 3.1);
 *   ORACLE_SCAN_BITS=b        the explicit recursion of eq. (3.13) is carried
 *                             in a b-bit significand: the Jacobian entries,
 *                             the residual entries and every correction are
 *                             rounded to b significant bits (to nearest) as
 *                             they enter or leave the recursion (b = 48: a
 *                             scan in pairs of 24-bit floats);
 *   and, through the compiler, FMA contraction of every a*b + c.
 *
 * Readings of the paper that this file takes (the paper is silent on them):
 *   - K in the paper counts residual evaluations; `iters` here counts Newton
 *     updates actually applied (paper K - 1).
 *   - implicit rule: the stopping quantity is ||(I - dg/dx_n)^{-1} h_n||_inf,
 *     the preconditioned residual (it reproduces the paper's implicit traces,
 *     e.g. 1/1.1 and 1/1.004 at iteration 0 from a zero guess).
 *   - converged iff ||h||_inf <= tol; a NaN or infinite residual entry ends
 *     the solve with status NONFINITE, checked before the tolerance.
 *   - guard (not in the paper, optional): after the Newton step is computed,
 *     q = first step index whose correction has an entry that is not finite
 *     or exceeds B in magnitude.  Entries before q take the Newton update;
 *     entries from q on are set to the last updated state (x0 if q = 0).
 *     Without the guard (plain method) a non-finite correction ends the
 *     solve with status NONFINITE and leaves the trajectory at the last
 *     iterate, whose residual was finite.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>

/* System and method identifiers (the numbers a caller passes). */
enum { OR_LORENZ63 = 1, OR_VDP = 2, OR_LINEAR_OSC = 3, OR_FKPP = 4, OR_LOGISTIC = 5,
       OR_DAHLQUIST = 6, OR_ROBERTSON = 7 };
enum { OR_EULER = 0, OR_RK4 = 1, OR_BACKWARD_EULER = 2, OR_TRAPEZOID = 3 };
enum { OR_OK = 0, OR_NOT_CONVERGED = 1, OR_NONFINITE = 2, OR_EINVAL = -1, OR_ENOMEM = -2 };

int oracle_nparams(int sys)
{
    switch (sys) {
    case OR_LORENZ63: return 3;   /* sigma, rho, beta */
    case OR_VDP: return 1;        /* mu */
    case OR_LINEAR_OSC: return 2; /* omega, zeta */
    case OR_FKPP: return 1;       /* D */
    case OR_LOGISTIC: return 2;   /* r, K */
    case OR_DAHLQUIST: return 1;  /* lambda */
    case OR_ROBERTSON: return 3;  /* k1, k2, k3 */
    default: return -1;
    }
}

static int dim_ok(int sys, int d)
{
    switch (sys) {
    case OR_LORENZ63: return d == 3;
    case OR_VDP: return d == 2;
    case OR_LINEAR_OSC: return d == 2;
    case OR_FKPP: return d >= 1;
    case OR_LOGISTIC: return d == 1;
    case OR_DAHLQUIST: return d == 1;
    case OR_ROBERTSON: return d == 3;
    default: return 0;
    }
}

/* ------------------------------------------------------------------------ */
/* Right-hand sides f(x) of dx/dt = f(x), eq. (2.1).                         */
/* ------------------------------------------------------------------------ */

/* Fisher-KPP on [0,1] by the method of lines: d interior nodes x_i = i/(d+1),
 * i = 1..d, spacing dx = 1/(d+1), Dirichlet zeros at both ends, three-point
 * second difference:  f_i = D (u_{i-1} - 2 u_i + u_{i+1}) / dx^2 + u_i (1 - u_i). */
static double fkpp_inv_dx2(int d)
{
    double dx = 1.0 / (double)(d + 1);
    return 1.0 / (dx * dx);
}

int oracle_rhs(int sys, const double *p, int d, const double *x, double *f)
{
    if (!dim_ok(sys, d)) return OR_EINVAL;
    switch (sys) {
    case OR_LORENZ63: {
        double s = p[0], r = p[1], b = p[2];
        f[0] = s * (x[1] - x[0]);
        f[1] = x[0] * (r - x[2]) - x[1];
        f[2] = x[0] * x[1] - b * x[2];
        break;
    }
    case OR_VDP: {
        /* second-order van der Pol written as (x, dx/dt) */
        double mu = p[0];
        f[0] = x[1];
        f[1] = mu * (1.0 - x[0] * x[0]) * x[1] - x[0];
        break;
    }
    case OR_LINEAR_OSC: {
        /* x'' + 2 zeta omega x' + omega^2 x = 0 written as (x, dx/dt) */
        double w = p[0], z = p[1];
        f[0] = x[1];
        f[1] = -w * w * x[0] - 2.0 * z * w * x[1];
        break;
    }
    case OR_FKPP: {
        double D = p[0], c = fkpp_inv_dx2(d);
        for (int i = 0; i < d; ++i) {
            double um = (i > 0) ? x[i - 1] : 0.0;
            double up = (i < d - 1) ? x[i + 1] : 0.0;
            f[i] = D * (um - 2.0 * x[i] + up) * c + x[i] * (1.0 - x[i]);
        }
        break;
    }
    case OR_LOGISTIC: {
        double r = p[0], K = p[1];
        f[0] = r * x[0] * (1.0 - x[0] / K);
        break;
    }
    case OR_DAHLQUIST:
        /* y' = lambda y (Sec. 4.2) */
        f[0] = p[0] * x[0];
        break;
    case OR_ROBERTSON: {
        /* Robertson's reaction (Sec. 4.2) */
        double k1 = p[0], k2 = p[1], k3 = p[2];
        f[0] = -k1 * x[0] + k3 * x[1] * x[2];
        f[1] = k1 * x[0] - k2 * x[1] * x[1] - k3 * x[1] * x[2];
        f[2] = k2 * x[1] * x[1];
        break;
    }
    }
    return OR_OK;
}

/* Dense Jacobian df/dx, row-major d x d. */
int oracle_rhs_jac(int sys, const double *p, int d, const double *x, double *J)
{
    if (!dim_ok(sys, d)) return OR_EINVAL;
    memset(J, 0, sizeof(double) * (size_t)d * (size_t)d);
    switch (sys) {
    case OR_LORENZ63: {
        double s = p[0], r = p[1], b = p[2];
        J[0] = -s;       J[1] = s;       J[2] = 0.0;
        J[3] = r - x[2]; J[4] = -1.0;    J[5] = -x[0];
        J[6] = x[1];     J[7] = x[0];    J[8] = -b;
        break;
    }
    case OR_VDP: {
        double mu = p[0];
        J[0] = 0.0;                          J[1] = 1.0;
        J[2] = -2.0 * mu * x[0] * x[1] - 1.0; J[3] = mu * (1.0 - x[0] * x[0]);
        break;
    }
    case OR_LINEAR_OSC: {
        double w = p[0], z = p[1];
        J[0] = 0.0;    J[1] = 1.0;
        J[2] = -w * w; J[3] = -2.0 * z * w;
        break;
    }
    case OR_FKPP: {
        double D = p[0], c = fkpp_inv_dx2(d);
        for (int i = 0; i < d; ++i) {
            J[(size_t)i * d + i] = -2.0 * D * c + 1.0 - 2.0 * x[i];
            if (i > 0) J[(size_t)i * d + i - 1] = D * c;
            if (i < d - 1) J[(size_t)i * d + i + 1] = D * c;
        }
        break;
    }
    case OR_LOGISTIC: {
        double r = p[0], K = p[1];
        J[0] = r * (1.0 - 2.0 * x[0] / K);
        break;
    }
    case OR_DAHLQUIST:
        J[0] = p[0];
        break;
    case OR_ROBERTSON: {
        double k1 = p[0], k2 = p[1], k3 = p[2];
        J[0] = -k1; J[1] = k3 * x[2];                       J[2] = k3 * x[1];
        J[3] = k1;  J[4] = -2.0 * k2 * x[1] - k3 * x[2];    J[5] = -k3 * x[1];
        J[6] = 0.0; J[7] = 2.0 * k2 * x[1];                 J[8] = 0.0;
        break;
    }
    }
    return OR_OK;
}

/* Parameter Jacobian df/dp, row-major d x P (P = oracle_nparams(sys)). */
int oracle_rhs_dparam(int sys, const double *p, int d, const double *x, double *G)
{
    if (!dim_ok(sys, d)) return OR_EINVAL;
    int P = oracle_nparams(sys);
    memset(G, 0, sizeof(double) * (size_t)d * (size_t)P);
    switch (sys) {
    case OR_LORENZ63:
        G[0 * 3 + 0] = x[1] - x[0];  /* df0/dsigma */
        G[1 * 3 + 1] = x[0];         /* df1/drho */
        G[2 * 3 + 2] = -x[2];        /* df2/dbeta */
        break;
    case OR_VDP:
        G[1] = (1.0 - x[0] * x[0]) * x[1];
        break;
    case OR_LINEAR_OSC: {
        double w = p[0], z = p[1];
        G[2 * 1 + 0] = -2.0 * w * x[0] - 2.0 * z * x[1];  /* df1/domega */
        G[2 * 1 + 1] = -2.0 * w * x[1];                   /* df1/dzeta */
        break;
    }
    case OR_FKPP: {
        double c = fkpp_inv_dx2(d);
        for (int i = 0; i < d; ++i) {
            double um = (i > 0) ? x[i - 1] : 0.0;
            double up = (i < d - 1) ? x[i + 1] : 0.0;
            G[i] = (um - 2.0 * x[i] + up) * c;
        }
        break;
    }
    case OR_LOGISTIC: {
        double r = p[0], K = p[1];
        G[0] = x[0] * (1.0 - x[0] / K);
        G[1] = r * x[0] * x[0] / (K * K);
        break;
    }
    case OR_DAHLQUIST:
        G[0] = x[0];
        break;
    case OR_ROBERTSON:
        G[0 * 3 + 0] = -x[0];
        G[1 * 3 + 0] = x[0];
        G[1 * 3 + 1] = -x[1] * x[1];
        G[2 * 3 + 1] = x[1] * x[1];
        G[0 * 3 + 2] = x[1] * x[2];
        G[1 * 3 + 2] = -x[1] * x[2];
        break;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* One-step maps phi(x) = x + g(x, h) and their Jacobians.                   */
/* ------------------------------------------------------------------------ */

/* Dense helpers: C = A B (n x m times m x k), all row-major. */
static void matmul(int n, int m, int k, const double *A, const double *B, double *C)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < k; ++j) {
            double s = 0.0;
            for (int l = 0; l < m; ++l) s += A[(size_t)i * m + l] * B[(size_t)l * k + j];
            C[(size_t)i * k + j] = s;
        }
}

/* Solves A y = b in place (b <- y) by Gaussian elimination with partial
 * pivoting; A (d x d, row-major) is overwritten.  Returns 0, or -1 for a
 * singular matrix. */
static int solve_dense(int d, double *A, double *b)
{
    for (int c = 0; c < d; ++c) {
        int piv = c;
        for (int r = c + 1; r < d; ++r)
            if (fabs(A[(size_t)r * d + c]) > fabs(A[(size_t)piv * d + c])) piv = r;
        if (A[(size_t)piv * d + c] == 0.0) return -1;
        if (piv != c) {
            for (int j = 0; j < d; ++j) {
                double t = A[(size_t)c * d + j];
                A[(size_t)c * d + j] = A[(size_t)piv * d + j];
                A[(size_t)piv * d + j] = t;
            }
            double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < d; ++r) {
            double m = A[(size_t)r * d + c] / A[(size_t)c * d + c];
            for (int j = c; j < d; ++j) A[(size_t)r * d + j] -= m * A[(size_t)c * d + j];
            b[r] -= m * b[c];
        }
    }
    for (int r = d - 1; r >= 0; --r) {
        double sacc = b[r];
        for (int j = r + 1; j < d; ++j) sacc -= A[(size_t)r * d + j] * b[j];
        b[r] = sacc / A[(size_t)r * d + r];
    }
    return 0;
}

/* Implicit rules x_n = x_{n-1} + g(x_{n-1}, x_n) (Sec. 3.4):
 *   backward Euler (eq. 2.5):  g = h f(x_n);
 *   trapezoidal rule (Sec. 3.4): g = (h/2) (f(x_{n-1}) + f(x_n)).
 * implicit_parts computes, for the states xp = x_{n-1} and xc = x_n,
 *   the residual h_n = xc - xp - g(xp, xc)                    (eq. 3.15),
 *   A_n = I - dg/dx_n, the diagonal block of eq. 3.16, and, if B is not
 *   NULL, B_n = I + dg/dx_{n-1}, minus the sub-diagonal block of eq. 3.16. */
static int is_implicit(int method) { return method == OR_BACKWARD_EULER || method == OR_TRAPEZOID; }

static void implicit_parts(int sys, int method, const double *p, int d, double h, const double *xp,
                           const double *xc, double *hn, double *A, double *B)
{
    double *f = (double *)malloc(sizeof(double) * d);
    double w = (method == OR_TRAPEZOID) ? 0.5 * h : h;   /* weight of f(x_n) in g */
    oracle_rhs(sys, p, d, xc, f);
    for (int i = 0; i < d; ++i) hn[i] = xc[i] - xp[i] - w * f[i];
    if (method == OR_TRAPEZOID) {
        oracle_rhs(sys, p, d, xp, f);
        for (int i = 0; i < d; ++i) hn[i] -= w * f[i];
    }
    oracle_rhs_jac(sys, p, d, xc, A);
    for (int i = 0; i < d * d; ++i) A[i] = -w * A[i];
    for (int i = 0; i < d; ++i) A[(size_t)i * d + i] += 1.0;
    if (B) {
        if (method == OR_TRAPEZOID) {
            oracle_rhs_jac(sys, p, d, xp, B);
            for (int i = 0; i < d * d; ++i) B[i] = w * B[i];
        } else {
            for (int i = 0; i < d * d; ++i) B[i] = 0.0;
        }
        for (int i = 0; i < d; ++i) B[(size_t)i * d + i] += 1.0;
    }
    free(f);
}

/*
 * phi(x) for the explicit Euler rule, eq. (2.2):  phi(x) = x + h f(x),
 *   dphi/dx = I + h df/dx,  dphi/dp = h df/dp;
 * or for the classical RK4 rule, eq. (2.3), with the tableau
 *   a21 = 1/2, a32 = 1/2, a43 = 1, b = (1/6, 1/3, 1/3, 1/6):
 *   y_i = x + h sum_j a_ij kappa_j,  kappa_i = f(y_i),  phi = x + h sum_i b_i kappa_i,
 * differentiated stage by stage (forward mode).
 * dphi_dx (d x d) and dphi_dp (d x P) may be NULL.
 */
int oracle_step(int sys, int method, const double *p, int d, double h, const double *x,
                double *phi, double *dphi_dx, double *dphi_dp)
{
    if (!dim_ok(sys, d)) return OR_EINVAL;
    int P = oracle_nparams(sys);
    size_t dd = (size_t)d * d, dp = (size_t)d * P;
    if (method == OR_EULER) {
        double *f = (double *)malloc(sizeof(double) * d);
        if (!f) return OR_ENOMEM;
        oracle_rhs(sys, p, d, x, f);
        for (int i = 0; i < d; ++i) phi[i] = x[i] + h * f[i];
        free(f);
        if (dphi_dx) {
            oracle_rhs_jac(sys, p, d, x, dphi_dx);
            for (size_t i = 0; i < dd; ++i) dphi_dx[i] *= h;
            for (int i = 0; i < d; ++i) dphi_dx[(size_t)i * d + i] += 1.0;
        }
        if (dphi_dp) {
            oracle_rhs_dparam(sys, p, d, x, dphi_dp);
            for (size_t i = 0; i < dp; ++i) dphi_dp[i] *= h;
        }
        return OR_OK;
    }
    if (method != OR_RK4) return OR_EINVAL;

    static const double a[4][4] = {{0, 0, 0, 0}, {0.5, 0, 0, 0}, {0, 0.5, 0, 0}, {0, 0, 1.0, 0}};
    static const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    double *kap = (double *)calloc((size_t)4 * d, sizeof(double));
    double *y = (double *)calloc((size_t)d, sizeof(double));
    double *Kx = (double *)calloc(4 * dd, sizeof(double)); /* d kappa_i / dx */
    double *Kp = (double *)calloc(4 * dp + 1, sizeof(double)); /* d kappa_i / dp */
    double *Yx = (double *)calloc(dd, sizeof(double));
    double *Yp = (double *)calloc(dp + 1, sizeof(double));
    double *Jf = (double *)calloc(dd, sizeof(double));
    double *Gf = (double *)calloc(dp + 1, sizeof(double));
    if (!kap || !y || !Kx || !Kp || !Yx || !Yp || !Jf || !Gf) {
        free(kap); free(y); free(Kx); free(Kp); free(Yx); free(Yp); free(Jf); free(Gf);
        return OR_ENOMEM;
    }
    for (int i = 0; i < 4; ++i) {
        /* stage argument y_i and its derivatives */
        for (int c = 0; c < d; ++c) {
            double s = 0.0;
            for (int j = 0; j < i; ++j) s += a[i][j] * kap[(size_t)j * d + c];
            y[c] = x[c] + h * s;
        }
        if (dphi_dx) {
            for (size_t e = 0; e < dd; ++e) {
                double s = 0.0;
                for (int j = 0; j < i; ++j) s += a[i][j] * Kx[(size_t)j * dd + e];
                Yx[e] = h * s;
            }
            for (int c = 0; c < d; ++c) Yx[(size_t)c * d + c] += 1.0;
        }
        if (dphi_dp) {
            for (size_t e = 0; e < dp; ++e) {
                double s = 0.0;
                for (int j = 0; j < i; ++j) s += a[i][j] * Kp[(size_t)j * dp + e];
                Yp[e] = h * s;
            }
        }
        oracle_rhs(sys, p, d, y, kap + (size_t)i * d);
        if (dphi_dx || dphi_dp) oracle_rhs_jac(sys, p, d, y, Jf);
        if (dphi_dx) matmul(d, d, d, Jf, Yx, Kx + (size_t)i * dd);
        if (dphi_dp) {
            oracle_rhs_dparam(sys, p, d, y, Gf);
            matmul(d, d, P, Jf, Yp, Kp + (size_t)i * dp);
            for (size_t e = 0; e < dp; ++e) Kp[(size_t)i * dp + e] += Gf[e];
        }
    }
    for (int c = 0; c < d; ++c) {
        double s = 0.0;
        for (int i = 0; i < 4; ++i) s += b[i] * kap[(size_t)i * d + c];
        phi[c] = x[c] + h * s;
    }
    if (dphi_dx) {
        for (size_t e = 0; e < dd; ++e) {
            double s = 0.0;
            for (int i = 0; i < 4; ++i) s += b[i] * Kx[(size_t)i * dd + e];
            dphi_dx[e] = h * s;
        }
        for (int c = 0; c < d; ++c) dphi_dx[(size_t)c * d + c] += 1.0;
    }
    if (dphi_dp) {
        for (size_t e = 0; e < dp; ++e) {
            double s = 0.0;
            for (int i = 0; i < 4; ++i) s += b[i] * Kp[(size_t)i * dp + e];
            dphi_dp[e] = h * s;
        }
    }
    free(kap); free(y); free(Kx); free(Kp); free(Yx); free(Yp); free(Jf); free(Gf);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Sequential solver and the residual of eq. (3.8).                          */
/* ------------------------------------------------------------------------ */

/* x_{n+1} = phi(x_n), n = 0..N-1; traj[n] holds x_{n+1}. */
int oracle_sequential(int sys, int method, const double *p, const double *x0, double h,
                      int64_t N, int d, double *traj)
{
    if (!dim_ok(sys, d) || N < 0) return OR_EINVAL;
    if (is_implicit(method)) {
        /* each step solves x_n - x_{n-1} - g(x_{n-1}, x_n) = 0 by Newton from x_{n-1},
         * to the last bit (correction below 1e-15 relative, at most 100 steps) */
        double *hn = (double *)malloc(sizeof(double) * d);
        double *A = (double *)malloc(sizeof(double) * (size_t)d * d);
        const double *prev = x0;
        for (int64_t n = 0; n < N; ++n) {
            double *y = traj + (size_t)n * d;
            memcpy(y, prev, sizeof(double) * d);
            for (int it = 0; it < 100; ++it) {
                implicit_parts(sys, method, p, d, h, prev, y, hn, A, NULL);
                if (solve_dense(d, A, hn)) break;
                double nrm = 0.0, ny = 0.0;
                for (int i = 0; i < d; ++i) {
                    y[i] -= hn[i];
                    if (fabs(hn[i]) > nrm) nrm = fabs(hn[i]);
                    if (fabs(y[i]) > ny) ny = fabs(y[i]);
                }
                if (nrm <= 1e-15 * ny || nrm == 0.0) break;
            }
            prev = y;
        }
        free(hn); free(A);
        return OR_OK;
    }
    const double *prev = x0;
    for (int64_t n = 0; n < N; ++n) {
        int rc = oracle_step(sys, method, p, d, h, prev, traj + (size_t)n * d, NULL, NULL);
        if (rc) return rc;
        prev = traj + (size_t)n * d;
    }
    return OR_OK;
}

/*
 * h_n = x_n - x_{n-1} - g_{n-1}(x_{n-1}) = x_n - phi(x_{n-1}), n = 1..N, eq. (3.8),
 * with x_0 the fixed initial value.  r[n-1] receives h_n (may be NULL).
 * Returns ||h||_inf through *res (NaN if any entry is NaN, else +inf if any
 * entry is infinite) and whether any entry was not finite through *nonfinite.
 */
int oracle_residual(int sys, int method, const double *p, const double *x0, double h,
                    int64_t N, int d, const double *traj, double *r, double *res, int *nonfinite)
{
    if (!dim_ok(sys, d) || N < 0) return OR_EINVAL;
    double *phi = (double *)malloc(sizeof(double) * d);
    double *A = (double *)malloc(sizeof(double) * (size_t)d * d);
    if (!phi || !A) { free(phi); free(A); return OR_ENOMEM; }
    double m = 0.0;
    int saw_nan = 0, nf = 0;
    for (int64_t n = 0; n < N; ++n) {
        const double *prev = (n == 0) ? x0 : traj + (size_t)(n - 1) * d;
#ifdef ORACLE_RESID_DIFF_FIRST
        if (method == OR_EULER) {
            /* rounding variant: h_n = (x_n - x_{n-1}) - h f(x_{n-1}) */
            oracle_rhs(sys, p, d, prev, phi);
            for (int c = 0; c < d; ++c) {
                double v = (traj[(size_t)n * d + c] - prev[c]) - h * phi[c];
                if (r) r[(size_t)n * d + c] = v;
                double a = fabs(v);
                if (!isfinite(v)) nf = 1;
                if (a != a) saw_nan = 1;
                else if (a > m) m = a;
            }
            continue;
        }
#endif
        if (is_implicit(method)) {
            /* implicit rule: the residual h_n of eq. 3.15 preconditioned by
             * (I - dg/dx_n)^{-1}, the quantity the paper's implicit residual
             * figure reports (reading taken here) */
            implicit_parts(sys, method, p, d, h, prev, traj + (size_t)n * d, phi, A, NULL);
            if (solve_dense(d, A, phi))
                for (int c = 0; c < d; ++c) phi[c] = NAN;
            for (int c = 0; c < d; ++c) phi[c] = traj[(size_t)n * d + c] - phi[c];
        } else {
            oracle_step(sys, method, p, d, h, prev, phi, NULL, NULL);
        }
        for (int c = 0; c < d; ++c) {
            double v = traj[(size_t)n * d + c] - phi[c];
            if (r) r[(size_t)n * d + c] = v;
            double a = fabs(v);
            if (!isfinite(v)) nf = 1;
            if (a != a) saw_nan = 1;
            else if (a > m) m = a;
        }
    }
    free(phi);
    free(A);
    if (res) *res = saw_nan ? NAN : m;
    if (nonfinite) *nonfinite = nf;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Affine elements, eqs. (3.2)-(3.4).                                        */
/* ------------------------------------------------------------------------ */

/* (A, b) = (A2, b2) (x) (A1, b1) = (A2 A1, A2 b1 + b2), eq. (3.3):
 * element 1 covers the earlier interval, element 2 the later one. */
int oracle_combine(int d, const double *A2, const double *b2, const double *A1, const double *b1,
                   double *A, double *b)
{
    if (d < 1) return OR_EINVAL;
    size_t dd = (size_t)d * d;
    double *tA = (double *)malloc(sizeof(double) * dd);
    double *tb = (double *)malloc(sizeof(double) * d);
    if (!tA || !tb) { free(tA); free(tb); return OR_ENOMEM; }
    matmul(d, d, d, A2, A1, tA);
    matmul(d, d, 1, A2, b1, tb);
    for (int i = 0; i < d; ++i) tb[i] += b2[i];
    memcpy(A, tA, sizeof(double) * dd);
    memcpy(b, tb, sizeof(double) * d);
    free(tA); free(tb);
    return OR_OK;
}

/*
 * States of the affine recursion z_{n+1} = F_n z_n + c_n started from
 * z_0 = 0 (eq. (3.2)), i.e. the b-parts of the prefix sums of eq. (3.1) over
 * the elements (F_n, c_n); element 0's matrix is replaced by 0 as in
 * eq. (3.4).  z[n] receives the state after element n:  z[0] = c_0,
 * z[n] = F_n z[n-1] + c_n.  A is [N][d][d], c and z are [N][d].
 */
int oracle_affine_scan(int64_t N, int d, const double *A, const double *c, double *z)
{
    if (N < 0 || d < 1) return OR_EINVAL;
    for (int64_t n = 0; n < N; ++n) {
        for (int i = 0; i < d; ++i) {
            double s = c[(size_t)n * d + i];
            if (n > 0) {
                for (int j = 0; j < d; ++j)
                    s += A[((size_t)n * d + i) * d + j] * z[(size_t)(n - 1) * d + j];
            }
            z[(size_t)n * d + i] = s;
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Newton's method, eqs. (3.8)-(3.13).                                       */
/* ------------------------------------------------------------------------ */

/* Sum of row . v over d entries, in the order the build selects (index order
 * by default; from the last index to the first in the ORACLE_SUM_REVERSED
 * rounding variant). */
static double row_dot(const double *row, const double *v, int d)
{
    double s = 0.0;
#ifdef ORACLE_SUM_REVERSED
    for (int j = d - 1; j >= 0; --j) s += row[j] * v[j];
#else
    for (int j = 0; j < d; ++j) s += row[j] * v[j];
#endif
    return s;
}

#if defined(ORACLE_SCAN_BITS) && ORACLE_SCAN_BITS > 0
/* v rounded to ORACLE_SCAN_BITS significant bits, to nearest (ties to even
 * in the default rounding mode); zero, infinities and NaN unchanged.
 * v = m 2^e with 0.5 <= |m| < 1, so m 2^b holds the b leading bits in its
 * integer part. */
static double scan_round(double v)
{
    if (v == 0.0 || !isfinite(v)) return v;
    int e;
    double m = frexp(v, &e);
    return ldexp(nearbyint(ldexp(m, ORACLE_SCAN_BITS)), e - ORACLE_SCAN_BITS);
}
#endif

#if defined(ORACLE_BLOCK) && ORACLE_BLOCK > 0
/*
 * Rounding variant (test builds only): the explicit recursion of eq. (3.13),
 *   dx[0] = -r[0],  dx[n] = J(x_n) dx[n-1] - r[n]   (0-based buffer index),
 * bracketed in blocks of ORACLE_BLOCK elements.  Element n is (F_n, c_n) with
 * F_0 = 0 (eq. 3.4), F_n = J(x_n) and c_n = -r[n]; each block's aggregate is
 * folded with eq. (3.3), the aggregates carry the correction from block to
 * block, and each block is replayed from its incoming vector.  By the
 * associativity of eq. (3.3) (Lemma 3.1) this is the same Newton step in
 * exact arithmetic.
 */
static int recursion_blocked(int sys, int method, const double *p, int d, double h, int64_t N,
                             const double *traj, const double *r, double *dx)
{
    const int64_t C = ORACLE_BLOCK;
    size_t dd = (size_t)d * d;
    double *P = (double *)malloc(sizeof(double) * dd), *tP = (double *)malloc(sizeof(double) * dd);
    double *F = (double *)malloc(sizeof(double) * dd), *phi = (double *)malloc(sizeof(double) * d);
    double *c = (double *)malloc(sizeof(double) * d), *tc = (double *)malloc(sizeof(double) * d);
    double *z = (double *)malloc(sizeof(double) * d), *v = (double *)malloc(sizeof(double) * d);
    double *tv = (double *)malloc(sizeof(double) * d);
    if (!P || !tP || !F || !phi || !c || !tc || !z || !v || !tv) {
        free(P); free(tP); free(F); free(phi); free(c); free(tc); free(z); free(v); free(tv);
        return OR_ENOMEM;
    }
    for (int i = 0; i < d; ++i) z[i] = 0.0;
    for (int64_t s0 = 0; s0 < N; s0 += C) {
        int64_t e0 = (s0 + C < N) ? s0 + C : N;
        /* aggregate of the block: (P, c) <- (F_n, c_n) o (P, c) */
        for (size_t i = 0; i < dd; ++i) P[i] = 0.0;
        for (int i = 0; i < d; ++i) { P[(size_t)i * d + i] = 1.0; c[i] = 0.0; }
        for (int64_t n = s0; n < e0; ++n) {
            if (n == 0) {
                for (size_t i = 0; i < dd; ++i) P[i] = 0.0;
                for (int i = 0; i < d; ++i) c[i] = -r[i];
                continue;
            }
            oracle_step(sys, method, p, d, h, traj + (size_t)(n - 1) * d, phi, F, NULL);
            for (int i = 0; i < d; ++i) {
                for (int j = 0; j < d; ++j) {
                    double sacc = 0.0;
                    for (int l = 0; l < d; ++l) sacc += F[(size_t)i * d + l] * P[(size_t)l * d + j];
                    tP[(size_t)i * d + j] = sacc;
                }
                tc[i] = row_dot(F + (size_t)i * d, c, d) - r[(size_t)n * d + i];
            }
            memcpy(P, tP, sizeof(double) * dd);
            memcpy(c, tc, sizeof(double) * d);
        }
        /* replay of the block from its incoming vector z */
        memcpy(v, z, sizeof(double) * d);
        for (int64_t n = s0; n < e0; ++n) {
            if (n == 0) {
                for (int i = 0; i < d; ++i) v[i] = -r[i];
            } else {
                oracle_step(sys, method, p, d, h, traj + (size_t)(n - 1) * d, phi, F, NULL);
                for (int i = 0; i < d; ++i) tv[i] = row_dot(F + (size_t)i * d, v, d) - r[(size_t)n * d + i];
                memcpy(v, tv, sizeof(double) * d);
            }
            memcpy(dx + (size_t)n * d, v, sizeof(double) * d);
        }
        /* incoming vector of the next block: the aggregate applied to z */
        for (int i = 0; i < d; ++i) tv[i] = row_dot(P + (size_t)i * d, z, d) + c[i];
        memcpy(z, tv, sizeof(double) * d);
    }
    free(P); free(tP); free(F); free(phi); free(c); free(tc); free(z); free(v); free(tv);
    return OR_OK;
}
#endif

/*
 * Solves h(xi) = 0 for xi = [x_1 .. x_N] (traj, [N][d]).
 *   guess     NULL: x_n = x0 for all n (constant guess); else the guess [N][d].
 *   guard_B   <= 0 (or not finite): the paper's plain Newton; > 0: the guard
 *             described in the header, with bound B.
 *   res_hist  NULL or room for max_iter + 1 values: ||h(xi^(k))||_inf per
 *             residual evaluation.
 *   iters     Newton updates applied; status OR_OK / OR_NOT_CONVERGED /
 *             OR_NONFINITE; guard_index = q of the last update (N if none cut).
 *   cut_hist  NULL or room for max_iter + 1 values: entry k receives the q of
 *             Newton step k (N if nothing was cut), for every step computed
 *             (including a plain solve's last, rejected step).
 * Each iteration:
 *   1. r = h(xi), res = ||r||_inf (eq. 3.8, Sec. 4 stopping quantity);
 *   2. non-finite residual -> NONFINITE; res <= tol -> OK;
 *      iteration count reached max_iter -> NOT_CONVERGED;
 *   3. Newton step by the affine recursion of eq. (3.13):
 *        dx_1 = -h_1,  dx_n = (I + dg_{n-1}/dx_{n-1}) dx_{n-1} - h_n,
 *      where I + dg/dx is the step map's Jacobian at x_{n-1};
 *   4. xi <- xi + dxi, eq. (3.11) (guarded as described when guard_B > 0).
 */
int oracle_newton(int sys, int method, const double *p, const double *x0, double h, int64_t N,
                  int d, double tol, int max_iter, double guard_B, const double *guess,
                  double *traj, double *res_hist, int32_t *iters, int32_t *status,
                  int64_t *guard_index, int64_t *cut_hist)
{
    if (!dim_ok(sys, d) || N < 1 || max_iter < 0 || !(tol >= 0.0) || !traj || !x0 || !p)
        return OR_EINVAL;
    int guarded = (guard_B > 0.0) && isfinite(guard_B);
    double cap = guarded ? guard_B : DBL_MAX;
    size_t nd = (size_t)N * d, dd = (size_t)d * d;
    double *r = (double *)malloc(sizeof(double) * nd);
    double *dx = (double *)malloc(sizeof(double) * nd);
    double *J = (double *)malloc(sizeof(double) * dd);
    double *Bm = (double *)malloc(sizeof(double) * dd);
    double *phi = (double *)malloc(sizeof(double) * d);
    if (!r || !dx || !J || !Bm || !phi) {
        free(r); free(dx); free(J); free(Bm); free(phi);
        return OR_ENOMEM;
    }

    if (guess) memcpy(traj, guess, sizeof(double) * nd);
    else for (int64_t n = 0; n < N; ++n) memcpy(traj + (size_t)n * d, x0, sizeof(double) * d);

    int it = 0, st = OR_NOT_CONVERGED;
    int64_t q_last = N;
    for (;;) {
        double res;
        int nf;
        oracle_residual(sys, method, p, x0, h, N, d, traj, r, &res, &nf);
        if (res_hist) res_hist[it] = res;
        if (nf) { st = OR_NONFINITE; break; }
        if (res <= tol) { st = OR_OK; break; }
        if (it == max_iter) { st = OR_NOT_CONVERGED; break; }

        /* Newton step, eq. (3.13): dx[n] holds Delta x_{n+1}. */
        for (int i = 0; i < d; ++i) dx[i] = -r[i];
        if (is_implicit(method)) {
            /* eq. 3.19:
             *   dx_n = (I - dg/dx_n)^{-1} [(I + dg/dx_{n-1}) dx_{n-1} - h_n]
             *        = A_n^{-1} B_n dx_{n-1} - r_n,
             * r_n the preconditioned residual above */
            for (int64_t n = 1; n < (int64_t)N; ++n) {
                const double *xp = traj + (size_t)(n - 1) * d;
                implicit_parts(sys, method, p, d, h, xp, traj + (size_t)n * d, phi, J, Bm);
                for (int i = 0; i < d; ++i) {
                    double sacc = 0.0;
                    for (int j = 0; j < d; ++j) sacc += Bm[(size_t)i * d + j] * dx[(size_t)(n - 1) * d + j];
                    phi[i] = sacc;
                }
                solve_dense(d, J, phi);
                for (int i = 0; i < d; ++i) dx[(size_t)n * d + i] = phi[i] - r[(size_t)n * d + i];
            }
        } else {
#if defined(ORACLE_BLOCK) && ORACLE_BLOCK > 0
            if (recursion_blocked(sys, method, p, d, h, N, traj, r, dx) != OR_OK) {
                free(r); free(dx); free(J); free(Bm); free(phi);
                return OR_ENOMEM;
            }
#elif defined(ORACLE_SCAN_BITS) && ORACLE_SCAN_BITS > 0
            for (int i = 0; i < d; ++i) dx[i] = scan_round(dx[i]);
            for (int64_t n = 1; n < (int64_t)N; ++n) {
                const double *xn = traj + (size_t)(n - 1) * d;
                oracle_step(sys, method, p, d, h, xn, phi, J, NULL);
                for (size_t i = 0; i < dd; ++i) J[i] = scan_round(J[i]);
                for (int i = 0; i < d; ++i)
                    dx[(size_t)n * d + i] =
                        scan_round(row_dot(J + (size_t)i * d, dx + (size_t)(n - 1) * d, d) -
                                   scan_round(r[(size_t)n * d + i]));
            }
#else
            for (int64_t n = 1; n < (int64_t)N; ++n) {
                const double *xn = traj + (size_t)(n - 1) * d;   /* x_n, state n (1-based) */
                oracle_step(sys, method, p, d, h, xn, phi, J, NULL);
                for (int i = 0; i < d; ++i)
                    dx[(size_t)n * d + i] = row_dot(J + (size_t)i * d, dx + (size_t)(n - 1) * d, d) -
                                            r[(size_t)n * d + i];
            }
#endif
        }
        /* first correction that is not finite (or exceeds the guard bound) */
        int64_t q = N;
        for (int64_t n = 0; n < N && q == N; ++n)
            for (int i = 0; i < d; ++i)
                if (!(fabs(dx[(size_t)n * d + i]) <= cap)) { q = n; break; }
        if (cut_hist) cut_hist[it] = q;
        if (!guarded && q < N) { st = OR_NONFINITE; break; }

        /* update, eq. (3.11) */
        for (int64_t n = 0; n < q; ++n)
            for (int i = 0; i < d; ++i) traj[(size_t)n * d + i] += dx[(size_t)n * d + i];
        for (int64_t n = q; n < N; ++n) {
            const double *src = (q > 0) ? traj + (size_t)(q - 1) * d : x0;
            memcpy(traj + (size_t)n * d, src, sizeof(double) * d);
        }
        q_last = q;
        ++it;
    }
    if (iters) *iters = it;
    if (status) *status = st;
    if (guard_index) *guard_index = q_last;
    free(r); free(dx); free(J); free(Bm); free(phi);
    return OR_OK;
}

/*
 * B independent IVPs of lengths N[b], solved one after another by
 * oracle_newton.  Trajectories are concatenated: IVP b occupies rows
 * offsets[b] .. offsets[b+1]-1 of traj ([sum N][d]), with offsets the
 * exclusive prefix sum of N.  res_out (nullable) receives each final
 * residual norm.
 */
int oracle_newton_batch(int sys, int method, int64_t B, const double *params, const double *x0,
                        const double *h, const int64_t *N, int d, double tol, int max_iter,
                        double guard_B, double *traj, int64_t *offsets, int32_t *iters,
                        int32_t *status, double *res_out)
{
    int P = oracle_nparams(sys);
    if (P < 0 || B < 0 || !dim_ok(sys, d)) return OR_EINVAL;
    double *hist = (double *)malloc(sizeof(double) * ((size_t)max_iter + 1));
    if (!hist) return OR_ENOMEM;
    int64_t off = 0;
    for (int64_t b = 0; b < B; ++b) {
        offsets[b] = off;
        int64_t gi;
        int rc = oracle_newton(sys, method, params + (size_t)b * P, x0 + (size_t)b * d, h[b], N[b],
                               d, tol, max_iter, guard_B, NULL, traj + (size_t)off * d, hist,
                               iters + b, status + b, &gi, NULL);
        if (rc) { free(hist); return rc; }
        if (res_out) res_out[b] = hist[iters[b]];
        off += N[b];
    }
    offsets[B] = off;
    free(hist);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Adjoint (reverse) recursion.                                              */
/* ------------------------------------------------------------------------ */

/*
 * For a loss L(x_1..x_N) of a trajectory that satisfies x_{n+1} = phi(x_n)
 * (the Newton root), with G_n = dL/dx_n given by grad_traj[n-1] (nullable)
 * plus grad_xN on G_N (nullable):
 *   lambda_N = G_N,  lambda_n = (dphi/dx(x_n))^T lambda_{n+1} + G_n,  n = N-1..1,
 *   dL/dx0 = (dphi/dx(x_0))^T lambda_1,
 *   dL/dp  = sum_{n=0}^{N-1} (dphi/dp(x_n))^T lambda_{n+1}.
 * This is the transposed form of the same affine recursion as eq. (3.13),
 * run backwards in time.
 */
int oracle_adjoint(int sys, int method, const double *p, const double *x0, double h, int64_t N,
                   int d, const double *traj, const double *grad_traj, const double *grad_xN,
                   double *grad_x0, double *grad_p)
{
    int P = oracle_nparams(sys);
    if (P < 0 || !dim_ok(sys, d) || N < 1) return OR_EINVAL;
    if (method != OR_EULER && method != OR_RK4) return OR_EINVAL;   /* explicit maps only */
    size_t dd = (size_t)d * d, dp = (size_t)d * P;
    double *lam = (double *)calloc((size_t)d, sizeof(double));
    double *nl = (double *)calloc((size_t)d, sizeof(double));
    double *J = (double *)calloc(dd, sizeof(double));
    double *G = (double *)calloc(dp, sizeof(double));
    double *phi = (double *)calloc((size_t)d, sizeof(double));
    if (!lam || !nl || !J || !G || !phi) {
        free(lam); free(nl); free(J); free(G); free(phi);
        return OR_ENOMEM;
    }
    for (int i = 0; i < P; ++i) grad_p[i] = 0.0;
    /* lambda_N */
    for (int i = 0; i < d; ++i) {
        double g = 0.0;
        if (grad_traj) g += grad_traj[(size_t)(N - 1) * d + i];
        if (grad_xN) g += grad_xN[i];
        lam[i] = g;
    }
    for (int64_t n = N - 1; n >= 0; --n) {
        const double *xn = (n == 0) ? x0 : traj + (size_t)(n - 1) * d;
        oracle_step(sys, method, p, d, h, xn, phi, J, G);
        /* dL/dp += (dphi/dp(x_n))^T lambda_{n+1} */
        for (int k = 0; k < P; ++k) {
            double s = 0.0;
            for (int i = 0; i < d; ++i) s += G[(size_t)i * P + k] * lam[i];
            grad_p[k] += s;
        }
        /* lambda_n = J^T lambda_{n+1} + G_n  (n >= 1);  dL/dx0 = J^T lambda_1 */
        for (int j = 0; j < d; ++j) {
            double s = 0.0;
            for (int i = 0; i < d; ++i) s += J[(size_t)i * d + j] * lam[i];
            if (n >= 1 && grad_traj) s += grad_traj[(size_t)(n - 1) * d + j];
            nl[j] = s;
        }
        memcpy(lam, nl, sizeof(double) * d);
    }
    memcpy(grad_x0, lam, sizeof(double) * d);
    free(lam); free(nl); free(J); free(G); free(phi);
    return OR_OK;
}
