/*
 * nls_oracle.c -- plain, slow, FP64 reference solver for batches of small
 * nonlinear systems F(u; p) = 0.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this library.  The GPU library never
 * includes, links or calls anything here, and nothing here is derived from
 * the GPU code: the residuals, the analytic Jacobians (no dual numbers), the
 * LU factorisation and the three globalisations are written out again from
 * the paper's definitions, one step after another, in the paper's order.
 *
 * Paper: "NonlinearSolve.jl: High-Performance and Robust Solvers for Systems
 * of Nonlinear Equations in Julia" (arXiv 2403.16341).
 *   Sec. 2, Eq. 1        problem statement: find u* with f(u*, theta) = 0
 *   Sec. 2.1             termination test ||f(u_k)||_inf <= abstol
 *   Sec. 2.1, Eq. 2      Newton-Raphson: J_k du = -f(u_k), u_{k+1} = u_k + du
 *   Sec. 2.2.1, Eq. 8-9  Armijo sufficient decrease on phi = 1/2 ||f||^2,
 *                        slope f^T J du; backtracking: alpha_0 = 1, alpha <- rho alpha
 *   Sec. 2.2.2, Eq. 13-15 trust-region model, ratio rho_k, radius update,
 *                        Powell's dogleg
 *   Sec. 3.2 (Fig. 5)    small dense systems use a native LU (partial pivoting)
 *   Sec. 2.2.1, Eq. 5    generalized Rosenbrock function
 *   Sec. 2.1, Eq. 3      Halley: a = Newton step, J b = H a a,
 *                        du = (a o a) / (a + b/2) elementwise
 *   Sec. 2.1, Eq. 4      Potra-Ptak: two solves with the same J_k,
 *                        y = u + du1, u_{k+1} = y + du2 with J_k du2 = -f(y)
 *   Sec. 2.2.2, Tab. 3   the NocedalWright radius update: Algorithm 4.1 of
 *                        Nocedal & Wright, Numerical Optimization (the
 *                        paper's reference for it)
 *   Sec. 3.1, Tab. 1     Broyden (identity start) and modified Broyden
 *                        (true Jacobian start), "good Broyden" update
 *
 * Readings where the paper gives no value (all listed in the design notes):
 *   backtracking c1 = 1e-4, rho = 1/2, at most 30 trials;
 *   trust region: Delta_0 = 1, accept iff rho_k > 0, expand (x2, capped at
 *   1e3) iff rho_k > 0.75, otherwise keep; on rejection shrink (x1/4) and
 *   reuse J and the Newton step; 32 rejections in a row -> TR_STALLED;
 *   Euclidean norm for the trust region; pivot ties go to the lowest row;
 *   an exactly zero or non-finite pivot is SINGULAR; the iteration count k
 *   counts loop passes (Jacobian uses, including rejected trust-region
 *   passes); Bratu's 1/h^2 is the exact integer (n+1)^2.
 *   NocedalWright: eta = 1e-4, Delta_0 = 1, Delta_max = 1e3, 32 rejections
 *   in a row -> TR_STALLED; "the step reaches the boundary" is the dogleg's
 *   branch C or D.
 *   Halley: where a_i + b_i/2 is exactly zero the component of the step is
 *   a_i (the Newton component).  Potra-Ptak: both substeps are taken in
 *   every pass, the convergence test is on f(u_{k+1}).  Broyden: full steps,
 *   no re-initialisation, the update is skipped for a zero step.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no fast-math, no FMA
 * contraction, so every operation is one IEEE double rounding).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { FAM_CUBIC = 0, FAM_BRATU = 1, FAM_SQUARE = 2, FAM_ROSENBROCK = 3 };
enum { ALG_NEWTON = 0, ALG_NEWTON_BACKTRACK = 1, ALG_TRUST_DOGLEG = 2, ALG_POTRA_PTAK = 4,
       ALG_HALLEY = 5, ALG_BROYDEN = 6, ALG_MOD_BROYDEN = 7, ALG_TRUST_DOGLEG_NW = 8 };
enum { ST_SUCCESS = 0, ST_MAXITERS = 1, ST_SINGULAR = 2, ST_NONFINITE = 3,
       ST_LS_FAILED = 4, ST_TR_STALLED = 5 };

/* Backtracking line search (Sec. 2.2.1). */
static const double LS_C1 = 1e-4;
static const double LS_RHO = 0.5;
static const int LS_MAX_TRIALS = 30;
/* Trust region, "Simple" radius update (Sec. 2.2.2). */
static const double TR_DELTA0 = 1.0;
static const double TR_ETA_EXPAND = 0.75;
static const double TR_GROW = 2.0;
static const double TR_SHRINK = 0.25;
static const double TR_DELTA_MAX = 1e3;
static const int TR_MAX_REJECTIONS = 32;
/* Trust region, NocedalWright radius update (Nocedal & Wright, Alg. 4.1). */
static const double TR_NW_ETA = 1e-4;

int oracle_n_params(int family, int n)
{
    switch (family) {
    case FAM_CUBIC: return n * n + n;
    case FAM_BRATU: return 1;
    case FAM_SQUARE: return n;
    case FAM_ROSENBROCK: return 0;
    default: return -1;
    }
}

/* ---------------------------------------------------------------- residuals */

/* F = f(u; p) for one instance; p is that instance's parameter vector. */
void oracle_residual(int family, int n, const double *p, const double *u, double *F)
{
    int i, j;
    if (family == FAM_CUBIC) {
        /* F_i = sum_j A_ij u_j + u_i^3 - b_i, A row-major in p, then b. */
        const double *A = p, *b = p + n * n;
        for (i = 0; i < n; i++) {
            double s = 0.0;
            for (j = 0; j < n; j++)
                s += A[i * n + j] * u[j];
            F[i] = s + u[i] * u[i] * u[i] - b[i];
        }
    } else if (family == FAM_BRATU) {
        /* F_i = (u_{i-1} - 2 u_i + u_{i+1}) / h^2 + lambda exp(u_i),
         * h = 1/(n+1), u_0 = u_{n+1} = 0 (1-based). */
        double lambda = p[0];
        double inv_h2 = (double)(n + 1) * (double)(n + 1);
        for (i = 0; i < n; i++) {
            double left = (i > 0) ? u[i - 1] : 0.0;
            double right = (i < n - 1) ? u[i + 1] : 0.0;
            F[i] = (left - 2.0 * u[i] + right) * inv_h2 + lambda * exp(u[i]);
        }
    } else if (family == FAM_SQUARE) {
        /* F_i = u_i^2 - p_i (the Sec. 2.3 example). */
        for (i = 0; i < n; i++)
            F[i] = u[i] * u[i] - p[i];
    } else { /* FAM_ROSENBROCK, Eq. 5 */
        F[0] = 1.0 - u[0];
        for (i = 1; i < n; i++)
            F[i] = 10.0 * (u[i] - u[i - 1] * u[i - 1]);
    }
}

/* Analytic Jacobian J_ij = dF_i/du_j, row-major. */
void oracle_jacobian(int family, int n, const double *p, const double *u, double *J)
{
    int i;
    memset(J, 0, sizeof(double) * (size_t)n * (size_t)n);
    if (family == FAM_CUBIC) {
        memcpy(J, p, sizeof(double) * (size_t)n * (size_t)n);
        for (i = 0; i < n; i++)
            J[i * n + i] += 3.0 * u[i] * u[i];
    } else if (family == FAM_BRATU) {
        double lambda = p[0];
        double inv_h2 = (double)(n + 1) * (double)(n + 1);
        for (i = 0; i < n; i++) {
            J[i * n + i] = -2.0 * inv_h2 + lambda * exp(u[i]);
            if (i > 0) J[i * n + i - 1] = inv_h2;
            if (i < n - 1) J[i * n + i + 1] = inv_h2;
        }
    } else if (family == FAM_SQUARE) {
        for (i = 0; i < n; i++)
            J[i * n + i] = 2.0 * u[i];
    } else {
        J[0] = -1.0;
        for (i = 1; i < n; i++) {
            J[i * n + i] = 10.0;
            J[i * n + i - 1] = -20.0 * u[i - 1];
        }
    }
}

/* Second directional derivative h = d^2/dt^2 F(u + t a) at t = 0, i.e. the
 * term H a a of Halley's method (Sec. 2.1, Eq. 3), from the closed-form
 * second derivatives of each family. */
void oracle_hvv(int family, int n, const double *p, const double *u, const double *a, double *h)
{
    int i;
    if (family == FAM_CUBIC) {
        /* the A u and b terms are linear; (u_i + t a_i)^3 gives 6 u_i a_i^2 */
        for (i = 0; i < n; i++)
            h[i] = 6.0 * u[i] * a[i] * a[i];
    } else if (family == FAM_BRATU) {
        /* the stencil is linear; lambda exp(u_i + t a_i) gives lambda exp(u_i) a_i^2 */
        for (i = 0; i < n; i++)
            h[i] = p[0] * exp(u[i]) * a[i] * a[i];
    } else if (family == FAM_SQUARE) {
        for (i = 0; i < n; i++)
            h[i] = 2.0 * a[i] * a[i];
    } else {
        /* F_1 is linear; -10 (u_{i-1} + t a_{i-1})^2 gives -20 a_{i-1}^2 */
        h[0] = 0.0;
        for (i = 1; i < n; i++)
            h[i] = -20.0 * a[i - 1] * a[i - 1];
    }
}

/* ---------------------------------------------------------------- dense LU */

/* In-place LU with partial pivoting: P A = L U, L unit lower (below the
 * diagonal), U upper.  piv[k] = row swapped with row k at step k.
 * Returns 0, or k+1 if the k-th pivot is zero or not finite. */
int oracle_lu_factor(int n, double *A, int *piv)
{
    int i, j, k;
    for (k = 0; k < n; k++) {
        int p = k;
        double best = fabs(A[k * n + k]);
        for (i = k + 1; i < n; i++) {
            double v = fabs(A[i * n + k]);
            if (v > best) { best = v; p = i; }
        }
        piv[k] = p;
        if (!(A[p * n + k] != 0.0) || !isfinite(A[p * n + k]))
            return k + 1;
        if (p != k) {
            for (j = 0; j < n; j++) {
                double t = A[k * n + j];
                A[k * n + j] = A[p * n + j];
                A[p * n + j] = t;
            }
        }
        for (i = k + 1; i < n; i++) {
            double l = A[i * n + k] / A[k * n + k];
            A[i * n + k] = l;
            for (j = k + 1; j < n; j++)
                A[i * n + j] -= l * A[k * n + j];
        }
    }
    return 0;
}

/* Solve A x = rhs from the factors (x may alias rhs). */
void oracle_lu_solve(int n, const double *LU, const int *piv, const double *rhs, double *x)
{
    int i, j, k;
    if (x != rhs)
        memcpy(x, rhs, sizeof(double) * (size_t)n);
    for (k = 0; k < n; k++) {
        if (piv[k] != k) {
            double t = x[k];
            x[k] = x[piv[k]];
            x[piv[k]] = t;
        }
    }
    for (i = 0; i < n; i++)
        for (j = 0; j < i; j++)
            x[i] -= LU[i * n + j] * x[j];
    for (i = n - 1; i >= 0; i--) {
        for (j = i + 1; j < n; j++)
            x[i] -= LU[i * n + j] * x[j];
        x[i] /= LU[i * n + i];
    }
}

/* ---------------------------------------------------------------- helpers */

static double norm_inf(int n, const double *v)
{
    double m = 0.0;
    int i;
    for (i = 0; i < n; i++)
        if (fabs(v[i]) > m) m = fabs(v[i]);
    return m;
}

static double dot(int n, const double *a, const double *b)
{
    double s = 0.0;
    int i;
    for (i = 0; i < n; i++)
        s += a[i] * b[i];
    return s;
}

static int all_finite(int n, const double *v)
{
    int i;
    for (i = 0; i < n; i++)
        if (!isfinite(v[i])) return 0;
    return 1;
}

static void matvec(int n, const double *J, const double *x, double *y)
{
    int i, j;
    for (i = 0; i < n; i++) {
        double s = 0.0;
        for (j = 0; j < n; j++)
            s += J[i * n + j] * x[j];
        y[i] = s;
    }
}

/* ---------------------------------------------------------------- dogleg */

/* Powell's dogleg step (Sec. 2.2.2) for the model
 *   m(d) = 1/2 ||F||^2 + d^T J^T F + 1/2 d^T J^T J d,   ||d||_2 <= Delta.
 * dN is the Newton step -J^{-1} F.  Writes the step to d and returns the
 * branch: 0 = full Newton step, 1 = steepest-descent direction cut at the
 * boundary, 2 = interpolation between the Cauchy point and dN. */
int oracle_dogleg(int n, const double *J, const double *F, const double *dN, double Delta,
                  double *d)
{
    int i;
    double *g, *Jg, *c, *w;
    double gg, JgJg, cc, nd, t;
    if (sqrt(dot(n, dN, dN)) <= Delta) {
        memcpy(d, dN, sizeof(double) * (size_t)n);
        return 0;
    }
    g = malloc(sizeof(double) * 4 * (size_t)n);
    Jg = g + n;
    c = g + 2 * n;
    w = g + 3 * n;
    /* gradient of the model at d = 0: g = J^T F */
    for (i = 0; i < n; i++) {
        int r;
        double s = 0.0;
        for (r = 0; r < n; r++)
            s += J[r * n + i] * F[r];
        g[i] = s;
    }
    matvec(n, J, g, Jg);
    gg = dot(n, g, g);
    JgJg = dot(n, Jg, Jg);
    /* minimiser of the model along -g (the Cauchy point) */
    for (i = 0; i < n; i++)
        c[i] = -(gg / JgJg) * g[i];
    cc = dot(n, c, c);
    if (sqrt(cc) >= Delta) {
        /* intersection of the direction -g with the sphere of radius Delta */
        nd = sqrt(gg);
        for (i = 0; i < n; i++)
            d[i] = -(Delta / nd) * g[i];
        free(g);
        return 1;
    }
    /* (1 - tau) c + tau dN with ||.|| = Delta: the largest tau in (0, 1) */
    for (i = 0; i < n; i++)
        w[i] = dN[i] - c[i];
    {
        double a = dot(n, w, w);
        double b = dot(n, c, w);
        double q = cc - Delta * Delta;
        t = (-b + sqrt(b * b - a * q)) / a;
    }
    for (i = 0; i < n; i++)
        d[i] = (1.0 - t) * c[i] + t * dN[i];
    free(g);
    return 2;
}

/* ---------------------------------------------------------------- Broyden */

/* "Good" Broyden rank-one update of a Jacobian approximation B (row-major):
 *     B <- B + (df - B du) du^T / (du^T du),
 * the least change (Frobenius norm) that satisfies the secant condition
 * B du = df.  No change when du is zero. */
void oracle_broyden_update(int n, double *B, const double *du, const double *df)
{
    int i, j;
    double dd = dot(n, du, du);
    double *r;
    if (!(dd != 0.0)) return;
    r = malloc(sizeof(double) * (size_t)n);
    matvec(n, B, du, r);
    for (i = 0; i < n; i++)
        r[i] = df[i] - r[i];
    for (i = 0; i < n; i++)
        for (j = 0; j < n; j++)
            B[i * n + j] += r[i] * du[j] / dd;
    free(r);
}

/* ---------------------------------------------------------------- solver */

typedef struct {
    int iters, nfev, status;
    double resid;
} oracle_result;

/* Optional per-iteration record: step length (line search), dogleg branch,
 * ratio rho_k and radius (trust region), ||F||_inf after the pass. */
typedef struct {
    double *alpha;
    int *branch;
    double *rho;
    double *radius;
    double *fnorm;
    int *trials;
} oracle_trace;

/* Test-only perturbation of the steps ("jitter"), off unless a caller asks
 * for it: every component of every linear-solve result is multiplied by
 * 1 + eps or 1 - eps, the sign drawn from a SplitMix64 stream (Steele, Lea
 * & Flood 2014) keyed by (seed, instance) and advanced once per component.
 * The parity tests use it to find the instances whose outcome changes under
 * perturbations of the size of the rounding of another correct solver
 * (another operation order, FMA; FP32 for mixed precision). */
typedef struct {
    double eps;
    uint64_t state;
} oracle_jitter;

static uint64_t splitmix64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

static void jitter_step(oracle_jitter *jt, int n, double *x)
{
    int i;
    if (!jt || jt->eps == 0.0) return;
    for (i = 0; i < n; i++)
        x[i] *= (splitmix64_next(&jt->state) >> 63) ? 1.0 + jt->eps : 1.0 - jt->eps;
}

static void solve_one(int family, int n, const double *p, double *u, int alg, double abstol,
                      int maxiters, oracle_result *res, const oracle_trace *tr, oracle_jitter *jt)
{
    size_t nn = (size_t)n * (size_t)n;
    double *J = malloc(sizeof(double) * (3 * nn + 9 * (size_t)n));
    double *LU = J + nn, *B = LU + nn;
    double *F = B + nn, *dN = F + n, *ut = dN + n, *Ft = ut + n, *Jd = Ft + n, *d = Jd + n,
           *rhs = d + n, *h = rhs + n, *bv = h + n;
    int *piv = malloc(sizeof(int) * (size_t)n);
    int i, k = 0, status = ST_MAXITERS, nfev = 0, need_jac = 1, rejections = 0;
    double Delta = TR_DELTA0;

    /* initial residual and convergence test (Sec. 2.1) */
    oracle_residual(family, n, p, u, F);
    nfev++;
    if (!all_finite(n, F)) {
        status = ST_NONFINITE;
        goto done;
    }
    if (norm_inf(n, F) <= abstol) {
        status = ST_SUCCESS;
        goto done;
    }
    if (alg == ALG_BROYDEN || alg == ALG_MOD_BROYDEN) {
        /* starting approximation (Tab. 1): the identity, or the true Jacobian */
        if (alg == ALG_MOD_BROYDEN) {
            oracle_jacobian(family, n, p, u, B);
        } else {
            memset(B, 0, sizeof(double) * nn);
            for (i = 0; i < n; i++)
                B[i * n + i] = 1.0;
        }
    }
    while (k < maxiters) {
        k++;
        if (alg == ALG_BROYDEN || alg == ALG_MOD_BROYDEN) {
            /* quasi-Newton step B du = -F, full step, then the good Broyden
             * update with du and df = F(u + du) - F(u) */
            memcpy(LU, B, sizeof(double) * nn);
            if (oracle_lu_factor(n, LU, piv) != 0) {
                status = ST_SINGULAR;
                goto done;
            }
            for (i = 0; i < n; i++)
                rhs[i] = -F[i];
            oracle_lu_solve(n, LU, piv, rhs, d);
            jitter_step(jt, n, d);
            for (i = 0; i < n; i++)
                ut[i] = u[i] + d[i];
            oracle_residual(family, n, p, ut, Ft);
            nfev++;
            for (i = 0; i < n; i++)
                h[i] = Ft[i] - F[i];
            oracle_broyden_update(n, B, d, h);
            memcpy(u, ut, sizeof(double) * (size_t)n);
            memcpy(F, Ft, sizeof(double) * (size_t)n);
            if (tr) { tr->alpha[k - 1] = 1.0; tr->trials[k - 1] = 1; }
        } else if (need_jac) {
            /* J_k and the Newton direction J_k dN = -F (Eq. 2) */
            oracle_jacobian(family, n, p, u, J);
            memcpy(LU, J, sizeof(double) * nn);
            if (oracle_lu_factor(n, LU, piv) != 0) {
                status = ST_SINGULAR;
                goto done;
            }
            for (i = 0; i < n; i++)
                rhs[i] = -F[i];
            oracle_lu_solve(n, LU, piv, rhs, dN);
            jitter_step(jt, n, dN);
        }
        if (alg == ALG_BROYDEN || alg == ALG_MOD_BROYDEN) {
            /* step taken above */
        } else if (alg == ALG_NEWTON) {
            for (i = 0; i < n; i++)
                u[i] = u[i] + dN[i];
            oracle_residual(family, n, p, u, F);
            nfev++;
            if (tr) { tr->alpha[k - 1] = 1.0; tr->trials[k - 1] = 1; }
        } else if (alg == ALG_NEWTON_BACKTRACK) {
            /* phi(alpha) = 1/2 ||F(u + alpha dN)||^2 must satisfy
             * phi(alpha) <= phi(0) + c1 alpha F^T J dN   (Eq. 8-9) */
            double phi0 = 0.5 * dot(n, F, F);
            double slope, alpha = 1.0;
            int m, accepted = 0;
            matvec(n, J, dN, Jd);
            slope = dot(n, F, Jd);
            for (m = 0; m < LS_MAX_TRIALS; m++) {
                for (i = 0; i < n; i++)
                    ut[i] = u[i] + alpha * dN[i];
                oracle_residual(family, n, p, ut, Ft);
                nfev++;
                if (all_finite(n, Ft) && 0.5 * dot(n, Ft, Ft) <= phi0 + LS_C1 * alpha * slope) {
                    accepted = 1;
                    break;
                }
                alpha = alpha * LS_RHO;
            }
            if (tr) { tr->alpha[k - 1] = accepted ? alpha : 0.0; tr->trials[k - 1] = m + accepted; }
            if (!accepted) {
                status = ST_LS_FAILED;
                goto done;
            }
            memcpy(u, ut, sizeof(double) * (size_t)n);
            memcpy(F, Ft, sizeof(double) * (size_t)n);
        } else if (alg == ALG_POTRA_PTAK) {
            /* Eq. 4: y = u + dN, then J_k du2 = -f(y) with the same factors,
             * u_{k+1} = y + du2 */
            for (i = 0; i < n; i++)
                ut[i] = u[i] + dN[i];
            oracle_residual(family, n, p, ut, Ft);
            nfev++;
            for (i = 0; i < n; i++)
                rhs[i] = -Ft[i];
            oracle_lu_solve(n, LU, piv, rhs, d);
            jitter_step(jt, n, d);
            for (i = 0; i < n; i++)
                u[i] = ut[i] + d[i];
            oracle_residual(family, n, p, u, F);
            nfev++;
            if (tr) { tr->alpha[k - 1] = 1.0; tr->trials[k - 1] = 1; }
        } else if (alg == ALG_HALLEY) {
            /* Eq. 3: a = dN, J_k b = H_k a a, du = (a o a) / (a + b/2) */
            oracle_hvv(family, n, p, u, dN, h);
            oracle_lu_solve(n, LU, piv, h, bv);
            jitter_step(jt, n, bv);
            for (i = 0; i < n; i++) {
                double den = dN[i] + 0.5 * bv[i];
                d[i] = (den != 0.0) ? (dN[i] * dN[i]) / den : dN[i];
            }
            for (i = 0; i < n; i++)
                u[i] = u[i] + d[i];
            oracle_residual(family, n, p, u, F);
            nfev++;
            if (tr) { tr->alpha[k - 1] = 1.0; tr->trials[k - 1] = 1; }
        } else {
            /* trust region with the dogleg step (Eq. 13-15) */
            double fF, ared, pred, rho;
            int branch = oracle_dogleg(n, J, F, dN, Delta, d);
            for (i = 0; i < n; i++)
                ut[i] = u[i] + d[i];
            oracle_residual(family, n, p, ut, Ft);
            nfev++;
            fF = dot(n, F, F);
            matvec(n, J, d, Jd);
            for (i = 0; i < n; i++)
                Jd[i] = F[i] + Jd[i];
            ared = fF - dot(n, Ft, Ft);
            pred = fF - dot(n, Jd, Jd);
            rho = (pred > 0.0 && all_finite(n, Ft)) ? ared / pred : -INFINITY;
            if (tr) { tr->branch[k - 1] = branch; tr->rho[k - 1] = rho; tr->radius[k - 1] = Delta; }
            if (alg == ALG_TRUST_DOGLEG_NW) {
                /* Nocedal & Wright, Algorithm 4.1: shrink when rho < 1/4,
                 * grow when rho > 3/4 and the step reached the boundary,
                 * accept when rho > eta (independently of the radius) */
                int accept = rho > TR_NW_ETA;
                if (rho < 0.25) {
                    Delta = 0.25 * Delta;
                } else if (rho > 0.75 && branch != 0) {
                    Delta = 2.0 * Delta;
                    if (Delta > TR_DELTA_MAX) Delta = TR_DELTA_MAX;
                }
                if (accept) {
                    memcpy(u, ut, sizeof(double) * (size_t)n);
                    memcpy(F, Ft, sizeof(double) * (size_t)n);
                    need_jac = 1;
                    rejections = 0;
                } else {
                    need_jac = 0;
                    rejections++;
                    if (rejections >= TR_MAX_REJECTIONS) {
                        status = ST_TR_STALLED;
                        goto done;
                    }
                }
            } else if (rho > 0.0) {
                memcpy(u, ut, sizeof(double) * (size_t)n);
                memcpy(F, Ft, sizeof(double) * (size_t)n);
                need_jac = 1;
                rejections = 0;
                if (rho > TR_ETA_EXPAND) {
                    Delta = TR_GROW * Delta;
                    if (Delta > TR_DELTA_MAX) Delta = TR_DELTA_MAX;
                }
            } else {
                Delta = TR_SHRINK * Delta;
                need_jac = 0;
                rejections++;
                if (rejections >= TR_MAX_REJECTIONS) {
                    status = ST_TR_STALLED;
                    goto done;
                }
            }
        }
        if (tr) tr->fnorm[k - 1] = norm_inf(n, F);
        if (!all_finite(n, F)) {
            status = ST_NONFINITE;
            goto done;
        }
        if (norm_inf(n, F) <= abstol) {
            status = ST_SUCCESS;
            goto done;
        }
    }
done:
    oracle_residual(family, n, p, u, F);
    res->resid = norm_inf(n, F);
    if (!all_finite(n, F)) res->resid = NAN;
    res->iters = k;
    res->nfev = nfev;
    res->status = status;
    free(piv);
    free(J);
}

/* Solve one instance, recording per-iteration data (arrays of maxiters). */
int oracle_solve_trace(int family, int n, const double *p, double *u, int alg, double abstol,
                       int maxiters, int *iters, double *resid, int *nfev, double *alpha,
                       int *trials, int *branch, double *rho, double *radius, double *fnorm)
{
    oracle_result r;
    oracle_trace t = {alpha, branch, rho, radius, fnorm, trials};
    solve_one(family, n, p, u, alg, abstol, maxiters, &r, &t, 0);
    *iters = r.iters;
    *resid = r.resid;
    *nfev = r.nfev;
    return r.status;
}

void oracle_solve_range_jitter(int family, int n, long k0, long k1, const double *params,
                               double *u, int alg, double abstol, int maxiters, int *status,
                               int *iters, double *resid, int *nfev, double eps, uint64_t seed);

/* Solve instances [k0, k1) of a batch stored instance-major:
 * params[k*E + e] (E = oracle_n_params) and u[k*n + i] (in/out). */
void oracle_solve_range(int family, int n, long k0, long k1, const double *params, double *u,
                        int alg, double abstol, int maxiters, int *status, int *iters,
                        double *resid, int *nfev)
{
    oracle_solve_range_jitter(family, n, k0, k1, params, u, alg, abstol, maxiters, status, iters,
                              resid, nfev, 0.0, 0);
}

/* As oracle_solve_range, with the steps of instance k perturbed by the
 * relative size eps (test infrastructure, see oracle_jitter); the sign
 * stream of instance k depends on (seed, k) only. */
void oracle_solve_range_jitter(int family, int n, long k0, long k1, const double *params,
                               double *u, int alg, double abstol, int maxiters, int *status,
                               int *iters, double *resid, int *nfev, double eps, uint64_t seed)
{
    long k;
    int E = oracle_n_params(family, n);
    for (k = k0; k < k1; k++) {
        oracle_result r;
        oracle_jitter jt;
        uint64_t key = seed;
        jt.eps = eps;
        jt.state = splitmix64_next(&key) ^ (uint64_t)k;
        solve_one(family, n, params + (size_t)k * (size_t)E, u + (size_t)k * (size_t)n, alg,
                  abstol, maxiters, &r, 0, &jt);
        status[k] = r.status;
        iters[k] = r.iters;
        resid[k] = r.resid;
        nfev[k] = r.nfev;
    }
}

/* Extra plain Newton steps from u while ||F||_inf keeps decreasing (at most
 * maxsteps); returns the final ||F||_inf.  Used to obtain a root accurate to
 * the rounding floor, against which solver outputs are compared. */
double oracle_polish(int family, int n, const double *p, double *u, int maxsteps)
{
    size_t nn = (size_t)n * (size_t)n;
    double *LU = malloc(sizeof(double) * (nn + 4 * (size_t)n));
    double *F = LU + nn, *d = F + n, *ut = d + n, *Ft = ut + n;
    int *piv = malloc(sizeof(int) * (size_t)n);
    int i, s;
    double fn;
    oracle_residual(family, n, p, u, F);
    fn = norm_inf(n, F);
    for (s = 0; s < maxsteps && isfinite(fn) && fn > 0.0; s++) {
        oracle_jacobian(family, n, p, u, LU);
        if (oracle_lu_factor(n, LU, piv) != 0) break;
        for (i = 0; i < n; i++)
            d[i] = -F[i];
        oracle_lu_solve(n, LU, piv, d, d);
        for (i = 0; i < n; i++)
            ut[i] = u[i] + d[i];
        oracle_residual(family, n, p, ut, Ft);
        if (!(norm_inf(n, Ft) < fn)) break;
        memcpy(u, ut, sizeof(double) * (size_t)n);
        memcpy(F, Ft, sizeof(double) * (size_t)n);
        fn = norm_inf(n, Ft);
    }
    free(piv);
    free(LU);
    return fn;
}

/* ---------------------------------------------------------------- sensitivity */

/* Adjoint sensitivity at a root u (Sec. 2.3, implicit function theorem):
 * with J = dF/du at u, du/dtheta = -J^{-1} dF/dtheta (the sign the printed
 * formula drops), so for a cotangent w = dL/du,
 *     dL/dtheta = -mu^T dF/dtheta,   J^T mu = w.
 * grad receives dL/dtheta in the family's parameter order (E values).
 * Returns 0, or 1 if J is singular. */
int oracle_adjoint(int family, int n, const double *p, const double *u, const double *w,
                   double *grad)
{
    size_t nn = (size_t)n * (size_t)n;
    double *J = malloc(sizeof(double) * (2 * nn + (size_t)n));
    double *Jt = J + nn, *mu = Jt + nn;
    int *piv = malloc(sizeof(int) * (size_t)n);
    int i, j, rc = 0;
    oracle_jacobian(family, n, p, u, J);
    for (i = 0; i < n; i++)
        for (j = 0; j < n; j++)
            Jt[i * n + j] = J[j * n + i];
    if (oracle_lu_factor(n, Jt, piv) != 0) {
        rc = 1;
        goto done;
    }
    oracle_lu_solve(n, Jt, piv, w, mu);
    if (family == FAM_CUBIC) {
        /* dF_i/dA_ij = u_j, dF_i/db_i = -1 */
        for (i = 0; i < n; i++) {
            for (j = 0; j < n; j++)
                grad[i * n + j] = -mu[i] * u[j];
            grad[n * n + i] = mu[i];
        }
    } else if (family == FAM_BRATU) {
        /* dF_i/dlambda = exp(u_i) */
        double s = 0.0;
        for (i = 0; i < n; i++)
            s += mu[i] * exp(u[i]);
        grad[0] = -s;
    } else if (family == FAM_SQUARE) {
        /* dF_i/dp_i = -1 */
        for (i = 0; i < n; i++)
            grad[i] = mu[i];
    }
done:
    free(piv);
    free(J);
    return rc;
}
