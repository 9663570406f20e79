/*
 * CPU ORACLE for the two-stage streaming NMF of Gu, Du & Billinge,
 * "A fast two-stage algorithm for non-negative matrix factorization in
 * streaming data" (arXiv 2101.08431).
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the CUDA library, and the library never calls
 * it.  Everything is plain FP64 C with triple loops, no blocking, no BLAS and
 * no threads, so that each function can be checked against the paper by eye.
 *
 * Conventions (Sec. 3.1, after eq. "eqn:kkt"):
 *   M  n x m, column-major with leading dimension ldm (M[i + ldm*j]);
 *   X  n x k, row-major (X[i*k + a])      -> this is x = vec(X^T);
 *   Y  k x m, column-major (Y[a + k*j])   -> this is y = vec(Y);
 *   R  (dual of X) stored like X, S (dual of Y) stored like Y.
 *
 * Readings of points the paper leaves open (each is also used, identically,
 * by the CUDA path, but implemented separately there):
 *   - NNLS entering tolerance: w_i > tol with
 *       tol = 10 * k * eps64 * (max|b| + max_i G_ii * max|y|);
 *   - Lawson-Hanson ties: the lowest index enters / leaves first;
 *   - Cholesky pivot <= 1e-14 * max_i G_ii: that variable is blocked (held at
 *     zero) for the rest of the solve;
 *   - an entering variable whose first least-squares value is <= 0 is
 *     blocked for the rest of the solve (cannot happen in exact arithmetic);
 *   - outer-iteration cap 5k + 10, after which the solve reports NOTCONV.
 *
 * Status codes match nothing on purpose: 0 ok, 1 bad argument,
 * 4 not converged, 6 non-finite number, 7 linear system not positive definite.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL 1
#define OR_NOTCONV 4
#define OR_ENUMERIC 6
#define OR_NOTPD 7

#define KMAX 32

static const double EPS64 = 2.220446049250313e-16;

/* ------------------------------------------------------------------------ */
/* NNLS: min_y 1/2 y^T G y - b^T y  s.t. y >= 0                             */
/* Problem "qp" (Sec. 2): with C = X and d = M_{:,j}, G = X^T X, b = X^T d; */
/* with C = Y^T and d = M_{i,:}^T, G = Y Y^T, b = Y d.                      */
/* Solved by the active-set method of Lawson and Hanson cited in Sec. 2,    */
/* started cold (empty passive set).                                        */
/* ------------------------------------------------------------------------ */

/* Solve G_PP z_P = b_P by Cholesky, the indices of P taken in ascending
 * order; z is zero outside P.  Returns -1 on success or the index whose pivot
 * fell below the threshold. */
static int chol_solve_subset(int k, const double *G, const double *b,
                             uint32_t P, double pivot_min, double *z)
{
    int idx[KMAX], p = 0;
    double L[KMAX][KMAX], v[KMAX];
    for (int i = 0; i < k; ++i)
        if (P & (1u << i)) idx[p++] = i;
    for (int c = 0; c < p; ++c) {
        double s = G[idx[c] * k + idx[c]];
        for (int l = 0; l < c; ++l) s -= L[c][l] * L[c][l];
        if (!(s > pivot_min)) return idx[c];
        L[c][c] = sqrt(s);
        for (int r = c + 1; r < p; ++r) {
            double t = G[idx[r] * k + idx[c]];
            for (int l = 0; l < c; ++l) t -= L[r][l] * L[c][l];
            L[r][c] = t / L[c][c];
        }
    }
    for (int c = 0; c < p; ++c) {           /* L v = b_P */
        double t = b[idx[c]];
        for (int l = 0; l < c; ++l) t -= L[c][l] * v[l];
        v[c] = t / L[c][c];
    }
    for (int i = 0; i < k; ++i) z[i] = 0.0;
    for (int c = p - 1; c >= 0; --c) {      /* L^T z_P = v */
        double t = v[c];
        for (int l = c + 1; l < p; ++l) t -= L[l][c] * z[idx[l]];
        z[idx[c]] = t / L[c][c];
    }
    return -1;
}

int oracle_nnls(int k, const double *G, const double *b, double *y,
                uint32_t *mask_out, int *outer_out)
{
    if (k < 1 || k > KMAX) return OR_EINVAL;
    double gmax = 0.0;
    for (int i = 0; i < k; ++i) {
        if (!isfinite(b[i])) return OR_ENUMERIC;
        if (G[i * k + i] > gmax) gmax = G[i * k + i];
    }
    const double pivot_min = 1e-14 * gmax;
    uint32_t P = 0, blocked = 0;
    double w[KMAX], z[KMAX];
    for (int i = 0; i < k; ++i) y[i] = 0.0;
    int status = OR_NOTCONV, outer;
    const int cap = 5 * k + 10;
    for (outer = 0; outer < cap; ++outer) {
        /* w = b - G y (the negative gradient) and the entering test */
        double bmax = 0.0, ymax = 0.0;
        for (int i = 0; i < k; ++i) {
            double t = b[i];
            for (int l = 0; l < k; ++l) t -= G[i * k + l] * y[l];
            w[i] = t;
            if (fabs(b[i]) > bmax) bmax = fabs(b[i]);
            if (y[i] > ymax) ymax = y[i];
        }
        const double tol = 10.0 * k * EPS64 * (bmax + gmax * ymax);
        int t_in = -1;
        double best = tol;
        for (int i = 0; i < k; ++i) {
            uint32_t bit = 1u << i;
            if ((P & bit) || (blocked & bit)) continue;
            if (w[i] > best) { best = w[i]; t_in = i; }
        }
        if (t_in < 0) { status = OR_OK; break; }
        P |= 1u << t_in;
        int first = 1;
        for (int inner = 0; inner <= k + 1; ++inner) {
            int f = chol_solve_subset(k, G, b, P, pivot_min, z);
            if (f >= 0) {                      /* singular direction: block it */
                P &= ~(1u << f);
                blocked |= 1u << f;
                y[f] = 0.0;
                first = 0;
                if (!P) break;
                continue;
            }
            if (first && !(z[t_in] > 0.0)) {   /* degenerate entering variable */
                P &= ~(1u << t_in);
                blocked |= 1u << t_in;
                break;
            }
            first = 0;
            int feasible = 1;
            for (int i = 0; i < k; ++i)
                if ((P & (1u << i)) && !(z[i] > 0.0)) feasible = 0;
            if (feasible) {
                for (int i = 0; i < k; ++i) y[i] = (P & (1u << i)) ? z[i] : 0.0;
                break;
            }
            /* step from y towards z until the first passive variable hits 0 */
            double alpha = 2.0;
            int q = -1;
            for (int i = 0; i < k; ++i) {
                if (!(P & (1u << i)) || z[i] > 0.0) continue;
                double a = y[i] / (y[i] - z[i]);
                if (a < alpha) { alpha = a; q = i; }
            }
            for (int i = 0; i < k; ++i)
                if (P & (1u << i)) y[i] += alpha * (z[i] - y[i]);
            y[q] = 0.0;
            P &= ~(1u << q);
            for (int i = 0; i < k; ++i)
                if ((P & (1u << i)) && !(y[i] > 0.0)) { y[i] = 0.0; P &= ~(1u << i); }
            if (!P) break;
        }
    }
    uint32_t mask = 0;
    for (int i = 0; i < k; ++i)
        if (y[i] > 0.0) mask |= 1u << i;
    if (mask_out) *mask_out = mask;
    if (outer_out) *outer_out = outer;
    return status;
}

/* Warm-started Lawson-Hanson (Sec. 2: the solution of the previous problem
 * seeds the next one, e.g. column j - 1 for column j).  y holds the warm start
 * on entry (y >= 0; its support is the initial passive set) and the solution
 * on exit.  The method is the cold-start solver's from a feasible point: the
 * inner loop first steps from y towards the least-squares solution on the
 * warm passive set, dropping variables that reach zero, then the outer loop
 * adds entering variables as before (same tolerance, ties, blocking and cap).
 * *outer_out: entering steps taken; *changes_out: variables that entered or
 * left the passive set.  The solution is unique (G positive definite), so it
 * agrees with the cold solve up to rounding; only the work differs. */
int oracle_nnls_warm(int k, const double *G, const double *b, double *y,
                     uint32_t *mask_out, int *outer_out, int *changes_out)
{
    if (k < 1 || k > KMAX) return OR_EINVAL;
    double gmax = 0.0;
    for (int i = 0; i < k; ++i) {
        if (!isfinite(b[i])) return OR_ENUMERIC;
        if (G[i * k + i] > gmax) gmax = G[i * k + i];
    }
    const double pivot_min = 1e-14 * gmax;
    uint32_t P = 0, blocked = 0;
    int changes = 0;
    for (int i = 0; i < k; ++i) {
        if (y[i] > 0.0) P |= 1u << i;
        else y[i] = 0.0;
    }
    double w[KMAX], z[KMAX];
    int status = OR_NOTCONV, outer = 0;
    const int cap = 5 * k + 10;
    int t_in = -1;                  /* no entering variable on the first pass */
    for (;;) {
        /* inner loop from the feasible y on P (t_in: the variable that just entered) */
        int first = t_in >= 0;
        for (int inner = 0; P && inner <= k + 1; ++inner) {
            int f = chol_solve_subset(k, G, b, P, pivot_min, z);
            if (f >= 0) {
                P &= ~(1u << f);
                blocked |= 1u << f;
                y[f] = 0.0;
                ++changes;
                first = 0;
                continue;
            }
            if (first && !(z[t_in] > 0.0)) {
                P &= ~(1u << t_in);
                blocked |= 1u << t_in;
                ++changes;
                break;
            }
            first = 0;
            int feasible = 1;
            for (int i = 0; i < k; ++i)
                if ((P & (1u << i)) && !(z[i] > 0.0)) feasible = 0;
            if (feasible) {
                for (int i = 0; i < k; ++i) y[i] = (P & (1u << i)) ? z[i] : 0.0;
                break;
            }
            double alpha = 2.0;
            int q = -1;
            for (int i = 0; i < k; ++i) {
                if (!(P & (1u << i)) || z[i] > 0.0) continue;
                double a = y[i] / (y[i] - z[i]);
                if (a < alpha) { alpha = a; q = i; }
            }
            for (int i = 0; i < k; ++i)
                if (P & (1u << i)) y[i] += alpha * (z[i] - y[i]);
            y[q] = 0.0;
            P &= ~(1u << q);
            ++changes;
            for (int i = 0; i < k; ++i)
                if ((P & (1u << i)) && !(y[i] > 0.0)) { y[i] = 0.0; P &= ~(1u << i); ++changes; }
        }
        if (!P)
            for (int i = 0; i < k; ++i) y[i] = 0.0;
        if (outer >= cap) break;
        /* outer step: w = b - G y and the entering test */
        double bmax = 0.0, ymax = 0.0;
        for (int i = 0; i < k; ++i) {
            double s = b[i];
            for (int l = 0; l < k; ++l) s -= G[i * k + l] * y[l];
            w[i] = s;
            if (fabs(b[i]) > bmax) bmax = fabs(b[i]);
            if (y[i] > ymax) ymax = y[i];
        }
        const double tol = 10.0 * k * EPS64 * (bmax + gmax * ymax);
        t_in = -1;
        double best = tol;
        for (int i = 0; i < k; ++i) {
            uint32_t bit = 1u << i;
            if ((P & bit) || (blocked & bit)) continue;
            if (w[i] > best) { best = w[i]; t_in = i; }
        }
        if (t_in < 0) { status = OR_OK; break; }
        P |= 1u << t_in;
        ++changes;
        ++outer;
    }
    uint32_t mask = 0;
    for (int i = 0; i < k; ++i)
        if (y[i] > 0.0) mask |= 1u << i;
    if (mask_out) *mask_out = mask;
    if (outer_out) *outer_out = outer;
    if (changes_out) *changes_out = changes;
    return status;
}

/* ------------------------------------------------------------------------ */
/* One ANLS sweep (Alg. "anls", Sec. 2), Y-update first, then X-update:     */
/*   Y_{:,j} = argmin_{y>=0} 1/2 ||X y - M_{:,j}||^2   for every column j;  */
/*   X_{i,:} = argmin_{x>=0} 1/2 ||Y^T x - M_{i,:}^T||^2  for every row i.  */
/* Products are formed straight from M, never from cached Grams.            */
/* ------------------------------------------------------------------------ */
int oracle_sweep(int64_t n, int64_t m, int k, const double *M, int64_t ldm,
                 double *X, double *Y, uint32_t *xmask, uint32_t *ymask,
                 int64_t *notconv_out)
{
    if (n < 1 || m < 1 || k < 1 || k > KMAX || ldm < n) return OR_EINVAL;
    double G[KMAX * KMAX];
    int64_t notconv = 0;
    int bad = OR_OK;
    /* G = X^T X */
    for (int a = 0; a < k; ++a)
        for (int c = 0; c < k; ++c) {
            double s = 0.0;
            for (int64_t i = 0; i < n; ++i) s += X[i * k + a] * X[i * k + c];
            G[a * k + c] = s;
        }
    /* The columns are independent problems (and so are the rows below): a
     * build with -fopenmp shares them among threads, each column computed
     * exactly as in the serial build; the default build ignores the pragma. */
    #pragma omp parallel for schedule(dynamic, 16) reduction(+ : notconv)
    for (int64_t j = 0; j < m; ++j) {
        double b[KMAX];
        for (int a = 0; a < k; ++a) {        /* b = X^T M_{:,j} */
            double s = 0.0;
            for (int64_t i = 0; i < n; ++i) s += X[i * k + a] * M[i + ldm * j];
            b[a] = s;
        }
        const int st = oracle_nnls(k, G, b, Y + k * j, ymask ? ymask + j : NULL, NULL);
        if (st == OR_NOTCONV) ++notconv;
        else if (st != OR_OK) {
            #pragma omp critical
            bad = st;
        }
    }
    if (bad != OR_OK) return bad;
    /* H = Y Y^T */
    double H[KMAX * KMAX];
    for (int a = 0; a < k; ++a)
        for (int c = 0; c < k; ++c) {
            double s = 0.0;
            for (int64_t j = 0; j < m; ++j) s += Y[a + k * j] * Y[c + k * j];
            H[a * k + c] = s;
        }
    #pragma omp parallel for schedule(dynamic, 16) reduction(+ : notconv)
    for (int64_t i = 0; i < n; ++i) {
        double b[KMAX];
        for (int a = 0; a < k; ++a) {        /* b = (M Y^T)_{i,:} */
            double s = 0.0;
            for (int64_t j = 0; j < m; ++j) s += M[i + ldm * j] * Y[a + k * j];
            b[a] = s;
        }
        const int st = oracle_nnls(k, H, b, X + i * k, xmask ? xmask + i : NULL, NULL);
        if (st == OR_NOTCONV) ++notconv;
        else if (st != OR_OK) {
            #pragma omp critical
            bad = st;
        }
    }
    if (bad != OR_OK) return bad;
    if (notconv_out) *notconv_out = notconv;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Objective of problem "prob" and the gradients of eq. "eqn:kkt":          */
/*   f = 1/2 ||XY - M||_F^2 from the residual itself;                        */
/*   graX = (XY - M) Y^T  (n x k, stored like X),                            */
/*   graY = X^T (XY - M)  (k x m, stored like Y).                            */
/* Either gradient pointer may be NULL.                                      */
/* ------------------------------------------------------------------------ */
double oracle_grad(int64_t n, int64_t m, int k, const double *M, int64_t ldm,
                   const double *X, const double *Y, double *graX, double *graY)
{
    double f = 0.0;
    if (graX) for (int64_t t = 0; t < n * k; ++t) graX[t] = 0.0;
    if (graY) for (int64_t t = 0; t < m * k; ++t) graY[t] = 0.0;
    for (int64_t j = 0; j < m; ++j)
        for (int64_t i = 0; i < n; ++i) {
            double res = -M[i + ldm * j];
            for (int a = 0; a < k; ++a) res += X[i * k + a] * Y[a + k * j];
            f += 0.5 * res * res;
            for (int a = 0; a < k; ++a) {
                if (graX) graX[i * k + a] += res * Y[a + k * j];
                if (graY) graY[a + k * j] += X[i * k + a] * res;
            }
        }
    return f;
}

double oracle_objective(int64_t n, int64_t m, int k, const double *M, int64_t ldm,
                        const double *X, const double *Y)
{
    return oracle_grad(n, m, k, M, ldm, X, Y, NULL, NULL);
}

/* KKT violation of an ANLS point (Sec. 5.1): with r = max(graX, 0) and
 * s = max(graY, 0), the error E(x, y, r, s; 0) of eq. "error" (2-norms) is
 *   E = max{ ||(min(graX,0), min(graY,0))||, ||(r o X, s o Y)|| }.
 * The relative figure divides the first term by s_g = ||M Y^T||_F + ||X^T M||_F
 * and the second by s_g * max(max X, max Y).
 * out[0] = E_abs, out[1] = relative KKT, out[2] = gradient-sign term,
 * out[3] = complementarity term, out[4] = s_g, out[5] = max(max X, max Y),
 * out[6] = f. */
int oracle_kkt(int64_t n, int64_t m, int k, const double *M, int64_t ldm,
               const double *X, const double *Y, double *out)
{
    if (n < 1 || m < 1 || k < 1 || k > KMAX || ldm < n) return OR_EINVAL;
    double *gX = (double *)malloc(sizeof(double) * n * k);
    double *gY = (double *)malloc(sizeof(double) * m * k);
    if (!gX || !gY) { free(gX); free(gY); return OR_EINVAL; }
    double f = oracle_grad(n, m, k, M, ldm, X, Y, gX, gY);
    double neg = 0.0, comp = 0.0, xymax = 0.0, pn = 0.0, bn = 0.0;
    for (int64_t t = 0; t < n * k; ++t) {
        double g = gX[t], r = g > 0.0 ? g : 0.0, mn = g < 0.0 ? g : 0.0;
        neg += mn * mn;
        comp += (r * X[t]) * (r * X[t]);
        if (X[t] > xymax) xymax = X[t];
    }
    for (int64_t t = 0; t < m * k; ++t) {
        double g = gY[t], s = g > 0.0 ? g : 0.0, mn = g < 0.0 ? g : 0.0;
        neg += mn * mn;
        comp += (s * Y[t]) * (s * Y[t]);
        if (Y[t] > xymax) xymax = Y[t];
    }
    /* ||M Y^T||_F and ||X^T M||_F straight from M */
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < k; ++a) {
            double s = 0.0;
            for (int64_t j = 0; j < m; ++j) s += M[i + ldm * j] * Y[a + k * j];
            pn += s * s;
        }
    for (int64_t j = 0; j < m; ++j)
        for (int a = 0; a < k; ++a) {
            double s = 0.0;
            for (int64_t i = 0; i < n; ++i) s += X[i * k + a] * M[i + ldm * j];
            bn += s * s;
        }
    double sg = sqrt(pn) + sqrt(bn);
    double e1 = sqrt(neg), e2 = sqrt(comp);
    out[0] = e1 > e2 ? e1 : e2;
    double r1 = sg > 0.0 ? e1 / sg : e1;
    double den2 = sg * xymax;
    double r2 = den2 > 0.0 ? e2 / den2 : e2;
    out[1] = r1 > r2 ? r1 : r2;
    out[2] = e1;
    out[3] = e2;
    out[4] = sg;
    out[5] = xymax;
    out[6] = f;
    free(gX);
    free(gY);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Stage 1 driver: ANLS sweeps until the relative step test of Sec. 4,      */
/*   ||(x_k,y_k) - (x_{k+1},y_{k+1})|| <= eps_STOL (1 + ||(x_k,y_k)||),     */
/* or until the relative KKT of the current point is <= kkt_target (a value */
/* <= 0 disables that test), or max_sweeps.  trace (may be NULL) receives   */
/* 4 numbers per evaluated point: f, E_abs, rel KKT, relative step.         */
/* ------------------------------------------------------------------------ */
int oracle_anls(int64_t n, int64_t m, int k, const double *M, int64_t ldm,
                double *X, double *Y, uint32_t *xmask, uint32_t *ymask,
                int max_sweeps, double stol, double kkt_target,
                double *trace, int *sweeps_out)
{
    if (n < 1 || m < 1 || k < 1 || k > KMAX || ldm < n) return OR_EINVAL;
    double *X0 = (double *)malloc(sizeof(double) * n * k);
    double *Y0 = (double *)malloc(sizeof(double) * m * k);
    if (!X0 || !Y0) { free(X0); free(Y0); return OR_EINVAL; }
    int t, st = OR_OK, evaluated = 0;
    double kk[7];
    for (t = 0; t < max_sweeps; ++t) {
        evaluated = 0;
        if (kkt_target > 0.0 || trace) {
            evaluated = 1;
            oracle_kkt(n, m, k, M, ldm, X, Y, kk);
            if (trace) {
                trace[4 * t + 0] = kk[6];
                trace[4 * t + 1] = kk[0];
                trace[4 * t + 2] = kk[1];
                trace[4 * t + 3] = 0.0;
            }
            if (kkt_target > 0.0 && kk[1] <= kkt_target) break;
        }
        evaluated = 0;
        memcpy(X0, X, sizeof(double) * n * k);
        memcpy(Y0, Y, sizeof(double) * m * k);
        int64_t nc = 0;
        st = oracle_sweep(n, m, k, M, ldm, X, Y, xmask, ymask, &nc);
        if (st != OR_OK) break;
        double d = 0.0, nx = 0.0;
        for (int64_t q = 0; q < n * k; ++q) {
            d += (X[q] - X0[q]) * (X[q] - X0[q]);
            nx += X0[q] * X0[q];
        }
        for (int64_t q = 0; q < m * k; ++q) {
            d += (Y[q] - Y0[q]) * (Y[q] - Y0[q]);
            nx += Y0[q] * Y0[q];
        }
        double step_rel = sqrt(d) / (1.0 + sqrt(nx));
        if (trace) trace[4 * t + 3] = step_rel;
        if (stol > 0.0 && step_rel <= stol) { ++t; break; }
    }
    if (st == OR_OK && trace && !evaluated) {   /* evaluate the last point too */
        oracle_kkt(n, m, k, M, ldm, X, Y, kk);
        trace[4 * t + 0] = kk[6];
        trace[4 * t + 1] = kk[0];
        trace[4 * t + 2] = kk[1];
        trace[4 * t + 3] = 0.0;
    }
    if (sweeps_out) *sweeps_out = t;
    free(X0);
    free(Y0);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Stage 2: the line-search interior point method (Alg. "alg:int" inside    */
/* Alg. "alg:fast", Sec. 3-4).                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n, m;
    int k;
    const double *M;
    int64_t ldm;
} prob_t;

/* E(x, y, r, s; mu) of eq. "error", 2-norms. */
static double ipm_error(const prob_t *p, const double *x, const double *y,
                        const double *r, const double *s, double mu,
                        const double *gX, const double *gY)
{
    int64_t nk = p->n * p->k, mk = p->m * p->k;
    double a = 0.0, c = 0.0;
    for (int64_t t = 0; t < nk; ++t) {
        a += (gX[t] - r[t]) * (gX[t] - r[t]);
        c += (r[t] * x[t] - mu) * (r[t] * x[t] - mu);
    }
    for (int64_t t = 0; t < mk; ++t) {
        a += (gY[t] - s[t]) * (gY[t] - s[t]);
        c += (s[t] * y[t] - mu) * (s[t] * y[t] - mu);
    }
    a = sqrt(a);
    c = sqrt(c);
    return a > c ? a : c;
}

/* Barrier merit function phi(x, y) of Sec. 3.1; +inf outside x, y > 0. */
static double ipm_phi(const prob_t *p, const double *x, const double *y, double mu)
{
    int64_t nk = p->n * p->k, mk = p->m * p->k;
    double lg = 0.0;
    for (int64_t t = 0; t < nk; ++t) {
        if (!(x[t] > 0.0)) return INFINITY;
        lg += log(x[t]);
    }
    for (int64_t t = 0; t < mk; ++t) {
        if (!(y[t] > 0.0)) return INFINITY;
        lg += log(y[t]);
    }
    return oracle_objective(p->n, p->m, p->k, p->M, p->ldm, x, y) - mu * lg;
}

/* In-place dense Cholesky of an N x N row-major SPD matrix (lower factor). */
static int dense_chol(int64_t N, double *A)
{
    for (int64_t c = 0; c < N; ++c) {
        double s = A[c * N + c];
        for (int64_t l = 0; l < c; ++l) s -= A[c * N + l] * A[c * N + l];
        if (!(s > 0.0) || !isfinite(s)) return OR_NOTPD;
        double d = sqrt(s);
        A[c * N + c] = d;
        for (int64_t r = c + 1; r < N; ++r) {
            double t = A[r * N + c];
            for (int64_t l = 0; l < c; ++l) t -= A[r * N + l] * A[c * N + l];
            A[r * N + c] = t / d;
        }
    }
    return OR_OK;
}

/* Primal-dual direction of eq. "eqn:equation": the reduced system eq. "eqn:p"
 *   [R1  Cb^T; Cb  R2] [dx; dy] = -grad phi
 * with R1 = blkdiag_n(Y Y^T) + rho I + Diag(x)^-1 Diag(r) and
 *      R2 = blkdiag_m(X^T X) + rho I + Diag(y)^-1 Diag(s),
 * solved as in Sec. 3.2 (eqs. "eqn:step", "eqn:step2"): Cholesky R1 = P^T P
 * block by block, W = Cb P^-1, Schur matrix R2 - W W^T (mk x mk, Cholesky),
 * then dx from the back substitution; finally dr, ds from the last two block
 * rows of eq. "eqn:equation".  Cb holds the Gauss-Newton blocks X_i^T Y_j^T
 * when full == 0 and, when full == 1, the blocks of C (plus the residual
 * (X_i Y_j - M_ij) I).  gX, gY are the gradients at (x, y).
 * Returns OR_NOTPD when a Cholesky factorisation fails. */
int oracle_ipm_direction(int64_t n, int64_t m, int k, const double *M, int64_t ldm,
                         const double *x, const double *y, const double *r,
                         const double *s, double mu, double rho, int full,
                         double *dx, double *dy, double *dr, double *ds)
{
    const int64_t nk = n * k, mk = m * k;
    double *gX = (double *)malloc(sizeof(double) * nk);
    double *gY = (double *)malloc(sizeof(double) * mk);
    double *L1 = (double *)malloc(sizeof(double) * n * k * k);   /* blocks of P^T */
    double *W = (double *)malloc(sizeof(double) * mk * nk);      /* Cb P^-1 */
    double *S = (double *)malloc(sizeof(double) * mk * mk);
    double *u = (double *)malloc(sizeof(double) * nk);
    double *rhs = (double *)malloc(sizeof(double) * mk);
    int st = OR_OK;
    if (!gX || !gY || !L1 || !W || !S || !u || !rhs) { st = OR_EINVAL; goto done; }
    oracle_grad(n, m, k, M, ldm, x, y, gX, gY);
    double YY[KMAX * KMAX], XX[KMAX * KMAX];
    for (int a = 0; a < k; ++a)
        for (int c = 0; c < k; ++c) {
            double t1 = 0.0, t2 = 0.0;
            for (int64_t j = 0; j < m; ++j) t1 += y[a + k * j] * y[c + k * j];
            for (int64_t i = 0; i < n; ++i) t2 += x[i * k + a] * x[i * k + c];
            YY[a * k + c] = t1;
            XX[a * k + c] = t2;
        }
    /* R1 blocks and their Cholesky factors L_i (R1_i = L_i L_i^T, P_i = L_i^T) */
    for (int64_t i = 0; i < n; ++i) {
        double *Li = L1 + i * k * k;
        for (int a = 0; a < k; ++a)
            for (int c = 0; c < k; ++c)
                Li[a * k + c] = YY[a * k + c] + (a == c ? rho + r[i * k + a] / x[i * k + a] : 0.0);
        if (dense_chol(k, Li) != OR_OK) { st = OR_NOTPD; goto done; }
    }
    /* b1 = -grad_x phi, u = P^-T b1 = L_i^-1 b1_i */
    for (int64_t i = 0; i < n; ++i) {
        const double *Li = L1 + i * k * k;
        for (int a = 0; a < k; ++a) {
            double t = -(gX[i * k + a] - mu / x[i * k + a]);
            for (int l = 0; l < a; ++l) t -= Li[a * k + l] * u[i * k + l];
            u[i * k + a] = t / Li[a * k + a];
        }
    }
    /* W block (j, i) = Cb_ji P_i^-1 = Cb_ji L_i^-T: each row w solves L_i w^T = c^T */
    for (int64_t j = 0; j < m; ++j)
        for (int64_t i = 0; i < n; ++i) {
            const double *Li = L1 + i * k * k;
            double res = -M[i + ldm * j];
            for (int a = 0; a < k; ++a) res += x[i * k + a] * y[a + k * j];
            for (int a = 0; a < k; ++a) {
                double *wrow = W + (j * k + a) * nk + i * k;
                for (int b = 0; b < k; ++b) {
                    double cab = x[i * k + a] * y[b + k * j];
                    if (full && a == b) cab += res;
                    double t = cab;
                    for (int l = 0; l < b; ++l) t -= Li[b * k + l] * wrow[l];
                    wrow[b] = t / Li[b * k + b];
                }
            }
        }
    /* Schur matrix S = R2 - W W^T and rhs = b2 - W u */
    for (int64_t p1 = 0; p1 < mk; ++p1) {
        int64_t j1 = p1 / k;
        int a1 = (int)(p1 % k);
        for (int64_t p2 = 0; p2 < mk; ++p2) {
            int64_t j2 = p2 / k;
            int a2 = (int)(p2 % k);
            double t = 0.0;
            if (j1 == j2) t = XX[a1 * k + a2] + (a1 == a2 ? rho + s[p1] / y[p1] : 0.0);
            const double *w1 = W + p1 * nk, *w2 = W + p2 * nk;
            for (int64_t q = 0; q < nk; ++q) t -= w1[q] * w2[q];
            S[p1 * mk + p2] = t;
        }
        double t = -(gY[p1] - mu / y[p1]);
        const double *w1 = W + p1 * nk;
        for (int64_t q = 0; q < nk; ++q) t -= w1[q] * u[q];
        rhs[p1] = t;
    }
    if (dense_chol(mk, S) != OR_OK) { st = OR_NOTPD; goto done; }
    for (int64_t c = 0; c < mk; ++c) {       /* L v = rhs */
        double t = rhs[c];
        for (int64_t l = 0; l < c; ++l) t -= S[c * mk + l] * dy[l];
        dy[c] = t / S[c * mk + c];
    }
    for (int64_t c = mk - 1; c >= 0; --c) {  /* L^T dy = v */
        double t = dy[c];
        for (int64_t l = c + 1; l < mk; ++l) t -= S[l * mk + c] * dy[l];
        dy[c] = t / S[c * mk + c];
    }
    /* dx = P^-1 (u - W^T dy) = L_i^-T (...) */
    for (int64_t q = 0; q < nk; ++q) {
        double t = u[q];
        for (int64_t p1 = 0; p1 < mk; ++p1) t -= W[p1 * nk + q] * dy[p1];
        dx[q] = t;
    }
    for (int64_t i = 0; i < n; ++i) {
        const double *Li = L1 + i * k * k;
        for (int a = k - 1; a >= 0; --a) {
            double t = dx[i * k + a];
            for (int l = a + 1; l < k; ++l) t -= Li[l * k + a] * dx[i * k + l];
            dx[i * k + a] = t / Li[a * k + a];
        }
    }
    /* Diag(r) dx + Diag(x) dr = mu e - Diag(r) x, likewise for (y, s) */
    for (int64_t q = 0; q < nk; ++q) dr[q] = mu / x[q] - r[q] - r[q] / x[q] * dx[q];
    for (int64_t q = 0; q < mk; ++q) ds[q] = mu / y[q] - s[q] - s[q] / y[q] * dy[q];
done:
    free(gX); free(gY); free(L1); free(W); free(S); free(u); free(rhs);
    return st;
}

/* Largest alpha in (0, 1] with v + alpha dv >= (1 - tau) v (eq. "eqn:alpha"). */
static double frac_to_boundary(int64_t N, const double *v, const double *dv, double tau)
{
    double a = 1.0;
    for (int64_t t = 0; t < N; ++t)
        if (dv[t] < 0.0) {
            double c = -tau * v[t] / dv[t];
            if (c < a) a = c;
        }
    return a;
}

/* Note on termination.  f(XD, D^-1 Y) = f(X, Y) for every positive diagonal
 * D, while the barrier terms change by -mu (n - m) sum_c log d_c; hence for
 * n != m the merit function phi is unbounded below along that orbit, the
 * boundedness hypothesis of Theorem "thm:converge" fails, and with 2-norms
 * the inner test E(.;mu) <= mu cannot hold before
 * ||X_c|| + ||Y_c|| + sqrt(n) + sqrt(m) >= |n - m| (each column c).  The
 * iterates then drift along the orbit and the Newton cap ends the run
 * (status NOTCONV).  The algorithm is implemented as printed regardless.
 *
 * Stage 2 started from the stage-1 point (X, Y), overwritten with the result.
 * Implements the transition of Sec. 4 (eqs. "upxy", "rho0", "rs", "mu",
 * "rho") and then Alg. "alg:fast": outer loop on mu, inner Newton loop with
 * the fraction-to-boundary rule (tau = 0.9), Armijo backtracking on phi
 * (eq. "eqn:armijo", eta = 0.5), predictor-based sigma (eqs. "eqn:muaff",
 * "eqn:mu"), and the Hessian switch at sigma <= sigma_c (Sec. 4).
 * stats: [0] E(.;0) at exit, [1] f, [2] Newton iterations, [3] outer
 * iterations, [4] final mu, [5] iterations that used the full Hessian,
 * [6] Armijo failures.  trace (may be NULL): 8 doubles per Newton iteration:
 * outer index, mu, phi before, phi after, 1 if the full Hessian was used,
 * accepted primal step alpha_1, dual step alpha_2, E(.;mu) before the step. */
int oracle_ipm(int64_t n, int64_t m, int k, const double *M, int64_t ldm,
               double *X, double *Y, double eps_tol, int max_newton,
               double *stats, double *trace, int trace_cap, int *ntrace)
{
    if (n < 1 || m < 1 || k < 1 || k > KMAX || ldm < n) return OR_EINVAL;
    const double tau = 0.9, eta = 0.5, sigma_c = 0.01;
    const int64_t nk = n * k, mk = m * k;
    prob_t p = {n, m, k, M, ldm};
    double *x = X, *y = Y;
    double *r = (double *)malloc(sizeof(double) * nk);
    double *s = (double *)malloc(sizeof(double) * mk);
    double *gX = (double *)malloc(sizeof(double) * nk);
    double *gY = (double *)malloc(sizeof(double) * mk);
    double *dx = (double *)malloc(sizeof(double) * nk);
    double *dy = (double *)malloc(sizeof(double) * mk);
    double *dr = (double *)malloc(sizeof(double) * nk);
    double *ds = (double *)malloc(sizeof(double) * mk);
    double *xt = (double *)malloc(sizeof(double) * nk);
    double *yt = (double *)malloc(sizeof(double) * mk);
    int st = OR_OK, it = 0, outer = 0, nfull = 0, nfail = 0, nt = 0;
    if (!r || !s || !gX || !gY || !dx || !dy || !dr || !ds || !xt || !yt) { st = OR_EINVAL; goto out; }

    /* transition: (x, y) := max{(x, y), rho0}, rho0 = 1e-6 max{(x, y)} */
    double vmax = 0.0;
    for (int64_t q = 0; q < nk; ++q) if (x[q] > vmax) vmax = x[q];
    for (int64_t q = 0; q < mk; ++q) if (y[q] > vmax) vmax = y[q];
    const double rho0 = 1e-6 * vmax;
    for (int64_t q = 0; q < nk; ++q) if (x[q] < rho0) x[q] = rho0;
    for (int64_t q = 0; q < mk; ++q) if (y[q] < rho0) y[q] = rho0;
    /* r = max|graX| e, s = max|graY| e */
    oracle_grad(n, m, k, M, ldm, x, y, gX, gY);
    double gxm = 0.0, gym = 0.0;
    for (int64_t q = 0; q < nk; ++q) if (fabs(gX[q]) > gxm) gxm = fabs(gX[q]);
    for (int64_t q = 0; q < mk; ++q) if (fabs(gY[q]) > gym) gym = fabs(gY[q]);
    if (!(gxm > 0.0)) gxm = EPS64;
    if (!(gym > 0.0)) gym = EPS64;
    for (int64_t q = 0; q < nk; ++q) r[q] = gxm;
    for (int64_t q = 0; q < mk; ++q) s[q] = gym;
    double mu = 0.0;
    for (int64_t q = 0; q < nk; ++q) mu += x[q] * r[q];
    for (int64_t q = 0; q < mk; ++q) mu += y[q] * s[q];
    mu /= (double)(nk + mk);
    const double rho = eps_tol;
    int flag = 0;
    double E0 = 0.0;

    for (outer = 0;; ++outer) {
        oracle_grad(n, m, k, M, ldm, x, y, gX, gY);
        E0 = ipm_error(&p, x, y, r, s, 0.0, gX, gY);
        if (E0 <= eps_tol) break;
        if (it >= max_newton || outer >= max_newton) { st = OR_NOTCONV; break; }
        const double eps_mu = mu;
        for (;;) {
            oracle_grad(n, m, k, M, ldm, x, y, gX, gY);
            const double e_mu = ipm_error(&p, x, y, r, s, mu, gX, gY);
            if (e_mu <= eps_mu) break;
            if (it >= max_newton) { st = OR_NOTCONV; break; }
            int used_full = 0, dst;
            double slope = 0.0;
            if (flag) {
                dst = oracle_ipm_direction(n, m, k, M, ldm, x, y, r, s, mu, rho, 1, dx, dy, dr, ds);
                if (dst == OR_OK) {
                    for (int64_t q = 0; q < nk; ++q) slope += dx[q] * (gX[q] - mu / x[q]);
                    for (int64_t q = 0; q < mk; ++q) slope += dy[q] * (gY[q] - mu / y[q]);
                }
                if (dst != OR_OK || !(slope < 0.0)) flag = 0;
                else used_full = 1;
            }
            if (!used_full) {
                dst = oracle_ipm_direction(n, m, k, M, ldm, x, y, r, s, mu, rho, 0, dx, dy, dr, ds);
                if (dst != OR_OK) { st = dst; goto out; }
                slope = 0.0;
                for (int64_t q = 0; q < nk; ++q) slope += dx[q] * (gX[q] - mu / x[q]);
                for (int64_t q = 0; q < mk; ++q) slope += dy[q] * (gY[q] - mu / y[q]);
            }
            double a1 = frac_to_boundary(nk, x, dx, tau);
            double t2 = frac_to_boundary(mk, y, dy, tau);
            if (t2 < a1) a1 = t2;
            double a2 = frac_to_boundary(nk, r, dr, tau);
            t2 = frac_to_boundary(mk, s, ds, tau);
            if (t2 < a2) a2 = t2;
            const double phi0 = ipm_phi(&p, x, y, mu);
            double phi1 = phi0;
            int accepted = 0;
            for (int bt = 0; bt < 60; ++bt, a1 *= 0.5) {
                for (int64_t q = 0; q < nk; ++q) xt[q] = x[q] + a1 * dx[q];
                for (int64_t q = 0; q < mk; ++q) yt[q] = y[q] + a1 * dy[q];
                phi1 = ipm_phi(&p, xt, yt, mu);
                if (phi1 <= phi0 + eta * a1 * slope) { accepted = 1; break; }
            }
            if (!accepted) { ++nfail; phi1 = phi0; a1 = 0.0; }
            for (int64_t q = 0; q < nk; ++q) { x[q] += a1 * dx[q]; r[q] += a2 * dr[q]; }
            for (int64_t q = 0; q < mk; ++q) { y[q] += a1 * dy[q]; s[q] += a2 * ds[q]; }
            if (trace && nt < trace_cap) {
                trace[8 * nt + 0] = outer;
                trace[8 * nt + 1] = mu;
                trace[8 * nt + 2] = phi0;
                trace[8 * nt + 3] = phi1;
                trace[8 * nt + 4] = used_full;
                trace[8 * nt + 5] = a1;
                trace[8 * nt + 6] = a2;
                trace[8 * nt + 7] = e_mu;
                ++nt;
            }
            nfull += used_full;
            ++it;
        }
        if (st != OR_OK) break;
        /* predictor (affine-scaling) direction, mu = 0, Gauss-Newton Hessian */
        int dst = oracle_ipm_direction(n, m, k, M, ldm, x, y, r, s, 0.0, rho, 0, dx, dy, dr, ds);
        if (dst != OR_OK) { st = dst; break; }
        double a1 = frac_to_boundary(nk, x, dx, 1.0), t2 = frac_to_boundary(mk, y, dy, 1.0);
        if (t2 < a1) a1 = t2;
        double a2 = frac_to_boundary(nk, r, dr, 1.0);
        t2 = frac_to_boundary(mk, s, ds, 1.0);
        if (t2 < a2) a2 = t2;
        double mu_aff = 0.0, mu_cur = 0.0;
        for (int64_t q = 0; q < nk; ++q) {
            mu_aff += (x[q] + a1 * dx[q]) * (r[q] + a2 * dr[q]);
            mu_cur += x[q] * r[q];
        }
        for (int64_t q = 0; q < mk; ++q) {
            mu_aff += (y[q] + a1 * dy[q]) * (s[q] + a2 * ds[q]);
            mu_cur += y[q] * s[q];
        }
        mu_aff /= (double)(nk + mk);
        mu_cur /= (double)(nk + mk);
        double ratio = mu_aff / mu_cur;
        double sigma = ratio * ratio * ratio;
        if (!(sigma < 0.99)) sigma = 0.99;
        if (sigma < 0.0) sigma = 0.0;
        mu *= sigma;
        flag = sigma <= sigma_c;
    }
    if (stats) {
        stats[0] = E0;
        stats[1] = oracle_objective(n, m, k, M, ldm, x, y);
        stats[2] = it;
        stats[3] = outer;
        stats[4] = mu;
        stats[5] = nfull;
        stats[6] = nfail;
    }
out:
    if (ntrace) *ntrace = nt;
    free(r); free(s); free(gX); free(gY); free(dx); free(dy); free(dr); free(ds);
    free(xt); free(yt);
    return st;
}

/* Alg. "alg:fast": stage-1 ANLS until the relative step test (eps_STOL),
 * then stage 2.  stats: [0..6] as oracle_ipm, [7] stage-1 sweeps. */
int oracle_two_stage(int64_t n, int64_t m, int k, const double *M, int64_t ldm,
                     double *X, double *Y, double stol, int max_sweeps,
                     double eps_tol, int max_newton, double *stats)
{
    int sweeps = 0;
    int st = oracle_anls(n, m, k, M, ldm, X, Y, NULL, NULL, max_sweeps, stol, 0.0,
                         NULL, &sweeps);
    if (st != OR_OK) return st;
    st = oracle_ipm(n, m, k, M, ldm, X, Y, eps_tol, max_newton, stats, NULL, 0, NULL);
    if (stats) stats[7] = sweeps;
    return st;
}
