/*
 * Reference oracle for batched unfolded ISTA / Step-LISTA / Oracle-ISTA on the
 * Lasso (Ablin, Moreau, Massias, Gramfort, "Learning step sizes for unfolded
 * sparse coding", arXiv 1905.11071).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct FP64 CPU
 * statement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product library
 * never does.  It shares no code, header or constant with the CUDA sources.
 *
 * Conventions
 *   D  : n x m dictionary, row-major (D[i*m + j] = D_ij).
 *   X  : N x n samples, row-major (sample i is X[i*n .. i*n+n-1]).
 *   Z  : N x m codes, row-major.
 *   Everything is double precision; the Python wrapper promotes the FP32
 *   inputs that the GPU consumes to double before calling in.
 *
 * Every routine follows the passage of the paper cited in its comment, in the
 * paper's order of operations: gradients are formed as D^T(Dz - x) with two
 * matrix-vector products (Eq. ista / Eq. pgd), never through a precomputed
 * Gram matrix, so the oracle does not share the GPU path's formulation.
 *
 * Parity-unpinned parts: none of the routines below is unpinned; the pins live
 * in tests/test_oracle_*.py (closed forms, invariants, brute force, finite
 * differences, an independent eigen-solver).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* sign(v) with sign(0) = 0 (Section 2, Notation). */
static double sgn(double v) { return v > 0.0 ? 1.0 : (v < 0.0 ? -1.0 : 0.0); }

/* Soft-thresholding ST(v, u) = sign(v) max(|v| - u, 0) (Section 1, after
 * Eq. ista). */
double orc_st(double v, double u)
{
    double a = fabs(v) - u;
    return a > 0.0 ? sgn(v) * a : 0.0;
}

/* r = D z - x  (n-vector). */
static void residual_Dz_minus_x(const double *D, int n, int m, const double *z,
                                const double *x, double *r)
{
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < m; ++j) s += D[(size_t)i * m + j] * z[j];
        r[i] = s - x[i];
    }
}

/* g = D^T r  (m-vector). */
static void Dt_times(const double *D, int n, int m, const double *r, double *g)
{
    for (int j = 0; j < m; ++j) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += D[(size_t)i * m + j] * r[i];
        g[j] = s;
    }
}

/* grad = D^T (D z - x): gradient of the smooth part of F_x (Eq. lasso);
 * work must hold n doubles. */
static void lasso_grad(const double *D, int n, int m, const double *x,
                       const double *z, double *grad, double *work)
{
    residual_Dz_minus_x(D, n, m, z, x, work);
    Dt_times(D, n, m, work, grad);
}

/* One proximal-gradient step with step alpha (Section 2 Notation and
 * Eq. pgd): out = psi_alpha(z, x) = ST(z - alpha D^T(Dz - x), alpha*lam).
 * work must hold n + m doubles.  out may not alias z. */
static void psi(const double *D, int n, int m, const double *x, double lam,
                double alpha, const double *z, double *out, double *work)
{
    double *grad = work + n;
    lasso_grad(D, n, m, x, z, grad, work);
    for (int j = 0; j < m; ++j) out[j] = orc_st(z[j] - alpha * grad[j], alpha * lam);
}

/* Lasso cost F_x(z) = 1/2 ||x - Dz||^2 + lam ||z||_1 (Eq. lasso).
 * work must hold n doubles. */
static double lasso_cost(const double *D, int n, int m, const double *x,
                         const double *z, double lam, double *work)
{
    residual_Dz_minus_x(D, n, m, z, x, work);
    double q = 0.0, l1 = 0.0;
    for (int i = 0; i < n; ++i) q += work[i] * work[i];
    for (int j = 0; j < m; ++j) l1 += fabs(z[j]);
    return 0.5 * q + lam * l1;
}

/* ------------------------------------------------------------------------ */
/* Batched Lasso quantities                                                  */
/* ------------------------------------------------------------------------ */

/* Per-sample objective F_{x_i}(z_i) (Eq. lasso) and duality gap.
 * The gap is not in the paper; it uses the standard Lasso dual: with
 * r = x - Dz and s = min(1, lam / ||D^T r||_inf), nu = s r is dual feasible
 * (||D^T nu||_inf <= lam) and the dual value is 1/2||x||^2 - 1/2||x - nu||^2.
 * gap may be NULL. */
void orc_objective(const double *D, int n, int m, const double *X, int N,
                   const double *Z, double lam, double *F, double *gap)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *cor = (double *)malloc(sizeof(double) * (size_t)m);
    for (int s = 0; s < N; ++s) {
        const double *x = X + (size_t)s * n;
        const double *z = Z + (size_t)s * m;
        F[s] = lasso_cost(D, n, m, x, z, lam, r);
        if (gap) {
            /* r = x - D z */
            residual_Dz_minus_x(D, n, m, z, x, r);
            for (int i = 0; i < n; ++i) r[i] = -r[i];
            Dt_times(D, n, m, r, cor);
            double ninf = 0.0;
            for (int j = 0; j < m; ++j) ninf = fabs(cor[j]) > ninf ? fabs(cor[j]) : ninf;
            double sc = (ninf > lam) ? lam / ninf : 1.0;
            double dual = 0.0, xx = 0.0;
            for (int i = 0; i < n; ++i) {
                double nu = sc * r[i];
                double d = x[i] - nu;
                xx += x[i] * x[i];
                dual += d * d;
            }
            dual = 0.5 * xx - 0.5 * dual;
            gap[s] = F[s] - dual;
        }
    }
    free(r);
    free(cor);
}

/* lambda_max(x) = ||D^T x||_inf per sample (Section 2, Framework). */
void orc_lambda_max(const double *D, int n, int m, const double *X, int N, double *out)
{
    double *g = (double *)malloc(sizeof(double) * (size_t)m);
    for (int s = 0; s < N; ++s) {
        Dt_times(D, n, m, X + (size_t)s * n, g);
        double v = 0.0;
        for (int j = 0; j < m; ++j) v = fabs(g[j]) > v ? fabs(g[j]) : v;
        out[s] = v;
    }
    free(g);
}

/* Gram quantities by definition: B = D^T D (m x m), C = X D (row i is
 * (D^T x_i)^T), xsq_i = ||x_i||^2.  (B appears through W_z = Id - D^T D / L in
 * Section 4; C is the D^T x term of the gradient in Eq. ista.) */
void orc_gram(const double *D, int n, int m, const double *X, int N,
              double *B, double *C, double *xsq)
{
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) {
            double s = 0.0;
            for (int i = 0; i < n; ++i) s += D[(size_t)i * m + a] * D[(size_t)i * m + b];
            B[(size_t)a * m + b] = s;
        }
    for (int s = 0; s < N; ++s) {
        const double *x = X + (size_t)s * n;
        double q = 0.0;
        for (int i = 0; i < n; ++i) q += x[i] * x[i];
        xsq[s] = q;
        for (int j = 0; j < m; ++j) {
            double v = 0.0;
            for (int i = 0; i < n; ++i) v += x[i] * D[(size_t)i * m + j];
            C[(size_t)s * m + j] = v;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Largest eigenvalue of a symmetric matrix: cyclic Jacobi rotations.        */
/* L = largest eigenvalue of D^T D (Section 1, after Eq. ista) and           */
/* L_S = largest eigenvalue of D_S^T D_S (Eq. spca) are both computed here.  */
/* ------------------------------------------------------------------------ */

/* Cyclic Jacobi eigenvalue iteration on a copy of the k x k symmetric matrix
 * A: each rotation zeroes one off-diagonal pair; sweeps repeat until the
 * off-diagonal mass is negligible.  Returns the largest diagonal entry of the
 * converged matrix.  work must hold k*k doubles. */
double orc_sym_max_eig(const double *A, int k, double *work)
{
    if (k <= 0) return 0.0;
    double *a = work;
    memcpy(a, A, sizeof(double) * (size_t)k * k);
    double fro = 0.0;
    for (size_t i = 0; i < (size_t)k * k; ++i) fro += a[i] * a[i];
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) off += 2.0 * a[(size_t)p * k + q] * a[(size_t)p * k + q];
        if (off <= 1e-30 * fro || off == 0.0) break;
        for (int p = 0; p < k - 1; ++p) {
            for (int q = p + 1; q < k; ++q) {
                double apq = a[(size_t)p * k + q];
                if (apq == 0.0) continue;
                double app = a[(size_t)p * k + p], aqq = a[(size_t)q * k + q];
                /* rotation angle that annihilates a_pq */
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0);
                double s = t * c;
                /* A <- J^T A J on rows/columns p and q */
                for (int r = 0; r < k; ++r) {
                    double arp = a[(size_t)r * k + p], arq = a[(size_t)r * k + q];
                    a[(size_t)r * k + p] = c * arp - s * arq;
                    a[(size_t)r * k + q] = s * arp + c * arq;
                }
                for (int r = 0; r < k; ++r) {
                    double apr = a[(size_t)p * k + r], aqr = a[(size_t)q * k + r];
                    a[(size_t)p * k + r] = c * apr - s * aqr;
                    a[(size_t)q * k + r] = s * apr + c * aqr;
                }
                a[(size_t)p * k + q] = 0.0;
                a[(size_t)q * k + p] = 0.0;
            }
        }
    }
    double best = a[0];
    for (int i = 1; i < k; ++i) best = a[(size_t)i * k + i] > best ? a[(size_t)i * k + i] : best;
    return best;
}

/* L_S = largest eigenvalue of D_S^T D_S for the index set S (Eq. spca), with
 * the convention L_{empty} = L supplied by the caller.  idx holds |S| column
 * indices.  work must hold 2*k*k doubles. */
static double support_lipschitz(const double *D, int n, int m, const int *idx, int k,
                                double L_empty, double *work)
{
    if (k == 0) return L_empty;
    double *G = work + (size_t)k * k;
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) {
            double s = 0.0;
            for (int i = 0; i < n; ++i) s += D[(size_t)i * m + idx[a]] * D[(size_t)i * m + idx[b]];
            G[(size_t)a * k + b] = s;
        }
    return orc_sym_max_eig(G, k, work);
}

/* L = largest eigenvalue of D^T D (Section 1, after Eq. ista). */
double orc_lipschitz(const double *D, int n, int m)
{
    int *idx = (int *)malloc(sizeof(int) * (size_t)m);
    double *work = (double *)malloc(sizeof(double) * 2 * (size_t)m * m);
    for (int j = 0; j < m; ++j) idx[j] = j;
    double L = support_lipschitz(D, n, m, idx, m, 0.0, work);
    free(idx);
    free(work);
    return L;
}

/* L_S for an explicit support given as a 0/1 mask of length m (Eq. spca). */
double orc_support_lipschitz(const double *D, int n, int m, const unsigned char *mask,
                             double L_empty)
{
    int *idx = (int *)malloc(sizeof(int) * (size_t)m);
    int k = 0;
    for (int j = 0; j < m; ++j)
        if (mask[j]) idx[k++] = j;
    double *work = (double *)malloc(sizeof(double) * 2 * (size_t)(k > 0 ? k : 1) * (k > 0 ? k : 1));
    double v = support_lipschitz(D, n, m, idx, k, L_empty, work);
    free(idx);
    free(work);
    return v;
}

/* ------------------------------------------------------------------------ */
/* Unfolded proximal gradient: ISTA, PGD with a step sequence, Step-LISTA.   */
/* ------------------------------------------------------------------------ */

/* T layers of Eq. pgd / Eq. steprec from z^(0) = 0 (Section 1 and Section 4,
 * Step-LISTA):  z^(t+1) = ST(z^(t) - alpha_t D^T(D z^(t) - x), alpha_t lam).
 * ISTA is alpha_t = 1/L for every t (Eq. ista).
 * Z (N x m) receives z^(T).  If Zall is not NULL it receives every iterate,
 * layout [t][sample][j] for t = 0..T. */
void orc_pgd(const double *D, int n, int m, const double *X, int N, double lam,
             const double *alpha, int T, double *Z, double *Zall)
{
    double *z = (double *)malloc(sizeof(double) * (size_t)m);
    double *zn = (double *)malloc(sizeof(double) * (size_t)m);
    double *work = (double *)malloc(sizeof(double) * (size_t)(n + m));
    for (int s = 0; s < N; ++s) {
        const double *x = X + (size_t)s * n;
        for (int j = 0; j < m; ++j) z[j] = 0.0;
        if (Zall) memcpy(Zall + (size_t)s * m, z, sizeof(double) * (size_t)m);
        for (int t = 0; t < T; ++t) {
            psi(D, n, m, x, lam, alpha[t], z, zn, work);
            memcpy(z, zn, sizeof(double) * (size_t)m);
            if (Zall) memcpy(Zall + ((size_t)(t + 1) * N + s) * m, z, sizeof(double) * (size_t)m);
        }
        memcpy(Z + (size_t)s * m, z, sizeof(double) * (size_t)m);
    }
    free(z);
    free(zn);
    free(work);
}

/* T layers of coupled LISTA (Eq. lista_layer, Section 4) from z^(0) = 0:
 *   z^(t+1) = ST(z^(t) - alpha_t W_t^T (D z^(t) - x), beta_t lam),
 * W_t = W + t*n*m (n x m, row-major like D), alpha_t, beta_t > 0.  Z: N x m. */
void orc_lista(const double *D, int n, int m, const double *X, int N, double lam,
               const double *W, const double *alpha, const double *beta, int T, double *Z)
{
    double *z = (double *)malloc(sizeof(double) * (size_t)m);
    double *v = (double *)malloc(sizeof(double) * (size_t)m);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    for (int s = 0; s < N; ++s) {
        const double *x = X + (size_t)s * n;
        for (int j = 0; j < m; ++j) z[j] = 0.0;
        for (int t = 0; t < T; ++t) {
            residual_Dz_minus_x(D, n, m, z, x, r);
            Dt_times(W + (size_t)t * n * m, n, m, r, v);
            for (int j = 0; j < m; ++j) z[j] = orc_st(z[j] - alpha[t] * v[j], beta[t] * lam);
        }
        memcpy(Z + (size_t)s * m, z, sizeof(double) * (size_t)m);
    }
    free(z);
    free(v);
    free(r);
}

/* ------------------------------------------------------------------------ */
/* Oracle-ISTA (Algorithm 1, Section 3).                                     */
/* ------------------------------------------------------------------------ */

/* The method.  Restricted to codes supported on S, the smooth part of F_x
 * has an L_S-Lipschitz gradient (Eq. spca), so the quadratic majorant of
 * F_x at z with curvature L_S bounds F_x from above at every point whose
 * support lies in S = supp(z) (the argument of Section 3 built on
 * Eq. majorization2).  Minimising that majorant is the proximal step with
 * step 1/L_S; its result is a certified descent step whenever its own
 * support stays inside S, condition (star).  When it leaves S the global
 * majorant with curvature L (an ISTA step) is used instead.  L_S is a
 * function of S alone, so one value is kept per sample and recomputed only
 * when S changes; the empty support takes L.
 *
 * This routine runs that method for T layers from z^(0) = 0, independently
 * per sample, with exact eigenvalues (cyclic Jacobi) and gradients formed as
 * D^T(Dz - x).
 * Outputs (every one but Z may be NULL): Z (N x m) = z^(T); LS (N) = the
 * L_S belonging to supp(z^(T-1)), the last support the method evaluated;
 * accepted (T) = per layer, the number of samples whose local step met
 * condition (star); decision (T x N) = that outcome per layer and sample;
 * Zall ((T+1) x N x m) = every iterate; margin (T x N) = for layer t and
 * sample s, how far the layer's decisions were from flipping: the smallest
 * distance of a pre-threshold value to its threshold among (i) the codes
 * outside S under the local step (which decide condition (star)) and (ii)
 * every code under the step actually taken (which decide the new support).
 * A layer whose margin is below the arithmetic's error scale can decide
 * differently in another precision; every later layer of that sample then
 * follows another trajectory. */

/* out = ST(z - step * grad, step * lam), coordinatewise; also returns
 * min_j ||z_j - step grad_j| - step lam| over the codes j with sel[j] != 0
 * (every code when sel is NULL). */
static double prox_step_with_margin(const double *z, const double *grad, int m, double step, double lam,
                                    const unsigned char *sel, double *out)
{
    double closest = INFINITY;
    for (int j = 0; j < m; ++j) {
        const double u = z[j] - step * grad[j];
        out[j] = orc_st(u, step * lam);
        const double d = fabs(fabs(u) - step * lam);
        if ((sel == NULL || sel[j]) && d < closest) closest = d;
    }
    return closest;
}

void orc_oista(const double *D, int n, int m, const double *X, int N, double lam,
               double L, int T, double *Z, double *LS, int *accepted, unsigned char *decision,
               double *Zall, double *margin)
{
    double *z = (double *)malloc(sizeof(double) * (size_t)m);
    double *cand = (double *)malloc(sizeof(double) * (size_t)m);
    double *fallback = (double *)malloc(sizeof(double) * (size_t)m);
    double *grad = (double *)malloc(sizeof(double) * (size_t)m);
    double *work = (double *)malloc(sizeof(double) * (size_t)n);
    double *ework = (double *)malloc(sizeof(double) * 2 * (size_t)m * m);
    int *idx = (int *)malloc(sizeof(int) * (size_t)m);
    unsigned char *S = (unsigned char *)malloc((size_t)m);
    unsigned char *offS = (unsigned char *)malloc((size_t)m);
    unsigned char *S_cached = (unsigned char *)malloc((size_t)m);
    if (accepted)
        for (int t = 0; t < T; ++t) accepted[t] = 0;
    for (int s = 0; s < N; ++s) {
        const double *x = X + (size_t)s * n;
        double L_S = L;
        int have_cache = 0;
        for (int j = 0; j < m; ++j) z[j] = 0.0;
        if (Zall) memcpy(Zall + (size_t)s * m, z, sizeof(double) * (size_t)m);
        for (int t = 0; t < T; ++t) {
            int k = 0;
            for (int j = 0; j < m; ++j) {
                S[j] = z[j] != 0.0;
                offS[j] = !S[j];
                if (S[j]) idx[k++] = j;
            }
            if (!have_cache || memcmp(S, S_cached, (size_t)m) != 0) {
                L_S = support_lipschitz(D, n, m, idx, k, L, ework);  /* L for the empty support */
                memcpy(S_cached, S, (size_t)m);
                have_cache = 1;
            }
            lasso_grad(D, n, m, x, z, grad, work);
            /* the step of the local majorant, and how close its codes off S came to their threshold */
            const double off_margin = prox_step_with_margin(z, grad, m, 1.0 / L_S, lam, offS, cand);
            int stays_in_S = 1;
            for (int j = 0; j < m; ++j)
                if (cand[j] != 0.0 && !S[j]) stays_in_S = 0;
            double taken_margin;
            if (stays_in_S) {
                taken_margin = prox_step_with_margin(z, grad, m, 1.0 / L_S, lam, NULL, cand);
                memcpy(z, cand, sizeof(double) * (size_t)m);
                if (accepted) accepted[t] += 1;
            } else {
                taken_margin = prox_step_with_margin(z, grad, m, 1.0 / L, lam, NULL, fallback);
                memcpy(z, fallback, sizeof(double) * (size_t)m);
            }
            if (decision) decision[(size_t)t * N + s] = (unsigned char)stays_in_S;
            if (margin) margin[(size_t)t * N + s] = off_margin < taken_margin ? off_margin : taken_margin;
            if (Zall) memcpy(Zall + ((size_t)(t + 1) * N + s) * m, z, sizeof(double) * (size_t)m);
            if (LS && t == T - 1) LS[s] = L_S;
        }
        memcpy(Z + (size_t)s * m, z, sizeof(double) * (size_t)m);
        if (LS && T == 0) LS[s] = L;
    }
    free(z); free(cand); free(fallback); free(grad); free(work); free(ework); free(idx);
    free(S); free(offS); free(S_cached);
}

/* ------------------------------------------------------------------------ */
/* Step-LISTA sub-gradient with respect to the step sizes.                   */
/* ------------------------------------------------------------------------ */

/* Loss: sum_i F_{x_i}(z_i^(T)) (the empirical form of Eq. unsupervised).
 * The paper obtains the sub-gradient by automatic differentiation of the
 * network (Appendix E); this is the same chain rule written by hand on
 * Eq. steprec, with the kink of ST at |u| = alpha*lam and of |z| at 0 taking
 * derivative 0 (sign(0) = 0):
 *   u^t   = z^t - alpha_t D^T(D z^t - x),   z^{t+1} = ST(u^t, alpha_t lam)
 *   dz^{t+1}/du^t      = diag(|u^t| > alpha_t lam)
 *   dz^{t+1}/dalpha_t  = mask_t * ( -D^T(D z^t - x) - lam sign(u^t) )
 *   du^t/dz^t          = Id - alpha_t D^T D
 *   dF/dz^T            = D^T(D z^T - x) + lam sign(z^T).
 * Backward sweep: G = dF/dz^T; for t = T-1..0: h = G * mask_t;
 * dalpha_t += <h, dz^{t+1}/dalpha_t>; G = h - alpha_t D^T D h.
 * Outputs dalpha (T) and *loss (the summed objective at z^(T)). */
void orc_slista_grad(const double *D, int n, int m, const double *X, int N, double lam,
                     const double *alpha, int T, double *dalpha, double *loss)
{
    double *zs = (double *)malloc(sizeof(double) * (size_t)(T + 1) * m);
    double *G = (double *)malloc(sizeof(double) * (size_t)m);
    double *h = (double *)malloc(sizeof(double) * (size_t)m);
    double *grad = (double *)malloc(sizeof(double) * (size_t)m);
    double *Bh = (double *)malloc(sizeof(double) * (size_t)m);
    double *work = (double *)malloc(sizeof(double) * (size_t)(n + m));
    double total = 0.0;
    for (int t = 0; t < T; ++t) dalpha[t] = 0.0;
    for (int s = 0; s < N; ++s) {
        const double *x = X + (size_t)s * n;
        for (int j = 0; j < m; ++j) zs[j] = 0.0;
        for (int t = 0; t < T; ++t)
            psi(D, n, m, x, lam, alpha[t], zs + (size_t)t * m, zs + (size_t)(t + 1) * m, work);
        const double *zT = zs + (size_t)T * m;
        total += lasso_cost(D, n, m, x, zT, lam, work);
        lasso_grad(D, n, m, x, zT, G, work);
        for (int j = 0; j < m; ++j) G[j] += lam * sgn(zT[j]);
        for (int t = T - 1; t >= 0; --t) {
            const double *zt = zs + (size_t)t * m;
            lasso_grad(D, n, m, x, zt, grad, work);
            double acc = 0.0;
            for (int j = 0; j < m; ++j) {
                double u = zt[j] - alpha[t] * grad[j];
                int on = fabs(u) > alpha[t] * lam;
                h[j] = on ? G[j] : 0.0;
                acc += h[j] * (-grad[j] - lam * sgn(u));
            }
            dalpha[t] += acc;
            /* D^T D h, as D^T applied to D h */
            for (int i = 0; i < n; ++i) {
                double v = 0.0;
                for (int j = 0; j < m; ++j) v += D[(size_t)i * m + j] * h[j];
                work[i] = v;
            }
            Dt_times(D, n, m, work, Bh);
            for (int j = 0; j < m; ++j) G[j] = h[j] - alpha[t] * Bh[j];
        }
    }
    if (loss) *loss = total;
    free(zs); free(G); free(h); free(grad); free(Bh); free(work);
}

/* ------------------------------------------------------------------------ */
/* Exact Lasso solution for small m by enumerating sign patterns.            */
/* ------------------------------------------------------------------------ */

/* Solve the k x k system A y = b by Gaussian elimination with partial
 * pivoting (A, b overwritten).  Returns 0 on success, -1 if singular. */
static int solve_dense(double *A, double *b, int k)
{
    for (int c = 0; c < k; ++c) {
        int p = c;
        for (int r = c + 1; r < k; ++r)
            if (fabs(A[(size_t)r * k + c]) > fabs(A[(size_t)p * k + c])) p = r;
        if (fabs(A[(size_t)p * k + c]) < 1e-13) return -1;
        if (p != c) {
            for (int j = 0; j < k; ++j) {
                double t = A[(size_t)c * k + j];
                A[(size_t)c * k + j] = A[(size_t)p * k + j];
                A[(size_t)p * k + j] = t;
            }
            double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int r = c + 1; r < k; ++r) {
            double f = A[(size_t)r * k + c] / A[(size_t)c * k + c];
            for (int j = c; j < k; ++j) A[(size_t)r * k + j] -= f * A[(size_t)c * k + j];
            b[r] -= f * b[c];
        }
    }
    for (int r = k - 1; r >= 0; --r) {
        double s = b[r];
        for (int j = r + 1; j < k; ++j) s -= A[(size_t)r * k + j] * b[j];
        b[r] = s / A[(size_t)r * k + r];
    }
    return 0;
}

/* The KKT conditions (Lemma 2.1, Eq. KKT) pin down z* once its sign pattern
 * s in {-1,0,+1}^m is known: on S = supp(s), D_S^T D_S z_S = D_S^T x - lam s_S,
 * and the candidate is optimal iff sign(z_S) = s_S and |D_j^T(x - Dz)| <= lam
 * off S.  All 3^m patterns are tried (m <= 12).  Returns the number of
 * patterns that satisfy the KKT conditions (1 for a unique solution), writes
 * the one with the smallest F_x into zout, or returns -1 if m is too large. */
int orc_lasso_bruteforce(const double *D, int n, int m, const double *x, double lam,
                         double *zout)
{
    if (m > 12 || m <= 0) return -1;
    int total = 1;
    for (int j = 0; j < m; ++j) total *= 3;
    double *A = (double *)malloc(sizeof(double) * (size_t)m * m);
    double *b = (double *)malloc(sizeof(double) * (size_t)m);
    double *z = (double *)malloc(sizeof(double) * (size_t)m);
    double *grad = (double *)malloc(sizeof(double) * (size_t)m);
    double *work = (double *)malloc(sizeof(double) * (size_t)(n + m));
    double *Dtx = (double *)malloc(sizeof(double) * (size_t)m);
    int *sg = (int *)malloc(sizeof(int) * (size_t)m);
    int *idx = (int *)malloc(sizeof(int) * (size_t)m);
    Dt_times(D, n, m, x, Dtx);
    int found = 0;
    double bestF = INFINITY;
    for (int code = 0; code < total; ++code) {
        int c = code, k = 0;
        for (int j = 0; j < m; ++j) {
            sg[j] = (c % 3) - 1;
            c /= 3;
            if (sg[j] != 0) idx[k++] = j;
        }
        for (int a = 0; a < k; ++a) {
            for (int bb = 0; bb < k; ++bb) {
                double s = 0.0;
                for (int i = 0; i < n; ++i) s += D[(size_t)i * m + idx[a]] * D[(size_t)i * m + idx[bb]];
                A[(size_t)a * k + bb] = s;
            }
            b[a] = Dtx[idx[a]] - lam * sg[idx[a]];
        }
        if (k > 0 && solve_dense(A, b, k) != 0) continue;
        for (int j = 0; j < m; ++j) z[j] = 0.0;
        int ok = 1;
        for (int a = 0; a < k; ++a) {
            z[idx[a]] = b[a];
            if (sgn(b[a]) != (double)sg[idx[a]]) ok = 0;
        }
        if (!ok) continue;
        lasso_grad(D, n, m, x, z, grad, work); /* D^T(Dz - x) */
        for (int j = 0; j < m; ++j)
            if (sg[j] == 0 && fabs(grad[j]) > lam * (1.0 + 1e-10)) { ok = 0; break; }
        if (!ok) continue;
        found += 1;
        double Fv = lasso_cost(D, n, m, x, z, lam, work);
        if (Fv < bestF) {
            bestF = Fv;
            memcpy(zout, z, sizeof(double) * (size_t)m);
        }
    }
    free(A); free(b); free(z); free(grad); free(work); free(Dtx); free(sg); free(idx);
    return found;
}

/* Largest violation of the KKT conditions (Lemma 2.1, Eq. KKT) at z for one
 * sample: on the support |D_j^T(x - Dz) - lam sign z_j|, off it
 * max(0, |D_j^T(x - Dz)| - lam). */
double orc_kkt_violation(const double *D, int n, int m, const double *x, const double *z,
                         double lam)
{
    double *grad = (double *)malloc(sizeof(double) * (size_t)m);
    double *work = (double *)malloc(sizeof(double) * (size_t)(n + m));
    lasso_grad(D, n, m, x, z, grad, work);
    double worst = 0.0;
    for (int j = 0; j < m; ++j) {
        double cj = -grad[j]; /* D_j^T (x - Dz) */
        double v = (z[j] != 0.0) ? fabs(cj - lam * sgn(z[j])) : fabs(cj) - lam;
        if (v > worst) worst = v;
    }
    free(grad);
    free(work);
    return worst;
}
