/*
 * Oracle for the sparse LU path: TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg may load this code.  The product path (the CUDA library) never calls
 * it and shares no code with it.
 *
 * What it computes (CKTSO, Section II-A, Algorithm 1, written for a CSC
 * matrix, i.e. the paper's row-major up-looking algorithm applied to the
 * transpose): a sequential left-looking Gilbert-Peierls LU factorization with
 * threshold partial pivoting,
 *
 *        P * A(:, Q) = L * U,   L unit lower triangular, U upper triangular,
 *
 * where Q is a given column order and P the row order chosen on the way.
 * For step k = 0..n-1 (column c = Q[k]):
 *   1. symbolic prediction: depth-first search from the rows of A(:,c)
 *      through the columns of L already computed; it yields the structure
 *      of column k and a topological order of the columns it depends on;
 *   2. x = A(:,c) scattered into a dense work vector (original row numbers);
 *   3. numerical update: for every dependency j in topological order,
 *      x(rows of L(:,j)) -= x(piv[j]) * L(:,j)   (one MAC per entry);
 *   4. threshold pivoting (Section II-A): among the rows of the structure
 *      that are not yet pivotal ("candidates"), the preferred row p (the
 *      previous pivot of this step, or the diagonal row c for a first
 *      factorization) is kept unless |x(p)| < eps * max |x(other candidates)|
 *      or x(p) == 0; otherwise the candidate of largest |x| becomes the pivot
 *      (ties: the row that comes first in the symmetric order Q);
 *   5. U(:,k) = x on the pivotal rows (diagonal last), L(:,k) = x on the
 *      other candidates divided by the pivot.
 * No candidate with a nonzero value => the matrix is singular.
 *
 * A re-factorization on an unchanged pattern (Section II-A, Algorithm 1 with
 * the symbolic and pivoting lines removed, checked as in Algorithms 3-5) is
 * defined as this factorization with the previous pivot sequence preferred:
 * when every preferred row passes the check this is exactly the
 * re-factorization without pivoting (same pattern, same permutation, hence
 * the same factors), and when one fails it is the factorization that the
 * restart with pivoting (Section IV-C/D) has to reproduce.
 *
 * Triangular solves follow Algorithm 2 (forward substitution with the unit
 * lower factor, then back substitution with U in reverse order).
 *
 * All arithmetic is IEEE binary64.  Compiled without FMA contraction so that
 * x86-64 and aarch64 builds give the same bits.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INPUT -1
#define ORC_ERR_SINGULAR -2
#define ORC_ERR_NOMEM -4

typedef struct {
    int n;
    /* strict lower factor, CSC, rows in step numbering, sorted */
    int *Lp, *Li;
    double *Lx;
    /* upper factor, CSC, rows in step numbering, sorted, diagonal last */
    int *Up, *Ui;
    double *Ux;
    int *piv;  /* piv[k] = original row that is pivotal at step k */
    int *Q;    /* Q[k] = original column of step k */
    int n_rejected; /* steps whose preferred row was not kept */
    int status;
    int bad_step;   /* step where a singular column was met, else -1 */
} orc_lu;

typedef struct {
    int *i;
    double *x;
    long long len, cap;
} vec_t;

static int vec_push(vec_t *v, int i, double x)
{
    if (v->len == v->cap) {
        long long cap = v->cap ? 2 * v->cap : 1024;
        int *ni = (int *)realloc(v->i, (size_t)cap * sizeof(int));
        if (!ni) return -1;
        v->i = ni;
        double *nx = (double *)realloc(v->x, (size_t)cap * sizeof(double));
        if (!nx) return -1;
        v->x = nx;
        v->cap = cap;
    }
    v->i[v->len] = i;
    v->x[v->len] = x;
    v->len++;
    return 0;
}

void orc_free(orc_lu *lu)
{
    if (!lu) return;
    free(lu->Lp); free(lu->Li); free(lu->Lx);
    free(lu->Up); free(lu->Ui); free(lu->Ux);
    free(lu->piv); free(lu->Q);
    free(lu);
}

/* sort (idx, val) pairs of one column by idx (insertion sort for short
 * columns, heap sort otherwise) */
static void sort_pairs(int *idx, double *val, long long m)
{
    if (m < 32) {
        for (long long a = 1; a < m; a++) {
            int ki = idx[a];
            double kv = val[a];
            long long b = a - 1;
            while (b >= 0 && idx[b] > ki) {
                idx[b + 1] = idx[b];
                val[b + 1] = val[b];
                b--;
            }
            idx[b + 1] = ki;
            val[b + 1] = kv;
        }
        return;
    }
    /* heap sort */
    for (long long s = m / 2 - 1; s >= 0; s--) {
        long long r = s;
        for (;;) {
            long long c = 2 * r + 1;
            if (c >= m) break;
            if (c + 1 < m && idx[c + 1] > idx[c]) c++;
            if (idx[r] >= idx[c]) break;
            int ti = idx[r]; idx[r] = idx[c]; idx[c] = ti;
            double tv = val[r]; val[r] = val[c]; val[c] = tv;
            r = c;
        }
    }
    for (long long e = m - 1; e > 0; e--) {
        int ti = idx[0]; idx[0] = idx[e]; idx[e] = ti;
        double tv = val[0]; val[0] = val[e]; val[e] = tv;
        long long r = 0;
        for (;;) {
            long long c = 2 * r + 1;
            if (c >= e) break;
            if (c + 1 < e && idx[c + 1] > idx[c]) c++;
            if (idx[r] >= idx[c]) break;
            ti = idx[r]; idx[r] = idx[c]; idx[c] = ti;
            tv = val[r]; val[r] = val[c]; val[c] = tv;
            r = c;
        }
    }
}

/*
 * Factorize.  prefer[k] = preferred pivot row (original numbering) of step
 * k, or NULL for the diagonal rows Q[k].  Returns a new orc_lu (status set);
 * NULL only when memory runs out.
 */
orc_lu *orc_factorize(int n, const int *Ap, const int *Ai, const double *Ax,
                      const int *Q, double eps, const int *prefer)
{
    orc_lu *lu = (orc_lu *)calloc(1, sizeof(orc_lu));
    if (!lu) return NULL;
    lu->n = n;
    lu->bad_step = -1;
    lu->status = ORC_OK;
    if (n < 1 || !Ap || !Ai || !Ax || !Q) { lu->status = ORC_ERR_INPUT; return lu; }

    int *pinv = (int *)malloc((size_t)n * sizeof(int));
    int *qinv = (int *)malloc((size_t)n * sizeof(int));
    int *mark = (int *)malloc((size_t)n * sizeof(int));
    int *stack = (int *)malloc((size_t)n * sizeof(int));
    int *pos = (int *)malloc((size_t)n * sizeof(int));
    int *topo = (int *)malloc((size_t)n * sizeof(int));
    double *x = (double *)calloc((size_t)n, sizeof(double));
    /* L columns while factorizing: original row numbers */
    long long *lbeg = (long long *)malloc((size_t)(n + 1) * sizeof(long long));
    long long *ubeg = (long long *)malloc((size_t)(n + 1) * sizeof(long long));
    vec_t L = {0}, U = {0};
    lu->piv = (int *)malloc((size_t)n * sizeof(int));
    lu->Q = (int *)malloc((size_t)n * sizeof(int));
    if (!pinv || !qinv || !mark || !stack || !pos || !topo || !x || !lbeg ||
        !ubeg || !lu->piv || !lu->Q) {
        lu->status = ORC_ERR_NOMEM;
        goto done;
    }
    for (int i = 0; i < n; i++) { pinv[i] = -1; qinv[i] = -1; mark[i] = -1; }
    for (int k = 0; k < n; k++) {
        if (Q[k] < 0 || Q[k] >= n || qinv[Q[k]] >= 0) { lu->status = ORC_ERR_INPUT; goto done; }
        qinv[Q[k]] = k;
        lu->Q[k] = Q[k];
    }
    lbeg[0] = 0;
    ubeg[0] = 0;

    for (int k = 0; k < n; k++) {
        int c = Q[k];
        /* ---- 1. symbolic prediction: DFS over the graph of L ---- */
        int ntopo = 0;
        for (int p = Ap[c]; p < Ap[c + 1]; p++) {
            int r0 = Ai[p];
            if (r0 < 0 || r0 >= n) { lu->status = ORC_ERR_INPUT; goto done; }
            if (mark[r0] == k) continue;
            int top = 0;
            stack[top] = r0;
            mark[r0] = k;
            pos[0] = 0;   /* pos[t] = next child offset of stack entry t */
            while (top >= 0) {
                int r = stack[top];
                int j = pinv[r];
                int pushed = 0;
                if (j >= 0) {
                    long long e = lbeg[j] + pos[top];
                    while (e < lbeg[j + 1]) {
                        int r2 = L.i[e];
                        e++;
                        if (mark[r2] != k) {
                            pos[top] = (int)(e - lbeg[j]);
                            mark[r2] = k;
                            top++;
                            stack[top] = r2;
                            pos[top] = 0;
                            pushed = 1;
                            break;
                        }
                    }
                    if (!pushed) pos[top] = (int)(lbeg[j + 1] - lbeg[j]);
                }
                if (!pushed) {
                    topo[ntopo++] = r;  /* postorder */
                    top--;
                }
            }
        }
        /* ---- 2. scatter A(:,c) ---- */
        for (int t = 0; t < ntopo; t++) x[topo[t]] = 0.0;
        for (int p = Ap[c]; p < Ap[c + 1]; p++) x[Ai[p]] = Ax[p];
        /* ---- 3. numerical update in topological order (reverse postorder) ---- */
        for (int t = ntopo - 1; t >= 0; t--) {
            int r = topo[t];
            int j = pinv[r];
            if (j < 0) continue;
            double xj = x[r];
            for (long long e = lbeg[j]; e < lbeg[j + 1]; e++)
                x[L.i[e]] -= L.x[e] * xj;
        }
        /* ---- 4. threshold pivoting with a preferred row ---- */
        int pref = prefer ? prefer[k] : c;
        int pref_cand = 0;
        double m = 0.0;        /* max |x| over candidates other than pref */
        int best = -1;         /* argmax |x| over all candidates, |x| > 0 */
        double best_abs = 0.0;
        for (int t = 0; t < ntopo; t++) {
            int r = topo[t];
            if (pinv[r] >= 0) continue;
            double a = fabs(x[r]);
            if (r == pref) pref_cand = 1;
            else if (a > m) m = a;
            if (a > best_abs || (a == best_abs && best >= 0 && a > 0.0 && qinv[r] < qinv[best])) {
                best = r;
                best_abs = a;
            }
        }
        int piv;
        if (pref_cand && x[pref] != 0.0 && fabs(x[pref]) >= eps * m) {
            piv = pref;
        } else {
            if (best < 0) {
                lu->status = ORC_ERR_SINGULAR;
                lu->bad_step = k;
                goto done;
            }
            piv = best;
            lu->n_rejected++;
        }
        double d = x[piv];
        /* ---- 5. store U(:,k) (pivotal rows, step numbers) and L(:,k) ---- */
        for (int t = 0; t < ntopo; t++) {
            int r = topo[t];
            if (pinv[r] >= 0) {
                if (vec_push(&U, pinv[r], x[r])) { lu->status = ORC_ERR_NOMEM; goto done; }
            }
        }
        if (vec_push(&U, k, d)) { lu->status = ORC_ERR_NOMEM; goto done; }
        for (int t = 0; t < ntopo; t++) {
            int r = topo[t];
            if (pinv[r] < 0 && r != piv) {
                if (vec_push(&L, r, x[r] / d)) { lu->status = ORC_ERR_NOMEM; goto done; }
            }
        }
        pinv[piv] = k;
        lu->piv[k] = piv;
        lbeg[k + 1] = L.len;
        ubeg[k + 1] = U.len;
    }

    /* ---- final CSC in step numbering, rows sorted ---- */
    lu->Lp = (int *)malloc((size_t)(n + 1) * sizeof(int));
    lu->Up = (int *)malloc((size_t)(n + 1) * sizeof(int));
    lu->Li = (int *)malloc((size_t)(L.len ? L.len : 1) * sizeof(int));
    lu->Lx = (double *)malloc((size_t)(L.len ? L.len : 1) * sizeof(double));
    lu->Ui = (int *)malloc((size_t)(U.len ? U.len : 1) * sizeof(int));
    lu->Ux = (double *)malloc((size_t)(U.len ? U.len : 1) * sizeof(double));
    if (!lu->Lp || !lu->Up || !lu->Li || !lu->Lx || !lu->Ui || !lu->Ux) {
        lu->status = ORC_ERR_NOMEM;
        goto done;
    }
    for (int k = 0; k <= n; k++) {
        lu->Lp[k] = (int)lbeg[k];
        lu->Up[k] = (int)ubeg[k];
    }
    for (long long e = 0; e < L.len; e++) {
        lu->Li[e] = pinv[L.i[e]];
        lu->Lx[e] = L.x[e];
    }
    for (long long e = 0; e < U.len; e++) {
        lu->Ui[e] = U.i[e];
        lu->Ux[e] = U.x[e];
    }
    for (int k = 0; k < n; k++) {
        sort_pairs(lu->Li + lbeg[k], lu->Lx + lbeg[k], lbeg[k + 1] - lbeg[k]);
        sort_pairs(lu->Ui + ubeg[k], lu->Ux + ubeg[k], ubeg[k + 1] - ubeg[k]);
    }

done:
    free(pinv); free(qinv); free(mark); free(stack); free(pos); free(topo);
    free(x); free(lbeg); free(ubeg);
    free(L.i); free(L.x); free(U.i); free(U.x);
    return lu;
}

int orc_status(const orc_lu *lu) { return lu->status; }
int orc_bad_step(const orc_lu *lu) { return lu->bad_step; }
int orc_rejected(const orc_lu *lu) { return lu->n_rejected; }
long long orc_nnz_l(const orc_lu *lu) { return lu->Lp ? lu->Lp[lu->n] : -1; }
long long orc_nnz_u(const orc_lu *lu) { return lu->Up ? lu->Up[lu->n] : -1; }

/* copy the factors out into caller arrays of the sizes reported above */
int orc_export(const orc_lu *lu, int *Lp, int *Li, double *Lx, int *Up,
               int *Ui, double *Ux, int *piv)
{
    if (lu->status != ORC_OK) return lu->status;
    int n = lu->n;
    memcpy(Lp, lu->Lp, (size_t)(n + 1) * sizeof(int));
    memcpy(Up, lu->Up, (size_t)(n + 1) * sizeof(int));
    memcpy(Li, lu->Li, (size_t)lu->Lp[n] * sizeof(int));
    memcpy(Lx, lu->Lx, (size_t)lu->Lp[n] * sizeof(double));
    memcpy(Ui, lu->Ui, (size_t)lu->Up[n] * sizeof(int));
    memcpy(Ux, lu->Ux, (size_t)lu->Up[n] * sizeof(double));
    memcpy(piv, lu->piv, (size_t)n * sizeof(int));
    return ORC_OK;
}

/*
 * Solve A x = b with the factors: y = L^-1 (P b), z = U^-1 y, x(Q) = z
 * (Algorithm 2 and its upper counterpart, column-oriented here).
 * x and b may not alias.
 */
int orc_solve(const orc_lu *lu, const double *b, double *x)
{
    if (lu->status != ORC_OK) return lu->status;
    int n = lu->n;
    double *y = (double *)malloc((size_t)n * sizeof(double));
    if (!y) return ORC_ERR_NOMEM;
    for (int k = 0; k < n; k++) y[k] = b[lu->piv[k]];
    for (int k = 0; k < n; k++) {
        double yk = y[k];
        for (int e = lu->Lp[k]; e < lu->Lp[k + 1]; e++) y[lu->Li[e]] -= lu->Lx[e] * yk;
    }
    for (int k = n - 1; k >= 0; k--) {
        int dpos = lu->Up[k + 1] - 1;   /* diagonal is the last entry */
        double zk = y[k] / lu->Ux[dpos];
        y[k] = zk;
        for (int e = lu->Up[k]; e < dpos; e++) y[lu->Ui[e]] -= lu->Ux[e] * zk;
    }
    for (int k = 0; k < n; k++) x[lu->Q[k]] = y[k];
    free(y);
    return ORC_OK;
}

/* the IEEE maximum: NaN if either argument is NaN */
static double max_nan(double m, double v)
{
    if (isnan(m) || isnan(v)) return NAN;
    return v > m ? v : m;
}

/*
 * Relative residual ||b - A x||_inf / (||A||_inf * ||x||_inf) of a CSC
 * matrix; out[0] = the ratio, out[1] = ||b - A x||_inf, out[2] = ||A||_inf,
 * out[3] = ||x||_inf.  A NaN in r, in a row sum of |A| or in x makes that
 * norm, and the ratio, NaN (the maximum of a set holding a NaN is NaN), so a
 * solution with a NaN entry never passes a residual bound.
 */
int orc_residual(int n, const int *Ap, const int *Ai, const double *Ax,
                 const double *x, const double *b, double *out)
{
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *rs = (double *)calloc((size_t)n, sizeof(double));
    if (!r || !rs) { free(r); free(rs); return ORC_ERR_NOMEM; }
    for (int i = 0; i < n; i++) r[i] = b[i];
    for (int c = 0; c < n; c++) {
        for (int p = Ap[c]; p < Ap[c + 1]; p++) {
            r[Ai[p]] -= Ax[p] * x[c];
            rs[Ai[p]] += fabs(Ax[p]);
        }
    }
    double rn = 0, an = 0, xn = 0;
    for (int i = 0; i < n; i++) {
        rn = max_nan(rn, fabs(r[i]));
        an = max_nan(an, rs[i]);
        xn = max_nan(xn, fabs(x[i]));
    }
    out[0] = (an > 0 && xn > 0) ? rn / (an * xn) : rn;
    out[1] = rn;
    out[2] = an;
    out[3] = xn;
    free(r);
    free(rs);
    return ORC_OK;
}
