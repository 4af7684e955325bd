/*
 * Plain FP64 CPU oracle for the KKT system of an equality-constrained
 * linear-quadratic optimal control problem.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA library and is deliberately slow and obvious: every routine is
 * a direct transcription of a definition, with plain loops.
 *
 * Problem (paper Sec. 2, eq. ocp-eq, E_j = I) and KKT system after elimination
 * of x_0 (eq. opt-cond-ocp-eq):
 *
 *   Q_N x^N - lambda^{N-1}                                 = b_x^N
 *   R_k u^k + S_k x^k + B_k^T lambda^k                     = b_u^k   (S_0 x^0 term absent)
 *   S_k^T u^k + Q_k x^k + A_k^T lambda^k - lambda^{k-1}    = b_x^k   (0 < k < N)
 *   B_k u^k + A_k x^k - x^{k+1}                            = b_lambda^k (A_0 x^0 term absent)
 *
 * where R_k, Q_k include the optional diagonal regularisation Sigma_k.  For
 * the original problem b = -(r~, q, f~) with r~^0 = r^0 + S_0 x_init and
 * f~^0 = f^0 + A_0 x_init.
 *
 * Vector layout (b, z, residuals): N records k = 0..N-1 of
 *   [ u^k (nu) | x^{k+1} (nx) | lambda^k (nx) ]
 * Matrix blocks are column-major; element (i,j) of a rows x cols block X is
 * X[i + j*rows].  Data layout per instance:
 *   Q (N+1) nx*nx, R N nu*nu, S N nu*nx, A N nx*nx, B N nx*nu,
 *   Sigma (N+1)*(nu+nx) records [Sigma_u | Sigma_x] or NULL.
 *
 * Parity status: every routine here is pinned by tests that do not reuse it
 * (dense brute force with a library solver, closed-form scalar Riccati, the
 * DARE fixed point, optimality of the primal trajectory by direct rollout,
 * central finite differences for the adjoint).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* small dense helpers (column-major)                                         */
/* ------------------------------------------------------------------------- */
#define IX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* C(m x n) = A^T (k x m)^T * B (k x n)   i.e. C = A^T B */
static void mat_tn(int m, int n, int k, const double *A, const double *B, double *C) {
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int t = 0; t < k; ++t) s += A[IX(t, i, k)] * B[IX(t, j, k)];
            C[IX(i, j, m)] = s;
        }
}

/* C(m x n) = A (m x k) * B (k x n) */
static void mat_nn(int m, int n, int k, const double *A, const double *B, double *C) {
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int t = 0; t < k; ++t) s += A[IX(i, t, m)] * B[IX(t, j, k)];
            C[IX(i, j, m)] = s;
        }
}

/* y(m) = A (m x n) x */
static void mat_vec(int m, int n, const double *A, const double *x, double *y) {
    for (int i = 0; i < m; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += A[IX(i, j, m)] * x[j];
        y[i] = s;
    }
}

/* y(n) = A^T x, A is m x n */
static void mat_tvec(int m, int n, const double *A, const double *x, double *y) {
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += A[IX(i, j, m)] * x[i];
        y[j] = s;
    }
}

/* In-place lower Cholesky factor of an SPD n x n matrix (upper part zeroed).
 * Returns 0, or 1 if a pivot is not positive and finite. */
static int cholesky(int n, double *M) {
    for (int j = 0; j < n; ++j) {
        double d = M[IX(j, j, n)];
        for (int t = 0; t < j; ++t) d -= M[IX(j, t, n)] * M[IX(j, t, n)];
        if (!(d > 0.0) || !isfinite(d)) return 1;
        d = sqrt(d);
        M[IX(j, j, n)] = d;
        for (int i = j + 1; i < n; ++i) {
            double s = M[IX(i, j, n)];
            for (int t = 0; t < j; ++t) s -= M[IX(i, t, n)] * M[IX(j, t, n)];
            M[IX(i, j, n)] = s / d;
        }
        for (int i = 0; i < j; ++i) M[IX(i, j, n)] = 0.0;
    }
    return 0;
}

/* Solve (L L^T) X = Y in place for nrhs columns of length n (ld n). */
static void chol_solve(int n, const double *L, int nrhs, double *Y) {
    for (int c = 0; c < nrhs; ++c) {
        double *y = Y + (size_t)c * n;
        for (int i = 0; i < n; ++i) {
            double s = y[i];
            for (int t = 0; t < i; ++t) s -= L[IX(i, t, n)] * y[t];
            y[i] = s / L[IX(i, i, n)];
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = y[i];
            for (int t = i + 1; t < n; ++t) s -= L[IX(t, i, n)] * y[t];
            y[i] = s / L[IX(i, i, n)];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* data access                                                                 */
/* ------------------------------------------------------------------------- */
typedef struct {
    int N, nx, nu;
    const double *Q, *R, *S, *A, *B, *Sigma;
} ocp_t;

static const double *blkQ(const ocp_t *p, int k) { return p->Q + (size_t)k * p->nx * p->nx; }
static const double *blkR(const ocp_t *p, int k) { return p->R + (size_t)k * p->nu * p->nu; }
static const double *blkS(const ocp_t *p, int k) { return p->S ? p->S + (size_t)k * p->nu * p->nx : NULL; }
static const double *blkA(const ocp_t *p, int k) { return p->A + (size_t)k * p->nx * p->nx; }
static const double *blkB(const ocp_t *p, int k) { return p->B + (size_t)k * p->nx * p->nu; }

/* effective R_k (+ Sigma_u^k) into out (nu x nu) */
static void effR(const ocp_t *p, int k, double *out) {
    int nu = p->nu;
    memcpy(out, blkR(p, k), sizeof(double) * nu * nu);
    if (p->Sigma)
        for (int i = 0; i < nu; ++i) out[IX(i, i, nu)] += p->Sigma[(size_t)k * (nu + p->nx) + i];
}

/* effective Q_k (+ Sigma_x^k) into out (nx x nx), k = 1..N */
static void effQ(const ocp_t *p, int k, double *out) {
    int nx = p->nx, nu = p->nu;
    memcpy(out, blkQ(p, k), sizeof(double) * nx * nx);
    if (p->Sigma)
        for (int i = 0; i < nx; ++i) out[IX(i, i, nx)] += p->Sigma[(size_t)k * (nu + nx) + nu + i];
}

static size_t rec(const ocp_t *p) { return (size_t)p->nu + 2 * (size_t)p->nx; }

/* ------------------------------------------------------------------------- */
/* right-hand side of the original problem (eq. opt-cond-ocp-eq)              */
/* ------------------------------------------------------------------------- */
void oracle_build_rhs(int N, int nx, int nu, const double *S, const double *A,
                      const double *q, const double *r, const double *c, const double *x0,
                      double *b) {
    size_t w = (size_t)nu + 2 * (size_t)nx;
    for (int k = 0; k < N; ++k) {
        double *bu = b + k * w, *bx = bu + nu, *bl = bx + nx;
        for (int i = 0; i < nu; ++i) bu[i] = -r[(size_t)k * nu + i];
        for (int i = 0; i < nx; ++i) bx[i] = -q[(size_t)(k + 1) * nx + i];
        for (int i = 0; i < nx; ++i) bl[i] = -c[(size_t)k * nx + i];
    }
    /* r~^0 = r^0 + S_0 x_init ; f~^0 = f^0 + A_0 x_init */
    for (int i = 0; i < nu; ++i) {
        double s = 0.0;
        if (S)
            for (int j = 0; j < nx; ++j) s += S[IX(i, j, nu)] * x0[j];
        b[i] -= s;
    }
    for (int i = 0; i < nx; ++i) {
        double s = 0.0;
        for (int j = 0; j < nx; ++j) s += A[IX(i, j, nx)] * x0[j];
        b[nu + nx + i] -= s;
    }
}

/* ------------------------------------------------------------------------- */
/* structured matrix-vector product y = K z (rows of eq. opt-cond-ocp-eq)    */
/* ------------------------------------------------------------------------- */
void oracle_kkt_matvec(int N, int nx, int nu, const double *Q, const double *R, const double *S,
                       const double *A, const double *B, const double *Sigma,
                       const double *z, double *y) {
    ocp_t p = {N, nx, nu, Q, R, S, A, B, Sigma};
    size_t w = rec(&p);
    double *M = malloc(sizeof(double) * (size_t)(nx > nu ? nx : nu) * (nx > nu ? nx : nu));
    double *t = malloc(sizeof(double) * (size_t)(nx > nu ? nx : nu));
    for (int k = 0; k < N; ++k) {
        const double *u = z + k * w;
        const double *xn = u + nu;            /* x^{k+1} */
        const double *lam = xn + nx;          /* lambda^k */
        const double *xk = k > 0 ? z + (k - 1) * w + nu : NULL; /* x^k */
        double *yu = y + k * w, *yx = yu + nu, *yl = yx + nx;
        /* row u^k: R_k u + S_k x^k + B_k^T lambda^k */
        effR(&p, k, M);
        mat_vec(nu, nu, M, u, yu);
        if (xk && S) {
            mat_vec(nu, nx, blkS(&p, k), xk, t);
            for (int i = 0; i < nu; ++i) yu[i] += t[i];
        }
        mat_tvec(nx, nu, blkB(&p, k), lam, t);
        for (int i = 0; i < nu; ++i) yu[i] += t[i];
        /* row x^{k+1} */
        int j = k + 1;
        effQ(&p, j, M);
        mat_vec(nx, nx, M, xn, yx);
        for (int i = 0; i < nx; ++i) yx[i] -= lam[i];
        if (j < N) {
            const double *un = z + j * w;               /* u^{j} */
            const double *ln = un + nu + nx;            /* lambda^{j} */
            if (S) {
                mat_tvec(nu, nx, blkS(&p, j), un, t);
                for (int i = 0; i < nx; ++i) yx[i] += t[i];
            }
            mat_tvec(nx, nx, blkA(&p, j), ln, t);
            for (int i = 0; i < nx; ++i) yx[i] += t[i];
        }
        /* row lambda^k: B_k u^k + A_k x^k - x^{k+1} */
        mat_vec(nx, nu, blkB(&p, k), u, yl);
        if (xk) {
            mat_vec(nx, nx, blkA(&p, k), xk, t);
            for (int i = 0; i < nx; ++i) yl[i] += t[i];
        }
        for (int i = 0; i < nx; ++i) yl[i] -= xn[i];
    }
    free(M);
    free(t);
}

/* y += |A| |x| (A m x n) and y += |A|^T |x| */
static void abs_mat_vec_add(int m, int n, const double *A, const double *x, double *y) {
    for (int i = 0; i < m; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += fabs(A[IX(i, j, m)]) * fabs(x[j]);
        y[i] += s;
    }
}
static void abs_mat_tvec_add(int m, int n, const double *A, const double *x, double *y) {
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += fabs(A[IX(i, j, m)]) * fabs(x[i]);
        y[j] += s;
    }
}

/* y = |K| |z|: the rows of oracle_kkt_matvec with every coefficient and every
 * entry of z replaced by its absolute value (the identity couplings of the
 * dynamics count +1).  Componentwise, an evaluation of b - K z in float64 with
 * any summation order is within gamma_m (|b| + |K| |z|) of the exact value,
 * gamma_m = m u / (1 - m u), m the most roundings on one term's path: the
 * terms of a row plus b, plus one for the diagonal entry, whose Sigma is
 * either added to Q_ii (R_ii) first or summed as a product of its own
 * (Higham, Accuracy and Stability of Numerical Algorithms, Sec. 3.1). */
void oracle_kkt_abs_matvec(int N, int nx, int nu, const double *Q, const double *R, const double *S,
                           const double *A, const double *B, const double *Sigma, const double *z, double *y) {
    ocp_t p = {N, nx, nu, Q, R, S, A, B, Sigma};
    size_t w = rec(&p);
    double *M = malloc(sizeof(double) * (size_t)(nx > nu ? nx : nu) * (nx > nu ? nx : nu));
    memset(y, 0, sizeof(double) * (size_t)N * w);
    for (int k = 0; k < N; ++k) {
        const double *u = z + k * w;
        const double *xn = u + nu;
        const double *lam = xn + nx;
        const double *xk = k > 0 ? z + (k - 1) * w + nu : NULL;
        double *yu = y + k * w, *yx = yu + nu, *yl = yx + nx;
        effR(&p, k, M);
        abs_mat_vec_add(nu, nu, M, u, yu);
        if (xk && S) abs_mat_vec_add(nu, nx, blkS(&p, k), xk, yu);
        abs_mat_tvec_add(nx, nu, blkB(&p, k), lam, yu);
        int j = k + 1;
        effQ(&p, j, M);
        abs_mat_vec_add(nx, nx, M, xn, yx);
        for (int i = 0; i < nx; ++i) yx[i] += fabs(lam[i]);
        if (j < N) {
            const double *un = z + j * w;
            const double *ln = un + nu + nx;
            if (S) abs_mat_tvec_add(nu, nx, blkS(&p, j), un, yx);
            abs_mat_tvec_add(nx, nx, blkA(&p, j), ln, yx);
        }
        abs_mat_vec_add(nx, nu, blkB(&p, k), u, yl);
        if (xk) abs_mat_vec_add(nx, nx, blkA(&p, k), xk, yl);
        for (int i = 0; i < nx; ++i) yl[i] += fabs(xn[i]);
    }
    free(M);
}

/* relative residual ||b - K z||_2 / ||b||_2 (returns ||b - Kz|| if b = 0) */
/* Relative KKT residual ||b - K z||_2 / ||b||_2 with every row evaluated in
 * plain float64 (products and sums rounded in the order of oracle_kkt_matvec,
 * Sigma already added to the diagonals of R and Q).  Its rounding error can
 * exceed the residual itself when the terms of a row cancel by many orders of
 * magnitude; oracle_kkt_residual below evaluates the same definition
 * accurately. */
double oracle_kkt_residual_fp64(int N, int nx, int nu, const double *Q, const double *R, const double *S,
                                const double *A, const double *B, const double *Sigma,
                                const double *z, const double *b, double *r_out) {
    size_t n = (size_t)N * ((size_t)nu + 2 * (size_t)nx);
    double *y = r_out ? r_out : malloc(sizeof(double) * n);
    oracle_kkt_matvec(N, nx, nu, Q, R, S, A, B, Sigma, z, y);
    double rn = 0.0, bn = 0.0;
    for (size_t i = 0; i < n; ++i) {
        y[i] = b[i] - y[i];
        rn += y[i] * y[i];
        bn += b[i] * b[i];
    }
    if (!r_out) free(y);
    rn = sqrt(rn);
    bn = sqrt(bn);
    return bn > 0.0 ? rn / bn : rn;
}

/* Error-free transformations: a + b = s + t exactly (Knuth's TwoSum) and
 * a b = p + e exactly (TwoProduct with a fused multiply-add; C99 fma is
 * correctly rounded). */
static void two_sum(double a, double b, double *s, double *t) {
    double x = a + b, bv = x - a;
    *s = x;
    *t = (a - (x - bv)) + (b - bv);
}

/* A row sum b_i - sum_j c_j v_j carried as hi + lo (Ogita, Rump and Oishi,
 * "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005), Dot2): the
 * result is as accurate as if computed in twice the working precision and
 * then rounded, |error| <= u |exact| + gamma_n^2 (|b_i| + sum |c_j v_j|). */
typedef struct { double hi, lo; } acc2_t;

static void acc2_sub_prod(acc2_t *a, double c, double v) {
    const double q = c * v, e = fma(c, v, -q); /* c v = q + e exactly */
    double s, t;
    two_sum(a->hi, -q, &s, &t);
    a->hi = s;
    a->lo += t - e;
}

static void acc2_sub_mat_vec(acc2_t *y, int m, int n, const double *M, const double *x) {
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) acc2_sub_prod(&y[i], M[IX(i, j, m)], x[j]);
}
static void acc2_sub_mat_tvec(acc2_t *y, int m, int n, const double *M, const double *x) {
    /* y (n) -= M^T x, M is m x n */
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < m; ++i) acc2_sub_prod(&y[j], M[IX(i, j, m)], x[i]);
}

/* Relative KKT residual ||b - K z||_2 / ||b||_2, the quantity the refinement
 * drives below its tolerance (eq. opt-cond-ocp-eq rows as in oracle_kkt_matvec,
 * Sigma_k as its own diagonal term, so K is the data exactly).  Every row is
 * accumulated with the compensated dot product above and rounded once; the
 * squared norms are then summed in plain float64 (relative error about
 * n u / 2, far below the quantity measured). */
double oracle_kkt_residual(int N, int nx, int nu, const double *Q, const double *R, const double *S,
                           const double *A, const double *B, const double *Sigma,
                           const double *z, const double *b, double *r_out) {
    ocp_t p = {N, nx, nu, Q, R, S, A, B, Sigma};
    size_t w = rec(&p), n = (size_t)N * w;
    acc2_t *y = malloc(sizeof(acc2_t) * n);
    for (size_t i = 0; i < n; ++i) {
        y[i].hi = b[i];
        y[i].lo = 0.0;
    }
    for (int k = 0; k < N; ++k) {
        const double *u = z + k * w;
        const double *xn = u + nu;
        const double *lam = xn + nx;
        const double *xk = k > 0 ? z + (k - 1) * w + nu : NULL;
        acc2_t *yu = y + k * w, *yx = yu + nu, *yl = yx + nx;
        /* row u^k: R_k u + Sigma_u u + S_k x^k + B_k^T lambda^k */
        acc2_sub_mat_vec(yu, nu, nu, blkR(&p, k), u);
        if (Sigma)
            for (int i = 0; i < nu; ++i) acc2_sub_prod(&yu[i], Sigma[(size_t)k * (nu + nx) + i], u[i]);
        if (xk && S) acc2_sub_mat_vec(yu, nu, nx, blkS(&p, k), xk);
        acc2_sub_mat_tvec(yu, nx, nu, blkB(&p, k), lam);
        /* row x^{k+1}: Q x - lambda^k (+ S^T u^{k+1} + A^T lambda^{k+1}) */
        int j = k + 1;
        acc2_sub_mat_vec(yx, nx, nx, blkQ(&p, j), xn);
        if (Sigma)
            for (int i = 0; i < nx; ++i) acc2_sub_prod(&yx[i], Sigma[(size_t)j * (nu + nx) + nu + i], xn[i]);
        for (int i = 0; i < nx; ++i) acc2_sub_prod(&yx[i], -1.0, lam[i]);
        if (j < N) {
            const double *un = z + j * w;
            const double *ln = un + nu + nx;
            if (S) acc2_sub_mat_tvec(yx, nu, nx, blkS(&p, j), un);
            acc2_sub_mat_tvec(yx, nx, nx, blkA(&p, j), ln);
        }
        /* row lambda^k: B u + A x^k - x^{k+1} */
        acc2_sub_mat_vec(yl, nx, nu, blkB(&p, k), u);
        if (xk) acc2_sub_mat_vec(yl, nx, nx, blkA(&p, k), xk);
        for (int i = 0; i < nx; ++i) acc2_sub_prod(&yl[i], -1.0, xn[i]);
    }
    double rn = 0.0, bn = 0.0;
    for (size_t i = 0; i < n; ++i) {
        const double r = y[i].hi + y[i].lo;
        if (r_out) r_out[i] = r;
        rn += r * r;
        bn += b[i] * b[i];
    }
    free(y);
    rn = sqrt(rn);
    bn = sqrt(bn);
    return bn > 0.0 ? rn / bn : rn;
}

/* ------------------------------------------------------------------------- */
/* dense KKT matrix (row-major dim x dim), same rows as above                */
/* ------------------------------------------------------------------------- */
int oracle_kkt_dense(int N, int nx, int nu, const double *Q, const double *R, const double *S,
                     const double *A, const double *B, const double *Sigma, double *K) {
    ocp_t p = {N, nx, nu, Q, R, S, A, B, Sigma};
    size_t w = rec(&p), n = (size_t)N * w;
    memset(K, 0, sizeof(double) * n * n);
#define KK(r, c) K[(size_t)(r) * n + (size_t)(c)]
    double *M = malloc(sizeof(double) * (size_t)(nx > nu ? nx : nu) * (nx > nu ? nx : nu));
    for (int k = 0; k < N; ++k) {
        size_t iu = k * w, ix = iu + nu, il = ix + nx;   /* u^k, x^{k+1}, lambda^k */
        size_t ixk = k > 0 ? (k - 1) * w + nu : 0;       /* x^k */
        /* row u^k */
        effR(&p, k, M);
        for (int a = 0; a < nu; ++a)
            for (int c = 0; c < nu; ++c) KK(iu + a, iu + c) = M[IX(a, c, nu)];
        if (k > 0 && S)
            for (int a = 0; a < nu; ++a)
                for (int c = 0; c < nx; ++c) KK(iu + a, ixk + c) = blkS(&p, k)[IX(a, c, nu)];
        for (int a = 0; a < nu; ++a)
            for (int c = 0; c < nx; ++c) KK(iu + a, il + c) = blkB(&p, k)[IX(c, a, nx)];
        /* row x^{k+1} */
        int j = k + 1;
        effQ(&p, j, M);
        for (int a = 0; a < nx; ++a)
            for (int c = 0; c < nx; ++c) KK(ix + a, ix + c) = M[IX(a, c, nx)];
        for (int a = 0; a < nx; ++a) KK(ix + a, il + a) = -1.0;
        if (j < N) {
            size_t iuj = j * w, ilj = iuj + nu + nx;
            if (S)
                for (int a = 0; a < nx; ++a)
                    for (int c = 0; c < nu; ++c) KK(ix + a, iuj + c) = blkS(&p, j)[IX(c, a, nu)];
            for (int a = 0; a < nx; ++a)
                for (int c = 0; c < nx; ++c) KK(ix + a, ilj + c) = blkA(&p, j)[IX(c, a, nx)];
        }
        /* row lambda^k */
        for (int a = 0; a < nx; ++a)
            for (int c = 0; c < nu; ++c) KK(il + a, iu + c) = blkB(&p, k)[IX(a, c, nx)];
        if (k > 0)
            for (int a = 0; a < nx; ++a)
                for (int c = 0; c < nx; ++c) KK(il + a, ixk + c) = blkA(&p, k)[IX(a, c, nx)];
        for (int a = 0; a < nx; ++a) KK(il + a, ix + a) = -1.0;
    }
#undef KK
    free(M);
    return 0;
}

/* Gaussian elimination with partial pivoting on a row-major n x n system. */
int oracle_dense_solve(int n, const double *K, const double *b, double *x) {
    double *M = malloc(sizeof(double) * (size_t)n * n);
    double *y = malloc(sizeof(double) * (size_t)n);
    memcpy(M, K, sizeof(double) * (size_t)n * n);
    memcpy(y, b, sizeof(double) * (size_t)n);
    int status = 0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        double best = fabs(M[(size_t)c * n + c]);
        for (int r = c + 1; r < n; ++r)
            if (fabs(M[(size_t)r * n + c]) > best) { best = fabs(M[(size_t)r * n + c]); piv = r; }
        if (!(best > 0.0)) { status = 1; break; }
        if (piv != c) {
            for (int t = 0; t < n; ++t) {
                double s = M[(size_t)c * n + t];
                M[(size_t)c * n + t] = M[(size_t)piv * n + t];
                M[(size_t)piv * n + t] = s;
            }
            double s = y[c]; y[c] = y[piv]; y[piv] = s;
        }
        for (int r = c + 1; r < n; ++r) {
            double f = M[(size_t)r * n + c] / M[(size_t)c * n + c];
            if (f == 0.0) continue;
            for (int t = c; t < n; ++t) M[(size_t)r * n + t] -= f * M[(size_t)c * n + t];
            y[r] -= f * y[c];
        }
    }
    if (!status)
        for (int r = n - 1; r >= 0; --r) {
            double s = y[r];
            for (int t = r + 1; t < n; ++t) s -= M[(size_t)r * n + t] * x[t];
            x[r] = s / M[(size_t)r * n + r];
        }
    free(M);
    free(y);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Textbook Riccati recursion with affine terms (paper Sec. 9.2,             */
/* eq. riccati-recursion-P), solving K z = b for nrhs right-hand sides.      */
/*                                                                             */
/* With r_k = -b_u^k, q_k = -b_x^k, c_k = -b_lambda^k and x^0 = 0 (x_init is  */
/* already folded into b):                                                     */
/*   P_N = Q_N, p_N = q_N                                                      */
/*   Huu = R + B^T P' B, Hux = S + B^T P' A, hu = r + B^T (P' c + p')          */
/*   K_k = -Huu^{-1} Hux, k_k = -Huu^{-1} hu                                   */
/*   P = Q + A^T P' A + Hux^T K_k,  p = q + A^T (P' c + p') + Hux^T k_k        */
/* forward: u = K x + k, x' = A x + B u + c, lambda^k = P_{k+1} x' + p_{k+1}.  */
/* Optional output Pout: P_k for k = 1..N ((N) blocks nx*nx, block k-1).      */
/* Returns 0, or 1 + k if Huu at stage k is not positive definite.            */
/* ------------------------------------------------------------------------- */
int oracle_riccati_solve(int N, int nx, int nu, const double *Q, const double *R, const double *S,
                         const double *A, const double *B, const double *Sigma,
                         int nrhs, const double *b, size_t b_stride, double *z, size_t z_stride,
                         double *Pout) {
    ocp_t p = {N, nx, nu, Q, R, S, A, B, Sigma};
    size_t w = rec(&p);
    size_t nx2 = (size_t)nx * nx;
    double *P = malloc(sizeof(double) * nx2 * (N + 1));          /* P_1..P_N at index k */
    double *pv = malloc(sizeof(double) * (size_t)nx * (N + 1) * nrhs);
    double *Kg = malloc(sizeof(double) * (size_t)nu * nx * N);   /* feedback K_k */
    double *kv = malloc(sizeof(double) * (size_t)nu * N * nrhs);
    double *Luu = malloc(sizeof(double) * (size_t)nu * nu);
    double *Hux = malloc(sizeof(double) * (size_t)nu * nx);
    double *PB = malloc(sizeof(double) * (size_t)nx * nu);
    double *PA = malloc(sizeof(double) * nx2);
    size_t mx = (size_t)(nx > nu ? nx : nu);
    double *T = malloc(sizeof(double) * mx * mx);
    double *v = malloc(sizeof(double) * (size_t)nx);
    double *hu = malloc(sizeof(double) * (size_t)nu * nrhs);
    double *xs = malloc(sizeof(double) * (size_t)nx);
    double *xn = malloc(sizeof(double) * (size_t)nx);
    int status = 0;

#define PVEC(k, c) (pv + ((size_t)(c) * (N + 1) + (k)) * nx)
#define KVEC(k, c) (kv + ((size_t)(c) * N + (k)) * nu)
    /* terminal */
    effQ(&p, N, P + nx2 * N);
    for (int c = 0; c < nrhs; ++c)
        for (int i = 0; i < nx; ++i) PVEC(N, c)[i] = -b[c * b_stride + (size_t)(N - 1) * w + nu + i];

    for (int k = N - 1; k >= 0; --k) {
        const double *Pn = P + nx2 * (k + 1);
        const double *Bk = blkB(&p, k), *Ak = blkA(&p, k);
        /* Huu = R + B^T P' B */
        mat_nn(nx, nu, nx, Pn, Bk, PB);
        mat_tn(nu, nu, nx, Bk, PB, Luu);
        effR(&p, k, T);
        for (size_t i = 0; i < (size_t)nu * nu; ++i) Luu[i] += T[i];
        /* hu = r + B^T (P' c + p') per rhs */
        for (int c = 0; c < nrhs; ++c) {
            const double *bl = b + c * b_stride + (size_t)k * w + nu + nx;   /* b_lambda^k = -c_k */
            for (int i = 0; i < nx; ++i) {
                double s = PVEC(k + 1, c)[i];
                for (int j = 0; j < nx; ++j) s += Pn[IX(i, j, nx)] * (-bl[j]);
                v[i] = s;
            }
            mat_tvec(nx, nu, Bk, v, hu + (size_t)c * nu);
            for (int i = 0; i < nu; ++i) hu[(size_t)c * nu + i] += -b[c * b_stride + (size_t)k * w + i];
        }
        if (cholesky(nu, Luu)) { status = 1 + k; goto done; }
        /* k_k = -Huu^{-1} hu */
        for (int c = 0; c < nrhs; ++c) {
            chol_solve(nu, Luu, 1, hu + (size_t)c * nu);
            for (int i = 0; i < nu; ++i) KVEC(k, c)[i] = -hu[(size_t)c * nu + i];
        }
        if (k == 0) break;   /* x^0 = 0: P_0 and p_0 are not needed */
        /* Hux = S + B^T P' A */
        mat_nn(nx, nx, nx, Pn, Ak, PA);
        mat_tn(nu, nx, nx, Bk, PA, Hux);
        if (S)
            for (size_t i = 0; i < (size_t)nu * nx; ++i) Hux[i] += blkS(&p, k)[i];
        /* K_k = -Huu^{-1} Hux */
        double *Kk = Kg + (size_t)nu * nx * k;
        memcpy(Kk, Hux, sizeof(double) * nu * nx);
        chol_solve(nu, Luu, nx, Kk);
        for (size_t i = 0; i < (size_t)nu * nx; ++i) Kk[i] = -Kk[i];
        /* P_k = Q + A^T P' A + Hux^T K_k */
        double *Pk = P + nx2 * k;
        mat_tn(nx, nx, nx, Ak, PA, Pk);
        mat_tn(nx, nx, nu, Hux, Kk, T);
        effQ(&p, k, PA);   /* reuse PA as scratch for Q_k */
        for (size_t i = 0; i < nx2; ++i) Pk[i] += T[i] + PA[i];
        /* symmetrise (the recursion is symmetric in exact arithmetic) */
        for (int i = 0; i < nx; ++i)
            for (int j = 0; j < i; ++j) {
                double s = 0.5 * (Pk[IX(i, j, nx)] + Pk[IX(j, i, nx)]);
                Pk[IX(i, j, nx)] = Pk[IX(j, i, nx)] = s;
            }
        /* p_k = q + A^T (P' c + p') + Hux^T k_k */
        for (int c = 0; c < nrhs; ++c) {
            const double *bl = b + c * b_stride + (size_t)k * w + nu + nx;
            for (int i = 0; i < nx; ++i) {
                double s = PVEC(k + 1, c)[i];
                for (int j = 0; j < nx; ++j) s += Pn[IX(i, j, nx)] * (-bl[j]);
                v[i] = s;
            }
            double *pk = PVEC(k, c);
            mat_tvec(nx, nx, Ak, v, pk);
            mat_tvec(nu, nx, Hux, KVEC(k, c), xn);
            const double *bx = b + c * b_stride + (size_t)(k - 1) * w + nu;   /* b_x^k */
            for (int i = 0; i < nx; ++i) pk[i] += xn[i] - bx[i];
        }
    }
    /* forward sweep */
    for (int c = 0; c < nrhs; ++c) {
        const double *bc = b + c * b_stride;
        double *zc = z + c * z_stride;
        for (int i = 0; i < nx; ++i) xs[i] = 0.0;   /* x^0 folded into b */
        for (int k = 0; k < N; ++k) {
            double *u = zc + k * w, *xo = u + nu, *lam = xo + nx;
            /* u^k = K_k x^k + k_k  (K_0 x^0 = 0) */
            for (int i = 0; i < nu; ++i) u[i] = KVEC(k, c)[i];
            if (k > 0) {
                const double *Kk = Kg + (size_t)nu * nx * k;
                for (int i = 0; i < nu; ++i)
                    for (int j = 0; j < nx; ++j) u[i] += Kk[IX(i, j, nu)] * xs[j];
            }
            /* x^{k+1} = A_k x^k + B_k u^k + c_k */
            for (int i = 0; i < nx; ++i) {
                double s = -bc[(size_t)k * w + nu + nx + i];
                if (k > 0)
                    for (int j = 0; j < nx; ++j) s += blkA(&p, k)[IX(i, j, nx)] * xs[j];
                for (int j = 0; j < nu; ++j) s += blkB(&p, k)[IX(i, j, nx)] * u[j];
                xo[i] = s;
            }
            /* lambda^k = P_{k+1} x^{k+1} + p_{k+1} */
            const double *Pn = P + nx2 * (k + 1);
            for (int i = 0; i < nx; ++i) {
                double s = PVEC(k + 1, c)[i];
                for (int j = 0; j < nx; ++j) s += Pn[IX(i, j, nx)] * xo[j];
                lam[i] = s;
            }
            memcpy(xs, xo, sizeof(double) * nx);
        }
    }
    if (Pout) memcpy(Pout, P + nx2, sizeof(double) * nx2 * N);
done:
#undef PVEC
#undef KVEC
    free(P); free(pv); free(Kg); free(kv); free(Luu); free(Hux); free(PB); free(PA);
    free(T); free(v); free(hu); free(xs); free(xn);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Adjoint of z = K^{-1} b(theta) for a loss gradient g = dL/dz.             */
/* w = K^{-1} g (K symmetric), then dL = w^T (db - dK z):                     */
/*   dq_k = -w_x^k (k=1..N), dr_k = -w_u^k, dc_k = -w_lambda^k,               */
/*   dQ_k = -sym(w_x^k x^k^T), dR_k = -sym(w_u^k u^k^T),                      */
/*   dS_k = -(w_u^k x^k^T + u^k w_x^k^T)  (k >= 1),  dS_0 = -w_u^0 x_init^T,  */
/*   dA_k = -(w_lambda^k x^k^T + lambda^k w_x^k^T) (k>=1), dA_0 = -w_l^0 x_init^T */
/*   dB_k = -(w_lambda^k u^k^T + lambda^k w_u^k^T),                           */
/*   dx_init = -S_0^T w_u^0 - A_0^T w_lambda^0,                                */
/*   dSigma_u^k = -w_u^k .* u^k, dSigma_x^k = -w_x^k .* x^k.                   */
/* Output arrays follow the data layout; entries that do not enter the KKT   */
/* system (dQ_0, dq_0, dSigma_x^0, dSigma_u^N) are zero.  Any output pointer  */
/* may be NULL.  Returns the status of the inner solve.                       */
/* ------------------------------------------------------------------------- */
int oracle_adjoint(int N, int nx, int nu, const double *Q, const double *R, const double *S,
                   const double *A, const double *B, const double *Sigma, const double *x0,
                   const double *z, const double *g, double *w_out,
                   double *dQ, double *dq, double *dR, double *dr, double *dS, double *dA,
                   double *dB, double *dc, double *dx0, double *dSigma) {
    ocp_t p = {N, nx, nu, Q, R, S, A, B, Sigma};
    size_t wr = rec(&p), n = (size_t)N * wr;
    double *w = w_out ? w_out : malloc(sizeof(double) * n);
    int status = oracle_riccati_solve(N, nx, nu, Q, R, S, A, B, Sigma, 1, g, n, w, n, NULL);
    if (status) goto out;
    if (dQ) memset(dQ, 0, sizeof(double) * (size_t)(N + 1) * nx * nx);
    if (dq) memset(dq, 0, sizeof(double) * (size_t)(N + 1) * nx);
    if (dSigma) memset(dSigma, 0, sizeof(double) * (size_t)(N + 1) * (nu + nx));
    for (int k = 0; k < N; ++k) {
        const double *u = z + k * wr, *lam = u + nu + nx;
        const double *xk = k > 0 ? z + (k - 1) * wr + nu : x0;   /* x^k (x_init at k=0) */
        const double *wu = w + k * wr, *wl = wu + nu + nx;
        const double *wxk = k > 0 ? w + (k - 1) * wr + nu : NULL;
        const double *xn = u + nu, *wxn = wu + nu;                 /* x^{k+1}, w_x^{k+1} */
        if (dr) for (int i = 0; i < nu; ++i) dr[(size_t)k * nu + i] = -wu[i];
        if (dc) for (int i = 0; i < nx; ++i) dc[(size_t)k * nx + i] = -wl[i];
        if (dq) for (int i = 0; i < nx; ++i) dq[(size_t)(k + 1) * nx + i] = -wxn[i];
        if (dR)
            for (int i = 0; i < nu; ++i)
                for (int j = 0; j < nu; ++j)
                    dR[(size_t)k * nu * nu + IX(i, j, nu)] = -0.5 * (wu[i] * u[j] + u[i] * wu[j]);
        if (dQ)
            for (int i = 0; i < nx; ++i)
                for (int j = 0; j < nx; ++j)
                    dQ[(size_t)(k + 1) * nx * nx + IX(i, j, nx)] = -0.5 * (wxn[i] * xn[j] + xn[i] * wxn[j]);
        if (dS)
            for (int i = 0; i < nu; ++i)
                for (int j = 0; j < nx; ++j)
                    dS[(size_t)k * nu * nx + IX(i, j, nu)] =
                        -(wu[i] * xk[j] + (wxk ? u[i] * wxk[j] : 0.0));
        if (dA)
            for (int i = 0; i < nx; ++i)
                for (int j = 0; j < nx; ++j)
                    dA[(size_t)k * nx * nx + IX(i, j, nx)] =
                        -(wl[i] * xk[j] + (wxk ? lam[i] * wxk[j] : 0.0));
        if (dB)
            for (int i = 0; i < nx; ++i)
                for (int j = 0; j < nu; ++j)
                    dB[(size_t)k * nx * nu + IX(i, j, nx)] = -(wl[i] * u[j] + lam[i] * wu[j]);
        if (dSigma) {
            for (int i = 0; i < nu; ++i) dSigma[(size_t)k * (nu + nx) + i] = -wu[i] * u[i];
            for (int i = 0; i < nx; ++i) dSigma[(size_t)(k + 1) * (nu + nx) + nu + i] = -wxn[i] * xn[i];
        }
    }
    if (dx0) {
        const double *wu0 = w, *wl0 = w + nu + nx;
        for (int j = 0; j < nx; ++j) {
            double s = 0.0;
            if (S)
                for (int i = 0; i < nu; ++i) s += S[IX(i, j, nu)] * wu0[i];
            for (int i = 0; i < nx; ++i) s += A[IX(i, j, nx)] * wl0[i];
            dx0[j] = -s;
        }
    }
out:
    if (!w_out) free(w);
    return status;
}
