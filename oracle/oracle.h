/* Plain FP64 CPU oracle (test infrastructure only; see oracle.c). */
#ifndef CYQ_ORACLE_H
#define CYQ_ORACLE_H
#include <stddef.h>

void oracle_build_rhs(int N, int nx, int nu, const double *S, const double *A,
                      const double *q, const double *r, const double *c, const double *x0,
                      double *b);
void oracle_kkt_matvec(int N, int nx, int nu, const double *Q, const double *R, const double *S,
                       const double *A, const double *B, const double *Sigma,
                       const double *z, double *y);
void oracle_kkt_abs_matvec(int N, int nx, int nu, const double *Q, const double *R, const double *S,
                           const double *A, const double *B, const double *Sigma, const double *z, double *y);
double oracle_kkt_residual(int N, int nx, int nu, const double *Q, const double *R, const double *S,
                           const double *A, const double *B, const double *Sigma,
                           const double *z, const double *b, double *r_out);
double oracle_kkt_residual_fp64(int N, int nx, int nu, const double *Q, const double *R, const double *S,
                                const double *A, const double *B, const double *Sigma,
                                const double *z, const double *b, double *r_out);
int oracle_kkt_dense(int N, int nx, int nu, const double *Q, const double *R, const double *S,
                     const double *A, const double *B, const double *Sigma, double *K);
int oracle_dense_solve(int n, const double *K, const double *b, double *x);
int oracle_riccati_solve(int N, int nx, int nu, const double *Q, const double *R, const double *S,
                         const double *A, const double *B, const double *Sigma,
                         int nrhs, const double *b, size_t b_stride, double *z, size_t z_stride,
                         double *Pout);
int oracle_adjoint(int N, int nx, int nu, const double *Q, const double *R, const double *S,
                   const double *A, const double *B, const double *Sigma, const double *x0,
                   const double *z, const double *g, double *w_out,
                   double *dQ, double *dq, double *dR, double *dr, double *dS, double *dA,
                   double *dB, double *dc, double *dx0, double *dSigma);
#endif
