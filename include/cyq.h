/*
 * cyq — factor and solve the KKT system of linear-quadratic optimal control
 * problems on one GB300 GPU (sm_103a).  C ABI; every compute call takes device
 * pointers and a CUDA stream and is stream-ordered (asynchronous).
 *
 * Method (arXiv 2512.09058, "Cyqlone"): the horizon of each problem is cut
 * into P segments; each segment is eliminated by a modified Riccati recursion
 * (Sec. 4.2, Alg. fact-mod-riccati), the segment couplings form a symmetric
 * positive definite block-tridiagonal Schur complement in the multipliers
 * lambda^{b_c} at the segment ends (Sec. 4.3, eq. schur-compl-example-4), and
 * that system is factored by cyclic reduction (Sec. 3.2.1, Sec. 4.4,
 * Alg. fact-parallel-riccati-cr, Alg. cr).  The solve is the forward/backward
 * substitution with the factor of eq. chol-fac-K-cyqlone.  P = 1 is the
 * factorized Riccati recursion with early elimination of u^0 (Sec. 4.2 footnote).
 *
 * ---------------------------------------------------------------------------
 * Problem and KKT system (Sec. 2, eq. ocp-eq and eq. opt-cond-ocp-eq, E_j = I).
 * Per instance: horizon N >= 1, nx >= 1 states, nu >= 1 inputs.  Unknowns
 *   z = (u^0, x^1, lambda^0, u^1, x^2, lambda^1, ..., u^{N-1}, x^N, lambda^{N-1})
 * i.e. N records of [ u^k (nu) | x^{k+1} (nx) | lambda^k (nx) ].  K z = b with
 *   R_k u^k + S_k x^k + B_k^T lambda^k                   = b_u^k  (no S_0 x^0 term)
 *   S_k^T u^k + Q_k x^k + A_k^T lambda^k - lambda^{k-1}  = b_x^k  (0 < k < N)
 *   Q_N x^N - lambda^{N-1}                               = b_x^N
 *   B_k u^k + A_k x^k - x^{k+1}                          = b_l^k  (no A_0 x^0 term)
 * where R_k and Q_k include the optional diagonal regularisation Sigma_k.
 * The vector b uses the same record layout as z (row of u^k, row of x^{k+1},
 * row of lambda^k).  cyq_build_rhs forms b = -(r~, q, f~) of the original
 * problem from (q, r, c, x_init).
 *
 * Data layout (float64, device, caller-owned).  Instances are concatenated
 * kind by kind in instance order; inside an instance the blocks follow stage
 * order and every block is column-major (element (i,j) at i + j*rows):
 *   Q      (N+1) blocks nx*nx  (Q_0 is not read)
 *   R      N blocks     nu*nu
 *   S      N blocks     nu*nx  (S_k in R^{nu x nx}; S_0 is not read)   may be NULL (S = 0)
 *   A      N blocks     nx*nx  (A_0 is not read)
 *   B      N blocks     nx*nu
 *   Sigma  (N+1) records of nu+nx: [Sigma_u^k | Sigma_x^k]; record 0's x part and
 *          record N's u part are not read                             may be NULL
 *   q (N+1)*nx, r N*nu, c N*nx, x_init nx   (cyq_build_rhs / cyq_solve_adjoint)
 *   b, z   sum_i N_i*(nu_i + 2 nx_i) per right-hand side; several right-hand
 *          sides are stored one after another (stride = that total).
 *
 * Ownership.  The caller owns data, b, z and gradient buffers; the handle
 * owns its factor and workspace (allocated once by cyq_create).  Data
 * pointers are BORROWED: the solve and the residual read A, B (and, in
 * refinement mode, every block) again, so the data must stay valid and
 * unchanged from cyq_factor until the last cyq_solve / cyq_solve_adjoint.
 *
 * Errors.  Host-detectable errors are returned immediately.  Numerical
 * errors found on the device (a non-positive or non-finite Cholesky pivot,
 * refinement that did not reach the tolerance) are written to a per-instance
 * device status word; cyq_get_instance_status synchronises the stream and
 * copies it.  No kernel traps, asserts or waits without a bound.
 */
#ifndef CYQ_H
#define CYQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum cyq_status {
    CYQ_OK = 0,
    CYQ_ERR_INVALID_ARG = 1,   /* bad size, NULL pointer, unsupported shape */
    CYQ_ERR_NOT_PD = 2,        /* a stage or coupling Cholesky pivot <= 0 or not finite */
    CYQ_ERR_NOT_CONVERGED = 3, /* refinement stopped above tol after it_max steps */
    CYQ_ERR_CUDA = 4,          /* a CUDA runtime call failed (message: cyq_last_error) */
    CYQ_ERR_TIMEOUT = 5,       /* a bounded device wait expired */
    CYQ_ERR_NO_FACTOR = 6,     /* solve called before a successful factor */
    CYQ_ERR_UNIMPLEMENTED = 7,
    CYQ_ERR_NO_DEVICE = 8,     /* no CUDA device visible */
    CYQ_ERR_UPDATE_RANK = 9    /* (instance status) a factorization update carried more columns than its
                                  workspace holds: factor this instance again */
} cyq_status;

typedef enum cyq_precision {
    CYQ_FP64 = 0,          /* factor and solve in float64 (+ float64 refinement if it_max > 0) */
    CYQ_FP32_REFINE = 1,   /* float32 factor/solve, float64 residual + iterative refinement */
    CYQ_FP64_IR32 = 2      /* float64 factor and solve; refinement corrections by float32 sweeps with a
                              float32 copy of the factor (written by the float64 factorization), float64
                              residual; instances still above tol after it_max steps get up to esc_max
                              float64 corrections with the same factor */
} cyq_precision;

/* Opaque handle (host object owning device workspace). */
typedef struct cyq_handle_s *cyq_handle;
/* ABI-compatible with cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *cyq_stream;

/* Host-side description, read (and copied) by cyq_create. */
typedef struct cyq_desc {
    int32_t batch;          /* number of independent instances, >= 1 */
    const int32_t *N;       /* host array [batch]: horizon of each instance, >= 1 */
    const int32_t *nx;      /* host array [batch]: states, >= 1 */
    const int32_t *nu;      /* host array [batch]: inputs, >= 1 */
    int32_t precision;      /* cyq_precision */
    int32_t P;              /* horizon segments per instance; 0 = automatic.  Clamped to N. */
    const int32_t *P_per_instance; /* optional host array [batch] overriding P (NULL = none) */
    int32_t max_nrhs;       /* largest nrhs passed to cyq_solve, >= 1 */
    int32_t it_max;         /* max refinement steps; 0 = plain solve (no residual); < 0: default 10 */
    double tol;             /* relative KKT residual target, default 1e-10 if <= 0 */
    int32_t device;         /* CUDA device ordinal (the caller's current device if < 0) */
    int32_t esc_max;        /* float32 mode: float64 corrections after re-factoring, in float64,
                               the instances still above tol after it_max steps; 0 = none,
                               < 0: default 3.  Not available (treated as 0) when the float64
                               stage factor of some size class does not fit in shared memory */
    int32_t recompute_factors; /* 0 (default): every stage factor is stored by cyq_factor and
                               reused by every solve and adjoint (store_factors_for_adjoint).
                               1: the batch is planned as recompute_chunks consecutive chunks of
                               instances that share one stage-factor workspace of the largest
                               chunk; cyq_factor keeps only the statuses and the coupling
                               factors, and every cyq_solve / cyq_solve_adjoint factors each
                               chunk again just before its sweeps (stage-factor memory / chunks,
                               one more factorization per call) */
    int32_t recompute_chunks;  /* chunks of the recompute mode (0: 4; at most batch) */
    int32_t early_escalation;  /* float32 mode, 1: after two float32 corrections the instances
                               whose residual contracts too slowly to reach tol in the remaining
                               ones stop the float32 corrections and are factored in float64 on a
                               second stream while the others continue.  0 (default): every
                               instance takes the it_max float32 corrections first (on the uneven
                               batch both take the same time) */
    int32_t certify;           /* 0 (default): an instance stops once its float64 residual
                               ||b - Kz|| / ||b|| <= tol.  1: it stops only once that residual plus
                               2 gamma_m || |b| + |K||z| || / ||b|| (m = 2 nx + nu + 3; Higham,
                               Accuracy and Stability of Numerical Algorithms, Sec. 3.1) is
                               <= tol: then every float64 evaluation of the residual of the
                               returned z, in any summation order, is <= tol.  For ill-conditioned
                               instances that bound can lie far above 1e-10 (they then end
                               NOT_CONVERGED) */
} cyq_desc;

/*
 * Plans segments and launch shapes for every instance and allocates the
 * handle's device workspace (factors, Schur complement blocks, coupling
 * vectors, refinement buffers).  The only call that allocates.
 * Errors: INVALID_ARG (sizes), CUDA (allocation), NO_DEVICE.
 */
cyq_status cyq_create(const cyq_desc *desc, cyq_handle *out);

/* Frees the workspace (after synchronising the device). NULL is a no-op. */
void cyq_destroy(cyq_handle h);

/*
 * Factor K (eq. chol-fac-K-cyqlone): segment Riccati factors (Alg.
 * fact-mod-riccati), Schur complement blocks (Alg. fact-parallel-riccati-cr,
 * compute-schur) and their cyclic-reduction factor (factor-schur).  All data
 * pointers are device float64 arrays in the layout above; S and Sigma may be
 * NULL.  Asynchronous on `stream`.  A failed pivot sets the instance status
 * to CYQ_ERR_NOT_PD.  Errors returned: INVALID_ARG (NULL Q/R/A/B), CUDA.
 */
cyq_status cyq_factor(cyq_handle h, const double *Q, const double *R, const double *S,
                      const double *A, const double *B, const double *Sigma, cyq_stream stream);

/*
 * Solve K z = b for nrhs right-hand sides (1 <= nrhs <= max_nrhs) with the
 * last factor.  b and z are device float64 arrays of nrhs * kkt_size
 * elements (kkt_size = sum_i N_i (nu_i + 2 nx_i)); they must not overlap.
 * it_max = 0: one forward/backward substitution in the factor's precision.
 * it_max > 0: that solve, then up to it_max steps of  r = b - K z (float64),
 * dz = K~^{-1} r (stored factor K~), z += dz, stopping per instance once
 * ||r_j|| / ||b_j|| <= tol for every right-hand side j; an instance still
 * above tol gets status CYQ_ERR_NOT_CONVERGED.  Every decision is taken on
 * the device (no host synchronisation), so the call can be captured in a
 * CUDA graph.  Errors returned: INVALID_ARG, NO_FACTOR, CUDA.
 */
cyq_status cyq_solve(cyq_handle h, const double *b, double *z, int32_t nrhs, cyq_stream stream);

/*
 * One forward/backward substitution with the stored factor, without residual
 * or refinement: dz = K~^{-1} r for nrhs right-hand sides, where K~ is the
 * factor a refinement correction uses (the handle's factor; in CYQ_FP64_IR32
 * mode its float32 copy).  This is the correction step of the refinement loop
 * of cyq_solve on its own (e.g. to apply the factor as a preconditioner).
 * r and dz as b and z of cyq_solve (must not overlap).  Asynchronous.
 * Errors returned: INVALID_ARG, NO_FACTOR, CUDA.
 */
cyq_status cyq_apply_factor(cyq_handle h, const double *r, double *dz, int32_t nrhs, cyq_stream stream);

/*
 * Factorization update (Sec. 6, Alg. fact-mod-riccati-update): turns the
 * stored factor into the factor of the KKT matrix whose stage matrices are
 *   H~_s = H_s + sum_r delta_{s,r} w_{s,r} w_{s,r}^T      (s = 0 .. N-1)
 * without factoring the data again (e.g. the constraint rows whose activity
 * changed between two augmented-Lagrangian Newton iterations, eq.
 * low-rank-update-Hj).  Stage s's matrix couples (u^s, x^s) for s >= 1 and
 * (u^0, x^N) for s = 0, so w_{s,r} has nu + nx entries [u part | x part]; at
 * s = 0 every row must be zero in its u part or in its x part (a row of D_0
 * or of C_N).  Each row is applied by sigma-orthogonal rotations (Givens for
 * delta > 0, hyperbolic for delta < 0) and carried to the earlier stages
 * through the dynamics, so the rank per stage grows with the rows added on the
 * way; the single coupling block is factored again.  One-segment handles only.
 *   Q, R, S: device float64 data of the updated problem (same layout as for
 *   cyq_factor; S may be NULL): the residual and refinement of later solves
 *   read them (A, B, Sigma of the last cyq_factor stay bound).
 *   w: device float64, per instance (in instance order) N * m_max rows of
 *   nu + nx entries, stage-major; delta: device float64, N * m_max per
 *   instance; a row with delta = 0 is skipped.
 * Instance status: CYQ_ERR_NOT_PD if a downdate leaves a stage matrix
 * indefinite, CYQ_ERR_UPDATE_RANK if a stage carries more than max(32, nx)
 * update columns (refactor that instance).  Asynchronous.  The factor of the
 * handle's precision is updated (and the float32 copy of CYQ_FP64_IR32).
 * Errors returned: INVALID_ARG, NO_FACTOR, UNIMPLEMENTED (more than one
 * segment), CUDA.
 */
cyq_status cyq_update_factor(cyq_handle h, const double *Q, const double *R, const double *S, const double *w,
                             const double *delta, int32_t m_max, cyq_stream stream);

/*
 * b = -(r~, q, f~) for one right-hand side of the original problem
 * (eq. opt-cond-ocp-eq: r~^0 = r^0 + S_0 x_init, f~^0 = f^0 + A_0 x_init),
 * using the data passed to the last cyq_factor.  q, r, c, x_init are device
 * float64 arrays in the layout above; b has kkt_size elements.  Asynchronous
 * on `stream`.  Errors: INVALID_ARG (NULL handle or array), NO_FACTOR, CUDA.
 */
cyq_status cyq_build_rhs(cyq_handle h, const double *q, const double *r, const double *c,
                         const double *x_init, double *b, cyq_stream stream);

/*
 * Float64 residual  res = b - K z  and per-instance relative residual
 * ||res||_2 / ||b||_2 (rel, device float64 array [batch], may be NULL; res may
 * be NULL).  Uses the data of the last cyq_factor.  One right-hand side; b, z
 * and res are device arrays of kkt_size elements.  Asynchronous on `stream`.
 * Errors: INVALID_ARG (NULL handle, b or z), NO_FACTOR (no cyq_factor yet), CUDA.
 */
cyq_status cyq_residual(cyq_handle h, const double *b, const double *z, double *res, double *rel,
                        cyq_stream stream);

/*
 * The same residual with every row evaluated compensated: each product split
 * exactly with a fused multiply-add and the row's sum carried in two parts
 * (the error-free transformations of Ogita, Rump and Oishi's Dot2), then
 * rounded once, so res and rel are as accurate as if computed in twice the
 * float64 precision.  Where a row's terms cancel by many orders of magnitude a
 * plain float64 evaluation (cyq_residual) can be as large as the residual
 * itself; this one is not.  About ten float64 instructions per term instead of
 * one.  Same arguments and errors as cyq_residual.
 */
cyq_status cyq_residual_compensated(cyq_handle h, const double *b, const double *z, double *res, double *rel,
                                    cyq_stream stream);

/*
 * Adjoint of z = K^{-1} b(theta) (implicit differentiation of K z = b).
 * Given z (the solution for the right-hand side built from x_init) and
 * dL_dz, solves K w = dL_dz with the stored factor (K is symmetric) and
 * returns dL/dtheta:
 *   dq_k = -w_x^k, dr_k = -w_u^k, dc_k = -w_l^k,
 *   dQ_k = -sym(w_x^k x^k^T), dR_k = -sym(w_u^k u^k^T),
 *   dS_k = -(w_u^k x^k^T + u^k w_x^k^T), dA_k = -(w_l^k x^k^T + lambda^k w_x^k^T),
 *   dB_k = -(w_l^k u^k^T + lambda^k w_u^k^T), with x^0 = x_init for k = 0
 *   (dS_0 = -w_u^0 x_init^T, dA_0 = -w_l^0 x_init^T), dx_init = -S_0^T w_u^0 - A_0^T w_l^0,
 *   dSigma_u^k = -w_u^k .* u^k, dSigma_x^k = -w_x^k .* x^k.
 * Every output is a device float64 array in the data layout (w: kkt_size);
 * entries that do not enter K (dQ_0, dq_0, dSigma_x^0, dSigma_u^N) are set to
 * zero; any output pointer may be NULL, except w on a handle that refines
 * (it_max > 0: the refinement's own vectors are in use).  One right-hand side.
 * Asynchronous on `stream`.  Errors: INVALID_ARG (NULL handle, x_init, z or
 * dL_dz; NULL w with it_max > 0), NO_FACTOR, the errors of cyq_solve, CUDA.
 */
cyq_status cyq_solve_adjoint(cyq_handle h, const double *x_init, const double *z, const double *dL_dz,
                             double *w, double *dQ, double *dq, double *dR, double *dr, double *dS,
                             double *dA, double *dB, double *dc, double *dx_init, double *dSigma,
                             cyq_stream stream);

/* Synchronises `stream` and copies the per-instance status words
 * (cyq_status values) into host_status[batch]. Returns the first non-OK one,
 * or INVALID_ARG (NULL handle or array) or CUDA. */
cyq_status cyq_get_instance_status(cyq_handle h, int32_t *host_status, cyq_stream stream);

/* Statistics of the last cyq_solve (host copy; synchronises `stream`). */
typedef struct cyq_stats {
    int32_t refine_steps;    /* corrections applied (max over instances) */
    double max_rel_residual; /* max over instances and rhs of ||b - Kz|| / ||b|| (-1 if it_max = 0) */
    double max_certified;    /* cyq_desc.certify = 1: max over instances and rhs of the certified
                                stop value ||b - Kz|| / ||b|| + 2 gamma_m || |b| + |K||z| || / ||b||,
                                m = 2 nx + nu + 3 (the largest value any float64 evaluation of the
                                residual of the returned z can give), evaluated where the residual
                                reached tol; -1 if it_max = 0 or certify = 0 */
    int32_t P_min, P_max;    /* segments per instance chosen by the plan */
    int64_t work_items;      /* (instance, segment) pairs */
} cyq_stats;
/* Errors: INVALID_ARG (NULL handle or out), CUDA. */
cyq_status cyq_get_stats(cyq_handle h, cyq_stats *out, cyq_stream stream);

/* Device bytes the handle allocated (its workspace: stage factors, coupling
 * blocks, refinement vectors, plans; the recompute mode's chunks included).
 * -1 for NULL.  Host-only, no synchronisation. */
int64_t cyq_workspace_bytes(cyq_handle h);

/* Number of float64 elements of one right-hand side (sum_i N_i (nu_i + 2 nx_i)). */
int64_t cyq_kkt_size(cyq_handle h);
/* Segments chosen for each instance (host array [batch]).  Errors: INVALID_ARG. */
cyq_status cyq_get_segments(cyq_handle h, int32_t *P_out);
/*
 * The stages of segment c of a horizon of N stages cut into P segments, in the
 * order the factorization processes them (Sec. 4.1, eq. block-matrix-example-4:
 * block column c >= 1 holds the stages b(c-1)+1 .. b(c), b(c) = floor(c N / P),
 * in reverse order; block column 0 holds stage 0, whose u^0 is paired with x^N,
 * then the last stages N-1 .. b(P-1)+1, indices taken modulo N).  *len receives
 * the count; stages (host, at least *len entries) may be NULL to ask for it.
 * The kernels walk their segments with the same rule.  Host only, no device.
 * Errors: INVALID_ARG (N < 1, P < 1, P > N, c outside 0..P-1, NULL len).
 */
cyq_status cyq_segment_stages(int32_t N, int32_t P, int32_t c, int32_t *stages, int32_t *len);
/*
 * Diagnostics: the stored factor of one stage (instance, stage s in 0..N-1),
 * copied to the host as (nu+nx) x (nu+nx) float64, column-major.  Its lower
 * triangle is the Cholesky factor [L^R 0; L^S L^Q] of the stage matrix H^_s of
 * Alg. fact-mod-riccati (stage 0 pairs u^0 with x^N); its strict upper triangle
 * holds L^{R-1} (and, at the first stage of a segment, L^{Q-1}), transposed.
 * Within segment 0, L^Q_s L^Q_s^T is the Riccati cost-to-go matrix P_s of
 * x^s (P_N for stage 0).  Synchronises the device.  Errors: INVALID_ARG,
 * NO_FACTOR, CUDA.
 */
cyq_status cyq_get_stage_factor(cyq_handle h, int32_t instance, int32_t stage, double *L_out);

/*
 * Diagnostics: the Cholesky pivot routine of the stage factorizations applied
 * element-wise: l[i] = sqrt(d[i]), il[i] = 1 / sqrt(d[i]) for positive finite
 * d (float64: a float32 estimate refined by a float64 series, with the library
 * routines outside [2^-120, 2^120]; float32: rsqrtf and one Newton step).
 * d, l, il (float64) and df, lf, ilf (float32) are device arrays of n
 * elements; either triple may be NULL.  Asynchronous on `stream`.
 * Errors: INVALID_ARG (n < 0, missing outputs), CUDA.
 */
cyq_status cyq_pivot_eval(const double *d, double *l, double *il, const float *df, float *lf, float *ilf,
                          int64_t n, cyq_stream stream);

/* Number of kernels launched by the last cyq_factor and cyq_solve calls. */
int64_t cyq_last_launch_count(cyq_handle h);

/*
 * Launch-shape autotuner (the paper tunes its SIMD width and segment count
 * per problem size, Sec. 5; here the GPU analogue).  For every size class of
 * the handle, times the stage factorization with 16, 32, 64 and 128 threads per
 * work item and the two solve sweeps with 32 to 256 threads per work item
 * (nrhs right-hand sides b), `reps` launches each (default 3 if < 1), with
 * CUDA events on `stream` (the stage factorization also with 16 threads, two
 * items per warp, where their shared memory fits in one CTA), and keeps the
 * fastest shapes in the handle: the
 * stage factor's for every later cyq_factor, the sweeps' for every later
 * cyq_solve with this nrhs.  Binds and factors the data like cyq_factor and
 * leaves the handle factored; z (nrhs * kkt_size) is scratch.  Synchronises
 * the stream.  Results do not depend on the shapes (the same arithmetic in
 * the same order per work item).  Errors: INVALID_ARG, CUDA.
 */
cyq_status cyq_autotune(cyq_handle h, const double *Q, const double *R, const double *S,
                        const double *A, const double *B, const double *Sigma, const double *b,
                        double *z, int32_t nrhs, int32_t reps, cyq_stream stream);

/* Launch shapes in use: threads per work item of the stage factor and of the
 * sweeps (for nrhs right-hand sides) per size class; arrays of *n_groups
 * entries (either may be NULL; call with both NULL to get *n_groups).
 * Errors: INVALID_ARG (NULL handle or n_groups). */
cyq_status cyq_get_launch_shapes(cyq_handle h, int32_t *n_groups, int32_t *factor_team,
                                 int32_t *sweep_team, int32_t nrhs);

/* Set the launch shapes explicitly (e.g. ones tuned earlier): arrays of one
 * entry per size class (cyq_get_launch_shapes gives the count); 0 restores
 * the default of that class; the sweep shapes apply to cyq_solve calls with
 * nrhs right-hand sides.  Either array may be NULL (left unchanged).
 * Allowed values: factor 16 (two items per warp, where their shared memory fits
 * in one CTA), 32, 64, 128; sweeps 32, 64, 128, 256.
 * Errors: INVALID_ARG. */
cyq_status cyq_set_launch_shapes(cyq_handle h, const int32_t *factor_team, const int32_t *sweep_team,
                                 int32_t nrhs);

/*
 * Segment-count tuner.  Starting from desc's segment counts (automatic where
 * desc->P = 0 and no P_per_instance), tries the counts scaled by 1/4, 1/2, 1,
 * 2 and 4 (clamped to [1, N_i]), each in a temporary handle: one untimed
 * factor + solve, then `reps` (default 2 if < 1) timed factor + solve with
 * nrhs right-hand sides b (refinement as set in desc).  Writes to P_out (host
 * array [batch], for use as desc->P_per_instance) the fastest counts among the
 * candidates that leave the fewest instances with a non-OK status (not solved
 * to desc->tol, or not positive definite).
 * Allocates and frees a handle per candidate (a candidate whose workspace
 * cannot be allocated is skipped); z is scratch; synchronises the stream.
 * Errors: INVALID_ARG, CUDA and the errors of cyq_create / cyq_solve.
 */
cyq_status cyq_tune_segments(const cyq_desc *desc, const double *Q, const double *R, const double *S,
                             const double *A, const double *B, const double *Sigma, const double *b,
                             double *z, int32_t nrhs, int32_t reps, cyq_stream stream, int32_t *P_out);

/*
 * Allocation-free factor + solve of ONE OCP in float64 (one segment, one
 * right-hand side).  The paper has no counterpart: this entry point exists
 * for callers that must not allocate device memory while they run (a
 * real-time control loop that allocates only at start-up, a host whose device
 * memory belongs to another runtime or allocator).  Its workspace is one fixed
 * array of 2^20 doubles (8 MiB) in the library's device image, held on every
 * GPU that loads the library until the process exits; it calls no allocator.
 *   Inputs: N, nx, nu and device float64 data Q, R, S (or NULL), A, B, Sigma
 *   (or NULL) of one instance in the layout above, and the right-hand side b
 *   (N (nu + 2 nx) elements).  Outputs: the solution z (same size, must not
 *   overlap b) and, if status is not NULL, one device int32 status word
 *   (CYQ_OK or CYQ_ERR_NOT_PD).
 *   Size limit: N (nu+nx)^2 + N nx (nu+nx) + N (nu+nx) + 5 nx^2 + 3 nx (+ padding) must
 *   not exceed 2^20 doubles; larger problems return CYQ_ERR_INVALID_ARG with
 *   the needed size in cyq_last_error().
 *   The workspace is shared by every call on a device and keeps the last
 *   call's contents: calls that overlap on the GPU (different streams or host
 *   threads) race and must be serialised.  The first call on a device looks up
 *   the workspace address with that device current and keeps it for the life
 *   of the process (a device reset after it is not supported).  The plan
 *   records are written on the device by a small kernel.  Asynchronous on `stream` (the data pointers must
 *   stay valid until it completes).
 */
cyq_status cyq_factor_solve_noalloc(int32_t N, int32_t nx, int32_t nu, const double *Q, const double *R,
                                    const double *S, const double *A, const double *B, const double *Sigma,
                                    const double *b, double *z, int32_t *status, cyq_stream stream);

/*
 * Parallel cyclic reduction for the last levels of the coupling solve (App. A,
 * Alg. pcr; Sec. 7.5.2).  With levels = T > 0 the cyclic reduction of the
 * segment couplings stops T levels early; the blocks left (every 2^(L-T)-th of
 * an instance's P blocks, L = ceil(log2 max P)) are then all eliminated into
 * both of their neighbours at each of the T remaining levels, which leaves
 * them decoupled: the solve runs those levels forward only, without back
 * substitution.  T is clamped to L; T = 0 restores plain cyclic reduction.
 * Instances with one segment are unaffected.  Re-plans the handle (device
 * allocations; the previous plan's buffers are released by cyq_destroy); the
 * next cyq_solve needs a new cyq_factor (NO_FACTOR until then).  The solution
 * is the same up to rounding.  Errors: INVALID_ARG, CUDA.
 */
cyq_status cyq_set_pcr_tail(cyq_handle h, int32_t levels);
/* Tail levels in use (after clamping).  Errors: INVALID_ARG. */
cyq_status cyq_get_pcr_tail(cyq_handle h, int32_t *levels);

/*
 * Float32 factor path (CYQ_FP32_REFINE handles).  With one_warp_per_item = 1
 * (the default) every segment that carries no A^cl (segment 0 of every
 * instance, i.e. whole horizons when P = 1) whose padded blocks satisfy
 * nu <= 32, nx <= 64 is factored in one persistent launch for the whole batch,
 * each by a team of 32, 64 or 128 threads chosen by the shared memory it needs
 * (the modified Riccati recursion of Alg. fact-mod-riccati and the segment's
 * compute-schur blocks, same stored factor layout; the flag's name dates from
 * one warp per item); the other segments, and every segment when
 * one_warp_per_item = 0, run the per-size-class kernels.  Both paths compute
 * the same factor up to float32 rounding (different summation order).  The next cyq_solve needs a new cyq_factor.  Errors: INVALID_ARG.
 */
cyq_status cyq_set_factor_path(cyq_handle h, int32_t one_warp_per_item);
/* The float32 factor path in use and the number of work items the persistent
 * launch covers (0 for float64 handles); either pointer may be NULL.
 * Errors: INVALID_ARG (NULL handle). */
cyq_status cyq_get_factor_path(cyq_handle h, int32_t *one_warp_per_item, int64_t *warp_items);

/* Selects the float32 sweep path: 1 = each sweep of a float32 solve is one
 * persistent launch over the whole batch (k_sweep_team), 0 = one launch per
 * size class.  Both run the same per-item code with the same order of
 * operations, so they give the same solution bit for bit; the factor is kept.
 * Errors: INVALID_ARG (NULL handle, a value other than 0 / 1, or 1 for a batch
 * without a persistent sweep plan). */
cyq_status cyq_set_sweep_path(cyq_handle h, int32_t persistent);

/* The float32 sweep path in use: 1 if each sweep of a float32 solve is one
 * persistent launch over the whole batch (k_sweep_team), 0 for the per-class
 * launches, and the number of work items the persistent launch covers (0 if it
 * has none); either pointer may be NULL.  Errors: INVALID_ARG (NULL handle). */
cyq_status cyq_get_sweep_path(cyq_handle h, int32_t *persistent, int64_t *items);

/*
 * Float32 mode: segments per instance of the float64 escalation plan (host
 * array [batch]).  Instances of 24 or more stages whose float64 stage blocks
 * with the A^cl propagation fit in shared memory get up to 16 segments there
 * (halved runs of at least 12 stages), so the float64 factor of an escalated
 * long instance spreads over several SMs; 0 everywhere when the escalation
 * runs on the handle's own plan (other precisions, recompute mode, short
 * horizons).  Errors: INVALID_ARG (NULL).
 */
cyq_status cyq_get_escalation_segments(cyq_handle h, int32_t *host_P);

/*
 * Newton system of the augmented Lagrangian inner problem (Sec. 5, eqs.
 * ocp-al, ocp-al-funcs, qpalm-ocp-hessians, newton-sys-with-x0, elim-x0).
 *
 * The QP adds to the OCP the constraints bl <= C_k x^k + D_k u^k <= bu
 * (0 <= k < N) and bl <= C_N x^N <= bu, relaxed with multiplier estimates y,
 * diagonal penalties Sigma_k and proximal terms (1/2)|x - xbar|^2 in the
 * Gamma_x^{-1} norm and (1/2)|u - ubar|^2 in the Gamma_u^{-1} norm.  At the
 * iterate (u, x), x^0 = x_init, stage k's rows w = C_k x^k + D_k u^k are active
 * where w + Sigma_k^{-1} y^k lies outside [bl, bu]; Sigma^J is Sigma on the
 * active rows and 0 elsewhere, y^ = y + Sigma (w - Pi(w + Sigma^{-1} y; [bl, bu])),
 * and the call writes
 *   Q~_k = Q_k + C_k^T Sigma^J C_k + Gamma_x^{-1}      (k = 0..N)
 *   R~_k = R_k + D_k^T Sigma^J D_k + Gamma_u^{-1},  S~_k = S_k + D_k^T Sigma^J C_k
 *   r~_k = R_k u^k + S_k x^k + r_k + D_k^T y^_k + Gamma_u^{-1}(u^k - ubar^k)
 *   q~_k = Q_k x^k + S_k^T u^k + q_k + C_k^T y^_k + Gamma_x^{-1}(x^k - xbar^k)
 *          (no S term at k = N)
 *   c~_k = B_k u^k + A_k x^k + f_k - x^{k+1}
 * in the data layout of the OCP, so that the Newton step (du, dx, lambda) is
 * cyq_factor(Q~, R~, S~, A, B, Sigma = NULL) and cyq_solve of
 * cyq_build_rhs(q~, r~, c~, x_init = 0) (dx^0 = 0).
 *
 * Layout (device float64 unless noted; per instance, instances concatenated
 * kind by kind; blocks column-major): C (N+1) blocks ny x nx, D N blocks
 * ny x nu, bl / bu / y / sigma (N+1) ny, gx nx and gu nu (diagonals of
 * Gamma_x^{-1} and Gamma_u^{-1}; NULL: no proximal term, then xbar / ubar are
 * not read), xbar (N+1) nx, ubar N nu; u N nu, x (N+1) nx (x^0 not read);
 * q, r, c (= f), x_init as for cyq_build_rhs.  ny is a HOST array [batch]
 * (rows per stage, >= 1).  Outputs: Q, R, S as the data, q (N+1) nx, r N nu,
 * c N nx, active (int32, 1 = active; may be NULL) and yhat (may be NULL)
 * (N+1) ny.  Every input pointer other than S, gx, gu, xbar, ubar must be
 * non-NULL, as must the six block and vector outputs; the outputs must not
 * overlap the inputs.  The handle supplies the dimensions (no factorization
 * needed).  Asynchronous on `stream`, except that the first call with a given
 * ny array synchronises the stream and uploads the per-instance offsets it
 * implies: make that call before capturing later ones in a CUDA graph.
 * Errors: INVALID_ARG (null pointer, ny < 1, N + 1 > 65535, a stage's
 * [D C] rows too large for shared memory), CUDA.
 */
typedef struct cyq_newton_in {
    const double *Q, *R, *S, *A, *B;
    const double *q, *r, *c, *x_init;
    const double *u, *x;
    const int32_t *ny;
    const double *C, *D, *bl, *bu, *y, *sigma;
    const double *gx, *gu, *xbar, *ubar;
} cyq_newton_in;
typedef struct cyq_newton_out {
    double *Q, *R, *S, *q, *r, *c;
    int32_t *active;
    double *yhat;
} cyq_newton_out;
cyq_status cyq_assemble_newton(cyq_handle h, const cyq_newton_in *in, const cyq_newton_out *out,
                               cyq_stream stream);

const char *cyq_status_string(cyq_status s);
/* Text of the last CUDA error seen by this thread's calls ("" if none). */
const char *cyq_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CYQ_H */
