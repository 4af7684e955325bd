// Internal declarations of the cyq CUDA library: plan records, segment
// geometry and the team-cooperative dense block primitives used by the
// kernels.  A "team" is one CTA of TEAM threads working on one unit of work
// (a horizon segment of one instance, or one cyclic-reduction block); all
// matrices live in shared memory, column-major with an explicit leading
// dimension, and have runtime sizes.
#pragma once

#include <cuda_runtime.h>
#include <type_traits>
#include <stdint.h>

#include <string>

namespace cyq {

// ---------------------------------------------------------------------------
// Plan records (device copies built by cyq_create)
// ---------------------------------------------------------------------------
struct Inst {
    int N, nx, nu, P;
    int item0;       // first work item of this instance
    int pad0;
    long long oQ, oR, oS, oA, oB, oSig;  // offsets into the data arrays (doubles)
    long long oZ;                        // offset into b / z (doubles)
    long long oL, oLB, oF;               // offsets into the factor arrays (elements)
    long long oDI;                       // offset into the reciprocal-diagonal array (N*(nx+nu) elements)
    long long oBA;                       // offset into the float32 [B A] copy (N*nx*(nx+nu) elements)
    long long oBlk;                      // offset of the P coupling blocks (nx*nx each)
    long long oVec;                      // offset of the P coupling vectors (nx each)
    long long oq, orv, oc, ox0;          // offsets of q ((N+1) nx), r (N nu), c (N nx), x_init (nx)
    long long oHf;                       // offset of the float32 stage matrices of segment 0 (padded tiles)
    long long oN;                        // stages of the instances before this one (sum of N)
    long long oNn;                       // sum of N (nu + nx) of the instances before this one
};

// Stage shapes (nx, nu) for which float32 kernels are also compiled with fixed
// dimensions (loops unrolled, index arithmetic folded); a launch whose work
// items all have one of these shapes uses them.  Entry 0 stands for any shape.
struct StageShape {
    int nx, nu;
};
constexpr StageShape kStageShapes[] = {{0, 0}, {8, 4}, {12, 4}, {24, 8}, {32, 16}};
constexpr int kNumStageShapes = sizeof(kStageShapes) / sizeof(kStageShapes[0]);
inline int stage_shape_index(int nx, int nu) {
    for (int i = 1; i < kNumStageShapes; ++i)
        if (kStageShapes[i].nx == nx && kStageShapes[i].nu == nu) return i;
    return 0;
}

struct Item {
    int inst, seg;
};

// Data pointers of the last factor call (borrowed, float64).
struct Data {
    const double *Q, *R, *S, *A, *B, *Sig;
};

// Device status codes (mirror cyq_status).
enum : int { ST_OK = 0, ST_NOT_PD = 2, ST_NOT_CONVERGED = 3, ST_RANK = 9 };

// Segment c of an instance with horizon N split into P segments: boundaries
// b(c) = floor(c N / P).  Segment c >= 1 holds stages b(c-1)+1 .. b(c);
// segment 0 holds stage 0 (u^0 paired with x^N) and stages b(P-1)+1 .. N-1.
// Stages are processed backward: s(t) = (b(c) - t) mod N, t = 0..len-1
// (Alg. fact-mod-riccati with indices reduced modulo N).
__host__ __device__ inline int seg_bound(int c, int N, int P) {
    return (int)(((long long)c * N) / P);
}
__host__ __device__ inline int seg_len(int c, int N, int P) {
    return c == 0 ? N - seg_bound(P - 1, N, P) : seg_bound(c, N, P) - seg_bound(c - 1, N, P);
}
__host__ __device__ inline int seg_stage(int c, int t, int N, int P) {
    int s = seg_bound(c, N, P) - t;
    return s < 0 ? s + N : s;
}
// Index of the state paired with stage s (x^s, or x^N for s = 0).
__host__ __device__ inline int xstate(int s, int N) { return s == 0 ? N : s; }

// ---------------------------------------------------------------------------
// Team primitives
// ---------------------------------------------------------------------------
__device__ __forceinline__ void team_sync() { __syncthreads(); }

// Compile-time loop: f(std::integral_constant<int, I>) for I = B .. E-1, so
// that register arrays are only ever indexed by constants.
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F &&f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// A team is the group of threads that works on one item: the whole CTA when
// TEAM >= 32, else TEAM consecutive lanes of a warp (several teams per warp,
// whose instructions then serve several items at once).  Thread index within
// the team, and a barrier over the team only.
template <int TEAM>
__device__ __forceinline__ int team_tid() {
    return TEAM >= 32 ? (int)threadIdx.x : (int)(threadIdx.x & (TEAM - 1));
}
template <int TEAM>
__device__ __forceinline__ void team_sync() {
    if constexpr (TEAM >= 32)
        __syncthreads();
    else
        __syncwarp(((1u << TEAM) - 1u) << (threadIdx.x & 31 & ~(TEAM - 1)));
}

// Element e of the lower triangle (diagonal included) of an n x n matrix in
// row order: row r holds r + 1 entries.  Returns (r, c) with c <= r.
__device__ __forceinline__ void tri_index(int e, int &r, int &c) {
    int rr = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while ((rr + 1) * (rr + 2) / 2 <= e) ++rr;
    while (rr * (rr + 1) / 2 > e) --rr;
    r = rr;
    c = e - rr * (rr + 1) / 2;
}

// Leading dimension of a shared-memory tile with `rows` rows: rounded up to an
// odd number, so that threads walking a row (stride = ld) hit distinct banks.
__host__ __device__ __forceinline__ int pad_ld(int rows) { return rows | 1; }

// Column-major walk of an m x n grid: element e = threadIdx.x, then steps of
// `step`; (r, c) advance without integer division.
__device__ __forceinline__ void rect_start(int e, int m, int &r, int &c) {
    c = e / m;
    r = e - c * m;
}
__device__ __forceinline__ void rect_advance(int &r, int &c, int m, int step) {
    r += step;
    while (r >= m) {
        r -= m;
        ++c;
    }
}

// Move (r, c) forward by `step` elements in that row order.  Threads start
// at tri_index(threadIdx.x) and step by the team size, so the mapping is
// computed once instead of once per element.
__device__ __forceinline__ void tri_advance(int &r, int &c, int step) {
    c += step;
    while (c > r) {
        c -= r + 1;
        ++r;
    }
}

// Cholesky pivots.  An FP64 instruction costs the same whether one or all 32
// lanes run it, and the library's double sqrt and division are sequences of
// ~10 and ~7 FP64 operations, so the pivot d -> (sqrt(d), 1/sqrt(d)) is built
// from a single-precision estimate and a short FP64 correction:
//   y0 = rsqrtf(d) (d truncated to float with integer operations),
//   e  = 1 - d y0^2,   y = y0 (1 + e/2 + 3e^2/8)
// (the series of (1-e)^{-1/2}; |e| < 2^-20 leaves a truncation error below
// 2^-60, so y is within ~1 ulp of 1/sqrt(d)), and sqrt(d) = d y.  Pivots
// outside [2^-120, 2^120] use the library routines.
__device__ __forceinline__ bool finite_pos(double d) { return d > 0.0 && d < 1.0 / 0.0; }
__device__ __forceinline__ bool finite_pos(float d) { return d > 0.0f && d < 1.0f / 0.0f; }

__device__ __forceinline__ void pivot(double d, double &l, double &il) {
    const int hi = __double2hiint(d), lo = __double2loint(d);
    const int ex = (hi >> 20) & 0x7ff;
    if (ex > 1023 - 120 && ex < 1023 + 120) {
        const int fbits = ((ex - 896) << 23) | ((hi & 0xfffff) << 3) | ((unsigned)lo >> 29);
        const float r = rsqrtf(__int_as_float(fbits));
        const int rb = __float_as_int(r);
        const int rex = ((rb >> 23) & 0xff) + 896;
        const double y0 = __hiloint2double((rex << 20) | ((rb & 0x7fffff) >> 3), (rb & 0x7) << 29);
        const double t = d * y0;
        const double e = fma(-t, y0, 1.0);
        const double c = fma(e, 0.375, 0.5);
        const double y = fma(y0, e * c, y0);
        il = y;
        l = d * y;
    } else {
        l = sqrt(d);
        il = 1.0 / l;
    }
}
__device__ __forceinline__ void pivot(float d, float &l, float &il) {
    float y = rsqrtf(d);
    y = y * fmaf(-0.5f * d * y, y, 1.5f);   // one Newton step
    il = y;
    l = d * y;
}

// Asynchronous global -> shared copies (8-byte elements, any alignment of doubles).
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <int TEAM>
__device__ __forceinline__ void async_copy_f64(double *dst, const double *src, int count) {
    for (int e = team_tid<TEAM>(); e < count; e += TEAM) cp_async8(dst + e, src + e);
}

// 16-byte asynchronous copies (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
// count doubles (even), dst and src 16-byte aligned, as pairs.
template <int TEAM>
__device__ __forceinline__ void async_copy_f64x2(double *dst, const double *src, int count) {
    for (int e = 2 * team_tid<TEAM>(); e < count; e += 2 * TEAM) cp_async16(dst + e, src + e);
}

// In-place lower Cholesky factor of the n x n matrix A (lower triangle read;
// upper triangle set to zero).  Right-looking: per column a pivot, a scaled
// column and a rank-1 update of the trailing lower triangle.  Every thread
// computes the pivot (an FP64 instruction costs the same on one lane as on
// all).  dinv[k] receives 1/L_kk when dinv is not null.  Returns false if a
// pivot was not positive and finite (that pivot is replaced by 1 so that the
// arithmetic stays finite).
template <typename T, int TEAM>
__device__ bool team_chol(T *A, int n, int ld, T *dinv = nullptr) {
    const int tid = team_tid<TEAM>();
    int r0, c0;
    tri_index(tid, r0, c0);
    bool ok = true;
    for (int k = 0; k < n; ++k) {
        T d = A[k + k * ld];
        if (!finite_pos(d)) { ok = false; d = T(1); }
        T l, il;
        pivot(d, l, il);
        team_sync<TEAM>();   // everyone has read A[k,k]
        if (tid == 0) {
            A[k + k * ld] = l;
            if (dinv) dinv[k] = il;
        }
        for (int i = k + 1 + tid; i < n; i += TEAM) A[i + k * ld] *= il;
        for (int i = tid; i < k; i += TEAM) A[i + k * ld] = T(0);   // upper part of column k
        team_sync<TEAM>();
        const int m = n - k - 1;                 // trailing size
        for (int r = r0, c = c0; r < m; tri_advance(r, c, TEAM)) {
            const int rr = r + k + 1, cc = c + k + 1;
            A[rr + cc * ld] = fma(-A[rr + k * ld], A[cc + k * ld], A[rr + cc * ld]);
        }
        team_sync<TEAM>();
    }
    return ok;
}

// X (m x n, ldx) := X * L^{-T}, L lower n x n (ldl): row-wise forward substitution
// (X L^T = Y).  One thread per row.  dinv (optional) holds 1/L_jj.
template <typename T, int TEAM>
__device__ void team_trsm_rlt(T *X, int m, int n, int ldx, const T *L, int ldl, const T *dinv = nullptr) {
    for (int r = team_tid<TEAM>(); r < m; r += TEAM) {
        for (int j = 0; j < n; ++j) {
            T s = X[r + j * ldx];
            for (int t = 0; t < j; ++t) s = fma(-X[r + t * ldx], L[j + t * ldl], s);
            X[r + j * ldx] = dinv ? s * dinv[j] : s / L[j + j * ldl];
        }
    }
    team_sync<TEAM>();
}

// Tinv (n x n, ldt) := L^{-1} for lower L (n x n, ldl); one thread per column.
template <typename T, int TEAM>
__device__ void team_trtri_lower(T *Tinv, int ldt, const T *L, int ldl, int n, const T *dinv = nullptr) {
    for (int c = team_tid<TEAM>(); c < n; c += TEAM) {
        for (int i = 0; i < c; ++i) Tinv[i + c * ldt] = T(0);
        for (int i = c; i < n; ++i) {
            T s = (i == c) ? T(1) : T(0);
            for (int t = c; t < i; ++t) s = fma(-L[i + t * ldl], Tinv[t + c * ldt], s);
            Tinv[i + c * ldt] = dinv ? s * dinv[i] : s / L[i + i * ldl];
        }
    }
    team_sync<TEAM>();
}

// C (m x n, ldc) (op)= A (m x k, lda) * B (k x n, ldb).  Mode: 0 assign, 1 add, -1 subtract.
template <typename T, int TEAM>
__device__ void team_gemm_nn(T *C, int ldc, const T *A, int lda, const T *B, int ldb, int m, int n, int k,
                             int mode) {
    int r, c;
    rect_start(team_tid<TEAM>(), m, r, c);
    for (; c < n; rect_advance(r, c, m, TEAM)) {
        T s = mode == 0 ? T(0) : C[r + c * ldc];
        const T *a = A + r, *b = B + c * ldb;
        if (mode >= 0) {
#pragma unroll 4
            for (int t = 0; t < k; ++t) s = fma(a[t * lda], b[t], s);
        } else {
#pragma unroll 4
            for (int t = 0; t < k; ++t) s = fma(-a[t * lda], b[t], s);
        }
        C[r + c * ldc] = s;
    }
    team_sync<TEAM>();
}

// C (m x n) (op)= A (m x k) * B^T (B is n x k, ldb).
template <typename T, int TEAM>
__device__ void team_gemm_nt(T *C, int ldc, const T *A, int lda, const T *B, int ldb, int m, int n, int k,
                             int mode) {
    int r, c;
    rect_start(team_tid<TEAM>(), m, r, c);
    for (; c < n; rect_advance(r, c, m, TEAM)) {
        T s = mode == 0 ? T(0) : C[r + c * ldc];
        const T *a = A + r, *b = B + c;
        if (mode >= 0) {
#pragma unroll 4
            for (int t = 0; t < k; ++t) s = fma(a[t * lda], b[t * ldb], s);
        } else {
#pragma unroll 4
            for (int t = 0; t < k; ++t) s = fma(-a[t * lda], b[t * ldb], s);
        }
        C[r + c * ldc] = s;
    }
    team_sync<TEAM>();
}

// Lower triangle of C (n x n) (op)= A A^T, A is n x k.
template <typename T, typename TC, int TEAM>
__device__ void team_syrk_lower(TC *C, int ldc, const T *A, int lda, int n, int k, int mode) {
    int r, c;
    tri_index(team_tid<TEAM>(), r, c);
    for (; r < n; tri_advance(r, c, TEAM)) {
        T s = T(0);
        const T *a = A + r, *b = A + c;
#pragma unroll 4
        for (int t = 0; t < k; ++t) s = fma(a[t * lda], b[t * lda], s);
        TC *o = C + r + c * ldc;
        *o = mode == 0 ? (TC)s : (mode > 0 ? *o + (TC)s : *o - (TC)s);
    }
    team_sync<TEAM>();
}

// Mirror the lower triangle of an n x n matrix into its upper triangle.
template <typename T, int TEAM>
__device__ void team_symmetrize(T *C, int ldc, int n) {
    const int cnt = n * n;
    for (int e = team_tid<TEAM>(); e < cnt; e += TEAM) {
        const int r = e % n, c = e / n;
        if (c > r) C[r + c * ldc] = C[c + r * ldc];
    }
    team_sync<TEAM>();
}

// ---------------------------------------------------------------------------
// Host launchers (defined in the kernel translation units)
// ---------------------------------------------------------------------------
struct Plan;   // host plan (api.cu)

struct FactorArgs {
    const Inst *inst;
    const Item *items;
    int n_items;
    Data data;
    void *L, *LB, *F;               // factor arrays (float or double)
    void *DI;                       // reciprocal diagonals of the stage factors
    void *BAf;                      // optional float32 copy of every stage's [B A]
    // optional float32 copies of the stored factor written by a float64 factorization
    // (L, L^B, A^cl / L^A, reciprocal diagonals), for float32 correction sweeps
    float *Lc, *LBc, *Fc, *DIc;
    double *Mf, *Mb, *Kc;           // Schur blocks (float64)
    double *U, *Y;                  // cyclic-reduction factor blocks (float64)
    int *status;
    bool stage_in_smem;             // copy each stage's raw blocks to shared memory (cp.async)
    bool need_G2;                   // some item propagates A^cl (P > 1): second [B^ A^] buffer
    const int *skip;                // optional per-instance flag: nonzero = do not factor this instance
    unsigned smem_team;             // shared-memory bytes per team (set by the launcher)
    const float *Hf;                // float32 stage matrices (persistent team factor; written by the ingest)
};

struct SolveArgs {
    const Inst *inst;
    const Item *items;
    int n_items;
    Data data;
    const void *L, *LB, *F, *DI;
    const void *BA;                 // float32 [B A] copies (float32 factors); float64 sweeps read the data
    const double *Mf, *Kc, *U, *Y;  // coupling factor (Mf holds the CR Cholesky blocks)
    const double *b;                // right-hand sides (float64)
    double *z;                      // solutions (float64)
    long long kkt;                  // elements per right-hand side
    int nrhs;
    double *dF, *dB, *lam;          // coupling vectors (float64), [rhs][P*nx]
    long long nvec;                 // coupling-vector elements per right-hand side
    const int *skip;                // optional per-instance flag: nonzero = leave this instance alone
    double *zacc;                   // optional: add the solution into zacc (z then holds intermediates only)
    int nbuf;                       // stage packages in shared memory: 2 = prefetch the next stage, 1 = fetch after use
};

// Level-parallel cyclic reduction plan: jobs (instance, block).  The
// eliminations of level l are jobs[elim_off[l] .. elim_off[l+1]) and its
// updates jobs[upd_off[l] .. upd_off[l+1]); all eliminations come first in
// the array, then all updates.
struct CrJob {
    int inst, k;
};
struct CrPlan {
    int n_inst = 0;                 // instances with P > 1
    const int *inst_list = nullptr; // device
    const CrJob *jobs = nullptr;    // device
    int levels = 0;                 // cyclic-reduction levels (before the parallel tail)
    int elim_off[33] = {0}, upd_off[33] = {0};
    // parallel cyclic reduction of the last levels (tail = 0: none, block 0 is the base):
    // the blocks left are every s0-th one; jobs (instance, tail index) of tail level t are
    // jobs[pcr_off[t] .. pcr_off[t+1]), every tail block is in jobs[pcr_off[tail] .. pcr_base_end)
    int tail = 0, s0 = 1;
    int pcr_off[33] = {0};
    int pcr_base_end = 0;
    const long long *oT_dev = nullptr;    // per instance: offset of its tail factor blocks (doubles)
    const long long *oV_dev = nullptr;    // per instance: offset of its tail vectors (doubles, per rhs)
    double *Lt = nullptr, *At = nullptr, *Bt = nullptr;   // tail L, A, B per (level, tail block)
    double *bt = nullptr;                 // tail vectors L^{-1} b, [rhs][nvt]
    long long nvt = 0;
};

cudaError_t launch_factor_segments(bool fp64, int team, int shape, size_t smem, const FactorArgs &a, cudaStream_t st);

// Float32 factor with one team of threads per item (segments without A^cl,
// padded blocks nu + nx <= 96, nx <= 64, nu <= 32) in one persistent launch: three item
// classes by shared memory (one team of 128 threads per CTA, two of 64 or four
// of 32); teams take items from their class's counter, then from the classes
// of smaller items.
constexpr int kTeamCtaThreads = 128;
// CTAs of the persistent float32 factor per SM (each with a third of the SM's shared memory)
constexpr int kFactorCtasPerSm = 3;
// CTAs of the persistent float32 sweeps per SM (deeper package rings matter more here
// than a third CTA: measured on the uneven batch, 10.5 ms per correction with two, 20 with three)
constexpr int kSweepCtasPerSm = 2;
constexpr int kWarpMaxNp = 96;        // padded nu + nx
// rows a team of class c covers in the Crout factorization (threads x rows per thread:
// 128 x 1, 64 x 2, 32 x 2)
constexpr int kTeamRows[3] = {128, 128, 64};
constexpr int kWarpMaxNxp = 64;       // padded nx
struct TeamPlanDev {
    const Item *items = nullptr;      // class 0, 1, 2 items (each sorted longest first)
    int off[3] = {0, 0, 0}, n[3] = {0, 0, 0};
    int *counter = nullptr;           // three queue heads (zeroed before each launch)
    int g0 = 0, g1 = 0;               // CTAs [0, g0) serve class 0, [g0, g0 + g1) class 1, the rest class 2
    int arena_floats = 0;             // shared memory per CTA (floats)
};
size_t warp_slot_bytes(int nx, int nu);
size_t warp_stage_floats(int nx, int nu);   // floats of one ingested stage matrix
// Ingest of the persistent team factor's stages: float32 stage matrices in the padded
// tile layout and float32 [B A]; one warp per chunk of stages of segment 0.
struct IngestChunk {
    int inst, t0, t1;
};
struct IngestArgs {
    const Inst *inst;
    const IngestChunk *chunks;
    int n_chunks;
    Data data;
    float *Hf;                      // stage matrices
    float *BAf;                     // [B A] copies (may be null)
};
cudaError_t launch_ingest_f32(const IngestArgs &g, cudaStream_t st);
// L^{R-1} of every stage of the one-team factor's segments into the stored factor.
cudaError_t launch_inv_R_f32(const IngestArgs &g, float *L, const float *DI, cudaStream_t st);
cudaError_t launch_factor_team(const FactorArgs &a, const TeamPlanDev &plan, int grid, cudaStream_t st);
cudaError_t launch_cr_factor_levels(const CrPlan &plan, int team, int nmax, const FactorArgs &a, cudaStream_t st,
                                    long long *launches);
size_t cr_tail_smem_bytes(int nmax);
cudaError_t launch_solve_backward(bool fp64, int team, int shape, size_t smem, const SolveArgs &a, cudaStream_t st);
cudaError_t launch_cr_solve(int n_inst_cr, const int *inst_list, int team, size_t smem, const SolveArgs &a,
                            cudaStream_t st);
cudaError_t launch_solve_forward(bool fp64, int team, int shape, size_t smem, const SolveArgs &a, cudaStream_t st);
cudaError_t launch_cr_solve_levels(const CrPlan &plan, int nmax, const SolveArgs &a, cudaStream_t st,
                                   long long *launches);

struct Chunk {
    int inst, k0, k1;   // records [k0, k1) of one instance
};

struct ResidArgs {
    const Inst *inst;
    const Chunk *chunks;
    int n_chunks;
    Data data;
    const double *b, *z;
    double *r;          // may be null (norms only)
    double *rr, *bb;    // accumulators of squared norms, [rhs][instance]
    const int *skip;    // optional per-instance flag: an instance runs iff skip[i] == run_if
    int run_if;
    const int *comp;    // optional per-instance flag: 1 = evaluate the rows compensated
    const int *sel;     // (set by the launcher) an instance runs iff sel[i] == sel_val
    int sel_val;
    long long kkt;      // elements per right-hand side
    int batch;
    bool need_bb;       // accumulate ||b||^2 too (false: bb already holds it)
    int max_nx;         // largest nx of the batch (launch choice)
};

struct GradArgs {
    const Inst *inst;
    const Chunk *chunks;
    const double *x0, *z, *w;
    double *dQ, *dq, *dR, *dr, *dS, *dA, *dB, *dc, *dSig;
};

cudaError_t launch_residual(const ResidArgs &a, int nrhs, cudaStream_t st);
// || |b| + |K| |z| ||^2 per instance and right-hand side into a.rr (instances with skip[i] == run_if)
cudaError_t launch_residual_scale(const ResidArgs &a, int nrhs, cudaStream_t st);
cudaError_t launch_certify(const Inst *inst, int batch, int nrhs, double *aa, const double *bb, const double *rel,
                           double *cert, int *done, double tol, cudaStream_t st);
// done[i] = done_value once every right-hand side of instance i is at or below tol;
// comp (optional): set to 1 where a residual in (tol, 100 tol] stayed above 0.8 of the last step's
cudaError_t launch_resid_finalize(int batch, int nrhs, double *rr, double *bb, double *rel, int *done, double tol,
                                  int *steps, int step, bool keep_bb, int done_value, int *comp, cudaStream_t st);
cudaError_t launch_mark_not_converged(int batch, const int *done, int *status, cudaStream_t st);
cudaError_t launch_clear_not_pd(int batch, const int *skip, int *status, cudaStream_t st);
cudaError_t launch_fill_int(int n, int *p, int v, cudaStream_t st);
cudaError_t launch_predict_escalation(int batch, int nrhs, const double *rel0, const double *rel, int *done, int *esc,
                                      double tol, int k, int left, cudaStream_t st);
cudaError_t launch_unpark(int batch, int *done, cudaStream_t st);
// Factorization update (update.cu): low-rank modifications of the stage matrices
// applied to the stored factor of one-segment instances.
struct UpdateArgs {
    const Inst *inst;
    const int *inst_list;           // instances to update
    int n_inst;
    Data data;                      // float64 data (the [B A] that carries the update between stages)
    void *L, *LB, *DI;              // stored factor (float or double)
    float *Lc, *LBc, *DIc;          // float32 copy to refresh (float64 factor with float32 corrections), or null
    double *Mf, *Mb;                // coupling block factor and M_bwd
    const double *w, *delta;        // update rows: instance, stage, row (m_max per stage); w has nu + nx entries
    int m_max;                      // rows per stage in w / delta
    int mcap;                       // update columns a stage can carry (workspace)
    int max_nx, max_nu;
    int *status;
};
template <typename T>
size_t update_smem_bytes(int nx, int nu, int mcap);
cudaError_t launch_update_factor(bool fp64, const UpdateArgs &u, cudaStream_t st);

// Newton-system assembly of the augmented Lagrangian inner problem (newton.cu).
struct AlmOff {
    long long oC, oD, oY;   // offsets of C, D and the per-row vectors (bl, bu, y, sigma, active, y^)
    long long ogx, ogu;     // offsets of the Gamma^{-1} diagonals
    int ny, pad;
};
struct NewtonArgs {
    const Inst *inst;
    const AlmOff *off;
    const double *Q, *R, *S, *A, *B, *q, *r, *f, *x0, *u, *x;
    const double *C, *D, *bl, *bu, *y, *sig, *gx, *gu, *xbar, *ubar;
    double *Qo, *Ro, *So, *qo, *ro, *co, *yhat;
    int *active;
};
size_t newton_smem_bytes(int ny, int nx, int nu);
cudaError_t launch_newton_assemble(const NewtonArgs &a, int batch, int max_stages, size_t smem, cudaStream_t st);

cudaError_t launch_build_rhs(const Inst *inst, int batch, const Data &d, const double *q, const double *r,
                             const double *c, const double *x0, double *b, long long z_lo, long long z_n,
                             cudaStream_t st);
cudaError_t launch_adjoint(const GradArgs &g, int n_chunks, int batch, const Data &d, double *dx0, cudaStream_t st);

size_t factor_smem_bytes(bool fp64, int nx, int nu, bool staged, bool need_G2);
cudaError_t launch_pivot_eval(const double *d, double *l, double *il, const float *df, float *lf, float *ilf,
                              long long n, cudaStream_t st);
size_t factor_stage_bytes(int nx, int nu);

// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device (cached per kernel and device, so repeated launches -- and
// launches recorded into a CUDA graph -- make no attribute calls).
cudaError_t ensure_smem(const void *kernel, size_t bytes);

// Sets the text returned by cyq_last_error() for the calling thread.
void set_last_error_message(const char *msg);
inline void set_last_error_message(const std::string &msg) { set_last_error_message(msg.c_str()); }
__host__ __device__ size_t solve_smem_bytes(bool fp64, int nx, int nu, int nrhs, int nbuf);
// Float32 sweeps of every item in one persistent launch (backward or forward).
cudaError_t launch_sweep_team(bool backward, const SolveArgs &a, const TeamPlanDev &plan, int grid, cudaStream_t st);

}  // namespace cyq
