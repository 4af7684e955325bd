// Float64 KKT residual, iterative-refinement bookkeeping, right-hand-side
// assembly and adjoint gradient assembly.
//
// Residual rows (paper eq. opt-cond-ocp-eq, E_j = I), record k of z:
//   u^k      : R_k u^k + S_k x^k + B_k^T lambda^k                       (no S_0 term)
//   x^{k+1}  : Q_{k+1} x^{k+1} - lambda^k + S_{k+1}^T u^{k+1} + A_{k+1}^T lambda^{k+1}
//              (the last two terms only for k+1 < N)
//   lambda^k : B_k u^k + A_k x^k - x^{k+1}                              (no A_0 term)
// with Sigma added to the diagonals of R and Q.  Work is split into chunks
// of records; each chunk adds its squared norms into per-instance float64
// accumulators.
#include "cyq_internal.cuh"

namespace cyq {


// Rows are processed one kind at a time (u rows, then lambda rows, then x rows)
// so that a warp runs one code path: a divergent FP64 instruction costs a
// full warp slot per path.  The order keeps the second read of B_k (u and lambda
// rows) and of A_k (lambda rows of record k, x rows of record k - 1) close to
// the first, while the chunk's blocks are still in L2.  Up to RG right-hand
// sides share every matrix load.
constexpr int RG = 4;

// Accumulation of one residual row, b - sum_j m_j z_j, by mode:
//   kResidPlain  float64 fused multiply-adds;
//   kResidScale  |b| + sum_j |m_j| |z_j| (the scale of the rounding error of any
//                float64 evaluation of the row);
//   kResidComp   compensated: every product split exactly into q + e with a
//                fused multiply-add, the sum carried as hi + lo with Knuth's
//                TwoSum (the error-free transformations of Ogita, Rump and
//                Oishi's Dot2, SIAM J. Sci. Comput. 26, 2005), so the row is
//                as accurate as if computed in twice the working precision and
//                rounded once.  Used where the plain evaluation's rounding is
//                as large as the residual itself (refinement at its noise
//                floor).  The _rn intrinsics keep the compiler from fusing or
//                reassociating the transformations.
constexpr int kResidPlain = 0, kResidScale = 1, kResidComp = 2;

template <int MODE>
struct RowAcc;

template <>
struct RowAcc<kResidPlain> {
    double v;
    __device__ __forceinline__ void init(double x) { v = x; }
    __device__ __forceinline__ void mac(double m, double zv) { v = fma(m, zv, v); }
    __device__ __forceinline__ double finish(double b) const { return b - v; }
};

template <>
struct RowAcc<kResidScale> {
    double v;
    __device__ __forceinline__ void init(double x) { v = fabs(x); }
    __device__ __forceinline__ void mac(double m, double zv) { v = fma(fabs(m), fabs(zv), v); }
    __device__ __forceinline__ double finish(double b) const { return fabs(b) + v; }
};

__device__ __forceinline__ void two_sum(double a, double b, double &s, double &t) {
    s = __dadd_rn(a, b);
    const double bv = __dsub_rn(s, a);
    t = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bv)), __dsub_rn(b, bv));
}

template <>
struct RowAcc<kResidComp> {
    double hi, lo;
    __device__ __forceinline__ void init(double x) {
        hi = x;
        lo = 0.0;
    }
    __device__ __forceinline__ void mac(double m, double zv) {
        const double q = __dmul_rn(m, zv), e = __fma_rn(m, zv, -q);   // m zv = q + e exactly
        double s, t;
        two_sum(hi, q, s, t);
        hi = s;
        lo = __dadd_rn(lo, __dadd_rn(t, e));
    }
    __device__ __forceinline__ double finish(double b) const {
        double d, t;
        two_sum(b, -hi, d, t);
        return __dadd_rn(d, __dsub_rn(t, lo));
    }
};

#define CYQ_ROW_UNROLL _Pragma("unroll 4")
#define CYQ_RESID_KERNEL k_residual_long_rows
#include "resid_rows.inc"
#undef CYQ_ROW_UNROLL
#undef CYQ_RESID_KERNEL
#define CYQ_ROW_UNROLL
#define CYQ_RESID_KERNEL k_residual_short_rows
#include "resid_rows.inc"
#undef CYQ_ROW_UNROLL
#undef CYQ_RESID_KERNEL

// Per instance: rel[r] = ||res_r|| / ||b_r|| for each right-hand side r; the
// instance is done once every right-hand side is at or below tol (refinement
// runs per instance).  Clears the accumulators (||b||^2 stays when keep_bb:
// b does not change between the refinement steps of one solve).  steps[i] records the number
// of corrections an instance received so far.
__global__ void k_resid_finalize(int batch, int nrhs, double *rr, double *bb, double *rel, int *done, double tol,
                                 int *steps, int step, bool keep_bb, int done_value, int *comp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= batch) return;
    if (done && done[i]) return;
    bool all = true, stalled = false;
    for (int r = 0; r < nrhs; ++r) {
        const long long j = (long long)r * batch + i;
        const double rn = sqrt(rr[j]), bn = sqrt(bb[j]);
        const double v = bn > 0.0 ? rn / bn : rn;
        // a correction that left a residual within a factor 100 above tol above 0.8 of the
        // previous one: the float64 evaluation's rounding (or a very slow contraction) limits
        // it; later evaluations of the instance are compensated (noise floors lie far below
        // 100 tol otherwise)
        if (comp && step > 0 && !(v <= tol) && v <= 100.0 * tol && v > 0.8 * rel[j]) stalled = true;
        if (rel) rel[j] = v;
        all = all && (v <= tol);
        rr[j] = 0.0;
        if (!keep_bb) bb[j] = 0.0;
    }
    if (done && all) done[i] = done_value;
    if (stalled) comp[i] = 1;
    if (steps) steps[i] = step;
}

// Certified stop.  Any float64 evaluation of b - K z, in any summation order,
// differs from the exact residual by at most gamma_m (|b| + |K| |z|)
// componentwise, m the number of terms of a row (Higham, Accuracy and
// Stability of Numerical Algorithms, Sec. 3.1: gamma_m = m u / (1 - m u),
// u = 2^-53).  A row of K z here has at most 2 nx + nu + 2 products (Sigma
// is added as a product of its own) and b one more term: m = 2 nx + nu + 3.
// So another evaluation of the same z (another program, another order) can
// read at most rel + 2 gamma_m || |b| + |K||z| || / ||b||.  Instances whose
// residual passed tol (done = 3) stop only if that sum is at or below tol too
// (done = 1), otherwise they take another correction (done = 0).  cert holds
// the sum; aa is cleared.
__global__ void k_certify(const Inst *inst, int batch, int nrhs, double *aa, const double *bb, const double *rel,
                          double *cert, int *done, double tol) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= batch || done[i] != 3) return;
    const Inst in = inst[i];
    const double u = 0x1p-53, m = 2.0 * in.nx + in.nu + 3.0;
    const double gamma = m * u / (1.0 - m * u);
    bool all = true;
    for (int r = 0; r < nrhs; ++r) {
        const long long j = (long long)r * batch + i;
        const double bn = sqrt(bb[j]);
        const double s = sqrt(aa[j]);
        const double c = rel[j] + 2.0 * gamma * (bn > 0.0 ? s / bn : s);
        cert[j] = c;
        all = all && (c <= tol);
        aa[j] = 0.0;
    }
    done[i] = all ? 1 : 0;
}

// Early float64 escalation (float32 refinement).  After `k` corrections the
// residual of every right-hand side has contracted from rel0 to rel; at that
// rate the `left` corrections still to come end at rel (rel / rel0)^(left / k).
// An instance that would stay above tol is parked (done = 2: the float32
// corrections skip it) and marked for a float64 factorization now (esc = 0;
// every other instance esc = 1, i.e. skipped by that factorization).
__global__ void k_predict_escalation(int batch, int nrhs, const double *rel0, const double *rel, int *done, int *esc,
                                     double tol, int k, int left) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= batch) return;
    bool park = false;
    if (!done[i]) {
        for (int r = 0; r < nrhs; ++r) {
            const long long j = (long long)r * batch + i;
            const double a = rel0[j], c = rel[j];
            if (!(c <= tol)) {
                const double rate = (a > 0.0 && c < a) ? pow(c / a, 1.0 / k) : 1.0;
                if (!(c * pow(rate, (double)left) <= tol)) park = true;
            }
        }
    }
    if (park) done[i] = 2;
    esc[i] = park ? 0 : 1;
}

// Instances about to be factored again in float64 (skip[i] == 0) lose a failed
// float32 pivot (status NOT_PD); the float64 factorization sets it again if its
// own pivot fails.
__global__ void k_clear_not_pd(int batch, const int *skip, int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < batch && !skip[i] && status[i] == ST_NOT_PD) status[i] = 0;
}

// Parked instances (done = 2) rejoin the refinement for the float64 corrections.
__global__ void k_unpark(int batch, int *done) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < batch && done[i] == 2) done[i] = 0;
}

// Instances still above tol after the last refinement step: status NOT_CONVERGED.
__global__ void k_mark_not_converged(int batch, const int *done, int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < batch && !done[i]) atomicCAS(status + i, 0, ST_NOT_CONVERGED);
}

// b = -(r~, q, f~) with r~^0 = r^0 + S_0 x_init and f~^0 = f^0 + A_0 x_init
// (eq. opt-cond-ocp-eq); one thread per element of b.
__device__ __forceinline__ int find_inst(const Inst *inst, int batch, long long e) {
    int lo = 0, hi = batch - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (inst[mid].oZ <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_build_rhs(const Inst *inst, int batch, Data d, const double *q, const double *r,
                            const double *c, const double *x0, double *b, long long z_lo, long long z_n) {
    for (long long e = z_lo + blockIdx.x * (long long)blockDim.x + threadIdx.x; e < z_lo + z_n;
         e += (long long)gridDim.x * blockDim.x) {
        const Inst in = inst[find_inst(inst, batch, e)];
        const int nx = in.nx, nu = in.nu, w = nu + 2 * nx;
        const long long loc = e - in.oZ;
        const int k = (int)(loc / w), row = (int)(loc % w);
        const double *xi = x0 + in.ox0;
        double v;
        if (row < nu) {
            v = r[in.orv + (long long)k * nu + row];
            if (k == 0 && d.S) {
                const double *S = d.S + in.oS;
                for (int j = 0; j < nx; ++j) v += S[row + j * nu] * xi[j];
            }
        } else if (row < nu + nx) {
            v = q[in.oq + (long long)(k + 1) * nx + (row - nu)];
        } else {
            const int i = row - nu - nx;
            v = c[in.oc + (long long)k * nx + i];
            if (k == 0) {
                const double *A = d.A + in.oA;
                for (int j = 0; j < nx; ++j) v += A[i + j * nx] * xi[j];
            }
        }
        b[e] = -v;
    }
}

// Adjoint gradients (implicit differentiation of K z = b), one CTA per chunk
// of records.  w = K^{-1} dL/dz is given; with x^0 = x_init:
//   dR_k = -sym(w_u u^T), dr_k = -w_u, dS_k = -(w_u x^{kT} + u w_x^{kT}),
//   dA_k = -(w_l x^{kT} + lambda w_x^{kT}), dB_k = -(w_l u^T + lambda w_u^T),
//   dc_k = -w_l, dQ_{k+1} = -sym(w_x x^T), dq_{k+1} = -w_x,
//   dSigma_u^k = -w_u .* u, dSigma_x^{k+1} = -w_x .* x
// (the w_x^k terms vanish for k = 0 since x^0 is fixed).

template <int TEAM>
__global__ void __launch_bounds__(TEAM) k_adjoint_grads(GradArgs g) {
    const Chunk ch = g.chunks[blockIdx.x];
    const Inst in = g.inst[ch.inst];
    const int nx = in.nx, nu = in.nu, wd = nu + 2 * nx, N = in.N;
    const double *z = g.z + in.oZ, *w = g.w + in.oZ, *xi = g.x0 + in.ox0;
    for (int k = ch.k0; k < ch.k1; ++k) {
        const double *u = z + (long long)k * wd, *xn = u + nu, *lam = xn + nx;
        const double *wu = w + (long long)k * wd, *wxn = wu + nu, *wl = wxn + nx;
        const double *xk = k > 0 ? u - wd + nu : xi;
        const double *wxk = k > 0 ? wu - wd + nu : nullptr;
        if (g.dR)
            for (int e = threadIdx.x; e < nu * nu; e += TEAM) {
                const int i = e % nu, j = e / nu;
                g.dR[in.oR + (long long)k * nu * nu + e] = -0.5 * (wu[i] * u[j] + u[i] * wu[j]);
            }
        if (g.dr)
            for (int i = threadIdx.x; i < nu; i += TEAM) g.dr[in.orv + (long long)k * nu + i] = -wu[i];
        if (g.dS)
            for (int e = threadIdx.x; e < nu * nx; e += TEAM) {
                const int i = e % nu, j = e / nu;
                g.dS[in.oS + (long long)k * nu * nx + e] = -(wu[i] * xk[j] + (wxk ? u[i] * wxk[j] : 0.0));
            }
        if (g.dA)
            for (int e = threadIdx.x; e < nx * nx; e += TEAM) {
                const int i = e % nx, j = e / nx;
                g.dA[in.oA + (long long)k * nx * nx + e] = -(wl[i] * xk[j] + (wxk ? lam[i] * wxk[j] : 0.0));
            }
        if (g.dB)
            for (int e = threadIdx.x; e < nx * nu; e += TEAM) {
                const int i = e % nx, j = e / nx;
                g.dB[in.oB + (long long)k * nx * nu + e] = -(wl[i] * u[j] + lam[i] * wu[j]);
            }
        if (g.dc)
            for (int i = threadIdx.x; i < nx; i += TEAM) g.dc[in.oc + (long long)k * nx + i] = -wl[i];
        if (g.dQ)
            for (int e = threadIdx.x; e < nx * nx; e += TEAM) {
                const int i = e % nx, j = e / nx;
                g.dQ[in.oQ + (long long)(k + 1) * nx * nx + e] = -0.5 * (wxn[i] * xn[j] + xn[i] * wxn[j]);
                if (k == 0) g.dQ[in.oQ + e] = 0.0;
            }
        if (g.dq)
            for (int i = threadIdx.x; i < nx; i += TEAM) {
                g.dq[in.oq + (long long)(k + 1) * nx + i] = -wxn[i];
                if (k == 0) g.dq[in.oq + i] = 0.0;
            }
        if (g.dSig) {
            double *ds = g.dSig + in.oSig;
            for (int i = threadIdx.x; i < nu; i += TEAM) ds[(long long)k * (nu + nx) + i] = -wu[i] * u[i];
            for (int i = threadIdx.x; i < nx; i += TEAM) ds[(long long)(k + 1) * (nu + nx) + nu + i] = -wxn[i] * xn[i];
            if (k == 0)
                for (int i = threadIdx.x; i < nx; i += TEAM) ds[nu + i] = 0.0;
            if (k == N - 1)
                for (int i = threadIdx.x; i < nu; i += TEAM) ds[(long long)N * (nu + nx) + i] = 0.0;
        }
    }
}

// dx_init = -S_0^T w_u^0 - A_0^T w_l^0 ; one thread per (instance, component).
__global__ void k_adjoint_dx0(const Inst *inst, int batch, Data d, const double *w, double *dx0) {
    const int ii = blockIdx.x;
    if (ii >= batch) return;
    const Inst in = inst[ii];
    const int nx = in.nx, nu = in.nu;
    const double *wu = w + in.oZ, *wl = wu + nu + nx;
    for (int j = threadIdx.x; j < nx; j += blockDim.x) {
        double acc = 0.0;
        if (d.S)
            for (int i = 0; i < nu; ++i) acc += d.S[in.oS + i + j * nu] * wu[i];
        for (int i = 0; i < nx; ++i) acc += d.A[in.oA + i + j * nx] * wl[i];
        dx0[in.ox0 + j] = -acc;
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <int NR, int MODE>
static void launch_residual_nr(const ResidArgs &a, int r_first, int groups, cudaStream_t st) {
    const dim3 grid(a.n_chunks, groups);
    if (a.max_nx >= 24)
        k_residual_long_rows<128, NR, MODE><<<grid, 128, 0, st>>>(a, r_first);
    else
        k_residual_short_rows<128, NR, MODE><<<grid, 128, 0, st>>>(a, r_first);
}

cudaError_t launch_residual(const ResidArgs &a, int nrhs, cudaStream_t st) {
    if (a.n_chunks == 0) return cudaSuccess;
    // plain rows for the instances without the compensated flag: full groups of RG
    // right-hand sides, then one launch for the remainder
    ResidArgs p = a;
    p.sel = a.comp;
    p.sel_val = 0;
    const int full = nrhs / RG, rest = nrhs % RG;
    if (full > 0) launch_residual_nr<RG, kResidPlain>(p, 0, full, st);
    switch (rest) {
        case 1: launch_residual_nr<1, kResidPlain>(p, full * RG, 1, st); break;
        case 2: launch_residual_nr<2, kResidPlain>(p, full * RG, 1, st); break;
        case 3: launch_residual_nr<3, kResidPlain>(p, full * RG, 1, st); break;
        default: break;
    }
    if (a.comp) {   // compensated rows for the flagged ones, one right-hand side per CTA row
        ResidArgs c = a;
        c.sel = a.comp;
        c.sel_val = 1;
        launch_residual_nr<1, kResidComp>(c, 0, nrhs, st);
    }
    return cudaGetLastError();
}

// One right-hand side per CTA row: the scale is evaluated once per instance
// and stop, on the instances about to stop.
cudaError_t launch_residual_scale(const ResidArgs &a, int nrhs, cudaStream_t st) {
    if (a.n_chunks == 0) return cudaSuccess;
    ResidArgs s = a;
    s.r = nullptr;
    s.need_bb = false;
    s.sel = nullptr;
    launch_residual_nr<1, kResidScale>(s, 0, nrhs, st);
    return cudaGetLastError();
}

cudaError_t launch_certify(const Inst *inst, int batch, int nrhs, double *aa, const double *bb, const double *rel,
                           double *cert, int *done, double tol, cudaStream_t st) {
    k_certify<<<(batch + 127) / 128, 128, 0, st>>>(inst, batch, nrhs, aa, bb, rel, cert, done, tol);
    return cudaGetLastError();
}

cudaError_t launch_resid_finalize(int batch, int nrhs, double *rr, double *bb, double *rel, int *done, double tol,
                                  int *steps, int step, bool keep_bb, int done_value, int *comp, cudaStream_t st) {
    k_resid_finalize<<<(batch + 127) / 128, 128, 0, st>>>(batch, nrhs, rr, bb, rel, done, tol, steps, step, keep_bb,
                                                          done_value, comp);
    return cudaGetLastError();
}

cudaError_t launch_predict_escalation(int batch, int nrhs, const double *rel0, const double *rel, int *done, int *esc,
                                      double tol, int k, int left, cudaStream_t st) {
    k_predict_escalation<<<(batch + 127) / 128, 128, 0, st>>>(batch, nrhs, rel0, rel, done, esc, tol, k, left);
    return cudaGetLastError();
}

__global__ void k_fill_int(int n, int *p, int v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

cudaError_t launch_fill_int(int n, int *p, int v, cudaStream_t st) {
    k_fill_int<<<(n + 127) / 128, 128, 0, st>>>(n, p, v);
    return cudaGetLastError();
}

cudaError_t launch_clear_not_pd(int batch, const int *skip, int *status, cudaStream_t st) {
    k_clear_not_pd<<<(batch + 127) / 128, 128, 0, st>>>(batch, skip, status);
    return cudaGetLastError();
}

cudaError_t launch_unpark(int batch, int *done, cudaStream_t st) {
    k_unpark<<<(batch + 127) / 128, 128, 0, st>>>(batch, done);
    return cudaGetLastError();
}

cudaError_t launch_mark_not_converged(int batch, const int *done, int *status, cudaStream_t st) {
    k_mark_not_converged<<<(batch + 127) / 128, 128, 0, st>>>(batch, done, status);
    return cudaGetLastError();
}

cudaError_t launch_build_rhs(const Inst *inst, int batch, const Data &d, const double *q, const double *r,
                             const double *c, const double *x0, double *b, long long z_lo, long long z_n,
                             cudaStream_t st) {
    long long blocks = (z_n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_build_rhs<<<(int)blocks, 256, 0, st>>>(inst, batch, d, q, r, c, x0, b, z_lo, z_n);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const GradArgs &g, int n_chunks, int batch, const Data &d, double *dx0, cudaStream_t st) {
    if (n_chunks > 0) k_adjoint_grads<128><<<n_chunks, 128, 0, st>>>(g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (dx0) k_adjoint_dx0<<<batch, 64, 0, st>>>(g.inst, batch, d, g.w, dx0);
    return cudaGetLastError();
}

}  // namespace cyq
