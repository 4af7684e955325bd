// Cyclic reduction of the block-tridiagonal Schur complement of the segment
// couplings (paper Sec. 3.2.1 eqs. cr-even / cr-odd, Sec. 4.4, App. A
// Alg. cr), always in float64.
//
// Block i (0 <= i < P) is the multiplier lambda^{b_i} at the end of segment i;
// the matrix is M_i = M_fwd,i + M_bwd,i on the diagonal and K_i (row i,
// column i-1) below it, in time order (the odd-even permutation of the paper
// is the elimination order, not a storage order).  Level l (stride s = 2^l)
// eliminates the blocks k = s, 3s, 5s, ...:
//   L_k = chol(M_k),  Y_k = K_{k+s} L_k^{-T},  U_k = K_k^T L_k^{-T}
// and updates the remaining blocks i = 0, 2s, 4s, ...:
//   M_i -= Y_{i-s} Y_{i-s}^T + U_{i+s} U_{i+s}^T,   K_i <- -Y_{i-s} U_{i-s}^T.
// Block 0 is factored last.  The solve is the matching forward substitution
// (b~_k = L_k^{-1} b_k, b_i -= Y_{i-s} b~_{i-s} + U_{i+s} b~_{i+s}) and back
// substitution (x_k = L_k^{-T}(b~_k - Y_k^T x_{k+s} - U_k^T x_{k-s})).
#include "cyq_internal.cuh"

namespace cyq {

namespace {

template <int TEAM>
__device__ void load_blk(double *dst, const double *src, int n, bool transpose) {
    for (int e = threadIdx.x; e < n * n; e += TEAM) {
        const int i = e % n, j = e / n;
        dst[e] = transpose ? src[j + i * n] : src[e];
    }
}

template <int TEAM>
__device__ void store_blk(double *dst, const double *src, int n) {
    for (int e = threadIdx.x; e < n * n; e += TEAM) dst[e] = src[e];
}

}  // namespace

// ---------------------------------------------------------------------------
// Level-parallel factorization: one launch per phase of each level, one CTA
// per block, so the O(P) eliminations of a level run on all SMs at once.
// ---------------------------------------------------------------------------

// M_c <- M_fwd,c + M_bwd,c for every block of every listed instance.
__global__ void k_cr_assemble(FactorArgs a, const int *inst_list, int n_inst) {
    const int ii = inst_list[blockIdx.y];
    if (a.skip && a.skip[ii]) return;
    const Inst in = a.inst[ii];
    const long long total = (long long)in.P * in.nx * in.nx;
    double *M = a.Mf + in.oBlk;
    const double *Mb = a.Mb + in.oBlk;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x)
        M[e] += Mb[e];
}

// Eliminate block k at stride s:  L_k = chol(M_k),  U_k = K_k^T L_k^{-T},  Y_k = K_{k+s} L_k^{-T}.
template <int TEAM>
__global__ void __launch_bounds__(TEAM) k_cr_eliminate(FactorArgs a, const CrJob *jobs, int s) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const CrJob job = jobs[blockIdx.x];
    if (a.skip && a.skip[job.inst]) return;
    const Inst in = a.inst[job.inst];
    const int P = in.P, n = in.nx, k = job.k;
    const long long nn = (long long)n * n;
    double *M = a.Mf + in.oBlk, *K = a.Kc + in.oBlk, *U = a.U + in.oBlk, *Y = a.Y + in.oBlk;
    double *W0 = reinterpret_cast<double *>(smem_raw), *W1 = W0 + nn, *W2 = W1 + nn, *dinv = W2 + nn;
    load_blk<TEAM>(W0, M + k * nn, n, false);
    load_blk<TEAM>(W1, K + k * nn, n, true);
    const bool hasY = k + s < P;
    if (hasY) load_blk<TEAM>(W2, K + (k + s) * nn, n, false);
    team_sync();
    const bool ok = team_chol<double, TEAM>(W0, n, n, dinv);
    store_blk<TEAM>(M + k * nn, W0, n);
    // both triangular solves in one pass: rows of U then rows of Y
    const int rows = hasY ? 2 * n : n;
    for (int r = threadIdx.x; r < rows; r += TEAM) {
        double *X = r < n ? W1 : W2;
        const int rr = r < n ? r : r - n;
        for (int j = 0; j < n; ++j) {
            double acc = X[rr + j * n];
            for (int t = 0; t < j; ++t) acc = fma(-X[rr + t * n], W0[j + t * n], acc);
            X[rr + j * n] = acc * dinv[j];
        }
    }
    team_sync();
    store_blk<TEAM>(U + k * nn, W1, n);
    if (hasY) store_blk<TEAM>(Y + k * nn, W2, n);
    if (!ok && threadIdx.x == 0) atomicCAS(a.status + job.inst, 0, ST_NOT_PD);
}

// Update block i at stride s:  M_i -= Y_{i-s} Y_{i-s}^T + U_{i+s} U_{i+s}^T,
// K_i <- -Y_{i-s} U_{i-s}^T (the fill coupling i and i-2s).
template <int TEAM>
__global__ void __launch_bounds__(TEAM) k_cr_update(FactorArgs a, const CrJob *jobs, int s) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const CrJob job = jobs[blockIdx.x];
    if (a.skip && a.skip[job.inst]) return;
    const Inst in = a.inst[job.inst];
    const int P = in.P, n = in.nx, i = job.k;
    const long long nn = (long long)n * n;
    double *M = a.Mf + in.oBlk, *K = a.Kc + in.oBlk;
    const double *U = a.U + in.oBlk, *Y = a.Y + in.oBlk;
    double *W0 = reinterpret_cast<double *>(smem_raw), *W1 = W0 + nn, *W2 = W1 + nn, *W3 = W2 + nn;
    const bool lo = i - s >= 0, hi = i + s < P, fill = i - 2 * s >= 0;
    if (lo) load_blk<TEAM>(W1, Y + (i - s) * nn, n, false);
    if (hi) load_blk<TEAM>(W2, U + (i + s) * nn, n, false);
    if (fill) load_blk<TEAM>(W3, U + (i - s) * nn, n, false);
    team_sync();
    // lower triangle of M_i minus the two symmetric products, straight from global
    const int cnt = n * (n + 1) / 2;
    double *Mi = M + i * nn;
    for (int e = threadIdx.x; e < cnt; e += TEAM) {
        int r, c;
        tri_index(e, r, c);
        double acc = Mi[r + c * n];
        if (lo)
            for (int t = 0; t < n; ++t) acc = fma(-W1[r + t * n], W1[c + t * n], acc);
        if (hi)
            for (int t = 0; t < n; ++t) acc = fma(-W2[r + t * n], W2[c + t * n], acc);
        W0[r + c * n] = acc;
    }
    if (fill) {
        double *Ki = K + i * nn;
        for (int e = threadIdx.x; e < n * n; e += TEAM) {
            const int r = e % n, c = e / n;
            double acc = 0.0;
            for (int t = 0; t < n; ++t) acc = fma(W1[r + t * n], W3[c + t * n], acc);
            Ki[e] = -acc;
        }
    }
    team_sync();
    for (int e = threadIdx.x; e < n * n; e += TEAM) {
        const int r = e % n, c = e / n;
        Mi[e] = r >= c ? W0[r + c * n] : W0[c + r * n];
    }
}

// Last block of every instance: L_0 = chol(M_0).
template <int TEAM>
__global__ void __launch_bounds__(TEAM) k_cr_base(FactorArgs a, const int *inst_list) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ii = inst_list[blockIdx.x];
    if (a.skip && a.skip[ii]) return;
    const Inst in = a.inst[ii];
    const int n = in.nx;
    double *M = a.Mf + in.oBlk;
    double *W0 = reinterpret_cast<double *>(smem_raw);
    load_blk<TEAM>(W0, M, n, false);
    team_sync();
    const bool ok = team_chol<double, TEAM>(W0, n, n);
    store_blk<TEAM>(M, W0, n);
    if (!ok && threadIdx.x == 0) atomicCAS(a.status + ii, 0, ST_NOT_PD);
}

cudaError_t launch_cr_factor_levels(const CrPlan &plan, int team, int nmax, const FactorArgs &a, cudaStream_t st,
                                    long long *launches) {
    if (plan.n_inst == 0) return cudaSuccess;
    cudaError_t e;
    const size_t nn = (size_t)nmax * nmax * sizeof(double);
    {
        dim3 grid(64, plan.n_inst);
        k_cr_assemble<<<grid, 256, 0, st>>>(a, plan.inst_list, plan.n_inst);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++*launches;
    }
    auto elim = team == 32 ? k_cr_eliminate<32> : k_cr_eliminate<128>;
    auto upd = team == 32 ? k_cr_update<32> : k_cr_update<128>;
    auto base = team == 32 ? k_cr_base<32> : k_cr_base<128>;
    const size_t se = 3 * nn + nmax * sizeof(double), su = 4 * nn;
    if ((e = ensure_smem((const void *)elim, se)) != cudaSuccess) return e;
    if ((e = ensure_smem((const void *)upd, su)) != cudaSuccess) return e;
    if ((e = ensure_smem((const void *)base, nn)) != cudaSuccess) return e;
    for (int l = 0; l < plan.levels; ++l) {
        const int s = 1 << l;
        const int ne = plan.elim_off[l + 1] - plan.elim_off[l], nu_ = plan.upd_off[l + 1] - plan.upd_off[l];
        if (ne > 0) {
            elim<<<ne, team, se, st>>>(a, plan.jobs + plan.elim_off[l], s);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            ++*launches;
        }
        if (nu_ > 0) {
            upd<<<nu_, team, su, st>>>(a, plan.jobs + plan.upd_off[l], s);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            ++*launches;
        }
    }
    base<<<plan.n_inst, team, nn, st>>>(a, plan.inst_list);
    ++*launches;
    return cudaGetLastError();
}

// Coupling right-hand side and cyclic-reduction solve, one CTA per instance:
//   rhs_c = d_fwd,c + d_bwd,(c+1 mod P) - b_lambda^{b_c},
// then M lambda = rhs; lambda^{b_c} is written into z and into the coupling
// vector used by the forward segment sweep.
template <int TEAM>
__global__ void __launch_bounds__(TEAM) k_cr_solve(SolveArgs a, const int *inst_list) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ii = inst_list[blockIdx.x];
    if (a.skip && a.skip[ii]) return;
    const Inst in = a.inst[ii];
    const int P = in.P, n = in.nx, N = in.N, nu = in.nu, nrhs = a.nrhs;
    const long long nn = (long long)n * n;
    const double *L = a.Mf + in.oBlk, *U = a.U + in.oBlk, *Y = a.Y + in.oBlk;
    double *v = reinterpret_cast<double *>(smem_raw);     // P * n * nrhs (block-major per rhs)
    double *di = v + (long long)P * n * nrhs;             // P * n reciprocal diagonals of the L_k
    const int w = nu + 2 * n;
    for (long long e = threadIdx.x; e < (long long)P * n; e += TEAM) {
        const int k = (int)(e / n), i = (int)(e % n);
        di[e] = 1.0 / L[k * nn + i + i * n];
    }
    // assemble right-hand sides
    for (long long e = threadIdx.x; e < (long long)nrhs * P * n; e += TEAM) {
        const int r = (int)(e / ((long long)P * n));
        const int rem = (int)(e % ((long long)P * n));
        const int c = rem / n, i = rem % n;
        const int bc = seg_bound(c, N, P);
        const double *dF = a.dF + r * a.nvec + in.oVec;
        const double *dB = a.dB + r * a.nvec + in.oVec;
        const double bl = a.b[r * a.kkt + in.oZ + (long long)bc * w + nu + n + i];
        v[e] = dF[c * n + i] + dB[((c + 1) % P) * n + i] - bl;
    }
    team_sync();
    int levels = 0;
    while ((1 << levels) < P) ++levels;
    // forward elimination
    for (int l = 0; l < levels; ++l) {
        const int s = 1 << l;
        // b~_k = L_k^{-1} b_k for eliminated k (one thread per (k, rhs))
        const int nk = (P - s + 2 * s - 1) / (2 * s);
        for (int job = threadIdx.x; job < nk * nrhs; job += TEAM) {
            const int k = s + (job % nk) * 2 * s, r = job / nk;
            double *x = v + (long long)r * P * n + (long long)k * n;
            const double *Lk = L + k * nn, *dk = di + (long long)k * n;
            for (int i = 0; i < n; ++i) {
                double acc = x[i];
                for (int t = 0; t < i; ++t) acc = fma(-Lk[i + t * n], x[t], acc);
                x[i] = acc * dk[i];
            }
        }
        team_sync();
        // b_i -= Y_{i-s} b~_{i-s} + U_{i+s} b~_{i+s}  (one thread per (i, row, rhs))
        const int ni = (P + 2 * s - 1) / (2 * s);
        for (int job = threadIdx.x; job < ni * n * nrhs; job += TEAM) {
            const int row = job % n, i = ((job / n) % ni) * 2 * s, r = job / (n * ni);
            double *vr = v + (long long)r * P * n;
            double acc = 0.0;
            if (i - s >= 0) {
                const double *Yk = Y + (i - s) * nn, *bt = vr + (long long)(i - s) * n;
                for (int t = 0; t < n; ++t) acc += Yk[row + t * n] * bt[t];
            }
            if (i + s < P) {
                const double *Uk = U + (i + s) * nn, *bt = vr + (long long)(i + s) * n;
                for (int t = 0; t < n; ++t) acc += Uk[row + t * n] * bt[t];
            }
            vr[(long long)i * n + row] -= acc;
        }
        team_sync();
    }
    // base block 0: x_0 = L_0^{-T} L_0^{-1} b_0
    for (int r = threadIdx.x; r < nrhs; r += TEAM) {
        double *x = v + (long long)r * P * n;
        for (int i = 0; i < n; ++i) {
            double acc = x[i];
            for (int t = 0; t < i; ++t) acc = fma(-L[i + t * n], x[t], acc);
            x[i] = acc * di[i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double acc = x[i];
            for (int t = i + 1; t < n; ++t) acc = fma(-L[t + i * n], x[t], acc);
            x[i] = acc * di[i];
        }
    }
    team_sync();
    // back substitution, coarse to fine
    for (int l = levels - 1; l >= 0; --l) {
        const int s = 1 << l;
        const int nk = (P - s + 2 * s - 1) / (2 * s);
        // tmp = b~_k - Y_k^T x_{k+s} - U_k^T x_{k-s}, then x_k = L_k^{-T} tmp
        for (int job = threadIdx.x; job < nk * nrhs; job += TEAM) {
            const int k = s + (job % nk) * 2 * s, r = job / nk;
            double *vr = v + (long long)r * P * n;
            double *x = vr + (long long)k * n;
            const double *Uk = U + k * nn, *Yk = Y + k * nn, *Lk = L + k * nn, *dk = di + (long long)k * n;
            const double *xp = vr + (long long)(k - s) * n;
            const double *xn = (k + s < P) ? vr + (long long)(k + s) * n : nullptr;
            for (int i = 0; i < n; ++i) {
                double acc = x[i];
                for (int t = 0; t < n; ++t) acc -= Uk[t + i * n] * xp[t];
                if (xn)
                    for (int t = 0; t < n; ++t) acc -= Yk[t + i * n] * xn[t];
                x[i] = acc;
            }
            for (int i = n - 1; i >= 0; --i) {
                double acc = x[i];
                for (int t = i + 1; t < n; ++t) acc = fma(-Lk[t + i * n], x[t], acc);
                x[i] = acc * dk[i];
            }
        }
        team_sync();
    }
    // scatter lambda^{b_c}
    for (long long e = threadIdx.x; e < (long long)nrhs * P * n; e += TEAM) {
        const int r = (int)(e / ((long long)P * n));
        const int rem = (int)(e % ((long long)P * n));
        const int c = rem / n, i = rem % n;
        const int bc = seg_bound(c, N, P);
        a.lam[r * a.nvec + in.oVec + rem] = v[e];
        const long long o = r * a.kkt + in.oZ + (long long)bc * w + nu + n + i;
        if (a.zacc) a.zacc[o] += v[e]; else a.z[o] = v[e];
    }
}

// ---------------------------------------------------------------------------
// Level-parallel solve (instances with many segments in a small batch): the
// single-CTA solve above runs a whole instance on one SM; here every level is
// one launch with one warp per (block, right-hand side), so the O(P) blocks of
// a level run on all SMs.  The coupling vector lam holds the right-hand side
// and, in place, the solution; the arithmetic is that of k_cr_solve.
// ---------------------------------------------------------------------------
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Block L (n x n, column-major) into shared memory and the reciprocals of its diagonal.
__device__ void crs_load_factor(double *Ls, double *di, const double *L, int n) {
    for (int e = threadIdx.x; e < n * n; e += 32) Ls[e] = L[e];
    __syncwarp();
    for (int i = threadIdx.x; i < n; i += 32) di[i] = 1.0 / Ls[i + i * n];
    __syncwarp();
}

// v := L^{-1} v (column-oriented forward substitution; row i belongs to lane i % 32).
__device__ void crs_forward(const double *Ls, const double *di, double *v, int n) {
    for (int t = 0; t < n; ++t) {
        if ((t & 31) == threadIdx.x) v[t] *= di[t];
        __syncwarp();
        const double xt = v[t];
        for (int i = t + 1 + ((threadIdx.x - t - 1) & 31); i < n; i += 32) v[i] = fma(-Ls[i + t * n], xt, v[i]);
    }
    __syncwarp();
}

// v := L^{-T} v (column-oriented back substitution).
__device__ void crs_backward(const double *Ls, const double *di, double *v, int n) {
    for (int t = n - 1; t >= 0; --t) {
        if ((t & 31) == threadIdx.x) v[t] *= di[t];
        __syncwarp();
        const double xt = v[t];
        for (int i = threadIdx.x; i < t; i += 32) v[i] = fma(-Ls[t + i * n], xt, v[i]);
    }
    __syncwarp();
}

__device__ __forceinline__ double *crs_vec(const SolveArgs &a, const Inst &in, int r, int k) {
    return a.lam + r * a.nvec + in.oVec + (long long)k * in.nx;
}

}  // namespace

// Right-hand side of the coupling system: rhs_c = d_fwd,c + d_bwd,(c+1 mod P) - b_lambda^{b_c}.
__global__ void k_crs_rhs(SolveArgs a, const int *inst_list) {
    const int ii = inst_list[blockIdx.y];
    if (a.skip && a.skip[ii]) return;
    const Inst in = a.inst[ii];
    const int P = in.P, n = in.nx, N = in.N, nu = in.nu, w = nu + 2 * n;
    const long long total = (long long)P * n * a.nrhs;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / ((long long)P * n));
        const int rem = (int)(e % ((long long)P * n));
        const int c = rem / n, i = rem % n;
        const int bc = seg_bound(c, N, P);
        const double *dF = a.dF + r * a.nvec + in.oVec, *dB = a.dB + r * a.nvec + in.oVec;
        const double bl = a.b[r * a.kkt + in.oZ + (long long)bc * w + nu + n + i];
        a.lam[r * a.nvec + in.oVec + rem] = dF[c * n + i] + dB[((c + 1) % P) * n + i] - bl;
    }
}

// Forward phase of level s, eliminated block k:  b~_k = L_k^{-1} b_k.
__global__ void __launch_bounds__(32) k_crs_forward(SolveArgs a, const CrJob *jobs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const CrJob job = jobs[blockIdx.x];
    if (a.skip && a.skip[job.inst]) return;
    const Inst in = a.inst[job.inst];
    const int n = in.nx, r = blockIdx.y;
    double *Ls = reinterpret_cast<double *>(smem_raw), *di = Ls + n * n, *v = di + n;
    crs_load_factor(Ls, di, a.Mf + in.oBlk + (long long)job.k * n * n, n);
    double *g = crs_vec(a, in, r, job.k);
    for (int i = threadIdx.x; i < n; i += 32) v[i] = g[i];
    __syncwarp();
    crs_forward(Ls, di, v, n);
    for (int i = threadIdx.x; i < n; i += 32) g[i] = v[i];
}

// Forward phase of level s, remaining block i:  b_i -= Y_{i-s} b~_{i-s} + U_{i+s} b~_{i+s}.
__global__ void __launch_bounds__(32) k_crs_update(SolveArgs a, const CrJob *jobs, int s) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const CrJob job = jobs[blockIdx.x];
    if (a.skip && a.skip[job.inst]) return;
    const Inst in = a.inst[job.inst];
    const int n = in.nx, P = in.P, i = job.k, r = blockIdx.y;
    const long long nn = (long long)n * n;
    double *xl = reinterpret_cast<double *>(smem_raw), *xh = xl + n;
    const bool lo = i - s >= 0, hi = i + s < P;
    if (lo) {
        const double *g = crs_vec(a, in, r, i - s);
        for (int t = threadIdx.x; t < n; t += 32) xl[t] = g[t];
    }
    if (hi) {
        const double *g = crs_vec(a, in, r, i + s);
        for (int t = threadIdx.x; t < n; t += 32) xh[t] = g[t];
    }
    __syncwarp();
    const double *Y = a.Y + in.oBlk + (i - s) * nn, *U = a.U + in.oBlk + (i + s) * nn;
    double *gi = crs_vec(a, in, r, i);
    for (int row = threadIdx.x; row < n; row += 32) {
        double acc = 0.0;
        if (lo)
            for (int t = 0; t < n; ++t) acc = fma(Y[row + t * n], xl[t], acc);
        if (hi)
            for (int t = 0; t < n; ++t) acc = fma(U[row + t * n], xh[t], acc);
        gi[row] -= acc;
    }
}

// Base block 0 of every listed instance:  x_0 = L_0^{-T} L_0^{-1} b_0.
__global__ void __launch_bounds__(32) k_crs_base(SolveArgs a, const int *inst_list) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ii = inst_list[blockIdx.x];
    if (a.skip && a.skip[ii]) return;
    const Inst in = a.inst[ii];
    const int n = in.nx, r = blockIdx.y;
    double *Ls = reinterpret_cast<double *>(smem_raw), *di = Ls + n * n, *v = di + n;
    crs_load_factor(Ls, di, a.Mf + in.oBlk, n);
    double *g = crs_vec(a, in, r, 0);
    for (int i = threadIdx.x; i < n; i += 32) v[i] = g[i];
    __syncwarp();
    crs_forward(Ls, di, v, n);
    crs_backward(Ls, di, v, n);
    for (int i = threadIdx.x; i < n; i += 32) g[i] = v[i];
}

// Back substitution of level s, eliminated block k:
//   x_k = L_k^{-T} (b~_k - U_k^T x_{k-s} - Y_k^T x_{k+s}).
__global__ void __launch_bounds__(32) k_crs_backward(SolveArgs a, const CrJob *jobs, int s) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const CrJob job = jobs[blockIdx.x];
    if (a.skip && a.skip[job.inst]) return;
    const Inst in = a.inst[job.inst];
    const int n = in.nx, P = in.P, k = job.k, r = blockIdx.y;
    const long long nn = (long long)n * n;
    double *Ls = reinterpret_cast<double *>(smem_raw), *di = Ls + n * n, *v = di + n, *xp = v + n, *xn = xp + n;
    crs_load_factor(Ls, di, a.Mf + in.oBlk + k * nn, n);
    const bool hasn = k + s < P;
    {
        const double *gp = crs_vec(a, in, r, k - s);
        for (int t = threadIdx.x; t < n; t += 32) xp[t] = gp[t];
        if (hasn) {
            const double *gn = crs_vec(a, in, r, k + s);
            for (int t = threadIdx.x; t < n; t += 32) xn[t] = gn[t];
        }
    }
    __syncwarp();
    const double *Uk = a.U + in.oBlk + k * nn, *Yk = a.Y + in.oBlk + k * nn;
    double *g = crs_vec(a, in, r, k);
    for (int i = threadIdx.x; i < n; i += 32) {
        double acc = g[i];
        for (int t = 0; t < n; ++t) acc -= Uk[t + i * n] * xp[t];
        if (hasn)
            for (int t = 0; t < n; ++t) acc -= Yk[t + i * n] * xn[t];
        v[i] = acc;
    }
    __syncwarp();
    crs_backward(Ls, di, v, n);
    for (int i = threadIdx.x; i < n; i += 32) g[i] = v[i];
}

// lambda^{b_c} of the solution into z (or added into zacc).
__global__ void k_crs_scatter(SolveArgs a, const int *inst_list) {
    const int ii = inst_list[blockIdx.y];
    if (a.skip && a.skip[ii]) return;
    const Inst in = a.inst[ii];
    const int P = in.P, n = in.nx, N = in.N, nu = in.nu, w = nu + 2 * n;
    const long long total = (long long)P * n * a.nrhs;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / ((long long)P * n));
        const int rem = (int)(e % ((long long)P * n));
        const int c = rem / n, i = rem % n;
        const int bc = seg_bound(c, N, P);
        const double x = a.lam[r * a.nvec + in.oVec + rem];
        const long long o = r * a.kkt + in.oZ + (long long)bc * w + nu + n + i;
        if (a.zacc) a.zacc[o] += x; else a.z[o] = x;
    }
}

cudaError_t launch_cr_solve_levels(const CrPlan &plan, int nmax, const SolveArgs &a, cudaStream_t st,
                                   long long *launches) {
    if (plan.n_inst == 0) return cudaSuccess;
    cudaError_t e;
    const int nr = a.nrhs;
    const size_t sm = ((size_t)nmax * nmax + 4 * (size_t)nmax) * sizeof(double);
    if ((e = ensure_smem((const void *)k_crs_forward, sm)) != cudaSuccess) return e;
    if ((e = ensure_smem((const void *)k_crs_base, sm)) != cudaSuccess) return e;
    if ((e = ensure_smem((const void *)k_crs_backward, sm)) != cudaSuccess) return e;
    k_crs_rhs<<<dim3(8, plan.n_inst), 256, 0, st>>>(a, plan.inst_list);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*launches;
    for (int l = 0; l < plan.levels; ++l) {
        const int s = 1 << l;
        const int ne = plan.elim_off[l + 1] - plan.elim_off[l], nu_ = plan.upd_off[l + 1] - plan.upd_off[l];
        if (ne > 0) {
            k_crs_forward<<<dim3(ne, nr), 32, sm, st>>>(a, plan.jobs + plan.elim_off[l]);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            ++*launches;
        }
        if (nu_ > 0) {
            k_crs_update<<<dim3(nu_, nr), 32, 2 * (size_t)nmax * sizeof(double), st>>>(
                a, plan.jobs + plan.upd_off[l], s);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            ++*launches;
        }
    }
    k_crs_base<<<dim3(plan.n_inst, nr), 32, sm, st>>>(a, plan.inst_list);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*launches;
    for (int l = plan.levels - 1; l >= 0; --l) {
        const int s = 1 << l;
        const int ne = plan.elim_off[l + 1] - plan.elim_off[l];
        if (ne > 0) {
            k_crs_backward<<<dim3(ne, nr), 32, sm, st>>>(a, plan.jobs + plan.elim_off[l], s);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            ++*launches;
        }
    }
    k_crs_scatter<<<dim3(8, plan.n_inst), 256, 0, st>>>(a, plan.inst_list);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_cr_solve(int n_inst_cr, const int *inst_list, int team, size_t smem, const SolveArgs &a,
                            cudaStream_t st) {
    if (n_inst_cr == 0) return cudaSuccess;
    cudaError_t e;
    if (team == 32) {
        e = ensure_smem((const void *)k_cr_solve<32>, smem);
        if (e != cudaSuccess) return e;
        k_cr_solve<32><<<n_inst_cr, 32, smem, st>>>(a, inst_list);
    } else {
        e = ensure_smem((const void *)k_cr_solve<128>, smem);
        if (e != cudaSuccess) return e;
        k_cr_solve<128><<<n_inst_cr, 128, smem, st>>>(a, inst_list);
    }
    return cudaGetLastError();
}

}  // namespace cyq
