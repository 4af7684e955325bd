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
