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

// Elimination of one block (shared by cyclic reduction and its parallel tail):
//   L = chol(M),  U = Klo^T L^{-T} (Klo: the block's coupling to its lower
//   neighbour, row = this block),  Y = Khi L^{-T} (Khi: the upper neighbour's
//   coupling to this block).  Klo / Khi null: that product is skipped.  L goes
//   to Lout, which may be M itself.  Returns false on a non-positive pivot.
template <int TEAM>
__device__ bool cr_eliminate_block(double *W0, const double *M, const double *Klo, const double *Khi, double *Lout,
                                   double *Uout, double *Yout, int n) {
    const long long nn = (long long)n * n;
    double *W1 = W0 + nn, *W2 = W1 + nn, *dinv = W2 + nn;
    load_blk<TEAM>(W0, M, n, false);
    if (Klo) load_blk<TEAM>(W1, Klo, n, true);
    if (Khi) load_blk<TEAM>(W2, Khi, n, false);
    team_sync();
    const bool ok = team_chol<double, TEAM>(W0, n, n, dinv);
    store_blk<TEAM>(Lout, W0, n);
    // both triangular solves in one pass: rows of U then rows of Y
    const int r0 = Klo ? 0 : n, rows = Khi ? 2 * n : n;
    for (int r = r0 + threadIdx.x; r < rows; r += TEAM) {
        double *X = r < n ? W1 : W2;
        const int rr = r < n ? r : r - n;
        for (int j = 0; j < n; ++j) {
            double acc = X[rr + j * n];
            for (int t = 0; t < j; ++t) acc = fma(-X[rr + t * n], W0[j + t * n], acc);
            X[rr + j * n] = acc * dinv[j];
        }
    }
    team_sync();
    if (Klo) store_blk<TEAM>(Uout, W1, n);
    if (Khi) store_blk<TEAM>(Yout, W2, n);
    return ok;
}

// Update of one remaining block: M -= Ylo Ylo^T + Uhi Uhi^T, and where Ufill is
// given, Kout = -Ylo Ufill^T (the fill coupling to the neighbour two strides down).
template <int TEAM>
__device__ void cr_update_block(double *W0, double *M, const double *Ylo, const double *Uhi, const double *Ufill,
                                double *Kout, int n) {
    const long long nn = (long long)n * n;
    double *W1 = W0 + nn, *W2 = W1 + nn, *W3 = W2 + nn;
    if (Ylo) load_blk<TEAM>(W1, Ylo, n, false);
    if (Uhi) load_blk<TEAM>(W2, Uhi, n, false);
    if (Ufill) load_blk<TEAM>(W3, Ufill, n, false);
    team_sync();
    // lower triangle of M minus the two symmetric products, straight from global
    const int cnt = n * (n + 1) / 2;
    for (int e = threadIdx.x; e < cnt; e += TEAM) {
        int r, c;
        tri_index(e, r, c);
        double acc = M[r + c * n];
        if (Ylo)
            for (int t = 0; t < n; ++t) acc = fma(-W1[r + t * n], W1[c + t * n], acc);
        if (Uhi)
            for (int t = 0; t < n; ++t) acc = fma(-W2[r + t * n], W2[c + t * n], acc);
        W0[r + c * n] = acc;
    }
    if (Ufill) {
        for (int e = threadIdx.x; e < n * n; e += TEAM) {
            const int r = e % n, c = e / n;
            double acc = 0.0;
            for (int t = 0; t < n; ++t) acc = fma(W1[r + t * n], W3[c + t * n], acc);
            Kout[e] = -acc;
        }
    }
    team_sync();
    for (int e = threadIdx.x; e < n * n; e += TEAM) {
        const int r = e % n, c = e / n;
        M[e] = r >= c ? W0[r + c * n] : W0[c + r * n];
    }
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
    const bool hasY = k + s < P;
    const bool ok = cr_eliminate_block<TEAM>(reinterpret_cast<double *>(smem_raw), M + k * nn, K + k * nn,
                                             hasY ? K + (k + s) * nn : nullptr, M + k * nn, U + k * nn,
                                             Y + k * nn, n);
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
    const bool lo = i - s >= 0, hi = i + s < P, fill = i - 2 * s >= 0;
    cr_update_block<TEAM>(reinterpret_cast<double *>(smem_raw), M + i * nn, lo ? Y + (i - s) * nn : nullptr,
                          hi ? U + (i + s) * nn : nullptr, fill ? U + (i - s) * nn : nullptr, K + i * nn, n);
}

// ---------------------------------------------------------------------------
// Parallel cyclic reduction of the last levels (paper App. A, Alg. pcr): the
// blocks left after the cyclic-reduction levels (every s0-th block, v of them
// per instance, tail index j = block / s0) are all eliminated into both of
// their neighbours at each tail level t (stride 2^t in tail indices), until
// no coupling is left; the right-hand side then needs no back substitution
// over these levels.  Per block and level:
//   L_j = chol(M_j),  A_j = E_{j+2^t} L_j^{-T},  B_j = E_j^T L_j^{-T}
//   M_j -= A_{j-2^t} A_{j-2^t}^T + B_{j+2^t} B_{j+2^t}^T,
//   E_j <- -A_{j-2^t} B_{j-2^t}^T   (E_j: coupling of j to j - stride),
// with L, A, B of every level kept for the solve (tail storage, per instance
// v x levels x 3 blocks).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pcr_count(int P, int s0) { return (P + s0 - 1) / s0; }

__device__ __forceinline__ double *pcr_blk(const CrPlan &p, double *base, const CrJob &job, int n, int v, int t, int j) {
    return base + p.oT_dev[job.inst] + ((long long)t * v + j) * n * n;
}

template <int TEAM>
__global__ void __launch_bounds__(TEAM) k_pcr_eliminate(FactorArgs a, CrPlan p, const CrJob *jobs, int t) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const CrJob job = jobs[blockIdx.x];
    if (a.skip && a.skip[job.inst]) return;
    const Inst in = a.inst[job.inst];
    const int n = in.nx, v = pcr_count(in.P, p.s0), j = job.k, sg = 1 << t;
    const long long nn = (long long)n * n;
    double *M = a.Mf + in.oBlk, *K = a.Kc + in.oBlk;
    const double *Klo = j - sg >= 0 ? K + (long long)j * p.s0 * nn : nullptr;
    const double *Khi = j + sg < v ? K + (long long)(j + sg) * p.s0 * nn : nullptr;
    const bool ok = cr_eliminate_block<TEAM>(reinterpret_cast<double *>(smem_raw), M + (long long)j * p.s0 * nn, Klo,
                                             Khi, pcr_blk(p, p.Lt, job, n, v, t, j), pcr_blk(p, p.Bt, job, n, v, t, j),
                                             pcr_blk(p, p.At, job, n, v, t, j), n);
    if (!ok && threadIdx.x == 0) atomicCAS(a.status + job.inst, 0, ST_NOT_PD);
}

template <int TEAM>
__global__ void __launch_bounds__(TEAM) k_pcr_update(FactorArgs a, CrPlan p, const CrJob *jobs, int t) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const CrJob job = jobs[blockIdx.x];
    if (a.skip && a.skip[job.inst]) return;
    const Inst in = a.inst[job.inst];
    const int n = in.nx, v = pcr_count(in.P, p.s0), j = job.k, sg = 1 << t;
    const long long nn = (long long)n * n;
    double *M = a.Mf + in.oBlk, *K = a.Kc + in.oBlk;
    const bool lo = j - sg >= 0, hi = j + sg < v, fill = j - 2 * sg >= 0;
    cr_update_block<TEAM>(reinterpret_cast<double *>(smem_raw), M + (long long)j * p.s0 * nn,
                          lo ? pcr_blk(p, p.At, job, n, v, t, j - sg) : nullptr,
                          hi ? pcr_blk(p, p.Bt, job, n, v, t, j + sg) : nullptr,
                          fill ? pcr_blk(p, p.Bt, job, n, v, t, j - sg) : nullptr, K + (long long)j * p.s0 * nn, n);
}

// Last factor of every tail block: L_j = chol(M_j) (in place).
template <int TEAM>
__global__ void __launch_bounds__(TEAM) k_pcr_base(FactorArgs a, CrPlan p, const CrJob *jobs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const CrJob job = jobs[blockIdx.x];
    if (a.skip && a.skip[job.inst]) return;
    const Inst in = a.inst[job.inst];
    const int n = in.nx;
    double *M = a.Mf + in.oBlk + (long long)job.k * p.s0 * n * n;
    double *W0 = reinterpret_cast<double *>(smem_raw);
    load_blk<TEAM>(W0, M, n, false);
    team_sync();
    const bool ok = team_chol<double, TEAM>(W0, n, n);
    store_blk<TEAM>(M, W0, n);
    if (!ok && threadIdx.x == 0) atomicCAS(a.status + job.inst, 0, ST_NOT_PD);
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
    if (plan.tail == 0) {
        base<<<plan.n_inst, team, nn, st>>>(a, plan.inst_list);
        ++*launches;
        return cudaGetLastError();
    }
    // parallel tail: every remaining block at every tail level, then each block's last factor
    auto pel = team == 32 ? k_pcr_eliminate<32> : k_pcr_eliminate<128>;
    auto pup = team == 32 ? k_pcr_update<32> : k_pcr_update<128>;
    auto pba = team == 32 ? k_pcr_base<32> : k_pcr_base<128>;
    if ((e = ensure_smem((const void *)pel, se)) != cudaSuccess) return e;
    if ((e = ensure_smem((const void *)pup, su)) != cudaSuccess) return e;
    if ((e = ensure_smem((const void *)pba, nn)) != cudaSuccess) return e;
    for (int t = 0; t < plan.tail; ++t) {
        const int nj = plan.pcr_off[t + 1] - plan.pcr_off[t];
        if (nj == 0) continue;
        pel<<<nj, team, se, st>>>(a, plan, plan.jobs + plan.pcr_off[t], t);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        pup<<<nj, team, su, st>>>(a, plan, plan.jobs + plan.pcr_off[t], t);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        *launches += 2;
    }
    const int nb = plan.pcr_base_end - plan.pcr_off[plan.tail];
    pba<<<nb, team, nn, st>>>(a, plan, plan.jobs + plan.pcr_off[plan.tail]);
    ++*launches;
    return cudaGetLastError();
}

size_t cr_tail_smem_bytes(int nmax) { return 4 * (size_t)nmax * nmax * sizeof(double); }

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

// Parallel tail of the solve, level t, every tail block j:  b~_j = L_j^{(t)-1} b_j
// (kept beside b_j: the neighbours' updates read it).
__global__ void __launch_bounds__(32) k_pcrs_forward(SolveArgs a, CrPlan p, const CrJob *jobs, int t) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const CrJob job = jobs[blockIdx.x];
    if (a.skip && a.skip[job.inst]) return;
    const Inst in = a.inst[job.inst];
    const int n = in.nx, r = blockIdx.y, v = pcr_count(in.P, p.s0), j = job.k;
    double *Ls = reinterpret_cast<double *>(smem_raw), *di = Ls + n * n, *w = di + n;
    crs_load_factor(Ls, di, pcr_blk(p, p.Lt, job, n, v, t, j), n);
    const double *g = crs_vec(a, in, r, j * p.s0);
    for (int i = threadIdx.x; i < n; i += 32) w[i] = g[i];
    __syncwarp();
    crs_forward(Ls, di, w, n);
    double *o = p.bt + r * p.nvt + p.oV_dev[job.inst] + (long long)j * n;
    for (int i = threadIdx.x; i < n; i += 32) o[i] = w[i];
}

// Parallel tail of the solve, level t:  b_j -= A_{j-2^t} b~_{j-2^t} + B_{j+2^t} b~_{j+2^t}.
__global__ void __launch_bounds__(32) k_pcrs_update(SolveArgs a, CrPlan p, const CrJob *jobs, int t) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const CrJob job = jobs[blockIdx.x];
    if (a.skip && a.skip[job.inst]) return;
    const Inst in = a.inst[job.inst];
    const int n = in.nx, r = blockIdx.y, v = pcr_count(in.P, p.s0), j = job.k, sg = 1 << t;
    double *xl = reinterpret_cast<double *>(smem_raw), *xh = xl + n;
    const bool lo = j - sg >= 0, hi = j + sg < v;
    const double *bt = p.bt + r * p.nvt + p.oV_dev[job.inst];
    if (lo)
        for (int i = threadIdx.x; i < n; i += 32) xl[i] = bt[(long long)(j - sg) * n + i];
    if (hi)
        for (int i = threadIdx.x; i < n; i += 32) xh[i] = bt[(long long)(j + sg) * n + i];
    __syncwarp();
    const double *A = lo ? pcr_blk(p, p.At, job, n, v, t, j - sg) : nullptr;
    const double *B = hi ? pcr_blk(p, p.Bt, job, n, v, t, j + sg) : nullptr;
    double *g = crs_vec(a, in, r, j * p.s0);
    for (int row = threadIdx.x; row < n; row += 32) {
        double acc = 0.0;
        if (lo)
            for (int c = 0; c < n; ++c) acc = fma(A[row + c * n], xl[c], acc);
        if (hi)
            for (int c = 0; c < n; ++c) acc = fma(B[row + c * n], xh[c], acc);
        g[row] -= acc;
    }
}

// Every tail block, decoupled after the last tail level:  x_j = L_j^{-T} L_j^{-1} b_j.
__global__ void __launch_bounds__(32) k_pcrs_base(SolveArgs a, CrPlan p, const CrJob *jobs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const CrJob job = jobs[blockIdx.x];
    if (a.skip && a.skip[job.inst]) return;
    const Inst in = a.inst[job.inst];
    const int n = in.nx, r = blockIdx.y;
    double *Ls = reinterpret_cast<double *>(smem_raw), *di = Ls + n * n, *w = di + n;
    crs_load_factor(Ls, di, a.Mf + in.oBlk + (long long)job.k * p.s0 * n * n, n);
    double *g = crs_vec(a, in, r, job.k * p.s0);
    for (int i = threadIdx.x; i < n; i += 32) w[i] = g[i];
    __syncwarp();
    crs_forward(Ls, di, w, n);
    crs_backward(Ls, di, w, n);
    for (int i = threadIdx.x; i < n; i += 32) g[i] = w[i];
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
    if (plan.tail == 0) {
        k_crs_base<<<dim3(plan.n_inst, nr), 32, sm, st>>>(a, plan.inst_list);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++*launches;
    } else {
        if ((e = ensure_smem((const void *)k_pcrs_forward, sm)) != cudaSuccess) return e;
        if ((e = ensure_smem((const void *)k_pcrs_base, sm)) != cudaSuccess) return e;
        for (int t = 0; t < plan.tail; ++t) {
            const int nj = plan.pcr_off[t + 1] - plan.pcr_off[t];
            if (nj == 0) continue;
            k_pcrs_forward<<<dim3(nj, nr), 32, sm, st>>>(a, plan, plan.jobs + plan.pcr_off[t], t);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            k_pcrs_update<<<dim3(nj, nr), 32, 2 * (size_t)nmax * sizeof(double), st>>>(
                a, plan, plan.jobs + plan.pcr_off[t], t);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            *launches += 2;
        }
        const int nb = plan.pcr_base_end - plan.pcr_off[plan.tail];
        k_pcrs_base<<<dim3(nb, nr), 32, sm, st>>>(a, plan, plan.jobs + plan.pcr_off[plan.tail]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++*launches;
    }
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
