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

// One CTA per instance: all levels in sequence (blocks in global memory,
// working copies in shared memory).
template <int TEAM>
__global__ void __launch_bounds__(TEAM) k_cr_factor(FactorArgs a, const int *inst_list) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ii = inst_list[blockIdx.x];
    const Inst in = a.inst[ii];
    const int P = in.P, n = in.nx;
    const long long nn = (long long)n * n;
    double *M = a.Mf + in.oBlk, *Mb = a.Mb + in.oBlk, *K = a.Kc + in.oBlk;
    double *U = a.U + in.oBlk, *Y = a.Y + in.oBlk;
    double *W0 = reinterpret_cast<double *>(smem_raw);  // n x n
    double *W1 = W0 + nn;                               // n x n
    double *W2 = W1 + nn;                               // n x n
    bool ok = true;

    for (long long e = threadIdx.x; e < P * nn; e += TEAM) M[e] += Mb[e];
    __threadfence_block();
    team_sync();

    for (int s = 1; s < P; s *= 2) {
        for (int k = s; k < P; k += 2 * s) {
            load_blk<TEAM>(W0, M + k * nn, n, false);
            team_sync();
            ok &= team_chol<double, TEAM>(W0, n, n);
            store_blk<TEAM>(M + k * nn, W0, n);
            // U_k = K_k^T L_k^{-T}
            load_blk<TEAM>(W1, K + k * nn, n, true);
            team_sync();
            team_trsm_rlt<double, TEAM>(W1, n, n, n, W0, n);
            store_blk<TEAM>(U + k * nn, W1, n);
            // Y_k = K_{k+s} L_k^{-T}
            if (k + s < P) {
                load_blk<TEAM>(W2, K + (k + s) * nn, n, false);
                team_sync();
                team_trsm_rlt<double, TEAM>(W2, n, n, n, W0, n);
                store_blk<TEAM>(Y + k * nn, W2, n);
            }
            __threadfence_block();
            team_sync();
        }
        for (int i = 0; i < P; i += 2 * s) {
            load_blk<TEAM>(W0, M + i * nn, n, false);
            team_sync();
            if (i - s >= 0) {
                load_blk<TEAM>(W1, Y + (i - s) * nn, n, false);
                team_sync();
                team_syrk_lower<double, double, TEAM>(W0, n, W1, n, n, n, -1);
                if (i - 2 * s >= 0) {
                    load_blk<TEAM>(W2, U + (i - s) * nn, n, false);
                    team_sync();
                    // K_i <- -Y_{i-s} U_{i-s}^T
                    double *Kn = K + i * nn;
                    for (int e = threadIdx.x; e < n * n; e += TEAM) {
                        const int r = e % n, c = e / n;
                        double acc = 0.0;
                        for (int t = 0; t < n; ++t) acc += W1[r + t * n] * W2[c + t * n];
                        Kn[e] = -acc;
                    }
                    team_sync();
                }
            }
            if (i + s < P) {
                load_blk<TEAM>(W1, U + (i + s) * nn, n, false);
                team_sync();
                team_syrk_lower<double, double, TEAM>(W0, n, W1, n, n, n, -1);
            }
            team_symmetrize<double, TEAM>(W0, n, n);
            store_blk<TEAM>(M + i * nn, W0, n);
            __threadfence_block();
            team_sync();
        }
    }
    load_blk<TEAM>(W0, M, n, false);
    team_sync();
    ok &= team_chol<double, TEAM>(W0, n, n);
    store_blk<TEAM>(M, W0, n);
    if (!ok && threadIdx.x == 0) atomicCAS(a.status + ii, 0, ST_NOT_PD);
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

size_t cr_smem_bytes(int nx) { return (size_t)3 * nx * nx * 8; }

cudaError_t launch_cr_factor(int n_inst_cr, const int *inst_list, int team, size_t smem, const FactorArgs &a,
                             cudaStream_t st) {
    if (n_inst_cr == 0) return cudaSuccess;
    cudaError_t e;
    if (team == 32) {
        e = cudaFuncSetAttribute(k_cr_factor<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_cr_factor<32><<<n_inst_cr, 32, smem, st>>>(a, inst_list);
    } else {
        e = cudaFuncSetAttribute(k_cr_factor<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_cr_factor<128><<<n_inst_cr, 128, smem, st>>>(a, inst_list);
    }
    return cudaGetLastError();
}

cudaError_t launch_cr_solve(int n_inst_cr, const int *inst_list, int team, size_t smem, const SolveArgs &a,
                            cudaStream_t st) {
    if (n_inst_cr == 0) return cudaSuccess;
    cudaError_t e;
    if (team == 32) {
        e = cudaFuncSetAttribute(k_cr_solve<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_cr_solve<32><<<n_inst_cr, 32, smem, st>>>(a, inst_list);
    } else {
        e = cudaFuncSetAttribute(k_cr_solve<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_cr_solve<128><<<n_inst_cr, 128, smem, st>>>(a, inst_list);
    }
    return cudaGetLastError();
}

}  // namespace cyq
