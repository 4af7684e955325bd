// Factorization updates (Sec. 6): the stored factor of K is modified in place
// into the factor of K~ = K + Upsilon S Upsilon^T, where every stage matrix
// changes by a low-rank term H~_s = H_s + sum_i delta_i w_i w_i^T (in the
// augmented Lagrangian, the rows of constraints whose activity changed,
// eq. low-rank-update-Hj), instead of factoring K~ from the data.
//
// Per stage, in the order of the factorization (Alg. fact-mod-riccati-update,
// Sec. 6.2), each update column w with sign sigma = sign(delta) (scaled by
// sqrt|delta|) is applied to the stage factor [L^R 0; L^S L^Q] (and, on the
// first stage of the segment, to the rows of L^B) by a sequence of
// sigma-orthogonal column rotations, one per pivot k:
//   r = sqrt(L_kk^2 + sigma w_k^2),  c = r / L_kk,  s = w_k / L_kk,
//   L_ik <- (L_ik + sigma s w_i) / c,  w_i <- c w_i - s L_ik   (i > k),
// which keeps L L^T + sigma w w^T invariant and annihilates w (a Givens
// rotation for sigma = +1, a hyperbolic one for sigma = -1).  After the nu
// input pivots the remaining x part of w is Phi^x: the cost-to-go L^Q L^Q^T
// changes by sigma Phi^x Phi^x^T, so the next stage's matrix H^ = H + [B A]^T
// L^Q L^Q^T [B A] receives the update column [B A]^T Phi^x with the same sign,
// besides its own new rows.  The rank carried from stage to stage grows by the
// rows added on the way.
//
// Stages before the first change in the order of the recursion keep their
// factor and are not touched.  Scope: instances with one segment (P = 1); the
// single coupling block
// M = L^B L^B^T + (L^Q L^Q^T)^{-1} of Sec. 4.3 is rebuilt from the updated
// factors and factored again (nx^3 / 2 flops), which is what the low-rank
// Schur-complement update of Sec. 6.3 and the cyclic-reduction update of
// Sec. 6.4 reduce to for one block.  The strictly upper parts of the stored
// factor (L^{R-1}, and L^{Q-1} at the segment start) and 1 / diag are
// recomputed for the updated stages.
#include <algorithm>

#include "cyq_internal.cuh"

namespace cyq {

namespace {

// Per-warp shared-memory layout (elements of T): stage factor (n x n, ld n|1),
// [B A] of the next stage (nx x n, ld nx), update columns (mcap x n), their
// x residuals Phi (mcap x nx), the L^B rows of the first stage (nx x nu),
// 1 / diag (n), signs (mcap), and the float64 coupling block (nx x nx).
struct UpdGeom {
    int n, nx, nu, ldl, mcap;
    size_t oL, oBA, oW, oPhi, oLB, oD, oSg, size;   // elements of T
    __host__ __device__ UpdGeom(int nx_, int nu_, int mcap_) {
        nx = nx_;
        nu = nu_;
        n = nx + nu;
        ldl = n | 1;
        mcap = mcap_;
        oL = 0;
        oBA = oL + (size_t)ldl * n;
        oW = oBA + (size_t)nx * n;
        oPhi = oW + (size_t)mcap * n;
        oLB = oPhi + (size_t)mcap * nx;
        oD = oLB + (size_t)nx * nu;
        oSg = oD + n;
        size = oSg + mcap;
    }
};

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c) { return fma(a, b, c); }

}  // namespace

template <typename T>
size_t update_smem_bytes(int nx, int nu, int mcap) {
    const UpdGeom G(nx, nu, mcap);
    size_t b = G.size * sizeof(T);
    b = (b + 15) / 16 * 16;
    return b + (size_t)nx * nx * sizeof(double);
}
template size_t update_smem_bytes<float>(int, int, int);
template size_t update_smem_bytes<double>(int, int, int);

namespace {

// One sigma-orthogonal rank-1 modification of the lower factor L (n x n, ld)
// and, when nb > 0, of the extra rows Lb (nb x nlead, ld nb) that take part in
// the first nlead pivots; w (n) and wb (nb) are annihilated.  dinv holds
// 1 / L_kk and is kept up to date.  When phi is not null it receives the x
// part w[nlead..n) as it stands after the first nlead pivots.  Returns false
// if a modified pivot is not positive and finite (a downdate that leaves the
// matrix indefinite).
template <typename T>
__device__ bool rank1(T *L, int n, int ld, T *dinv, T *w, T sigma, int nlead, T *Lb, int nb, T *wb, T *phi,
                      int nphi) {
    const int lane = (int)(threadIdx.x & 31);
    bool ok = true;
    for (int k = 0; k < n; ++k) {
        if (k == nlead && phi) {
            for (int i = lane; i < nphi; i += 32) phi[i] = w[nlead + i];
        }
        const T lkk = L[k + k * ld], wk = w[k], dk = dinv[k];
        T d2 = fma_t(sigma * wk, wk, lkk * lkk);
        if (!finite_pos(d2)) {
            ok = false;
            d2 = lkk * lkk;
        }
        T r, ir;
        pivot(d2, r, ir);
        const T c = r * dk, s = wk * dk, ic = lkk * ir, ss = sigma * s;
        __syncwarp();   // every lane has read L_kk, w_k and 1 / L_kk
        for (int i = k + 1 + lane; i < n; i += 32) {
            const T li = (L[i + k * ld] + ss * w[i]) * ic;
            L[i + k * ld] = li;
            w[i] = fma_t(c, w[i], -s * li);
        }
        if (k < nlead)
            for (int j = lane; j < nb; j += 32) {
                const T lj = (Lb[j + k * nb] + ss * wb[j]) * ic;
                Lb[j + k * nb] = lj;
                wb[j] = fma_t(c, wb[j], -s * lj);
            }
        if (lane == 0) {
            L[k + k * ld] = r;
            dinv[k] = ir;
            w[k] = T(0);
        }
        __syncwarp();
    }
    if (n == nlead && phi) {
        for (int i = lane; i < nphi; i += 32) phi[i] = T(0);
    }
    return ok;
}

// Stored factor of a stage from the working tile: lower triangle, L^{R-1}
// (transposed) above the R diagonal, zeros elsewhere; 1 / diag.
template <typename T>
__device__ void store_stage(T *Ls, T *DIs, const T *L, int n, int nu, int ld, const T *dinv, float *Lc, float *DIc) {
    const int lane = (int)(threadIdx.x & 31);
    for (int e = lane; e < n * n; e += 32) {
        const int b = e / n, a = e - b * n;
        Ls[e] = a >= b ? L[a + b * ld] : T(0);
    }
    for (int i = lane; i < n; i += 32) DIs[i] = dinv[i];
    __syncwarp();
    // L^{R-1}: column cc by lane cc (forward substitution), entry (cc, i) = (L^{R-1})_{i,cc}
    for (int cc = lane; cc < nu; cc += 32)
        for (int i = cc + 1; i < nu; ++i) {
            T acc = T(0);
            for (int k = cc; k < i; ++k) acc = fma_t(-L[i + k * ld], k == cc ? dinv[cc] : Ls[cc + k * n], acc);
            Ls[cc + i * n] = acc * dinv[i];
        }
    if (Lc) {   // the float32 copy of a float64 factor (float32 corrections)
        __syncwarp();
        for (int e = lane; e < n * n; e += 32) Lc[e] = (float)Ls[e];
        for (int i = lane; i < n; i += 32) DIc[i] = (float)dinv[i];
    }
}

template <typename T>
__global__ void __launch_bounds__(32) k_update_factor(UpdateArgs u) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ii = blockIdx.x;
    if (ii >= u.n_inst) return;
    const int inst = u.inst_list[ii];
    const Inst in = u.inst[inst];
    if (in.P != 1) return;   // the host accepts one-segment handles only
    const int lane = (int)(threadIdx.x & 31);
    const int N = in.N, nx = in.nx, nu = in.nu, n = nx + nu;
    const UpdGeom G(nx, nu, u.mcap);
    T *sm = reinterpret_cast<T *>(smem_raw);
    T *L = sm + G.oL, *BA = sm + G.oBA, *W = sm + G.oW, *Phi = sm + G.oPhi, *LB = sm + G.oLB, *dinv = sm + G.oD,
      *sg = sm + G.oSg;
    double *M = reinterpret_cast<double *>(smem_raw + (G.size * sizeof(T) + 15) / 16 * 16);
    const int ld = G.ldl;
    T *Lg = reinterpret_cast<T *>(u.L) + in.oL;
    T *DIg = reinterpret_cast<T *>(u.DI) + in.oDI;
    T *LBg = reinterpret_cast<T *>(u.LB) + in.oLB;
    const long long rbase = in.oN * u.m_max;    // rows of this instance: [stage][m_max]
    const long long wbase = in.oNn * u.m_max;   // their entries: [stage][m_max][nu + nx]
    bool ok = true, rank_over = false;
    bool lb_loaded = false;
    int mp = 0;   // columns carried from the previous stage (their Phi and signs)
    for (int t = 0; t < N; ++t) {
        const int s = seg_stage(0, t, N, 1);
        // a stage without carried columns and without rows of its own keeps its factor
        // (every stage before the first change in the order of the recursion)
        if (mp == 0) {
            bool any = false;
            for (int r = 0; r < u.m_max; ++r) any |= u.delta[rbase + (long long)s * u.m_max + r] != 0.0;
            if (!any) continue;
        }
        // the stage factor and 1 / diag into the working tile
        for (int e = lane; e < n * n; e += 32) {
            const int b = e / n, a = e - b * n;
            if (a >= b) L[a + b * ld] = Lg[(long long)s * n * n + e];
        }
        for (int i = lane; i < n; i += 32) dinv[i] = DIg[(long long)s * n + i];
        if (t == 0) {
            for (int e = lane; e < nx * nu; e += 32) LB[e] = LBg[(long long)s * nx * nu + e];
            lb_loaded = true;
        }
        // [B A] of this stage (the carried columns enter through it): float64 data
        if (t > 0 && mp > 0) {
            const double *B = u.data.B + in.oB + (long long)s * nx * nu;
            const double *A = u.data.A + in.oA + (long long)s * nx * nx;
            for (int e = lane; e < nx * n; e += 32) BA[e] = (T)(e < nx * nu ? B[e] : A[e - nx * nu]);
        }
        __syncwarp();
        // update columns: [B A]^T Phi of the carried columns, then this stage's own rows
        int m = 0;
        for (int j = 0; j < mp; ++j) {
            for (int a = lane; a < n; a += 32) {
                T acc = T(0);
                for (int k = 0; k < nx; ++k) acc = fma_t(BA[k + a * nx], Phi[j * nx + k], acc);
                W[m * n + a] = acc;
            }
            if (lane == 0) sg[m] = sg[j];
            ++m;
        }
        __syncwarp();
        for (int r = 0; r < u.m_max; ++r) {
            const long long ro = (long long)s * u.m_max + r;
            const double dl = u.delta[rbase + ro];
            if (dl == 0.0) continue;
            if (m >= G.mcap) {
                rank_over = true;   // more columns than the workspace carries: refactor this instance
                continue;
            }
            const double sq = sqrt(fabs(dl));
            for (int a = lane; a < n; a += 32) W[m * n + a] = (T)(sq * u.w[wbase + ro * n + a]);
            if (lane == 0) sg[m] = dl > 0.0 ? T(1) : T(-1);
            ++m;
        }
        __syncwarp();
        // apply them one by one; the x residuals after the nu input pivots are carried on
            for (int j = 0; j < m; ++j) {
            T *wj = W + (size_t)j * n;
            // the L^B rows of the first stage take part in the input pivots with zero update entries
            T *wbj = nullptr;
            if (t == 0) {
                wbj = BA;   // scratch (no [B A] is read at the first stage)
                for (int i = lane; i < nx; i += 32) wbj[i] = T(0);
                __syncwarp();
            }
            ok &= rank1<T>(L, n, ld, dinv, wj, sg[j], nu, t == 0 ? LB : nullptr, t == 0 ? nx : 0, wbj,
                           Phi + (size_t)j * nx, nx);
        }
        mp = m;
        __syncwarp();
        store_stage<T>(Lg + (long long)s * n * n, DIg + (long long)s * n, L, n, nu, ld, dinv,
                       u.Lc ? u.Lc + in.oL + (long long)s * n * n : nullptr,
                       u.DIc ? u.DIc + in.oDI + (long long)s * n : nullptr);
        if (t == 0)
            for (int e = lane; e < nx * nu; e += 32) {
                LBg[(long long)s * nx * nu + e] = LB[e];
                if (u.LBc) u.LBc[in.oLB + (long long)s * nx * nu + e] = (float)LB[e];
            }
        __syncwarp();
        if (t == N - 1) {
            // the coupling block: T = L^{Q-1} (in the W tile), its strict lower part (transposed)
            // into the stored Q block, M_bwd = T^T T, M = L^B L^B^T + M_bwd, float64 Cholesky
            const T *LQ = L + nu + nu * ld;
            const T *dq = dinv + nu;
            T *Ti = W;   // nx x nx, ld nx (mcap >= nx is checked by the host)
            if (!lb_loaded) {   // the first stage kept its factor: its L^B rows from the store
                const int s0 = seg_stage(0, 0, N, 1);
                for (int e = lane; e < nx * nu; e += 32) LB[e] = LBg[(long long)s0 * nx * nu + e];
            }
            for (int cc = lane; cc < nx; cc += 32) {
                for (int i = 0; i < cc; ++i) Ti[i + cc * nx] = T(0);
                for (int i = cc; i < nx; ++i) {
                    T v = (i == cc) ? T(1) : T(0);
                    for (int k = cc; k < i; ++k) v = fma_t(-LQ[i + k * ld], Ti[k + cc * nx], v);
                    Ti[i + cc * nx] = v * dq[i];
                }
            }
            __syncwarp();
            T *Lq = Lg + (long long)s * n * n + nu + nu * n;
            float *Lqc = u.Lc ? u.Lc + in.oL + (long long)s * n * n + nu + nu * n : nullptr;
            for (int e = lane; e < nx * nx; e += 32) {
                const int cc = e / nx, i = e - cc * nx;
                if (i > cc) {
                    Lq[cc + i * n] = Ti[i + cc * nx];
                    if (Lqc) Lqc[cc + i * n] = (float)Ti[i + cc * nx];
                }
            }
            double *Mbg = u.Mb + in.oBlk;
            double *Mfg = u.Mf + in.oBlk;
            for (int e = lane; e < nx * nx; e += 32) {
                const int j = e / nx, i = e - j * nx;
                const int k0 = i > j ? i : j;
                T v = T(0);
                for (int k = k0; k < nx; ++k) v = fma_t(Ti[k + i * nx], Ti[k + j * nx], v);
                T f = T(0);
                for (int k = 0; k < nu; ++k) f = fma_t(LB[(i > j ? i : j) + k * nx], LB[(i > j ? j : i) + k * nx], f);
                Mbg[e] = (double)v;
                M[e] = (double)f + (double)v;
            }
            __syncwarp();
            for (int k = 0; k < nx; ++k) {
                double d = M[k + k * nx];
                if (!finite_pos(d)) {
                    ok = false;
                    d = 1.0;
                }
                double l, il;
                pivot(d, l, il);
                __syncwarp();
                if (lane == 0) M[k + k * nx] = l;
                for (int i = k + 1 + lane; i < nx; i += 32) M[i + k * nx] *= il;
                for (int i = lane; i < k; i += 32) M[i + k * nx] = 0.0;
                __syncwarp();
                for (int j = k + 1; j < nx; ++j) {
                    const double ljk = M[j + k * nx];
                    for (int i = j + lane; i < nx; i += 32) M[i + j * nx] = fma(-M[i + k * nx], ljk, M[i + j * nx]);
                }
                __syncwarp();
            }
            for (int e = lane; e < nx * nx; e += 32) Mfg[e] = M[e];
        }
        __syncwarp();
    }
    if (lane == 0) {
        if (rank_over) atomicCAS(u.status + inst, 0, ST_RANK);
        else if (!ok) atomicCAS(u.status + inst, 0, ST_NOT_PD);
    }
}

}  // namespace

cudaError_t launch_update_factor(bool fp64, const UpdateArgs &u, cudaStream_t st) {
    if (u.n_inst == 0) return cudaSuccess;
    const size_t smem = fp64 ? update_smem_bytes<double>(u.max_nx, u.max_nu, u.mcap)
                             : update_smem_bytes<float>(u.max_nx, u.max_nu, u.mcap);
    cudaError_t e;
    if (fp64) {
        e = ensure_smem((const void *)k_update_factor<double>, smem);
        if (e != cudaSuccess) return e;
        k_update_factor<double><<<u.n_inst, 32, smem, st>>>(u);
    } else {
        e = ensure_smem((const void *)k_update_factor<float>, smem);
        if (e != cudaSuccess) return e;
        k_update_factor<float><<<u.n_inst, 32, smem, st>>>(u);
    }
    return cudaGetLastError();
}

}  // namespace cyq
