// Segment factorization: the modified Riccati recursion of one horizon
// segment (paper Sec. 4.2, Alg. fact-mod-riccati) followed by that segment's
// contribution to the Schur complement of the coupling multipliers
// (Sec. 4.3, Alg. fact-parallel-riccati-cr, function compute-schur).
//
// One CTA ("team") per (instance, segment).  Per stage j, processed backward:
//   chol [R^ S^; S^T Q^] = [L^R 0; L^S L^Q]                       (potrf)
//   L^B = B^ L^{R-T},  A^cl = A^ - L^B L^{S T}                      (trsm, gemm)
//   [B^ A^]_{j-1} = A^cl [B A]_{j-1}                                (gemm, P > 1)
//   V = [B A]_{j-1}^T L^Q,  H^_{j-1} = H_{j-1} + V V^T              (trmm, syrk)
// and at the first stage j1 of the segment
//   L^A = A^cl L^{Q-T},  M_fwd = sum_j L^B_j L^B_j^T + L^A L^A^T,
//   M_bwd = L^{Q-T} L^{Q-1} = (L^Q L^Q^T)^{-1},  K = -L^A L^{Q-1}.
// The Schur blocks are written in float64 whatever the factor precision.
// With a single segment the coupling block M = M_fwd + M_bwd is also
// Cholesky-factored here (float64), which is the whole cyclic reduction.
#include "cyq_internal.cuh"

namespace cyq {

namespace {

template <typename T>
__device__ __forceinline__ size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Lower triangle of the stage Hessian [R S; S^T Q] (+ Sigma) of stage s.
template <typename T, int TEAM>
__device__ void load_stage_hessian(T *H, int ld, const Data &d, const Inst &in, int s) {
    const int nx = in.nx, nu = in.nu, N = in.N;
    const int xq = xstate(s, N);
    const double *R = d.R + in.oR + (long long)s * nu * nu;
    const double *Q = d.Q + in.oQ + (long long)xq * nx * nx;
    for (int e = threadIdx.x; e < nu * nu; e += TEAM) {
        const int i = e % nu, j = e / nu;
        if (i >= j) H[i + j * ld] = (T)R[e];
    }
    for (int e = threadIdx.x; e < nx * nx; e += TEAM) {
        const int i = e % nx, j = e / nx;
        if (i >= j) H[(nu + i) + (nu + j) * ld] = (T)Q[e];
    }
    // S_s is nu x nx (element (j,i) at j + i*nu); its transpose fills rows nu.., cols 0..nu-1
    if (s != 0 && d.S) {
        const double *S = d.S + in.oS + (long long)s * nu * nx;
        for (int e = threadIdx.x; e < nu * nx; e += TEAM) {
            const int j = e % nu, i = e / nu;
            H[(nu + i) + j * ld] = (T)S[e];
        }
    } else {
        for (int e = threadIdx.x; e < nu * nx; e += TEAM) {
            const int j = e % nu, i = e / nu;
            H[(nu + i) + j * ld] = T(0);
        }
    }
    if (d.Sig) {
        const double *su = d.Sig + in.oSig + (long long)s * (nu + nx);
        const double *sx = d.Sig + in.oSig + (long long)xq * (nu + nx) + nu;
        team_sync();
        for (int i = threadIdx.x; i < nu; i += TEAM) H[i + i * ld] += (T)su[i];
        for (int i = threadIdx.x; i < nx; i += TEAM) H[(nu + i) + (nu + i) * ld] += (T)sx[i];
    }
}

// [B_s A_s] (nx x (nu+nx), ld nx); A_0 is replaced by zero (x^0 is eliminated).
template <typename T, int TEAM>
__device__ void load_BA(T *BA, const Data &d, const Inst &in, int s) {
    const int nx = in.nx, nu = in.nu;
    const double *B = d.B + in.oB + (long long)s * nx * nu;
    for (int e = threadIdx.x; e < nx * nu; e += TEAM) BA[e] = (T)B[e];
    if (s != 0) {
        const double *A = d.A + in.oA + (long long)s * nx * nx;
        for (int e = threadIdx.x; e < nx * nx; e += TEAM) BA[nx * nu + e] = (T)A[e];
    } else {
        for (int e = threadIdx.x; e < nx * nx; e += TEAM) BA[nx * nu + e] = T(0);
    }
}

template <typename T, int TEAM>
__device__ void store_block(T *dst, const T *src, int rows, int cols, int ld) {
    for (int e = threadIdx.x; e < rows * cols; e += TEAM) dst[e] = src[(e % rows) + (e / rows) * ld];
}

template <typename T, int TEAM>
__device__ void store_block_f64(double *dst, const T *src, int rows, int cols, int ld, double scale) {
    for (int e = threadIdx.x; e < rows * cols; e += TEAM) dst[e] = scale * (double)src[(e % rows) + (e / rows) * ld];
}

}  // namespace

template <typename T, int TEAM>
__global__ void __launch_bounds__(TEAM) k_factor_segments(FactorArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
        const Item wi = a.items[item];
        const Inst in = a.inst[wi.inst];
        const int N = in.N, nx = in.nx, nu = in.nu, P = in.P, c = wi.seg;
        const int nux = nx + nu;
        const int len = seg_len(c, N, P);

        T *H = reinterpret_cast<T *>(smem_raw);    // nux x nux (stage Hessian -> factor)
        T *BA = H + nux * nux;                     // nx x nux  ([B A] of the next stage)
        T *G = BA + nx * nux;                      // nx x nux  ([B^ A^] -> [L^B A^cl])
        T *G2 = G + nx * nux;                      // nx x nux  (next [B^ A^])
        T *V = G2 + nx * nux;                      // nux x nx
        size_t off = (size_t)(V + nux * nx - H) * sizeof(T);
        off = (off + 15) / 16 * 16;
        double *Mf = reinterpret_cast<double *>(smem_raw + off);   // nx x nx float64 accumulator

        T *Lg = reinterpret_cast<T *>(a.L) + in.oL;
        T *LBg = reinterpret_cast<T *>(a.LB) + in.oLB;
        T *Fg = reinterpret_cast<T *>(a.F) + in.oF;

        int s = seg_stage(c, 0, N, P);
        load_stage_hessian<T, TEAM>(H, nux, a.data, in, s);
        load_BA<T, TEAM>(G, a.data, in, s);
        for (int e = threadIdx.x; e < nx * nx; e += TEAM) Mf[e] = 0.0;
        team_sync();

        bool ok = true;
        for (int t = 0; t < len; ++t) {
            s = seg_stage(c, t, N, P);
            const bool hasG = (t == 0) || (c >= 1);
            const bool last = (t == len - 1);
            ok &= team_chol<T, TEAM>(H, nux, nux);
            store_block<T, TEAM>(Lg + (long long)s * nux * nux, H, nux, nux, nux);
            if (hasG) {
                // L^B = B^ L^{R-T}
                team_trsm_rlt<T, TEAM>(G, nx, nu, nx, H, nux);
                // A^cl = A^ - L^B L^{S T}   (L^S = rows nu.. of columns 0..nu-1)
                team_gemm_nt<T, TEAM>(G + nx * nu, nx, G, nx, H + nu, nux, nx, nx, nu, -1);
                store_block<T, TEAM>(LBg + (long long)s * nx * nu, G, nx, nu, nx);
                team_syrk_lower<T, double, TEAM>(Mf, nx, G, nx, nx, nu, +1);
                if (c >= 1 && !last) store_block<T, TEAM>(Fg + (long long)s * nx * nx, G + nx * nu, nx, nx, nx);
            }
            if (!last) {
                const int s2 = seg_stage(c, t + 1, N, P);
                load_BA<T, TEAM>(BA, a.data, in, s2);
                team_sync();
                // V = [B A]^T L^Q : V[a][j] = sum_{k >= j} BA[k][a] L^Q[k][j]
                const T *LQ = H + nu + nu * nux;
                for (int e = threadIdx.x; e < nux * nx; e += TEAM) {
                    const int aa = e % nux, j = e / nux;
                    T acc = T(0);
                    for (int k = j; k < nx; ++k) acc += BA[k + aa * nx] * LQ[k + j * nux];
                    V[aa + j * nux] = acc;
                }
                if (c >= 1) {
                    // [B^ A^]_{s2} = A^cl [B A]_{s2}
                    team_gemm_nn<T, TEAM>(G2, nx, G + nx * nu, nx, BA, nx, nx, nux, nx, 0);
                } else {
                    team_sync();
                }
                load_stage_hessian<T, TEAM>(H, nux, a.data, in, s2);
                team_sync();
                team_syrk_lower<T, T, TEAM>(H, nux, V, nux, nux, nx, +1);
                T *tmp = G; G = G2; G2 = tmp;
            } else {
                const T *LQ = H + nu + nu * nux;
                T *LA = G + nx * nu;
                if (c >= 1) {
                    // L^A = A^cl L^{Q-T}, stored in place of A^cl of the first stage
                    team_trsm_rlt<T, TEAM>(LA, nx, nx, nx, LQ, nux);
                    store_block<T, TEAM>(Fg + (long long)s * nx * nx, LA, nx, nx, nx);
                    team_syrk_lower<T, double, TEAM>(Mf, nx, LA, nx, nx, nx, +1);
                }
                // Tinv = L^{Q -1}
                T *Ti = V;
                team_trtri_lower<T, TEAM>(Ti, nx, LQ, nux, nx);
                // M_bwd = Tinv^T Tinv  -> BA (full symmetric)
                T *Mb = BA;
                for (int e = threadIdx.x; e < nx * nx; e += TEAM) {
                    const int i = e % nx, j = e / nx;
                    const int k0 = i > j ? i : j;
                    T acc = T(0);
                    for (int k = k0; k < nx; ++k) acc += Ti[k + i * nx] * Ti[k + j * nx];
                    Mb[e] = acc;
                }
                team_sync();
                const int cb = (c - 1 + P) % P;
                store_block_f64<T, TEAM>(a.Mb + in.oBlk + (long long)cb * nx * nx, Mb, nx, nx, nx, 1.0);
                if (c >= 1) {
                    // K = -L^A Tinv (row lambda^{b_c}, column lambda^{b_{c-1}})
                    T *Kb = G2;
                    for (int e = threadIdx.x; e < nx * nx; e += TEAM) {
                        const int i = e % nx, j = e / nx;
                        T acc = T(0);
                        for (int k = j; k < nx; ++k) acc += LA[i + k * nx] * Ti[k + j * nx];
                        Kb[e] = -acc;
                    }
                    team_sync();
                    store_block_f64<T, TEAM>(a.Kc + in.oBlk + (long long)c * nx * nx, Kb, nx, nx, nx, 1.0);
                }
                team_symmetrize<double, TEAM>(Mf, nx, nx);
                if (P == 1) {
                    // single coupling block: M = M_fwd + M_bwd, factor it (float64)
                    for (int e = threadIdx.x; e < nx * nx; e += TEAM) Mf[e] += (double)Mb[e];
                    team_sync();
                    ok &= team_chol<double, TEAM>(Mf, nx, nx);
                }
                double *dst = a.Mf + in.oBlk + (long long)c * nx * nx;
                for (int e = threadIdx.x; e < nx * nx; e += TEAM) dst[e] = Mf[e];
            }
        }
        if (!ok && threadIdx.x == 0) atomicCAS(a.status + wi.inst, 0, ST_NOT_PD);
        team_sync();
    }
}

size_t factor_smem_bytes(bool fp64, int nx, int nu) {
    const size_t nux = (size_t)nx + nu;
    const size_t el = fp64 ? 8 : 4;
    size_t off = (nux * nux + 3 * nx * nux + nux * nx) * el;
    off = (off + 15) / 16 * 16;
    return off + (size_t)nx * nx * 8;
}

template <typename T, int TEAM>
static cudaError_t launch_factor_t(size_t smem, const FactorArgs &a, cudaStream_t st) {
    auto k = k_factor_segments<T, TEAM>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<a.n_items, TEAM, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_factor_segments(bool fp64, int team, size_t smem, const FactorArgs &a, cudaStream_t st) {
    if (a.n_items == 0) return cudaSuccess;
    if (fp64) {
        if (team == 32) return launch_factor_t<double, 32>(smem, a, st);
        if (team == 64) return launch_factor_t<double, 64>(smem, a, st);
        return launch_factor_t<double, 128>(smem, a, st);
    }
    if (team == 32) return launch_factor_t<float, 32>(smem, a, st);
    if (team == 64) return launch_factor_t<float, 64>(smem, a, st);
    return launch_factor_t<float, 128>(smem, a, st);
}

}  // namespace cyq
