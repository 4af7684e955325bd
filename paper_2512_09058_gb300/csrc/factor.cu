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
//
// When they fit, the raw blocks of the next stage (R, S, Q, Sigma, B, A) are
// copied into shared memory (cp.async) while the current stage is factored;
// the current stage's copy is consumed by the end of the previous step, so
// one buffer suffices.  H^ = H + V V^T is assembled directly from that copy,
// or from global memory for blocks too large to stage.
#include <algorithm>

#include "cyq_internal.cuh"

namespace cyq {

namespace {

// Raw stage record in shared memory (float64): R (nu x nu) | S (nu x nx) |
// Q (nx x nx) | Sigma_u (nu) | Sigma_x (nx) | B (nx x nu) | A (nx x nx).
// [B A] is contiguous and column-major with leading dimension nx.
struct StageLayout {
    int oR, oS, oQ, oSu, oSx, oB, oA, size;
    __device__ StageLayout(int nx, int nu) {
        oR = 0;
        oS = oR + nu * nu;
        oQ = oS + nu * nx;
        oSu = oQ + nx * nx;
        oSx = oSu + nu;
        oB = oSx + nx;
        oA = oB + nx * nu;
        size = oA + nx * nx;
        size = (size + 1) & ~1;
    }
};

// Issue the asynchronous copy of stage s's raw blocks.
template <int TEAM>
__device__ void prefetch_stage(double *buf, const StageLayout &L, const Data &d, const Inst &in, int s) {
    const int nx = in.nx, nu = in.nu, N = in.N, xq = xstate(s, N);
    async_copy_f64<TEAM>(buf + L.oR, d.R + in.oR + (long long)s * nu * nu, nu * nu);
    if (s != 0 && d.S) async_copy_f64<TEAM>(buf + L.oS, d.S + in.oS + (long long)s * nu * nx, nu * nx);
    async_copy_f64<TEAM>(buf + L.oQ, d.Q + in.oQ + (long long)xq * nx * nx, nx * nx);
    if (d.Sig) {
        async_copy_f64<TEAM>(buf + L.oSu, d.Sig + in.oSig + (long long)s * (nu + nx), nu);
        async_copy_f64<TEAM>(buf + L.oSx, d.Sig + in.oSig + (long long)xq * (nu + nx) + nu, nx);
    }
    async_copy_f64<TEAM>(buf + L.oB, d.B + in.oB + (long long)s * nx * nu, nx * nu);
    if (s != 0) async_copy_f64<TEAM>(buf + L.oA, d.A + in.oA + (long long)s * nx * nx, nx * nx);
    cp_async_commit();
}

// Zero the parts of a stage record that the copy does not fill (S_0, A_0, Sigma).
template <int TEAM>
__device__ void stage_zero_fill(double *buf, const StageLayout &L, const Data &d, const Inst &in, int s) {
    const int nx = in.nx, nu = in.nu;
    if (s == 0 || !d.S)
        for (int e = team_tid<TEAM>(); e < nu * nx; e += TEAM) buf[L.oS + e] = 0.0;
    if (!d.Sig)
        for (int e = team_tid<TEAM>(); e < nu + nx; e += TEAM) buf[L.oSu + e] = 0.0;
    if (s == 0)
        for (int e = team_tid<TEAM>(); e < nx * nx; e += TEAM) buf[L.oA + e] = 0.0;
}

// Where the blocks of one stage are read from: the shared-memory copy, or
// global memory directly when the copy would not fit.  Null S / A / Sigma
// pointers stand for zero blocks (S_0, A_0, no regularisation).
struct StageSrc {
    const double *R, *S, *Q, *Su, *Sx, *B, *A;
};

__device__ __forceinline__ StageSrc stage_src_smem(const double *buf, const StageLayout &L) {
    return StageSrc{buf + L.oR, buf + L.oS, buf + L.oQ, buf + L.oSu, buf + L.oSx, buf + L.oB, buf + L.oA};
}

__device__ __forceinline__ StageSrc stage_src_global(const Data &d, const Inst &in, int s) {
    const int nx = in.nx, nu = in.nu, N = in.N, xq = xstate(s, N);
    StageSrc r;
    r.R = d.R + in.oR + (long long)s * nu * nu;
    r.S = (s != 0 && d.S) ? d.S + in.oS + (long long)s * nu * nx : nullptr;
    r.Q = d.Q + in.oQ + (long long)xq * nx * nx;
    r.Su = d.Sig ? d.Sig + in.oSig + (long long)s * (nu + nx) : nullptr;
    r.Sx = d.Sig ? d.Sig + in.oSig + (long long)xq * (nu + nx) + nu : nullptr;
    r.B = d.B + in.oB + (long long)s * nx * nu;
    r.A = s != 0 ? d.A + in.oA + (long long)s * nx * nx : nullptr;
    return r;
}

// Element (a, b), a >= b, of the stage Hessian [R S; S^T Q] + diag(Sigma).
__device__ __forceinline__ double stage_H(const StageSrc &src, int nu, int nx, int a, int b) {
    if (a < nu) return src.R[a + b * nu] + ((a == b && src.Su) ? src.Su[a] : 0.0);
    if (b < nu) return src.S ? src.S[b + (a - nu) * nu] : 0.0;
    const int i = a - nu, j = b - nu;
    return src.Q[i + j * nx] + ((i == j && src.Sx) ? src.Sx[i] : 0.0);
}

// [B A] (nx x (nu+nx)) of a stage into T storage with leading dimension ld.
template <typename T, int TEAM>
__device__ void fill_BA(T *BA, int ld, const StageSrc &src, int nx, int nu) {
    int r, c;
    rect_start(team_tid<TEAM>(), nx, r, c);
    for (; c < nu; rect_advance(r, c, nx, TEAM)) BA[r + c * ld] = (T)src.B[r + c * nx];
    rect_start(team_tid<TEAM>(), nx, r, c);
    for (; c < nx; rect_advance(r, c, nx, TEAM)) BA[r + (nu + c) * ld] = src.A ? (T)src.A[r + c * nx] : T(0);
}

template <typename T, int TEAM>
__device__ void store_block(T *dst, const T *src, int rows, int cols, int ld) {
    int r, c;
    rect_start(team_tid<TEAM>(), rows, r, c);
    for (; c < cols; rect_advance(r, c, rows, TEAM)) dst[r + c * rows] = src[r + c * ld];
}

// Float32 copy of a block a float64 factorization stores (dst may be null).
template <typename T, int TEAM>
__device__ void store_block_f32(float *dst, const T *src, int rows, int cols, int ld) {
    if (!dst) return;
    int r, c;
    rect_start(team_tid<TEAM>(), rows, r, c);
    for (; c < cols; rect_advance(r, c, rows, TEAM)) dst[r + c * rows] = (float)src[r + c * ld];
}

template <typename T, int TEAM>
__device__ void store_block_f64(double *dst, const T *src, int rows, int cols, int ld) {
    int r, c;
    rect_start(team_tid<TEAM>(), rows, r, c);
    for (; c < cols; rect_advance(r, c, rows, TEAM)) dst[r + c * rows] = (double)src[r + c * ld];
}

}  // namespace

// Shared-memory tiles of one work item (T = factor precision).  Every tile
// has an odd leading dimension (pad_ld) except the aliased raw [B A] copy.
struct FactorTiles {
    int ldH, ldV, ldG, ldT;
    size_t nH, nVG, nG, nBA;   // elements
    __host__ __device__ FactorTiles(int nx, int nu, bool need_G2, bool ba_alias) {
        const int nux = nx + nu;
        ldH = pad_ld(nux);
        ldV = pad_ld(nux);
        ldG = pad_ld(nx);
        ldT = pad_ld(nx);
        nH = (size_t)ldH * nux;
        const size_t nV = (size_t)ldV * nx, nGg = (size_t)ldG * nux;
        // without A^cl propagation [B^ A^] lives only until V is formed: one shared tile
        nVG = need_G2 ? nV : (nV > nGg ? nV : nGg);
        nG = need_G2 ? 2 * nGg : 0;
        nBA = ba_alias ? 0 : nGg;
    }
};


// Interior stages t0 <= t < t1 of a segment that carries no A^cl (segment 0):
// float32, one warp, a stage shape fixed at compile time with NU + NX <= 32.
// Lane i holds row i of the current stage matrix in registers, and columns
// reach the other lanes through shuffles, so a stage needs no shared-memory
// round trips and no block barriers.  Entered with H^_{s(t0)} in the H tile
// (leading dimension ldH); leaves H^_{s(t1)} there.  Every value is formed by
// the same operations in the same order as in the shared-memory path below
// (potrf, L^{R-1}, V = [B A]^T L^Q, H^ = H + V V^T), so the results agree.
// Largest nu + nx of the register path (a 32-row matrix and V no longer fit in
// the registers of one thread without spilling).
constexpr int kRegisterRows = 24;

// Interior stages t0 <= t < t1 of a segment that carries no A^cl (segment 0):
// float32, one warp, a stage shape fixed at compile time with NU + NX <= 32.
// Lane i holds row i of the current stage matrix in registers, and columns
// reach the other lanes through shuffles, so a stage needs no shared-memory
// round trips and no block barriers.  Entered with H^_{s(t0)} in the H tile
// (leading dimension ldH); leaves H^_{s(t1)} there.  Every value is formed by
// the same operations in the same order as in the shared-memory path below
// (potrf, L^{R-1}, V = [B A]^T L^Q, H^ = H + V V^T), so the results agree.
template <int NX, int NU>
__device__ __forceinline__ bool stages_in_registers(float *H, int ldH, float *Vs, double *buf, const StageLayout &SL,
                                                    const FactorArgs &a, const Inst &in, int c, int t0, int t1,
                                                    float *Lg, float *DIg, float *BAg) {
    constexpr int NUX = NX + NU;
    constexpr unsigned FULL = 0xffffffffu;
    static_assert(NUX <= 32, "one row per lane");
    static_assert(NX % 4 == 0, "rows of V as 16-byte vectors");
    const int lane = threadIdx.x;
    const int N = in.N, P = in.P;
    float h[NUX];
    static_for<0, NUX>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        h[j] = (lane < NUX && j <= lane) ? H[lane + j * ldH] : 0.0f;
    });
    bool ok = true;
    for (int t = t0; t < t1; ++t) {
        const int s = seg_stage(c, t, N, P), s2 = seg_stage(c, t + 1, N, P);
        prefetch_stage<32>(buf, SL, a.data, in, s2);   // lands while this stage is factored
        // Cholesky, right-looking: column k is scaled by the lanes that own its rows,
        // then row j of column k is broadcast for the rank-1 update of column j
        float dl = 1.0f;
        static_for<0, NUX>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            float d = __shfl_sync(FULL, h[k], k);
            if (!finite_pos(d)) {
                ok = false;
                d = 1.0f;
            }
            float l, il;
            pivot(d, l, il);
            if (lane == k) {
                h[k] = l;
                dl = il;
            } else if (lane > k) {
                h[k] *= il;
            }
            static_for<k + 1, NUX>([&](auto jc) {
                constexpr int j = decltype(jc)::value;
                const float ljk = __shfl_sync(FULL, h[k], j);
                if (lane >= j) h[j] = fmaf(-h[k], ljk, h[j]);
            });
        });
        // X = L^{R-1}, row m of X in lane m: X[m][k] = -1/L_mm sum_{q=k}^{m-1} L[m][q] X[q][k]
        float x[NU], acc[NU];
        static_for<0, NU>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            x[k] = acc[k] = 0.0f;
        });
        static_for<0, NU>([&](auto mc) {
            constexpr int m = decltype(mc)::value;
            if (lane == m) {
                static_for<0, m>([&](auto kc) {
                    constexpr int k = decltype(kc)::value;
                    x[k] = -acc[k] * dl;
                });
                x[m] = dl;
            }
            static_for<0, m + 1>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                const float xm = __shfl_sync(FULL, x[k], m);
                if (lane > m) acc[k] = fmaf(h[m], xm, acc[k]);
            });
        });
        // stored factor: lower triangle, X transposed above the diagonal of the R block, zeros elsewhere
        float *Ls = Lg + (long long)s * NUX * NUX;
        if (lane < NUX) {
            static_for<0, NUX>([&](auto jc) {
                constexpr int j = decltype(jc)::value;
                if (j <= lane)
                    Ls[lane + j * NUX] = h[j];
                else if (!(lane < NU && j < NU))
                    Ls[lane + j * NUX] = 0.0f;
            });
            DIg[(long long)s * NUX + lane] = dl;
        }
        if (lane < NU) {
            static_for<0, NU>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                if (k < lane) Ls[k + lane * NUX] = x[k];
            });
        }
        // raw blocks of stage s2
        stage_zero_fill<32>(buf, SL, a.data, in, s2);
        cp_async_wait_all();
        __syncwarp();
        const StageSrc src = stage_src_smem(buf, SL);
        // V = [B A]^T L^Q, row `lane`: v[j] = sum_{k >= j} BA[k][lane] L^Q[k][j]
        float v[NX];
        static_for<0, NX>([&](auto jc) { v[decltype(jc)::value] = 0.0f; });
        const double *bacol = lane < NU ? src.B + lane * NX : src.A + (lane - NU) * NX;   // column `lane` of [B A]
        float *badst = (BAg && lane < NUX) ? BAg + (long long)s2 * NX * NUX + lane * NX : nullptr;
        static_for<0, NX>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            const float ba = lane < NUX ? (float)bacol[k] : 0.0f;
            if (badst) badst[k] = ba;
            static_for<0, k + 1>([&](auto jc) {
                constexpr int j = decltype(jc)::value;
                const float lq = __shfl_sync(FULL, h[NU + j], NU + k);
                v[j] = fmaf(ba, lq, v[j]);
            });
        });
        // H^_{s2} = H_{s2} + V V^T, row `lane`; rows of V are read back from shared
        // memory as 16-byte broadcasts
        if (lane < NUX) {
            static_for<0, NX / 4>([&](auto qc) {
                constexpr int j = 4 * decltype(qc)::value;
                *reinterpret_cast<float4 *>(Vs + lane * NX + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            });
        }
        __syncwarp();
        const int ra = lane < NU ? lane : 0, qa = lane >= NU && lane < NUX ? lane - NU : 0;
        static_for<0, NUX>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            // raw entry (lane, b), lane >= b: R, S^T or Q, plus Sigma on the diagonal (float64, as stage_H)
            double raw;
            if constexpr (b < NU)
                raw = lane < NU ? src.R[ra + b * NU] + (lane == b ? src.Su[b] : 0.0) : src.S[b + qa * NU];
            else
                raw = src.Q[qa + (b - NU) * NX] + (lane == b ? src.Sx[b - NU] : 0.0);
            float hb = (lane < NUX && b <= lane) ? (float)raw : 0.0f;
            static_for<0, NX / 4>([&](auto qc) {
                constexpr int j = 4 * decltype(qc)::value;
                const float4 vb = *reinterpret_cast<const float4 *>(Vs + b * NX + j);
                hb = fmaf(v[j], vb.x, hb);
                hb = fmaf(v[j + 1], vb.y, hb);
                hb = fmaf(v[j + 2], vb.z, hb);
                hb = fmaf(v[j + 3], vb.w, hb);
            });
            h[b] = b <= lane ? hb : 0.0f;
        });
        __syncwarp();   // every lane has read the stage copy and V before they are overwritten
    }
    if (lane < NUX) {
        static_for<0, NUX>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            if (j <= lane) H[lane + j * ldH] = h[j];
        });
    }
    __syncwarp();
    return ok;
}

template <typename T, int TEAM, int NXC, int NUC>
__global__ void __launch_bounds__(TEAM < 32 ? 32 : TEAM) k_factor_segments(FactorArgs a) {
    extern __shared__ __align__(16) unsigned char smem_all[];
    // TEAM < 32: 32 / TEAM teams per CTA (one warp), each with its own item and
    // its own a.smem_team bytes of shared memory
    constexpr int TPC = TEAM < 32 ? 32 / TEAM : 1;
    const int team = TEAM < 32 ? (int)threadIdx.x / TEAM : 0;
    const int tid = team_tid<TEAM>();
    unsigned char *smem_raw = smem_all + (size_t)team * a.smem_team;
    for (int item = blockIdx.x * TPC + team; item < a.n_items; item += gridDim.x * TPC) {
        const Item wi = a.items[item];
        if (a.skip && a.skip[wi.inst]) continue;
        const Inst in = a.inst[wi.inst];
        // NXC / NUC > 0: kernel compiled for that stage shape (every item of the launch has it)
        const int nx = NXC > 0 ? NXC : in.nx, nu = NUC > 0 ? NUC : in.nu;
        const int N = in.N, P = in.P, c = wi.seg;
        const int nux = nx + nu;
        const int len = seg_len(c, N, P);
        const StageLayout SL(nx, nu);
        const bool propagate = c >= 1;   // segment 0 never carries A^cl (A_0 = 0, S_0 = 0)

        const bool staged = a.stage_in_smem;
        // [B A] of the next stage: aliased to the staged float64 copy, or
        // converted into its own shared-memory tile.
        const bool ba_alias = staged && sizeof(T) == 8;
        const FactorTiles TL(nx, nu, a.need_G2, ba_alias);
        const int ldH = TL.ldH, ldV = TL.ldV, ldG = TL.ldG, ldT = TL.ldT;
        double *buf = reinterpret_cast<double *>(smem_raw);         // raw stage copy (staged mode)
        double *Mf = buf + (staged ? SL.size : 0);                   // nx x nx float64 accumulator
        T *H = reinterpret_cast<T *>(Mf + nx * nx);                  // nux x nux (stage Hessian -> factor)
        T *V = H + TL.nH;                                            // nux x nx
        // [B^ A^] -> [L^B A^cl]; without propagation it shares V's tile (used before V is formed)
        T *G = a.need_G2 ? V + TL.nVG : V;                           // nx x nux
        T *G2 = G + (a.need_G2 ? TL.nG / 2 : 0);                     // nx x nux  (next [B^ A^], P > 1)
        T *BAc = V + TL.nVG + TL.nG;                                 // nx x nux  ([B A] tile)
        T *dinv = BAc + TL.nBA;                                      // nux
        const int ldBA = ba_alias ? nx : ldG;

        T *Lg = reinterpret_cast<T *>(a.L) + in.oL;
        // float64 factorization that also writes a float32 copy for float32 correction sweeps
        const bool copy32 = sizeof(T) == 8 && a.Lc != nullptr;
        T *LBg = reinterpret_cast<T *>(a.LB) + in.oLB;
        T *Fg = reinterpret_cast<T *>(a.F) + in.oF;
        T *DIg = reinterpret_cast<T *>(a.DI) + in.oDI;

        // first stage: H^ = H and [B^ A^] = [B A]
        int s = seg_stage(c, 0, N, P);
        StageSrc src;
        if (staged) {
            prefetch_stage<TEAM>(buf, SL, a.data, in, s);
            stage_zero_fill<TEAM>(buf, SL, a.data, in, s);
            cp_async_wait_all();
            src = stage_src_smem(buf, SL);
        } else {
            src = stage_src_global(a.data, in, s);
        }
        for (int e = tid; e < nx * nx; e += TEAM) Mf[e] = 0.0;
        team_sync<TEAM>();
        {
            int r, q;
            tri_index(tid, r, q);
            for (; r < nux; tri_advance(r, q, TEAM)) H[r + q * ldH] = (T)stage_H(src, nu, nx, r, q);
            fill_BA<T, TEAM>(G, ldG, src, nx, nu);
        }
        team_sync<TEAM>();

        bool ok = true;
        for (int t = 0; t < len; ++t) {
            if constexpr (sizeof(T) == 4 && TEAM == 32 && NXC > 0 && NXC % 4 == 0 && NXC + NUC <= kRegisterRows) {
                // V's tile (>= nux * nx floats) holds the rows of V; it must be 16-byte aligned
                if (t == 1 && !propagate && staged && len > 2 && (reinterpret_cast<size_t>(V) & 15) == 0) {
                    ok &= stages_in_registers<NXC, NUC>(reinterpret_cast<float *>(H), ldH,
                                                        reinterpret_cast<float *>(V), buf, SL, a, in, c, 1,
                                                        len - 1, reinterpret_cast<float *>(Lg),
                                                        reinterpret_cast<float *>(DIg),
                                                        reinterpret_cast<float *>(a.BAf) + (a.BAf ? in.oBA : 0));
                    t = len - 1;   // the last stage closes the segment below
                }
            }
            s = seg_stage(c, t, N, P);
            const bool hasG = (t == 0) || propagate;
            const bool last = (t == len - 1);
            int s2 = 0;
            if (!last) {
                s2 = seg_stage(c, t + 1, N, P);
                // the copy of the next stage overlaps with the factorization below
                if (staged) prefetch_stage<TEAM>(buf, SL, a.data, in, s2);
            }
            ok &= team_chol<T, TEAM>(H, nux, ldH, dinv);
            // L^{R-1} (strictly lower part) into the free upper triangle of the R block,
            // transposed: entry (k, i), k < i, holds (L^{R-1})_{ik}.  The solve sweeps
            // then apply L^{R-1} and L^{R-T} as parallel matrix-vector products.
            for (int cc = tid; cc < nu; cc += TEAM)
                for (int i = cc + 1; i < nu; ++i) {
                    T acc = T(0);
                    for (int k = cc; k < i; ++k)
                        acc = fma(-H[i + k * ldH], k == cc ? dinv[cc] : H[cc + k * ldH], acc);
                    H[cc + i * ldH] = acc * dinv[i];
                }
            team_sync<TEAM>();
            store_block<T, TEAM>(Lg + (long long)s * nux * nux, H, nux, nux, ldH);
            for (int i = tid; i < nux; i += TEAM) DIg[(long long)s * nux + i] = dinv[i];
            if (copy32) {
                store_block_f32<T, TEAM>(a.Lc + in.oL + (long long)s * nux * nux, H, nux, nux, ldH);
                for (int i = tid; i < nux; i += TEAM) a.DIc[in.oDI + (long long)s * nux + i] = (float)dinv[i];
            }
            if (hasG) {
                // L^B = B^ L^{R-T}
                team_trsm_rlt<T, TEAM>(G, nx, nu, ldG, H, ldH, dinv);
                // A^cl = A^ - L^B L^{S T}   (L^S = rows nu.. of columns 0..nu-1)
                team_gemm_nt<T, TEAM>(G + ldG * nu, ldG, G, ldG, H + nu, ldH, nx, nx, nu, -1);
                store_block<T, TEAM>(LBg + (long long)s * nx * nu, G, nx, nu, ldG);
                if (copy32) store_block_f32<T, TEAM>(a.LBc + in.oLB + (long long)s * nx * nu, G, nx, nu, ldG);
                team_syrk_lower<T, double, TEAM>(Mf, nx, G, ldG, nx, nu, +1);
                if (propagate && !last) {
                    store_block<T, TEAM>(Fg + (long long)s * nx * nx, G + ldG * nu, nx, nx, ldG);
                    if (copy32) store_block_f32<T, TEAM>(a.Fc + in.oF + (long long)s * nx * nx, G + ldG * nu, nx, nx, ldG);
                }
            }
            if (!last) {
                if (staged) {
                    stage_zero_fill<TEAM>(buf, SL, a.data, in, s2);
                    cp_async_wait_all();
                    team_sync<TEAM>();   // every thread's copies have landed
                    src = stage_src_smem(buf, SL);
                } else {
                    src = stage_src_global(a.data, in, s2);
                }
                const T *BA;
                if (ba_alias) {
                    BA = reinterpret_cast<const T *>(src.B);
                    if (copy32)   // float32 [B A] of stage s2 for the float32 correction sweeps
                        store_block_f32<T, TEAM>(reinterpret_cast<float *>(a.BAf) + in.oBA + (long long)s2 * nx * nux, BA,
                                                 nx, nux, nx);
                } else {
                    fill_BA<T, TEAM>(BAc, ldBA, src, nx, nu);
                    team_sync<TEAM>();
                    BA = BAc;
                    // float32 copy for the solve sweeps (no conversions there)
                    if (a.BAf)
                        store_block_f32<T, TEAM>(reinterpret_cast<float *>(a.BAf) + in.oBA + (long long)s2 * nx * nux,
                                                 BAc, nx, nux, ldBA);
                }
                // V = [B A]^T L^Q : V[a][j] = sum_{k >= j} BA[k][a] L^Q[k][j]
                const T *LQ = H + nu + nu * ldH;
                {
                    int aa, j;
                    rect_start(tid, nux, aa, j);
                    for (; j < nx; rect_advance(aa, j, nux, TEAM)) {
                        const T *ba = BA + aa * ldBA, *lq = LQ + j * ldH;
                        T acc = T(0);
#pragma unroll 4
                        for (int k = j; k < nx; ++k) acc = fma(ba[k], lq[k], acc);
                        V[aa + j * ldV] = acc;
                    }
                }
                if (propagate) {
                    // [B^ A^]_{s2} = A^cl [B A]_{s2}
                    team_gemm_nn<T, TEAM>(G2, ldG, G + ldG * nu, ldG, BA, ldBA, nx, nux, nx, 0);
                } else {
                    team_sync<TEAM>();
                }
                // H^_{s2} = H_{s2} + V V^T  (lower triangle, straight from the raw record)
                {
                    int r, q;
                    tri_index(tid, r, q);
                    for (; r < nux; tri_advance(r, q, TEAM)) {
                        T acc = (T)stage_H(src, nu, nx, r, q);
                        const T *vr = V + r, *vq = V + q;
#pragma unroll 4
                        for (int k = 0; k < nx; ++k) acc = fma(vr[k * ldV], vq[k * ldV], acc);
                        H[r + q * ldH] = acc;
                    }
                }
                team_sync<TEAM>();
                if (a.need_G2) {
                    T *tmp = G; G = G2; G2 = tmp;
                }
            } else {
                const T *LQ = H + nu + nu * ldH;
                const T *dq = dinv + nu;
                T *LA = G + ldG * nu;
                if (propagate) {
                    // L^A = A^cl L^{Q-T}, stored in place of A^cl of the first stage
                    team_trsm_rlt<T, TEAM>(LA, nx, nx, ldG, LQ, ldH, dq);
                    store_block<T, TEAM>(Fg + (long long)s * nx * nx, LA, nx, nx, ldG);
                    if (copy32) store_block_f32<T, TEAM>(a.Fc + in.oF + (long long)s * nx * nx, LA, nx, nx, ldG);
                    team_syrk_lower<T, double, TEAM>(Mf, nx, LA, ldG, nx, nx, +1);
                }
                // Tinv = L^{Q -1}  (in V's tile; L^Q is not needed after this)
                T *Ti = V;
                team_trtri_lower<T, TEAM>(Ti, ldT, LQ, ldH, nx, dq);
                // and its strictly lower part, transposed, into the upper triangle of the
                // stored Q block of this (first) stage, for the sweeps' end-of-segment solves
                {
                    T *Lq = Lg + (long long)s * nux * nux + nu + nu * nux;
                    int i, cc;
                    rect_start(tid, nx, i, cc);
                    for (; cc < nx; rect_advance(i, cc, nx, TEAM))
                        if (i > cc) {
                            Lq[cc + i * nux] = Ti[i + cc * ldT];
                            if (copy32)
                                a.Lc[in.oL + (long long)s * nux * nux + nu + nu * nux + cc + i * nux] = (float)Ti[i + cc * ldT];
                        }
                }
                // M_bwd = Tinv^T Tinv  (full symmetric, in the H tile, leading dimension ldT)
                T *Mb = H;
                {
                    int i, j;
                    rect_start(tid, nx, i, j);
                    for (; j < nx; rect_advance(i, j, nx, TEAM)) {
                        const int k0 = i > j ? i : j;
                        T acc = T(0);
                        for (int k = k0; k < nx; ++k) acc = fma(Ti[k + i * ldT], Ti[k + j * ldT], acc);
                        Mb[i + j * ldT] = acc;
                    }
                }
                team_sync<TEAM>();
                const int cb = (c - 1 + P) % P;
                store_block_f64<T, TEAM>(a.Mb + in.oBlk + (long long)cb * nx * nx, Mb, nx, nx, ldT);
                team_symmetrize<double, TEAM>(Mf, nx, nx);
                if (P == 1) {
                    // single coupling block: M = M_fwd + M_bwd, factor it (float64)
                    int i, j;
                    rect_start(tid, nx, i, j);
                    for (; j < nx; rect_advance(i, j, nx, TEAM)) Mf[i + j * nx] += (double)Mb[i + j * ldT];
                    team_sync<TEAM>();
                    ok &= team_chol<double, TEAM>(Mf, nx, nx);
                }
                double *dst = a.Mf + in.oBlk + (long long)c * nx * nx;
                for (int e = tid; e < nx * nx; e += TEAM) dst[e] = Mf[e];
                if (propagate) {
                    // K = -L^A Tinv (row lambda^{b_c}, column lambda^{b_{c-1}}), reusing the H tile
                    team_sync<TEAM>();   // M_bwd has been read
                    T *Kb = H;
                    int i, j;
                    rect_start(tid, nx, i, j);
                    for (; j < nx; rect_advance(i, j, nx, TEAM)) {
                        T acc = T(0);
                        for (int k = j; k < nx; ++k) acc = fma(LA[i + k * ldG], Ti[k + j * ldT], acc);
                        Kb[i + j * ldT] = -acc;
                    }
                    team_sync<TEAM>();
                    store_block_f64<T, TEAM>(a.Kc + in.oBlk + (long long)c * nx * nx, Kb, nx, nx, ldT);
                }
            }
        }
        if (!ok && tid == 0) atomicCAS(a.status + wi.inst, 0, ST_NOT_PD);
        team_sync<TEAM>();
    }
}

// ---------------------------------------------------------------------------
// Float64 stage factor, two items per warp, for small stage shapes fixed at
// compile time (NU + NX <= 16) and segments without A^cl (one segment per
// instance).
//
// Each FP64 unit serves one SM sub-partition and takes ~64 cycles per warp
// instruction whether 1 or 32 lanes are active, while a dependent FP64 chain
// waits ~70 cycles: with one warp per sub-partition the float64 factor is
// bound by the FP64 warp instructions and by the other instructions between
// them.  Here a team of 16 threads owns an item, so every FP64 instruction
// serves two items, and four warps per CTA put one warp on each
// sub-partition.  The lower triangle of the stage matrix lives in registers,
// its entries dealt out column-major over the team (entry f to thread f % 16,
// slot f / 16): the entries a pivot still updates are a suffix of that order,
// so few lanes idle, and each column reaches the team through shared memory
// once per pivot.
//
// The arithmetic of every entry is that of the shared-memory path above
// (team_chol, L^{R-1}, trsm, syrk, V, H^ = H + V V^T, trtri, M_bwd, the
// coupling Cholesky) in the same order, so the stored factor is bit for bit
// the same.
// ---------------------------------------------------------------------------
namespace {

constexpr int kPairTeam = 16;          // threads per item
constexpr int kPairItemsPerCta = 8;    // four warps

// Positive and finite (the test of finite_pos on the bits, without FP64 instructions).
__device__ __forceinline__ bool pos_finite_bits(double d) {
    const int hi = __double2hiint(d), lo = __double2loint(d);
    return hi >= 0 && (hi | lo) != 0 && ((hi >> 20) & 0x7ff) != 0x7ff;
}

// The raw blocks of stage s as 16-byte copies: every block of the compiled
// shapes has an even number of doubles; `pairs` says that the instance's
// blocks start on 16-byte boundaries (else 8-byte copies).
template <int NX, int NU>
__device__ void prefetch_stage_pairs(double *buf, const StageLayout &L, const Data &d, const Inst &in, int s,
                                     bool pairs) {
    if (!pairs) {
        prefetch_stage<kPairTeam>(buf, L, d, in, s);
        return;
    }
    const int N = in.N, xq = xstate(s, N);
    async_copy_f64x2<kPairTeam>(buf + L.oR, d.R + in.oR + (long long)s * NU * NU, NU * NU);
    if (s != 0 && d.S) async_copy_f64x2<kPairTeam>(buf + L.oS, d.S + in.oS + (long long)s * NU * NX, NU * NX);
    async_copy_f64x2<kPairTeam>(buf + L.oQ, d.Q + in.oQ + (long long)xq * NX * NX, NX * NX);
    if (d.Sig) {
        async_copy_f64x2<kPairTeam>(buf + L.oSu, d.Sig + in.oSig + (long long)s * (NU + NX), NU);
        async_copy_f64x2<kPairTeam>(buf + L.oSx, d.Sig + in.oSig + (long long)xq * (NU + NX) + NU, NX);
    }
    async_copy_f64x2<kPairTeam>(buf + L.oB, d.B + in.oB + (long long)s * NX * NU, NX * NU);
    if (s != 0) async_copy_f64x2<kPairTeam>(buf + L.oA, d.A + in.oA + (long long)s * NX * NX, NX * NX);
    cp_async_commit();
}

// x + 0.0 without an FP64 instruction (-0 becomes +0, everything else is unchanged).
__device__ __forceinline__ double plus_zero(double x) {
    return __double_as_longlong(x) == (long long)0x8000000000000000ULL ? 0.0 : x;
}

// Per-item shared memory (doubles): raw stage record | H tile | V (row-major) |
// L^B | M_fwd | 1/diag | two column buffers.
template <int NX, int NU>
struct PairLayout {
    static constexpr int NUX = NX + NU;
    static constexpr int ldH = NUX | 1, ldVr = (NX + 3) & ~1, ldG = NX | 1, ldT = NX | 1;
    static constexpr int raw = (NU * NU + NU * NX + NX * NX + NUX + NX * NU + NX * NX + 1) & ~1;
    static constexpr int oH = raw;
    static constexpr int oV = (oH + ldH * NUX + 1) & ~1;
    static constexpr int oG = oV + NUX * ldVr;
    static constexpr int oMf = oG + ldG * NU;
    static constexpr int oD = oMf + NX * NX;
    static constexpr int oC = oD + NUX;
    static constexpr int size = (oC + 2 * NUX + 1) & ~1;
    static constexpr int ntri = NUX * (NUX + 1) / 2;
    static constexpr int slots = (ntri + kPairTeam - 1) / kPairTeam;
    static constexpr size_t bytes = (size_t)kPairItemsPerCta * size * 8;
    static_assert(NUX <= kPairTeam, "one row of V per thread");
    static_assert(NX % 2 == 0 && NU % 2 == 0, "rows of V and the raw blocks as 16-byte pairs");
    static_assert(ldT * NX <= NUX * ldVr && ldT * NX <= ldH * NUX, "L^{Q-1} and M_bwd reuse the V and H tiles");
};

// Column-major position f of a lower-triangle entry of an n x n matrix: (row, column).
__device__ __forceinline__ void colmajor_entry(int f, int n, int &r, int &c) {
    c = 0;
    while (f >= n - c) {
        f -= n - c;
        ++c;
    }
    r = c + f;
}

template <int NX, int NU>
__global__ void __launch_bounds__(kPairTeam * kPairItemsPerCta) k_factor_pairs(FactorArgs a) {
    using LY = PairLayout<NX, NU>;
    constexpr int NUX = LY::NUX, ldH = LY::ldH, ldVr = LY::ldVr, ldG = LY::ldG, ldT = LY::ldT;
    constexpr int NT = LY::ntri, NS = LY::slots;
    extern __shared__ __align__(16) unsigned char smem_all[];
    const int team = threadIdx.x / kPairTeam, q = threadIdx.x % kPairTeam;
    const int item = blockIdx.x * kPairItemsPerCta + team;
    if (item >= a.n_items) return;   // the team leaves as a whole; only team barriers follow
    const Item wi = a.items[item];
    if (a.skip && a.skip[wi.inst]) return;
    const Inst in = a.inst[wi.inst];
    const int N = in.N, P = in.P, c = wi.seg;
    const int len = seg_len(c, N, P);
    const StageLayout SL(NX, NU);
    const unsigned tmask = 0xffffu << (threadIdx.x & 16);
    const int tbase = threadIdx.x & 16;
    double *buf = reinterpret_cast<double *>(smem_all) + (size_t)team * LY::size;
    double *H = buf + LY::oH, *V = buf + LY::oV, *G = buf + LY::oG, *Mf = buf + LY::oMf, *dinv = buf + LY::oD;
    double *colbuf = buf + LY::oC;
    double *Lg = reinterpret_cast<double *>(a.L) + in.oL;
    double *LBg = reinterpret_cast<double *>(a.LB) + in.oLB;
    double *DIg = reinterpret_cast<double *>(a.DI) + in.oDI;
    const bool copy32 = a.Lc != nullptr;
    const Data &dd = a.data;
    const bool pairs = ((reinterpret_cast<size_t>(dd.R) | reinterpret_cast<size_t>(dd.S) |
                         reinterpret_cast<size_t>(dd.Q) | reinterpret_cast<size_t>(dd.Sig) |
                         reinterpret_cast<size_t>(dd.B) | reinterpret_cast<size_t>(dd.A)) & 15) == 0 &&
                       ((in.oR | in.oS | in.oQ | in.oSig | in.oB | in.oA) & 1) == 0;

    // this thread's entries of the stage matrix: (row, column) and the raw-record
    // offsets of R / S^T / Q and of Sigma (diagonal entries)
    int er[NS], ec[NS], eraw[NS], esig[NS];
    static_for<0, NS>([&](auto mc) {
        constexpr int m = decltype(mc)::value;
        const int f = q + kPairTeam * m;
        int r = 0, cc = 0;
        if (f < NT) colmajor_entry(f, NUX, r, cc);
        er[m] = r;
        ec[m] = cc;
        if (r < NU) {
            eraw[m] = SL.oR + r + cc * NU;
            esig[m] = SL.oSu + r;
        } else if (cc < NU) {
            eraw[m] = SL.oS + cc + (r - NU) * NU;
            esig[m] = -1;
        } else {
            eraw[m] = SL.oQ + (r - NU) + (cc - NU) * NX;
            esig[m] = SL.oSx + r - NU;
        }
    });
    // raw entry of the stage Hessian (stage_H's arithmetic: R and Q entries get
    // Sigma on the diagonal and + 0.0 elsewhere, S entries nothing)
    auto raw_entry = [&](int m) -> double {
        const double v = buf[eraw[m]];
        if (esig[m] < 0) return v;
        return er[m] == ec[m] ? v + buf[esig[m]] : plus_zero(v);
    };

    // first stage: H^ = H, B^ = B
    int s = seg_stage(c, 0, N, P);
    prefetch_stage_pairs<NX, NU>(buf, SL, a.data, in, s, pairs);
    stage_zero_fill<kPairTeam>(buf, SL, a.data, in, s);
    cp_async_wait_all();
    for (int e = q; e < NX * NX; e += kPairTeam) Mf[e] = 0.0;
    team_sync<kPairTeam>();
    double h[NS];
    static_for<0, NS>([&](auto mc) {
        constexpr int m = decltype(mc)::value;
        h[m] = (q + kPairTeam * m < NT) ? raw_entry(m) : 0.0;
    });
    for (int e = q; e < NX * NU; e += kPairTeam) G[e % NX + (e / NX) * ldG] = buf[SL.oB + e];
    team_sync<kPairTeam>();

    bool ok = true;
    for (int t = 0; t < len; ++t) {
        s = seg_stage(c, t, N, P);
        const bool last = (t == len - 1);
        int s2 = 0;
        if (!last) {
            s2 = seg_stage(c, t + 1, N, P);
            prefetch_stage_pairs<NX, NU>(buf, SL, a.data, in, s2, pairs);   // lands while this stage is factored
        }
        // Cholesky in registers (team_chol's arithmetic)
        double myil = 0.0;
        static_for<0, NUX>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            constexpr int Fk = k * NUX - k * (k - 1) / 2;               // entry (k, k)
            constexpr int Fk1 = (k + 1) * NUX - (k + 1) * k / 2;        // first entry of column k + 1
            double *col = colbuf + (k & 1) * NUX;
            double d = __shfl_sync(tmask, h[Fk / kPairTeam], tbase + Fk % kPairTeam);
            if (!pos_finite_bits(d)) {
                ok = false;
                d = 1.0;
            }
            double l, il;
            pivot(d, l, il);
            if (q == k) myil = il;
            if (q == Fk % kPairTeam) h[Fk / kPairTeam] = l;
            // column k below the diagonal: scale, then publish
            static_for<(Fk + 1) / kPairTeam, (Fk1 - 1) / kPairTeam + 1>([&](auto mc) {
                constexpr int m = decltype(mc)::value;
                const int f = q + kPairTeam * m;
                if (f > Fk && f < Fk1) {
                    h[m] *= il;
                    col[er[m]] = h[m];
                }
            });
            team_sync<kPairTeam>();
            // trailing update: the entries of columns k+1.. (a suffix of the slots)
            if constexpr (Fk1 < NT) {
                static_for<Fk1 / kPairTeam, NS>([&](auto mc) {
                    constexpr int m = decltype(mc)::value;
                    const int f = q + kPairTeam * m;
                    if (f >= Fk1 && f < NT) h[m] = fma(-col[er[m]], col[ec[m]], h[m]);
                });
            }
        });
        // the factor into the H tile (lower triangle) and 1/diag
        static_for<0, NS>([&](auto mc) {
            constexpr int m = decltype(mc)::value;
            if (q + kPairTeam * m < NT) H[er[m] + ec[m] * ldH] = h[m];
        });
        if (q < NUX) dinv[q] = myil;
        team_sync<kPairTeam>();
        // L^{R-1}, transposed into the upper triangle of the R block (column q of it)
        if (q < NU) {
            for (int i = q + 1; i < NU; ++i) {
                double acc = 0.0;
                for (int k = q; k < i; ++k) acc = fma(-H[i + k * ldH], k == q ? dinv[q] : H[q + k * ldH], acc);
                H[q + i * ldH] = acc * dinv[i];
            }
        }
        team_sync<kPairTeam>();
        if (q < NUX) {
            // row q of the stored factor: lower triangle, L^{R-1} above the R diagonal, zeros
            double *Ls = Lg + (long long)s * NUX * NUX + q;
            float *Lcs = copy32 ? a.Lc + in.oL + (long long)s * NUX * NUX + q : nullptr;
            static_for<0, NUX>([&](auto cc_) {
                constexpr int cc = decltype(cc_)::value;
                const bool keep = q >= cc || cc < NU;
                const double v = keep ? H[q + cc * ldH] : 0.0;
                Ls[cc * NUX] = v;
                if (Lcs) Lcs[cc * NUX] = keep ? (float)v : 0.0f;
            });
            DIg[(long long)s * NUX + q] = dinv[q];
            if (copy32) a.DIc[in.oDI + (long long)s * NUX + q] = (float)dinv[q];
        }
        if (t == 0) {
            // L^B = B^ L^{R-T} (one row per thread), then M_fwd = L^B L^B^T (lower)
            if (q < NX) {
                for (int j = 0; j < NU; ++j) {
                    double v = G[q + j * ldG];
                    for (int k = 0; k < j; ++k) v = fma(-G[q + k * ldG], H[j + k * ldH], v);
                    G[q + j * ldG] = v * dinv[j];
                }
            }
            team_sync<kPairTeam>();
            for (int e = q; e < NX * NU; e += kPairTeam) {
                const double v = G[e % NX + (e / NX) * ldG];
                LBg[(long long)s * NX * NU + e] = v;
                if (copy32) a.LBc[in.oLB + (long long)s * NX * NU + e] = (float)v;
            }
            for (int e = q; e < NX * (NX + 1) / 2; e += kPairTeam) {
                int r, cc;
                tri_index(e, r, cc);
                double v = 0.0;
#pragma unroll
                for (int k = 0; k < NU; ++k) v = fma(G[r + k * ldG], G[cc + k * ldG], v);
                Mf[r + cc * NX] = Mf[r + cc * NX] + v;
            }
            team_sync<kPairTeam>();
        }
        if (!last) {
            stage_zero_fill<kPairTeam>(buf, SL, a.data, in, s2);
            cp_async_wait_all();
            team_sync<kPairTeam>();   // every thread's copies have landed
            const double *BA = buf + SL.oB;   // [B A] of stage s2, column-major, leading dimension NX
            if (copy32 && a.BAf) {
                float *dst = reinterpret_cast<float *>(a.BAf) + in.oBA + (long long)s2 * NX * NUX;
                for (int e = q; e < NX * NUX; e += kPairTeam) dst[e] = (float)BA[e];
            }
            // V = [B A]^T L^Q, row q: V[q][j] = sum_{k >= j} BA[k][q] L^Q[k][j]
            if (q < NUX) {
                const double *LQ = H + NU + NU * ldH;
                double ba[NX], v[NX];
                static_for<0, NX>([&](auto kc) { ba[decltype(kc)::value] = BA[decltype(kc)::value + q * NX]; });
                static_for<0, NX>([&](auto jc) {
                    constexpr int j = decltype(jc)::value;
                    double acc = 0.0;
                    static_for<j, NX>([&](auto kc) {
                        constexpr int k = decltype(kc)::value;
                        acc = fma(ba[k], LQ[k + j * ldH], acc);
                    });
                    v[j] = acc;
                });
                static_for<0, NX / 2>([&](auto jc) {
                    constexpr int j = 2 * decltype(jc)::value;
                    *reinterpret_cast<double2 *>(V + q * ldVr + j) = make_double2(v[j], v[j + 1]);
                });
            }
            team_sync<kPairTeam>();
            // H^_{s2} = H_{s2} + V V^T, this thread's entries, into registers
            static_for<0, NS>([&](auto mc) {
                constexpr int m = decltype(mc)::value;
                if (q + kPairTeam * m < NT) {
                    double acc = raw_entry(m);
                    const double *vr = V + er[m] * ldVr, *vc = V + ec[m] * ldVr;
                    static_for<0, NX / 2>([&](auto kc) {
                        constexpr int k = 2 * decltype(kc)::value;
                        const double2 x = *reinterpret_cast<const double2 *>(vr + k);
                        const double2 y = *reinterpret_cast<const double2 *>(vc + k);
                        acc = fma(x.x, y.x, acc);
                        acc = fma(x.y, y.y, acc);
                    });
                    h[m] = acc;
                }
            });
            team_sync<kPairTeam>();   // the raw record and V have been read
        } else {
            // close the segment: L^{Q-1} (one column per thread), M_bwd, coupling block
            const double *LQ = H + NU + NU * ldH;
            const double *dq = dinv + NU;
            double *Ti = V;
            if (q < NX) {
                for (int i = 0; i < q; ++i) Ti[i + q * ldT] = 0.0;
                for (int i = q; i < NX; ++i) {
                    double v = (i == q) ? 1.0 : 0.0;
                    for (int k = q; k < i; ++k) v = fma(-LQ[i + k * ldH], Ti[k + q * ldT], v);
                    Ti[i + q * ldT] = v * dq[i];
                }
            }
            team_sync<kPairTeam>();
            {
                double *Lq = Lg + (long long)s * NUX * NUX + NU + NU * NUX;
                float *Lqc = copy32 ? a.Lc + in.oL + (long long)s * NUX * NUX + NU + NU * NUX : nullptr;
                for (int e = q; e < NX * NX; e += kPairTeam) {
                    const int i = e % NX, cc = e / NX;
                    if (i > cc) {
                        Lq[cc + i * NUX] = Ti[i + cc * ldT];
                        if (Lqc) Lqc[cc + i * NUX] = (float)Ti[i + cc * ldT];
                    }
                }
            }
            double *Mb = H;   // M_bwd = L^{Q-T} L^{Q-1}, leading dimension ldT
            for (int e = q; e < NX * NX; e += kPairTeam) {
                const int i = e % NX, j = e / NX;
                const int k0 = i > j ? i : j;
                double v = 0.0;
                for (int k = k0; k < NX; ++k) v = fma(Ti[k + i * ldT], Ti[k + j * ldT], v);
                Mb[i + j * ldT] = v;
            }
            team_sync<kPairTeam>();
            const int cb = (c - 1 + P) % P;
            for (int e = q; e < NX * NX; e += kPairTeam)
                a.Mb[in.oBlk + (long long)cb * NX * NX + e] = Mb[e % NX + (e / NX) * ldT];
            team_symmetrize<double, kPairTeam>(Mf, NX, NX);
            if (P == 1) {
                for (int e = q; e < NX * NX; e += kPairTeam) Mf[e] += Mb[e % NX + (e / NX) * ldT];
                team_sync<kPairTeam>();
                ok &= team_chol<double, kPairTeam>(Mf, NX, NX);
            }
            double *dst = a.Mf + in.oBlk + (long long)c * NX * NX;
            for (int e = q; e < NX * NX; e += kPairTeam) dst[e] = Mf[e];
        }
    }
    if (!ok && q == 0) atomicCAS(a.status + wi.inst, 0, ST_NOT_PD);
}

template <int NX, int NU>
cudaError_t launch_factor_pairs(const FactorArgs &a, cudaStream_t st) {
    using LY = PairLayout<NX, NU>;
    auto k = k_factor_pairs<NX, NU>;
    cudaError_t e = ensure_smem((const void *)k, LY::bytes);
    if (e != cudaSuccess) return e;
    k<<<(a.n_items + kPairItemsPerCta - 1) / kPairItemsPerCta, kPairTeam * kPairItemsPerCta, LY::bytes, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

// Diagnostics: the stage factor's pivot routine (sqrt(d), 1/sqrt(d)) applied
// element-wise, float64 and float32, so that its accuracy can be tested.
__global__ void k_pivot_eval(const double *d, double *l, double *il, const float *df, float *lf, float *ilf,
                             long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (d) {
            double a, b;
            pivot(d[i], a, b);
            l[i] = a;
            il[i] = b;
        }
        if (df) {
            float a, b;
            pivot(df[i], a, b);
            lf[i] = a;
            ilf[i] = b;
        }
    }
}

cudaError_t launch_pivot_eval(const double *d, double *l, double *il, const float *df, float *lf, float *ilf,
                              long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    k_pivot_eval<<<(int)blocks, 256, 0, st>>>(d, l, il, df, lf, ilf, n);
    return cudaGetLastError();
}

size_t factor_stage_bytes(int nx, int nu) {
    const size_t nux = (size_t)nx + nu;
    size_t stage = (size_t)nu * nu + (size_t)nu * nx + (size_t)nx * nx + nux + (size_t)nx * nu + (size_t)nx * nx;
    stage = (stage + 1) & ~(size_t)1;
    return stage * 8;
}

size_t factor_smem_bytes(bool fp64, int nx, int nu, bool staged, bool need_G2) {
    const size_t nux = (size_t)nx + nu;
    const size_t el = fp64 ? 8 : 4;
    const FactorTiles TL(nx, nu, need_G2, staged && fp64);
    size_t bytes = (staged ? factor_stage_bytes(nx, nu) : 0) + (size_t)nx * nx * 8;
    bytes += (TL.nH + TL.nVG + TL.nG + TL.nBA + nux) * el;
    return (bytes + 15) / 16 * 16;
}

template <typename T, int TEAM, int NXC = 0, int NUC = 0>
static cudaError_t launch_factor_t(size_t smem, const FactorArgs &a0, cudaStream_t st) {
    constexpr int TPC = TEAM < 32 ? 32 / TEAM : 1;
    FactorArgs a = a0;
    a.smem_team = (unsigned)((smem + 15) / 16 * 16);
    const size_t total = (size_t)a.smem_team * TPC;
    auto k = k_factor_segments<T, TEAM, NXC, NUC>;
    cudaError_t e = ensure_smem((const void *)k, total);
    if (e != cudaSuccess) return e;
    k<<<(a.n_items + TPC - 1) / TPC, TEAM < 32 ? 32 : TEAM, total, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_factor_segments(bool fp64, int team, int shape, size_t smem, const FactorArgs &a, cudaStream_t st) {
    if (a.n_items == 0) return cudaSuccess;
    if (team == 16 && fp64 && !a.need_G2 && a.stage_in_smem) {
        // every item is a whole horizon (no A^cl): two items per warp, compiled stage shapes
        if (shape == 1) return launch_factor_pairs<kStageShapes[1].nx, kStageShapes[1].nu>(a, st);
        if (shape == 2) return launch_factor_pairs<kStageShapes[2].nx, kStageShapes[2].nu>(a, st);
    }
    if (team == 16) return fp64 ? launch_factor_t<double, 16>(smem, a, st) : launch_factor_t<float, 16>(smem, a, st);
    if (fp64) {
        if (team == 32) return launch_factor_t<double, 32>(smem, a, st);
        if (team == 64) return launch_factor_t<double, 64>(smem, a, st);
        return launch_factor_t<double, 128>(smem, a, st);
    }
    if (team == 32) {
        switch (shape) {   // float32, one warp: kernels compiled for the listed stage shapes (kStageShapes)
            case 1: return launch_factor_t<float, 32, kStageShapes[1].nx, kStageShapes[1].nu>(smem, a, st);
            case 2: return launch_factor_t<float, 32, kStageShapes[2].nx, kStageShapes[2].nu>(smem, a, st);
            case 3: return launch_factor_t<float, 32, kStageShapes[3].nx, kStageShapes[3].nu>(smem, a, st);
            case 4: return launch_factor_t<float, 32, kStageShapes[4].nx, kStageShapes[4].nu>(smem, a, st);
            default: return launch_factor_t<float, 32>(smem, a, st);
        }
    }
    if (team == 64) return launch_factor_t<float, 64>(smem, a, st);
    return launch_factor_t<float, 128>(smem, a, st);
}

}  // namespace cyq
