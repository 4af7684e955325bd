// Float32 stage factorization of the segments that carry no A^cl (every
// segment of a one-segment instance, and segment 0 of any instance): the
// modified Riccati recursion of Alg. fact-mod-riccati without its propagation
// terms (Sec. 4.2; for P = 1 the factorized Riccati recursion), followed by the
// segment's Schur-complement contribution (compute-schur) and, for one-segment
// instances, the float64 Cholesky factor of the single coupling block.
//
// Ingest (k_ingest_f32): every stage's data is converted once, by a streaming
// kernel with all lanes busy, into float32: the stage matrix
// [R S; S^T Q] + diag(Sigma) in the padded tile layout of the factor (lower
// triangle) and [B A] (the copy the float32 sweeps read).  Double-to-float
// conversions run on the FP64 pipe; here they leave the stage recursion.
//
// Factor (k_factor_team): one team of 32, 64 or 128 threads per work item,
// one persistent launch for the whole batch.  The host sorts the items by
// cost (longest first) into three classes by the shared memory they need;
// the CTAs of the launch come in three configurations (one team of 128
// threads, two of 64 or four of 32, each team with its slot of the CTA's
// arena), the number of CTAs of each configuration in proportion to its
// class's work.  Every team takes items from its class's device counter and,
// when that class is exhausted, from the classes of smaller items, so the
// GPU stays busy to the end and no team waits for another.  Per stage:
//   potrf   left-looking Crout in blocks of 4 columns: each thread owns rows
//           tid, tid + T and accumulates 4 columns at a time from its own row
//           entries and a float4 broadcast of the block rows; the 4 x 4
//           diagonal block is factored by its warp with shuffles, the other
//           rows solve against it (two team barriers per block column);
//   V       V = [B A]^T L^Q, one row of V per thread (its column of [B A] in
//           registers, L^Q columns as float4 broadcasts, four columns of V
//           at a time), written in place of that column;
//   H^      H^ = H + V V^T on 4 x 4 register tiles of the lower triangle,
//           dealt out evenly over the team (two float4 rows of V per
//           operand, 64 FMAs per 8 shared-memory loads).
// Dimensions are padded to multiples of 4 with decoupled identity rows and
// columns (u padding between the u and x blocks, x padding at the end), which
// leave the factor of the real entries unchanged.  The next stage's stage
// matrix and [B A] are copied to shared memory with cp.async while the
// current stage is factored.
#include <algorithm>

#include "cyq_internal.cuh"

namespace cyq {

namespace {


// Tile index of real index a of the stage vector [u | x] (u padded to nup).
__device__ __forceinline__ int tile_of(int a, int nu, int nup) { return a < nu ? a : a - nu + nup; }

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// A team of T threads (a whole number of warps) inside a CTA: thread index,
// and a barrier over the team only (a named barrier; a warp barrier for T = 32).
template <int T>
struct Team {
    int tid, bar;
    __device__ __forceinline__ void sync() const {
        if constexpr (T == 32)
            __syncwarp();
        else
            asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(T) : "memory");
    }
};

}  // namespace

// Geometry of one item (in floats).  Slot layout:
//   dinv (np) | 4 x 4 block scratch (16) | H (np x np, column-major, ld np) |
//   BV (np x ldb: columns of [B A] of the next stage, then rows of V in place)
// (the next stage matrix is read from its ingested tile in global memory while
// H^ is formed, so that three CTAs fit on an SM)
// and at the end of the segment: the float64 coupling block (nx x nx) from
// the start of H, L^{Q-1} (nxp x nxp, ld nxp) behind both H and that block.
// The ingested stage matrices use the H layout (np x np per stage, lower
// triangle).
struct WarpGeom {
    int nx, nu, nux, nup, nxp, np, ldb;
    int oD, oK, oH, oBV, oT, size;
    __host__ __device__ WarpGeom(int nx_, int nu_) {
        nx = nx_;
        nu = nu_;
        nux = nx + nu;
        nup = (nu + 3) & ~3;
        nxp = (nx + 3) & ~3;
        np = nup + nxp;
        ldb = nxp + 4;
        oD = 0;
        oK = np;
        oH = np + 16;                          // np is a multiple of 4: every tile starts 16-byte aligned
        oBV = oH + np * np;
        const int main_end = oBV + np * ldb;
        const int mfloats = 2 * nxp * nxp;     // float64 nx x nx block (ld nx) fits in 2 nxp^2 floats
        oT = oH + (np * np > mfloats ? np * np : mfloats);
        const int last_end = oT + nxp * nxp;
        size = ((main_end > last_end ? main_end : last_end) + 3) & ~3;
    }
};

size_t warp_slot_bytes(int nx, int nu) { return (size_t)WarpGeom(nx, nu).size * 4; }
size_t warp_stage_floats(int nx, int nu) {
    const WarpGeom G(nx, nu);
    return (size_t)G.np * G.np;
}

namespace {

// ---------------------------------------------------------------------------
// Ingest: float32 stage matrices (padded tile layout) and [B A] copies
// ---------------------------------------------------------------------------
// A streaming pass bound by load latency: four blocks per SM (64 registers a
// thread) keep a third more loads in flight than three.
__global__ void __launch_bounds__(256, 4) k_ingest_f32(IngestArgs g) {
    const int w = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    if (w >= g.n_chunks) return;
    const IngestChunk ch = g.chunks[w];
    const int lane = (int)(threadIdx.x & 31);
    const Inst in = g.inst[ch.inst];
    const int N = in.N, P = in.P, nx = in.nx, nu = in.nu, nux = nx + nu;
    const WarpGeom G(nx, nu);
    const int np = G.np, nup = G.nup;
    const Data &d = g.data;
    for (int t = ch.t0; t < ch.t1; ++t) {
        const int s = seg_stage(0, t, N, P), xq = xstate(s, N);
        const double *R = d.R + in.oR + (long long)s * nu * nu;
        const double *S = (s != 0 && d.S) ? d.S + in.oS + (long long)s * nu * nx : nullptr;
        const double *Q = d.Q + in.oQ + (long long)xq * nx * nx;
        const double *Su = d.Sig ? d.Sig + in.oSig + (long long)s * nux : nullptr;
        const double *Sx = d.Sig ? d.Sig + in.oSig + (long long)xq * nux + nu : nullptr;
        float *Ht = g.Hf + in.oHf + (long long)s * np * np;
        // the tile column-major and flat over the lanes, four entries per lane at a time:
        // their sources first, then all loads, then the conversions (eight loads in flight
        // per lane); entries above the diagonal are not written (never read)
        int tq = 0, tr = lane;
        while (tr >= np) {
            tr -= np;
            ++tq;
        }
        for (int e0 = lane; e0 < np * np; e0 += 128) {
            const double *src[4], *sga[4];
            float cv[4];
            bool st[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                st[u] = e0 + 32 * u < np * np && tr >= tq;
                src[u] = nullptr;
                sga[u] = nullptr;
                cv[u] = 0.0f;
                if (st[u]) {
                    const bool padq = (tq >= nu && tq < nup) || tq >= nup + nx;
                    const bool padr = (tr >= nu && tr < nup) || tr >= nup + nx;
                    if (padq || padr) {
                        cv[u] = tr == tq ? 1.0f : 0.0f;
                    } else if (tr < nu) {
                        src[u] = R + tr + tq * nu;
                        if (tr == tq && Su) sga[u] = Su + tr;
                    } else if (tq < nu) {
                        if (S) src[u] = S + tq + (tr - nup) * nu;
                    } else {
                        const int i = tr - nup, j = tq - nup;
                        src[u] = Q + i + j * nx;
                        if (i == j && Sx) sga[u] = Sx + i;
                    }
                }
                tr += 32;
                while (tr >= np) {
                    tr -= np;
                    ++tq;
                }
            }
            double x[4], y[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                x[u] = src[u] ? __ldg(src[u]) : 0.0;
                y[u] = sga[u] ? __ldg(sga[u]) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (st[u]) Ht[e0 + 32 * u] = src[u] ? (float)(x[u] + y[u]) : cv[u];
        }
        if (t > 0 && g.BAf) {
            // [B A] of the stages whose predecessor propagates into them (all but the first)
            const double *B = d.B + in.oB + (long long)s * nx * nu;
            const double *A = d.A + in.oA + (long long)s * nx * nx;
            float *o = g.BAf + in.oBA + (long long)s * nx * nux;
            const int nb = nx * nu, n = nx * nux;
#pragma unroll 4
            for (int e = lane; e < n; e += 32) o[e] = (float)(e < nb ? __ldg(B + e) : __ldg(A + e - nb));
        }
    }
}

// ---------------------------------------------------------------------------
// Factor
// ---------------------------------------------------------------------------
// Lower triangle of an np x np tile (ld np, 16-byte aligned) from global memory
// to shared memory with 16-byte asynchronous copies (column q from row q & ~3).
template <int T>
__device__ __forceinline__ void fetch_tile_lower(float *dst, const float *src, int np, const Team<T> &tm) {
    const int nc = np >> 2;
    for (int q = tm.tid; q < np; q += T)
        for (int c = q >> 2; c < nc; ++c) cp_async16(dst + q * np + 4 * c, src + q * np + 4 * c);
}

// Columns of [B A] of stage s (float32 copy, nx x nux, ld nx) into the BV tile
// (column ta at ta * ldb); 16-byte copies where a column allows them.
template <int T>
__device__ __forceinline__ void fetch_BV(float *BV, const float *BA, const WarpGeom &G, const Team<T> &tm) {
    const int nx = G.nx, nu = G.nu, nup = G.nup, ldb = G.ldb;
    const bool al = (reinterpret_cast<size_t>(BA) & 15) == 0 && (nx & 3) == 0;
    if (al) {
        const int per = nx >> 2, n = G.nux * per;
        for (int e = tm.tid; e < n; e += T) {
            const int a = e / per, c = e - a * per;
            cp_async16(BV + tile_of(a, nu, nup) * ldb + 4 * c, BA + a * nx + 4 * c);
        }
    } else {
        const int n = G.nux * nx;
        for (int e = tm.tid; e < n; e += T) {
            const int a = e / nx, k = e - a * nx;
            cp_async4(BV + tile_of(a, nu, nup) * ldb + k, BA + e);
        }
    }
}

// Float64 Cholesky of an n x n matrix (ld) by a team (right-looking, one pivot
// at a time, the pivot routine of the stage factor); upper part zeroed.
template <int T>
__device__ bool team_chol_f64(double *A, int n, int ld, const Team<T> &tm) {
    bool ok = true;
    for (int k = 0; k < n; ++k) {
        double d = A[k + k * ld];
        if (!finite_pos(d)) {
            ok = false;
            d = 1.0;
        }
        double l, il;
        pivot(d, l, il);
        tm.sync();   // everyone has read A[k,k]
        if (tm.tid == 0) A[k + k * ld] = l;
        for (int i = k + 1 + tm.tid; i < n; i += T) A[i + k * ld] *= il;
        for (int i = tm.tid; i < k; i += T) A[i + k * ld] = 0.0;
        tm.sync();
        const int m = n - k - 1;
        for (int e = tm.tid; e < m * m; e += T) {
            const int jj = e / m, ii = e - jj * m;
            if (ii < jj) continue;
            const int i = ii + k + 1, j = jj + k + 1;
            A[i + j * ld] = fma(-A[i + k * ld], A[j + k * ld], A[i + j * ld]);
        }
        tm.sync();
    }
    return ok;
}

// Left-looking blocked Crout factorization of the padded np x np matrix in H
// (column-major, ld np; lower triangle read and overwritten with L) by a team
// whose threads own rows tid + T m, m < RPT.  dinv receives 1 / L_kk.  Returns
// false if a pivot was not positive and finite (that pivot is replaced by 1).
template <int T, int RPT>
__device__ bool team_crout(float *H, int np, float *dinv, float *dblk, const Team<T> &tm) {
    const int ld = np, tid = tm.tid, lane = tid & 31;
    bool ok = true;
    for (int q0 = 0; q0 < np; q0 += 4) {
        float acc[RPT][4];
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
            const int r = tid + T * m;
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[m][j] = (r < np && r >= q0 + j) ? H[(q0 + j) * ld + r] : 0.0f;
        }
        // acc[r][j] -= sum_{k < q0} L[r][k] L[q0+j][k], even and odd k in two partial sums
        // (q0 is a multiple of 4, so the number of terms is even)
        float accb[RPT][4];
#pragma unroll
        for (int m = 0; m < RPT; ++m)
#pragma unroll
            for (int j = 0; j < 4; ++j) accb[m][j] = 0.0f;
        bool active = false;   // some own row at or below the block
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
            const int r = tid + T * m;
            active = active || (r < np && r >= q0);
        }
#pragma unroll 2
        for (int k = 0; k < (active ? q0 : 0); k += 2) {
            const float *ck = H + k * ld, *ck1 = ck + ld;
            const float4 lq = *reinterpret_cast<const float4 *>(ck + q0);
            const float4 lq1 = *reinterpret_cast<const float4 *>(ck1 + q0);
#pragma unroll
            for (int m = 0; m < RPT; ++m) {
                const int r = tid + T * m;
                if (r < np && r >= q0) {
                    const float lr = ck[r], lr1 = ck1[r];
                    acc[m][0] = fmaf(-lr, lq.x, acc[m][0]);
                    acc[m][1] = fmaf(-lr, lq.y, acc[m][1]);
                    acc[m][2] = fmaf(-lr, lq.z, acc[m][2]);
                    acc[m][3] = fmaf(-lr, lq.w, acc[m][3]);
                    accb[m][0] = fmaf(-lr1, lq1.x, accb[m][0]);
                    accb[m][1] = fmaf(-lr1, lq1.y, accb[m][1]);
                    accb[m][2] = fmaf(-lr1, lq1.z, accb[m][2]);
                    accb[m][3] = fmaf(-lr1, lq1.w, accb[m][3]);
                }
            }
        }
#pragma unroll
        for (int m = 0; m < RPT; ++m)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[m][j] += accb[m][j];
        // the 4 x 4 diagonal block: rows q0..q0+3 are owned by threads o..o+3 (one warp), slot md;
        // the owners publish their rows, and every lane of that warp factors the block
        // (the same operations on every lane, no shuffles in the chain of pivots)
        const int md = q0 / T, o = q0 - md * T, l0 = o & 31;
        if ((tid >> 5) == (o >> 5)) {
            const int bi = lane - l0;   // this lane's row in the block (0..3), else outside
            if (bi >= 0 && bi < 4) {
                float4 row = make_float4(acc[0][0], acc[0][1], acc[0][2], acc[0][3]);
#pragma unroll
                for (int m = 1; m < RPT; ++m)
                    if (md == m) row = make_float4(acc[m][0], acc[m][1], acc[m][2], acc[m][3]);
                *reinterpret_cast<float4 *>(dblk + 4 * bi) = row;
            }
            __syncwarp();
            float b[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 x = *reinterpret_cast<const float4 *>(dblk + 4 * i);
                b[i][0] = x.x;
                b[i][1] = x.y;
                b[i][2] = x.z;
                b[i][3] = x.w;
            }
            float il4[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float d = b[j][j];
                if (!finite_pos(d)) {
                    ok = false;
                    d = 1.0f;
                }
                float l, il;
                pivot(d, l, il);
                b[j][j] = l;
                il4[j] = il;
#pragma unroll
                for (int i = j + 1; i < 4; ++i) b[i][j] *= il;
#pragma unroll
                for (int jj = j + 1; jj < 4; ++jj)
#pragma unroll
                    for (int i = jj; i < 4; ++i) b[i][jj] = fmaf(-b[i][j], b[jj][j], b[i][jj]);
            }
            if (bi >= 0 && bi < 4) {
                dinv[q0 + bi] = bi == 0 ? il4[0] : (bi == 1 ? il4[1] : (bi == 2 ? il4[2] : il4[3]));
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float v = bi == 0 ? b[0][j] : (bi == 1 ? b[1][j] : (bi == 2 ? b[2][j] : b[3][j]));
                    if (bi >= j) H[(q0 + j) * ld + q0 + bi] = v;
                }
            }
            __syncwarp();   // dblk is free again
        }
        tm.sync();
        // the rows below the block: solve against its 4 x 4 factor
        const float4 c0 = *reinterpret_cast<const float4 *>(H + q0 * ld + q0);
        const float4 c1 = *reinterpret_cast<const float4 *>(H + (q0 + 1) * ld + q0);
        const float4 c2 = *reinterpret_cast<const float4 *>(H + (q0 + 2) * ld + q0);
        const float4 dv = *reinterpret_cast<const float4 *>(dinv + q0);
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
            const int r = tid + T * m;
            if (r < np && r >= q0 + 4) {
                const float x0 = acc[m][0] * dv.x;
                const float x1 = fmaf(-x0, c0.y, acc[m][1]) * dv.y;
                const float x2 = fmaf(-x1, c1.z, fmaf(-x0, c0.z, acc[m][2])) * dv.z;
                const float x3 = fmaf(-x2, c2.w, fmaf(-x1, c1.w, fmaf(-x0, c0.w, acc[m][3]))) * dv.w;
                H[q0 * ld + r] = x0;
                H[(q0 + 1) * ld + r] = x1;
                H[(q0 + 2) * ld + r] = x2;
                H[(q0 + 3) * ld + r] = x3;
            }
        }
        tm.sync();
    }
    return ok;
}

// V = [B A]^T L^Q in place: column ta of BV ([B A], nxp entries) becomes row ta
// of V: V[ta][j] = sum_{k >= j} BA[k][ta] LQ[k][j], four j at a time.  L^Q is
// the nxp x nxp block of H at (nup, nup); only its lower triangle is read.
template <int T, int NXP>
__device__ void team_form_V(float *BV, const float *H, const WarpGeom &G, const Team<T> &tm) {
    const int np = G.np, nxp = G.nxp, ldb = G.ldb, ld = G.np;
    const float *LQ = H + G.nup * ld + G.nup;
    for (int ta = tm.tid; ta < np; ta += T) {
        float *col = BV + ta * ldb;
        float ba[NXP];
#pragma unroll
        for (int k = 0; k < NXP; k += 4) {
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < nxp) x = *reinterpret_cast<const float4 *>(col + k);
            ba[k] = x.x;
            ba[k + 1] = x.y;
            ba[k + 2] = x.z;
            ba[k + 3] = x.w;
        }
        for (int j0 = 0; j0 < nxp; j0 += 4) {
            const float *q0 = LQ + j0 * ld, *q1 = q0 + ld, *q2 = q1 + ld, *q3 = q2 + ld;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
            for (int kc = 0; kc < NXP; kc += 4) {
                if (kc < nxp && kc >= j0) {
                    const float4 l0 = *reinterpret_cast<const float4 *>(q0 + kc);
                    const float4 l1 = *reinterpret_cast<const float4 *>(q1 + kc);
                    const float4 l2 = *reinterpret_cast<const float4 *>(q2 + kc);
                    const float4 l3 = *reinterpret_cast<const float4 *>(q3 + kc);
                    if (kc == j0) {
                        // diagonal chunk: column j0 + jj takes rows k >= j0 + jj only
                        a0 = fmaf(ba[kc], l0.x, a0);
                        a0 = fmaf(ba[kc + 1], l0.y, a0);
                        a0 = fmaf(ba[kc + 2], l0.z, a0);
                        a0 = fmaf(ba[kc + 3], l0.w, a0);
                        a1 = fmaf(ba[kc + 1], l1.y, a1);
                        a1 = fmaf(ba[kc + 2], l1.z, a1);
                        a1 = fmaf(ba[kc + 3], l1.w, a1);
                        a2 = fmaf(ba[kc + 2], l2.z, a2);
                        a2 = fmaf(ba[kc + 3], l2.w, a2);
                        a3 = fmaf(ba[kc + 3], l3.w, a3);
                    } else {
                        a0 = fmaf(ba[kc], l0.x, a0);
                        a1 = fmaf(ba[kc], l1.x, a1);
                        a2 = fmaf(ba[kc], l2.x, a2);
                        a3 = fmaf(ba[kc], l3.x, a3);
                        a0 = fmaf(ba[kc + 1], l0.y, a0);
                        a1 = fmaf(ba[kc + 1], l1.y, a1);
                        a2 = fmaf(ba[kc + 1], l2.y, a2);
                        a3 = fmaf(ba[kc + 1], l3.y, a3);
                        a0 = fmaf(ba[kc + 2], l0.z, a0);
                        a1 = fmaf(ba[kc + 2], l1.z, a1);
                        a2 = fmaf(ba[kc + 2], l2.z, a2);
                        a3 = fmaf(ba[kc + 2], l3.z, a3);
                        a0 = fmaf(ba[kc + 3], l0.w, a0);
                        a1 = fmaf(ba[kc + 3], l1.w, a1);
                        a2 = fmaf(ba[kc + 3], l2.w, a2);
                        a3 = fmaf(ba[kc + 3], l3.w, a3);
                    }
                }
            }
            *reinterpret_cast<float4 *>(col + j0) = make_float4(a0, a1, a2, a3);
        }
    }
}

// H^ = Hn + V V^T (lower triangle, tile indices; Hn is the next stage matrix's
// ingested tile in global memory, read at the start of each 4 x 4 tile so that
// the loads overlap the products) on 4 x 4 tiles (block row bi >= block column
// bj) dealt out over the team.
template <int T, int NXP>
__device__ void team_form_H(float *H, const float *__restrict__ Hn, const float *BV, const WarpGeom &G,
                            const Team<T> &tm) {
    const int nb = G.np >> 2, nxp = G.nxp, ldb = G.ldb, ld = G.np;
    const int ntiles = nb * (nb + 1) / 2;
    int bi, bj;
    tri_index(tm.tid, bi, bj);
    for (int e = tm.tid; e < ntiles; e += T, tri_advance(bi, bj, T)) {
        const float *r0 = BV + (4 * bi) * ldb, *c0 = BV + (4 * bj) * ldb;
        float a[4][4];
        // column 4 bj + j, rows 4 bi .. 4 bi + 3 of Hn (16-byte aligned: np, ld are multiples of 4)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float4 h = __ldg(reinterpret_cast<const float4 *>(Hn + (4 * bj + j) * ld + 4 * bi));
            a[0][j] = h.x;
            a[1][j] = h.y;
            a[2][j] = h.z;
            a[3][j] = h.w;
        }
#pragma unroll
        for (int kc = 0; kc < NXP; kc += 4) {
            if (kc < nxp) {
                float4 x[4], y[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    x[i] = *reinterpret_cast<const float4 *>(r0 + i * ldb + kc);
                    y[i] = *reinterpret_cast<const float4 *>(c0 + i * ldb + kc);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float s = a[i][j];
                        s = fmaf(x[i].x, y[j].x, s);
                        s = fmaf(x[i].y, y[j].y, s);
                        s = fmaf(x[i].z, y[j].z, s);
                        s = fmaf(x[i].w, y[j].w, s);
                        a[i][j] = s;
                    }
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int o = (4 * bj + j) * ld + 4 * bi;
            if (bi != bj) {
                *reinterpret_cast<float4 *>(H + o) = make_float4(a[0][j], a[1][j], a[2][j], a[3][j]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (i >= j) H[o + i] = a[i][j];
            }
        }
    }
}

// L^{R-1} of every stage of the covered segments, after the factorization (it
// is only read by the solve sweeps, so it leaves the stage recursion): one
// warp per chunk of stages; the stored L^R block of a stage is copied to
// shared memory, lane cc keeps column cc of L^{R-1} in registers (zero above
// the diagonal, 1/L_cc on it) and forms the rows below by forward substitution
//   X[i][cc] = -(1/L_ii) sum_{k < i} L[i][k] X[k][cc]
// (the entries L[i][k] as broadcasts), and writes X[i][cc] transposed into the
// free upper triangle of the stored R block, as the per-class factor does.
template <int NUB>
__device__ __forceinline__ void warp_inv_R(float *Ls, const float *DIs, float *Rs, int nu, int nux) {
    const int cc = (int)(threadIdx.x & 31);
    for (int e = cc; e < nu * nu; e += 32) {
        const int k = e / nu, i = e - k * nu;
        Rs[i + k * NUB] = Ls[i + k * nux];
    }
    __syncwarp();
    float x[NUB];
#pragma unroll
    for (int k = 0; k < NUB; ++k) x[k] = (k == cc && k < nu) ? DIs[k] : 0.0f;
#pragma unroll
    for (int i = 1; i < NUB; ++i) {
        if (i < nu) {
            float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
            for (int k = 0; k < i; ++k) {
                const float l = Rs[i + k * NUB];
                if (k & 1) s1 = fmaf(l, x[k], s1);
                else s0 = fmaf(l, x[k], s0);
            }
            const float v = -(s0 + s1) * DIs[i];
            if (i > cc) x[i] = v;
        }
    }
#pragma unroll
    for (int i = 1; i < NUB; ++i)
        if (i < nu && i > cc) Ls[cc + i * nux] = x[i];
    __syncwarp();   // the shared copy is reused by the next stage
}

__global__ void __launch_bounds__(256) k_inv_R_f32(IngestArgs g, float *L, const float *DI) {
    __shared__ float rs[8][32 * 32];
    const int wl = (int)(threadIdx.x >> 5);
    const int w = (int)(blockIdx.x * 8 + wl);
    if (w >= g.n_chunks) return;
    const IngestChunk ch = g.chunks[w];
    const Inst in = g.inst[ch.inst];
    const int N = in.N, P = in.P, nu = in.nu, nux = in.nx + in.nu;
    if (nu < 2) return;
    for (int t = ch.t0; t < ch.t1; ++t) {
        const int s = seg_stage(0, t, N, P);
        float *Ls = L + in.oL + (long long)s * nux * nux;
        const float *DIs = DI + in.oDI + (long long)s * nux;
        if (nu <= 8)
            warp_inv_R<8>(Ls, DIs, rs[wl], nu, nux);
        else if (nu <= 16)
            warp_inv_R<16>(Ls, DIs, rs[wl], nu, nux);
        else
            warp_inv_R<32>(Ls, DIs, rs[wl], nu, nux);
    }
}

// Stored factor of stage s (nux x nux, column-major, real indices): lower
// triangle, L^{R-1} above the R diagonal, zeros elsewhere; and 1 / diag.
template <int T>
__device__ void team_store_L(float *Ls, float *DIs, const float *H, const float *dinv, const WarpGeom &G,
                             const Team<T> &tm) {
    const int nux = G.nux, nu = G.nu, nup = G.nup, ld = G.np;
    int a, b;
    rect_start(tm.tid, nux, a, b);
    for (; b < nux; rect_advance(a, b, nux, T)) {
        const int ta = tile_of(a, nu, nup), tb = tile_of(b, nu, nup);
        const bool keep = a >= b || (a < nu && b < nu);
        Ls[a + b * nux] = keep ? H[tb * ld + ta] : 0.0f;
    }
    for (int i = tm.tid; i < nux; i += T) DIs[i] = dinv[tile_of(i, nu, nup)];
}

template <int T, int RPT, int NXP>
__device__ void team_factor_item(const FactorArgs &a, const Item wi, float *slot, const Team<T> &tm) {
    const int tid = tm.tid;
    const Inst in = a.inst[wi.inst];
    const int N = in.N, P = in.P, c = wi.seg;
    const int len = seg_len(c, N, P);
    const WarpGeom G(in.nx, in.nu);
    const int nx = G.nx, nu = G.nu, nux = G.nux, nup = G.nup, nxp = G.nxp, np = G.np, ld = G.np;
    float *dinv = slot + G.oD, *H = slot + G.oH, *BV = slot + G.oBV;
    float *dblk = slot + G.oK;   // 4 x 4 diagonal block of the Crout factorization
    float *Lg = reinterpret_cast<float *>(a.L) + in.oL;
    float *DIg = reinterpret_cast<float *>(a.DI) + in.oDI;
    float *LBg = reinterpret_cast<float *>(a.LB) + in.oLB;
    const float *Hg = a.Hf + in.oHf;
    const float *BAg = reinterpret_cast<const float *>(a.BAf) + in.oBA;
    double *Mfg = a.Mf + in.oBlk + (long long)c * nx * nx;

    // zero padding of the [B A] tile (kept zero: V rows / columns of the padding vanish)
    for (int e = tid; e < np * G.ldb; e += T) BV[e] = 0.0f;
    // first stage: H^ = H
    int s = seg_stage(c, 0, N, P);
    fetch_tile_lower<T>(H, Hg + (long long)s * np * np, np, tm);
    cp_async_commit();
    bool ok = true;
    for (int t = 0; t < len; ++t) {
        s = seg_stage(c, t, N, P);
        const bool last = t == len - 1;
        const int s2 = last ? 0 : seg_stage(c, t + 1, N, P);
        if (t > 0 && !last) {
            // the next stage's [B A] lands while this stage is factored
            fetch_BV<T>(BV, BAg + (long long)s2 * nx * nux, G, tm);
            cp_async_commit();
            cp_async_wait_one();   // (no older group is pending)
        } else {
            cp_async_wait_all();
        }
        tm.sync();
        ok &= team_crout<T, RPT>(H, np, dinv, dblk, tm);
        team_store_L<T>(Lg + (long long)s * nux * nux, DIg + (long long)s * nux, H, dinv, G, tm);
        if (t == 0) {
            // L^B = B L^{R-T} of the segment's first stage (scratch in BV, ld nxp + 1), then
            // M_fwd = L^B L^B^T into the float64 coupling block (full symmetric)
            const int ldg = nxp + 1;
            const double *B0 = a.data.B + in.oB + (long long)s * nx * nu;
            for (int e = tid; e < nx * nu; e += T) {
                const int j = e / nx, i = e - j * nx;
                BV[i + j * ldg] = (float)B0[e];
            }
            tm.sync();
            for (int i = tid; i < nx; i += T)
                for (int j = 0; j < nu; ++j) {
                    float v = BV[i + j * ldg];
                    for (int k = 0; k < j; ++k) v = fmaf(-BV[i + k * ldg], H[j + k * ld], v);
                    BV[i + j * ldg] = v * dinv[j];
                }
            tm.sync();
            float *LBs = LBg + (long long)s * nx * nu;
            for (int e = tid; e < nx * nu; e += T) {
                const int j = e / nx, i = e - j * nx;
                LBs[e] = BV[i + j * ldg];
            }
            for (int e = tid; e < nx * nx; e += T) {
                const int j = e / nx, i = e - j * nx;
                if (i < j) continue;
                float v = 0.0f;
                for (int k = 0; k < nu; ++k) v = fmaf(BV[i + k * ldg], BV[j + k * ldg], v);
                Mfg[i + j * nx] = (double)v;
                Mfg[j + i * nx] = (double)v;
            }
            tm.sync();
            for (int e = tid; e < np * G.ldb; e += T) BV[e] = 0.0f;   // restore the zero padding
            tm.sync();
            if (!last) {
                fetch_BV<T>(BV, BAg + (long long)s2 * nx * nux, G, tm);
                cp_async_commit();
            }
        }
        if (!last) {
            cp_async_wait_all();
            tm.sync();
            team_form_V<T, NXP>(BV, H, G, tm);
            tm.sync();
            team_form_H<T, NXP>(H, Hg + (long long)s2 * np * np, BV, G, tm);
            tm.sync();
        } else {
            // close the segment: T = L^{Q-1}, its strict lower part (transposed) into the
            // stored Q block, M_bwd = T^T T, and for one segment the coupling Cholesky
            const float *LQ = H + nup * ld + nup;
            const float *dq = dinv + nup;
            float *Ti = slot + G.oT;   // ld nxp
            for (int cc = tid; cc < nx; cc += T) {
                for (int i = 0; i < cc; ++i) Ti[i + cc * nxp] = 0.0f;
                for (int i = cc; i < nx; ++i) {
                    float v = (i == cc) ? 1.0f : 0.0f;
                    for (int k = cc; k < i; ++k) v = fmaf(-LQ[i + k * ld], Ti[k + cc * nxp], v);
                    Ti[i + cc * nxp] = v * dq[i];
                }
            }
            tm.sync();
            float *Lq = Lg + (long long)s * nux * nux + nu + nu * nux;
            {
                int i, cc;
                rect_start(tid, nx, i, cc);
                for (; cc < nx; rect_advance(i, cc, nx, T))
                    if (i > cc) Lq[cc + i * nux] = Ti[i + cc * nxp];
            }
            const int cb = (c - 1 + P) % P;
            double *Mbg = a.Mb + in.oBlk + (long long)cb * nx * nx;
            double *M = reinterpret_cast<double *>(slot + G.oH);   // ld nx
            {
                int i, j;
                rect_start(tid, nx, i, j);
                for (; j < nx; rect_advance(i, j, nx, T)) {
                    const int k0 = i > j ? i : j;
                    float v = 0.0f;
                    for (int k = k0; k < nx; ++k) v = fmaf(Ti[k + i * nxp], Ti[k + j * nxp], v);
                    Mbg[i + j * nx] = (double)v;
                    if (P == 1) M[i + j * nx] = Mfg[i + j * nx] + (double)v;
                }
            }
            tm.sync();
            if (P == 1) {
                ok &= team_chol_f64<T>(M, nx, nx, tm);
                for (int e = tid; e < nx * nx; e += T) Mfg[e] = M[e];
            }
            tm.sync();
        }
    }
    if (!ok) atomicCAS(a.status + wi.inst, 0, ST_NOT_PD);
}

// One CTA configuration: TEAMS teams of T threads, every team with its slot of
// the arena, taking items from the counter of class `cls` until it is empty.
template <int T, int RPT>
__device__ void team_loop(const FactorArgs &a, const TeamPlanDev &plan, int cls, float *arena, int *cmd) {
    constexpr int TEAMS = kTeamCtaThreads / T;
    const int tmi = threadIdx.x / T;
    Team<T> tm;
    tm.tid = threadIdx.x - tmi * T;
    tm.bar = 1 + tmi;
    float *slot = arena + (size_t)tmi * (plan.arena_floats / TEAMS);
    for (;;) {
        if (tm.tid == 0) cmd[tmi] = atomicAdd(plan.counter + cls, 1);
        tm.sync();
        const int idx = cmd[tmi];
        tm.sync();   // the command word is read before it is rewritten
        if (idx >= plan.n[cls]) break;
        const Item wi = plan.items[plan.off[cls] + idx];
        if (!(a.skip && a.skip[wi.inst])) {
            const int nxp = (a.inst[wi.inst].nx + 3) & ~3;
            if (nxp <= 16)
                team_factor_item<T, RPT, 16>(a, wi, slot, tm);
            else if (nxp <= 32)
                team_factor_item<T, RPT, 32>(a, wi, slot, tm);
            else
                team_factor_item<T, RPT, 64>(a, wi, slot, tm);
        }
        tm.sync();   // the slot is reused by the next item
    }
}

// Every CTA starts with the configuration of the class it is assigned to and,
// once that class's counter is exhausted, re-forms its teams for the other
// classes in turn (largest items first), so that no SM idles while items are
// left.  Class c items run with teams of 128 >> c threads (c = 0, 1, 2).
__global__ void __launch_bounds__(kTeamCtaThreads, kFactorCtasPerSm) k_factor_team(FactorArgs a, TeamPlanDev plan) {
    extern __shared__ __align__(16) unsigned char smem_all[];
    __shared__ int cmd[4];
    float *arena = reinterpret_cast<float *>(smem_all);
    const int first = (int)blockIdx.x < plan.g0 ? 0 : ((int)blockIdx.x < plan.g0 + plan.g1 ? 1 : 2);
    for (int step = 0; step < 3; ++step) {
        const int cls = step == 0 ? first : (first == 0 ? step : step - 1 + (step - 1 >= first ? 1 : 0));
        if (plan.n[cls] > 0) {
            if (cls == 0)
                team_loop<128, 1>(a, plan, 0, arena, cmd);
            else if (cls == 1)
                team_loop<64, 2>(a, plan, 1, arena, cmd);
            else
                team_loop<32, 2>(a, plan, 2, arena, cmd);
        }
        __syncthreads();   // every team of the CTA has left the configuration and its slots
    }
}

}  // namespace

cudaError_t launch_ingest_f32(const IngestArgs &g, cudaStream_t st) {
    if (g.n_chunks == 0) return cudaSuccess;
    k_ingest_f32<<<(g.n_chunks + 7) / 8, 256, 0, st>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_inv_R_f32(const IngestArgs &g, float *L, const float *DI, cudaStream_t st) {
    if (g.n_chunks == 0) return cudaSuccess;
    k_inv_R_f32<<<(g.n_chunks + 7) / 8, 256, 0, st>>>(g, L, DI);
    return cudaGetLastError();
}

cudaError_t launch_factor_team(const FactorArgs &a, const TeamPlanDev &plan, int grid, cudaStream_t st) {
    if (grid <= 0) return cudaSuccess;
    const size_t arena = (size_t)plan.arena_floats * 4;
    cudaError_t e = ensure_smem((const void *)k_factor_team, arena);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(plan.counter, 0, 3 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_factor_team<<<grid, kTeamCtaThreads, arena, st>>>(a, plan);
    return cudaGetLastError();
}

}  // namespace cyq
