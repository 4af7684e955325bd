// Segment sweeps of the solve with the factor of eq. chol-fac-K-cyqlone.
//
// For a segment with outgoing coupling multiplier mu = lambda^{b_c} and
// incoming nu = lambda^{b_{c-1}}, the stage variables are eliminated backward
// exactly as in the factorization, now carrying the affine terms of the
// right-hand side b (h = -(b_u, b_x), dynamics offsets c = -b_lambda):
//   rho_j = L^{R-1} h^_u,   p_j = h^_x - L^S rho_j,
//   g    += -L^B_j rho_j (+ A^cl_j c_{j-1} when the segment propagates A^cl),
//   h^_{j-1} = h_{j-1} + [B A]_{j-1}^T (L^Q_j L^Q_j^T c_{j-1} + p_j),
// and at the first stage j1 (y = L^{Q-1} p_{j1}):
//   d_bwd = L^{Q-T} y,   d_fwd = g - L^A y.
// These are the segment's contributions to the coupling right-hand side
//   M lambda_c = d_fwd,c + d_bwd,c+1 - b_lambda^{b_c}
// (solved by cyclic reduction).  The forward sweep then recovers
//   x^{j1} = -L^{Q-T}(L^{Q-1}(p_{j1} - nu) + L^{A T} mu),
//   u^j     = -L^{R-T}(L^{S T} x^j + rho_j + L^{B T}_j mu),
//   lambda^{j-1} = L^Q_j L^Q_j^T x^j + p_j + A^{cl T}_j mu   (interior stages),
//   x^{j+1} = A_j x^j + B_j u^j + c_j.
// rho_j and p_j are parked in the u / x slots of z between the two sweeps.
//
// The factor stores L^{R-1} (every stage) and L^{Q-1} (first stage of each
// segment) in the free upper triangle of L, so every triangular solve here is
// a parallel matrix-vector product.
//
// Work per stage is split into three barrier-separated phases; products
// whose rows are independent of each other share a phase.  Each stage's
// package (factor blocks, [B A], and the right-hand-side / parked vector
// entries the stage reads) is copied to shared memory with cp.async up to
// three stages ahead, in a ring of up to four packages (or right after use
// when a single package is all that fits).  The float32 sweeps read a float32 copy of [B A]
// written by the factorization and convert the package's float64 vector
// entries once on arrival, so no conversion sits inside a dot product.
// One CTA per (instance, segment); nrhs right-hand sides share each block.
#include "cyq_internal.cuh"

namespace cyq {

namespace {

// The threads that sweep one work item: the whole CTA (bar = 0, the per-class
// launches), or a team of TEAM threads inside a persistent CTA (named barrier
// bar; a warp barrier for TEAM = 32).
struct SweepCtx {
    int tid, bar;
};
template <int TEAM>
__device__ __forceinline__ void sweep_sync(const SweepCtx &c) {
    if constexpr (TEAM == 32) {
        if (c.bar == 0) __syncthreads();
        else __syncwarp();
    } else {
        if (c.bar == 0) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(c.bar), "n"(TEAM) : "memory");
    }
}

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

// count elements global -> shared; 16-byte copies when both ends and the
// length allow it.
template <typename T, int TEAM>
__device__ void async_copy(T *dst, const T *src, int count, int tid) {
    const int bytes = count * (int)sizeof(T);
    if (((reinterpret_cast<unsigned long long>(src) | reinterpret_cast<unsigned long long>(dst)) & 15) == 0 &&
        (bytes & 15) == 0) {
        char *d = reinterpret_cast<char *>(dst);
        const char *g = reinterpret_cast<const char *>(src);
        for (int e = tid; e < bytes / 16; e += TEAM) cp_async16(d + 16 * e, g + 16 * e);
        return;
    }
    for (int e = tid; e < count; e += TEAM) {
        if (sizeof(T) == 8)
            cp_async8(dst + e, src + e);
        else
            cp_async4(dst + e, src + e);
    }
}

// Column-major walk over the (row, right-hand side) pairs of an n x nrhs
// grid: the thread's first pair and the step, computed once per work item.
// Pair 0 goes to thread `first` (the assignment wraps around the team), so
// that two products of one phase can start on different warps.
struct Walk {
    int i0, r0, di, dr, n;
    __device__ __forceinline__ void init(int n_, int team, int tid, int first = 0) {
        n = n_;
        const int vt = (tid - first + team) % team;
        r0 = vt / n;
        i0 = vt - r0 * n;
        dr = team / n;
        di = team - dr * n;
    }
    __device__ __forceinline__ void next(int &i, int &r) const {
        i += di;
        r += dr;
        if (i >= n) {
            i -= n;
            ++r;
        }
    }
};

__host__ __device__ __forceinline__ size_t align16(size_t b) { return (b + 15) / 16 * 16; }

constexpr int kPairMaxNx = 16;

// Two dot products with one accumulator, one FMA per step: the n1 terms
// a1[q*sa1] b1[q] starting from init1, then the n2 terms a2[q*sa2] b2[q]
// starting from init2 (n2 may be 0).  Each product sums its terms in the
// same order as a loop of its own.  A thread that owns rows i and n-1-i of a
// triangular product this way has n+1 terms, whatever i: the lanes of a warp
// stay equally busy (one FP64 instruction costs a whole warp slot).
template <typename T>
__device__ __forceinline__ void dot2(const T *a1, int sa1, const T *b1, int n1, T init1, const T *a2, int sa2,
                                     const T *b2, int n2, T init2, T &o1, T &o2) {
    T acc = init1, first = init1;
    const int n = n1 + n2;
    for (int m = 0; m < n; ++m) {
        if (m == n1) {
            first = acc;
            acc = init2;
        }
        const bool sec = m >= n1;
        const int q = sec ? m - n1 : m;
        acc = fma(sec ? a2[q * sa2] : a1[q * sa1], sec ? b2[q] : b1[q], acc);
    }
    o1 = n2 > 0 ? first : acc;
    o2 = acc;
}

// Wait until at most n of this thread's committed cp.async groups are pending.
__device__ __forceinline__ void cp_async_wait_pending(int n) {
    if (n <= 0)
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    else if (n == 1)
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    else
        asm volatile("cp.async.wait_group 2;\n" ::: "memory");
}

// Per-stage package in shared memory.
template <typename T>
struct Package {
    double *vb;          // nrhs records of nux + nx float64 vector entries
    T *L, *D, *LB, *F;   // (nu+nx)^2 (ld nu+nx), nu+nx, nx*nu, nx*nx
    T *BA;               // nx x (nu+nx), ld nx ([B A])
};

template <typename T>
__device__ Package<T> carve_package(unsigned char *&p, int nx, int nu, int nrhs) {
    const size_t nux = nx + nu;
    Package<T> k;
    k.vb = reinterpret_cast<double *>(p); p += align16((nux + nx) * nrhs * 8);
    k.L = reinterpret_cast<T *>(p);       p += align16(nux * nux * sizeof(T));
    k.D = reinterpret_cast<T *>(p);       p += align16(nux * sizeof(T));
    k.LB = reinterpret_cast<T *>(p);      p += align16((size_t)nx * nu * sizeof(T));
    k.F = reinterpret_cast<T *>(p);       p += align16((size_t)nx * nx * sizeof(T));
    k.BA = reinterpret_cast<T *>(p);      p += align16((size_t)nx * nux * sizeof(T));
    return k;
}

__host__ __device__ size_t package_bytes(bool fp64, int nx, int nu, int nrhs) {
    const size_t nux = (size_t)nx + nu, el = fp64 ? 8 : 4;
    return align16((nux + nx) * nrhs * 8) + align16(nux * nux * el) + align16(nux * el) +
           align16((size_t)nx * nu * el) + align16((size_t)nx * nx * el) + align16((size_t)nx * nux * el);
}

// Factor blocks of stage s (L^B / the A^cl block only where the sweep uses them).
template <typename T, int TEAM>
__device__ void fetch_factor(const Package<T> &k, const SolveArgs &a, const Inst &in, int s, bool wantLB,
                             bool wantF, int tid) {
    const int nx = in.nx, nu = in.nu, nux = nx + nu;
    async_copy<T, TEAM>(k.L, reinterpret_cast<const T *>(a.L) + in.oL + (long long)s * nux * nux, nux * nux, tid);
    async_copy<T, TEAM>(k.D, reinterpret_cast<const T *>(a.DI) + in.oDI + (long long)s * nux, nux, tid);
    if (wantLB)
        async_copy<T, TEAM>(k.LB, reinterpret_cast<const T *>(a.LB) + in.oLB + (long long)s * nx * nu, nx * nu, tid);
    if (wantF)
        async_copy<T, TEAM>(k.F, reinterpret_cast<const T *>(a.F) + in.oF + (long long)s * nx * nx, nx * nx, tid);
}

// [B A] of stage s (s > 0): the float32 copy, or the float64 data itself.
template <typename T, int TEAM>
__device__ void fetch_BA(const Package<T> &k, const SolveArgs &a, const Inst &in, int s, int tid) {
    const int nx = in.nx, nu = in.nu, nux = nx + nu;
    if (sizeof(T) == 4) {
        async_copy<T, TEAM>(k.BA, reinterpret_cast<const T *>(a.BA) + in.oBA + (long long)s * nx * nux, nx * nux, tid);
    } else {
        double *d = reinterpret_cast<double *>(k.BA);
        async_copy<double, TEAM>(d, a.data.B + in.oB + (long long)s * nx * nu, nx * nu, tid);
        async_copy<double, TEAM>(d + nx * nu, a.data.A + in.oA + (long long)s * nx * nx, nx * nx, tid);
    }
}

// Vectors of one work item (T), each nrhs copies.
template <typename T>
struct Vecs {
    T *hh, *rho, *wv, *tv, *pv, *gmu, *cv, *xa, *xb;
    T *nb;      // float32: the package's vector entries after conversion (two buffers of nbs)
    int nbs;
};

template <typename T>
__device__ Vecs<T> carve_vecs(unsigned char *p, int nx, int nu, int nrhs) {
    const int nux = nx + nu, nv = nux + nx;
    T *q = reinterpret_cast<T *>(p);
    Vecs<T> v;
    v.hh = q;  q += nux * nrhs;
    v.rho = q; q += nu * nrhs;
    v.wv = q;  q += nx * nrhs;
    v.tv = q;  q += nx * nrhs;
    v.pv = q;  q += nx * nrhs;
    v.gmu = q; q += nx * nrhs;
    v.cv = q;  q += nx * nrhs;
    v.xa = q;  q += nx * nrhs;
    v.xb = q;  q += nx * nrhs;
    v.nb = q;
    v.nbs = nv * nrhs;
    return v;
}

__host__ __device__ size_t vecs_bytes(bool fp64, int nx, int nu, int nrhs) {
    const size_t nux = (size_t)nx + nu;
    return (nux + nu + 7 * (size_t)nx + 2 * (nux + nx)) * nrhs * (fp64 ? 8 : 4);
}

// Vector entries of the package as T: float64 reads them in place; float32
// converts the entries this thread copied itself (visible to it after its own
// cp.async wait) into nb; the barrier that follows publishes them.
template <typename T>
__device__ __forceinline__ const T *package_vectors(const Package<T> &K, const Vecs<T> &v, int buf, const Walk &Wv,
                                                    int nrhs, int nv) {
    if (sizeof(T) == 8) return reinterpret_cast<const T *>(K.vb);
    T *nb = v.nb + buf * v.nbs;
    for (int i = Wv.i0, r = Wv.r0; r < nrhs; Wv.next(i, r)) nb[i + r * nv] = (T)K.vb[i + r * nv];
    return nb;
}

}  // namespace

__host__ __device__ size_t solve_smem_bytes(bool fp64, int nx, int nu, int nrhs, int nbuf) {
    return align16(nbuf * package_bytes(fp64, nx, nu, nrhs)) + vecs_bytes(fp64, nx, nu, nrhs);
}

template <typename T, int TEAM, int NXC, int NUC>
__device__ void sweep_backward_item(const SolveArgs &a, const Item wi, unsigned char *smem_raw, const SweepCtx ctx, const int nbuf_in) {
    const int tid = ctx.tid;
    const Inst in = a.inst[wi.inst];
    // NXC / NUC > 0: kernel compiled for that stage shape (every item of the launch has it)
    const int nx = NXC > 0 ? NXC : in.nx, nu = NUC > 0 ? NUC : in.nu;
    const int N = in.N, P = in.P, c = wi.seg, nrhs = a.nrhs;
    const int nux = nx + nu, nv = nux + nx, w = nu + 2 * nx;
    const int len = seg_len(c, N, P);
    // Wp: pairs of rows (i, nx-1-i) of the triangular products, in float64 for small
    // nx, where unequal row lengths leave most lanes of an FP64 instruction idle
    // (the pairing costs ALU work per step, which float32 and large nx do not repay)
    const bool pair = sizeof(T) == 8 && nx <= kPairMaxNx;
    const int half = (nx + 1) / 2;
    Walk Wu, Wx, Wux, Wv, Wp;
    Wu.init(nu, TEAM, tid);
    Wx.init(nx, TEAM, tid);
    Wux.init(nux, TEAM, tid);
    Wv.init(nv, TEAM, tid);
    // the paired triangular products start on the second warp: the first one has the
    // u rows of the same phase
    Wp.init(half, TEAM, tid, TEAM >= 64 ? 32 : 0);
    // when the u rows and the pairs each fit one warp, the first warp also forms the
    // pairs' p = h_x - L^S rho right after rho (its own rows: a warp barrier suffices),
    // which leaves the second warp only the products that need w
    const bool early_p = pair && TEAM >= 64 && nu * nrhs <= 32 && half * nrhs <= 32;
    Walk Wq;
    Wq.init(half, TEAM, tid);
    // ring of nbuf packages: the package of processing step u sits in slot u % nbuf
    // and is fetched D = nbuf - 1 steps ahead (right after use when nbuf == 1)
    const size_t pbytes = package_bytes(sizeof(T) == 8, nx, nu, nrhs);
    const int nbuf = nbuf_in, D = nbuf_in - 1;
    auto package = [&](int u) {
        unsigned char *q = smem_raw + (size_t)(u % nbuf) * pbytes;
        return carve_package<T>(q, nx, nu, nrhs);
    };
    const Vecs<T> v = carve_vecs<T>(smem_raw + align16(nbuf_in * pbytes), nx, nu, nrhs);
    const double *b = a.b + in.oZ;
    double *z = a.z + in.oZ;

    // package t: factor blocks of stage s(t); [B A] of stage s(t+1) and its
    // right-hand-side entries (b_u, b_x of h_{s(t+1)}, then b_lambda = -c)
    auto fetch = [&](int t) {
        if (t >= len) {   // an empty group keeps the count of groups in flight uniform
            cp_async_commit();
            return;
        }
        const int s = seg_stage(c, t, N, P);
        const Package<T> K = package(t);
        fetch_factor<T, TEAM>(K, a, in, s, (t == 0) || (c >= 1), c >= 1, tid);
        if (t < len - 1) {
            const int s2 = seg_stage(c, t + 1, N, P), xq2 = xstate(s2, N);
            fetch_BA<T, TEAM>(K, a, in, s2, tid);
            for (int i = Wv.i0, r = Wv.r0; r < nrhs; Wv.next(i, r)) {
                const double *br = b + r * a.kkt;
                const double *src = i < nu    ? br + (long long)s2 * w + i
                                    : i < nux ? br + (long long)(xq2 - 1) * w + i
                                              : br + (long long)s2 * w + nu + (i - nu);
                cp_async8(K.vb + i + r * nv, src);
            }
        }
        cp_async_commit();
    };
    for (int u = 0; u < (D > 0 ? D : 1); ++u) fetch(u);
    {
        const int s = seg_stage(c, 0, N, P), xq = xstate(s, N);
        for (int i = Wux.i0, r = Wux.r0; r < nrhs; Wux.next(i, r)) {
            const double *br = b + r * a.kkt;
            v.hh[i + r * nux] = -(T)(i < nu ? br[(long long)s * w + i] : br[(long long)(xq - 1) * w + i]);
        }
        for (int e = tid; e < nx * nrhs; e += TEAM) v.gmu[e] = T(0);
    }
    for (int t = 0; t < len; ++t) {
        const int s = seg_stage(c, t, N, P), xq = xstate(s, N);
        const bool hasG = (t == 0) || (c >= 1);
        const bool last = t == len - 1;
        const Package<T> K = package(t);
        cp_async_wait_pending(D > 0 ? D - 1 : 0);   // this step's package has landed
        const T *nb = last ? nullptr : package_vectors<T>(K, v, t & 1, Wv, nrhs, nv);
        sweep_sync<TEAM>(ctx);
        if (D > 0) fetch(t + D);   // into the slot read by the previous step
        const T *Ls = K.L, *Ds = K.D;
        const T *LQ = Ls + nu + nu * nux, *DQ = Ds + nu;

        // phase 1: rho = L^{R-1} h_u (stored inverse);  w = L^{Q T} c
        for (int i = Wu.i0, r = Wu.r0; r < nrhs; Wu.next(i, r)) {
            const T *hu = v.hh + r * nux;
            T acc = Ds[i] * hu[i];
#pragma unroll 4
            for (int k = 0; k < i; ++k) acc = fma(Ls[k + i * nux], hu[k], acc);
            v.rho[i + r * nu] = acc;
        }
        if (early_p && tid < 32) {
            __syncwarp();   // rho of every right-hand side (all on this warp)
            for (int ip = Wq.i0, r = Wq.r0; r < nrhs; Wq.next(ip, r)) {
                const int i1 = ip, i2 = nx - 1 - ip;
                const T *ro = v.rho + r * nu;
                T p1 = v.hh[r * nux + nu + i1], p2 = v.hh[r * nux + nu + i2];
#pragma unroll 4
                for (int k = 0; k < nu; ++k) {
                    p1 = fma(-Ls[(nu + i1) + k * nux], ro[k], p1);
                    p2 = fma(-Ls[(nu + i2) + k * nux], ro[k], p2);
                }
                v.pv[i1 + r * nx] = p1;
                v.pv[i2 + r * nx] = p2;
            }
        }
        if (!last && pair) {
            for (int jp = Wp.i0, r = Wp.r0; r < nrhs; Wp.next(jp, r)) {
                const int j1 = jp, j2 = nx - 1 - jp;
                const T *cr = nb + r * nv + nux;   // b_lambda = -c
                T w1, w2;
                dot2(LQ + j1 + j1 * nux, 1, cr + j1, nx - j1, T(0), LQ + j2 + j2 * nux, 1, cr + j2,
                     j2 != j1 ? nx - j2 : 0, T(0), w1, w2);
                v.wv[j1 + r * nx] = -w1;
                if (j2 != j1) v.wv[j2 + r * nx] = -w2;
            }
        } else if (!last) {
            for (int j = Wx.i0, r = Wx.r0; r < nrhs; Wx.next(j, r)) {
                const T *cr = nb + r * nv + nux;   // b_lambda = -c
                T acc = T(0);
#pragma unroll 4
                for (int k = j; k < nx; ++k) acc = fma(LQ[k + j * nux], cr[k], acc);
                v.wv[j + r * nx] = -acc;
            }
        }
        sweep_sync<TEAM>(ctx);
        // phase 2: p = h_x - L^S rho (parked);  g -= L^B rho;  t = L^Q w + p;  g += A^cl c
        for (int i = Wu.i0, r = Wu.r0; r < nrhs; Wu.next(i, r))
            z[r * a.kkt + (long long)s * w + i] = (double)v.rho[i + r * nu];
        for (int ip = Wp.i0, r = Wp.r0; r < nrhs && pair; Wp.next(ip, r)) {
            const int i1 = ip, i2 = nx - 1 - ip;
            const bool two = i2 != i1;
            const T *ro = v.rho + r * nu;
            T p1, p2;
            if (early_p) {
                p1 = v.pv[i1 + r * nx];
                p2 = v.pv[i2 + r * nx];
            } else {
                p1 = v.hh[r * nux + nu + i1];
                p2 = v.hh[r * nux + nu + i2];
#pragma unroll 4
                for (int k = 0; k < nu; ++k) {
                    p1 = fma(-Ls[(nu + i1) + k * nux], ro[k], p1);
                    p2 = fma(-Ls[(nu + i2) + k * nux], ro[k], p2);
                }
            }
            z[r * a.kkt + (long long)(xq - 1) * w + nu + i1] = (double)p1;
            if (two) z[r * a.kkt + (long long)(xq - 1) * w + nu + i2] = (double)p2;
            T g1 = v.gmu[i1 + r * nx], g2 = v.gmu[i2 + r * nx];
            if (hasG) {
#pragma unroll 4
                for (int k = 0; k < nu; ++k) {
                    g1 = fma(-K.LB[i1 + k * nx], ro[k], g1);
                    g2 = fma(-K.LB[i2 + k * nx], ro[k], g2);
                }
            }
            if (!last) {
                const T *wr = v.wv + r * nx;
                T t1, t2;
                dot2(LQ + i1, nux, wr, i1 + 1, p1, LQ + i2, nux, wr, two ? i2 + 1 : 0, p2, t1, t2);
                v.tv[i1 + r * nx] = t1;
                if (two) v.tv[i2 + r * nx] = t2;
                if (c >= 1) {
                    const T *cr = nb + r * nv + nux;
#pragma unroll 4
                    for (int k = 0; k < nx; ++k) {
                        g1 = fma(-K.F[i1 + k * nx], cr[k], g1);
                        g2 = fma(-K.F[i2 + k * nx], cr[k], g2);
                    }
                }
            } else {
                v.pv[i1 + r * nx] = p1;
                if (two) v.pv[i2 + r * nx] = p2;
            }
            v.gmu[i1 + r * nx] = g1;
            if (two) v.gmu[i2 + r * nx] = g2;
        }
        for (int i = Wx.i0, r = Wx.r0; r < nrhs && !pair; Wx.next(i, r)) {
            const T *ro = v.rho + r * nu;
            T pacc = v.hh[r * nux + nu + i];
#pragma unroll 4
            for (int k = 0; k < nu; ++k) pacc = fma(-Ls[(nu + i) + k * nux], ro[k], pacc);
            z[r * a.kkt + (long long)(xq - 1) * w + nu + i] = (double)pacc;
            T g = v.gmu[i + r * nx];
            if (hasG) {
#pragma unroll 4
                for (int k = 0; k < nu; ++k) g = fma(-K.LB[i + k * nx], ro[k], g);
            }
            if (!last) {
                const T *wr = v.wv + r * nx;
                T acc = pacc;
#pragma unroll 4
                for (int j = 0; j <= i; ++j) acc = fma(LQ[i + j * nux], wr[j], acc);
                v.tv[i + r * nx] = acc;
                if (c >= 1) {
                    const T *cr = nb + r * nv + nux;
#pragma unroll 4
                    for (int k = 0; k < nx; ++k) g = fma(-K.F[i + k * nx], cr[k], g);
                }
            } else {
                v.pv[i + r * nx] = pacc;
            }
            v.gmu[i + r * nx] = g;
        }
        sweep_sync<TEAM>(ctx);
        if (!last) {
            // phase 3: h^_{s2} = h_{s2} + [B A]^T t
            for (int aa = Wux.i0, r = Wux.r0; r < nrhs; Wux.next(aa, r)) {
                const T *tr = v.tv + r * nx;
                const T *col = K.BA + aa * nx;
                T acc = -nb[aa + r * nv];
#pragma unroll 4
                for (int k = 0; k < nx; ++k) acc = fma(col[k], tr[k], acc);
                v.hh[aa + r * nux] = acc;
            }
            if (D == 0) {
                sweep_sync<TEAM>(ctx);   // the single package is free again
                fetch(t + 1);
            }
        } else {
            // y = L^{Q-1} p  (inverse stored above the diagonal of the segment's first Q block)
            for (int i = Wx.i0, r = Wx.r0; r < nrhs; Wx.next(i, r)) {
                const T *pr = v.pv + r * nx;
                T acc = DQ[i] * pr[i];
#pragma unroll 4
                for (int k = 0; k < i; ++k) acc = fma(LQ[k + i * nux], pr[k], acc);
                v.wv[i + r * nx] = acc;
            }
            sweep_sync<TEAM>(ctx);
            // d_bwd = L^{Q-T} y ;  d_fwd = g - L^A y
            for (int i = Wx.i0, r = Wx.r0; r < nrhs; Wx.next(i, r)) {
                const T *y = v.wv + r * nx;
                T db = DQ[i] * y[i];
#pragma unroll 4
                for (int k = i + 1; k < nx; ++k) db = fma(LQ[i + k * nux], y[k], db);
                T df = v.gmu[i + r * nx];
                if (c >= 1) {
#pragma unroll 4
                    for (int k = 0; k < nx; ++k) df = fma(-K.F[i + k * nx], y[k], df);
                }
                a.dF[r * a.nvec + in.oVec + (long long)c * nx + i] = (double)df;
                a.dB[r * a.nvec + in.oVec + (long long)c * nx + i] = (double)db;
            }
            sweep_sync<TEAM>(ctx);   // shared memory is reused by the next work item
        }
    }
}

template <typename T, int TEAM, int NXC, int NUC>
__global__ void __launch_bounds__(TEAM) k_solve_backward(SolveArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
        const Item wi = a.items[item];
        if (a.skip && a.skip[wi.inst]) continue;
        sweep_backward_item<T, TEAM, NXC, NUC>(a, wi, smem_raw, SweepCtx{(int)threadIdx.x, 0}, a.nbuf);
    }
}

template <typename T, int TEAM, int NXC, int NUC>
__device__ void sweep_forward_item(const SolveArgs &a, const Item wi, unsigned char *smem_raw, const SweepCtx ctx, const int nbuf_in) {
    const int tid = ctx.tid;
    const Inst in = a.inst[wi.inst];
    // NXC / NUC > 0: kernel compiled for that stage shape (every item of the launch has it)
    const int nx = NXC > 0 ? NXC : in.nx, nu = NUC > 0 ? NUC : in.nu;
    const int N = in.N, P = in.P, c = wi.seg, nrhs = a.nrhs;
    const int nux = nx + nu, nv = nux + nx, w = nu + 2 * nx;
    const int len = seg_len(c, N, P);
    // Wp: pairs of rows (i, nx-1-i) of the triangular products, in float64 for small
    // nx, where unequal row lengths leave most lanes of an FP64 instruction idle
    // (the pairing costs ALU work per step, which float32 and large nx do not repay)
    const bool pair = sizeof(T) == 8 && nx <= kPairMaxNx;
    const int half = (nx + 1) / 2;
    Walk Wu, Wx, Wv, Wp;
    Wu.init(nu, TEAM, tid);
    Wx.init(nx, TEAM, tid);
    Wv.init(nv, TEAM, tid);
    // the paired triangular products start on the second warp: the first one has the
    // u rows of the same phase
    Wp.init(half, TEAM, tid, TEAM >= 64 ? 32 : 0);
    // ring of nbuf packages: the package of processing step u sits in slot u % nbuf
    // and is fetched D = nbuf - 1 steps ahead (right after use when nbuf == 1)
    const size_t pbytes = package_bytes(sizeof(T) == 8, nx, nu, nrhs);
    const int nbuf = nbuf_in, D = nbuf_in - 1;
    auto package = [&](int u) {
        unsigned char *q = smem_raw + (size_t)(u % nbuf) * pbytes;
        return carve_package<T>(q, nx, nu, nrhs);
    };
    const Vecs<T> v = carve_vecs<T>(smem_raw + align16(nbuf_in * pbytes), nx, nu, nrhs);
    T *mu = v.gmu, *nuv = v.cv;   // coupling multipliers
    const double *b = a.b + in.oZ;
    double *z = a.z + in.oZ;
    double *zacc = a.zacc ? a.zacc + in.oZ : nullptr;

    // package for processing step t (time order: t = len-1 .. 0): factor blocks
    // and [B A] of stage s(t), its parked rho / p and b_lambda = -c
    auto fetch = [&](int u) {
        const int t = len - 1 - u;
        if (t < 0) {   // an empty group keeps the count of groups in flight uniform
            cp_async_commit();
            return;
        }
        const int s = seg_stage(c, t, N, P), xq = xstate(s, N);
        const Package<T> K = package(u);
        fetch_factor<T, TEAM>(K, a, in, s, (t == 0) || (c >= 1), c >= 1, tid);
        if (t > 0) fetch_BA<T, TEAM>(K, a, in, s, tid);
        for (int i = Wv.i0, r = Wv.r0; r < nrhs; Wv.next(i, r)) {
            if (i >= nux && t == 0) continue;
            const double *src = i < nu    ? z + r * a.kkt + (long long)s * w + i
                                : i < nux ? z + r * a.kkt + (long long)(xq - 1) * w + i
                                          : b + r * a.kkt + (long long)s * w + nu + (i - nu);
            cp_async8(K.vb + i + r * nv, src);
        }
        cp_async_commit();
    };
    for (int u = 0; u < (D > 0 ? D : 1); ++u) fetch(u);
    for (int e = tid; e < nx * nrhs; e += TEAM) {
        const int i = e % nx, r = e / nx;
        const double *lr = a.lam + r * a.nvec + in.oVec;
        mu[e] = (T)lr[(long long)c * nx + i];
        nuv[e] = (T)lr[(long long)((c - 1 + P) % P) * nx + i];
    }
    T *xv = v.xa, *xn = v.xb;
    for (int t = len - 1; t >= 0; --t) {
        const int s = seg_stage(c, t, N, P), xq = xstate(s, N);
        const bool hasG = (t == 0) || (c >= 1);
        const bool first = t == len - 1;
        const int u = len - 1 - t;
        const Package<T> K = package(u);
        cp_async_wait_pending(D > 0 ? D - 1 : 0);   // this step's package has landed
        const T *nb = package_vectors<T>(K, v, t & 1, Wv, nrhs, nv);
        sweep_sync<TEAM>(ctx);
        if (D > 0) fetch(u + D);   // into the slot read by the previous step
        const T *Ls = K.L, *Ds = K.D;
        const T *LQ = Ls + nu + nu * nux, *DQ = Ds + nu;
        if (first) {
            // x^{j1} = -L^{Q-T} (L^{Q-1}(p - nu) + L^{A T} mu)
            for (int i = Wx.i0, r = Wx.r0; r < nrhs; Wx.next(i, r)) {
                const T *pr = nb + r * nv + nu, *nr = nuv + r * nx, *mr = mu + r * nx;
                T acc = DQ[i] * (pr[i] - nr[i]);
                for (int k = 0; k < i; ++k) acc = fma(LQ[k + i * nux], pr[k] - nr[k], acc);
                if (c >= 1) {
#pragma unroll 4
                    for (int k = 0; k < nx; ++k) acc = fma(K.F[k + i * nx], mr[k], acc);
                }
                v.wv[i + r * nx] = acc;
            }
            sweep_sync<TEAM>(ctx);
            for (int i = Wx.i0, r = Wx.r0; r < nrhs; Wx.next(i, r)) {
                const T *y = v.wv + r * nx;
                T acc = DQ[i] * y[i];
#pragma unroll 4
                for (int k = i + 1; k < nx; ++k) acc = fma(LQ[i + k * nux], y[k], acc);
                xv[i + r * nx] = -acc;
            }
            sweep_sync<TEAM>(ctx);
        }
        // phase 1: v = L^{S T} x + rho + L^{B T} mu ;  w = L^{Q T} x (interior stages) ;  x out
        for (int k = Wu.i0, r = Wu.r0; r < nrhs; Wu.next(k, r)) {
            const T *x = xv + r * nx, *mr = mu + r * nx;
            T acc = nb[k + r * nv];
#pragma unroll 4
            for (int i = 0; i < nx; ++i) acc = fma(Ls[(nu + i) + k * nux], x[i], acc);
            if (hasG) {
#pragma unroll 4
                for (int i = 0; i < nx; ++i) acc = fma(K.LB[i + k * nx], mr[i], acc);
            }
            v.hh[k + r * nux] = acc;
        }
        for (int jp = Wp.i0, r = Wp.r0; r < nrhs && pair; Wp.next(jp, r)) {
            const int j1 = jp, j2 = nx - 1 - jp;
            const bool two = j2 != j1;
            const T *x = xv + r * nx;
            if (!first) {
                T w1, w2;
                dot2(LQ + j1 + j1 * nux, 1, x + j1, nx - j1, T(0), LQ + j2 + j2 * nux, 1, x + j2,
                     two ? nx - j2 : 0, T(0), w1, w2);
                v.wv[j1 + r * nx] = w1;
                if (two) v.wv[j2 + r * nx] = w2;
            }
            const long long o = r * a.kkt + (long long)(xq - 1) * w + nu;
            if (zacc) {
                atomicAdd(zacc + o + j1, (double)x[j1]);
                if (two) atomicAdd(zacc + o + j2, (double)x[j2]);
            } else {
                z[o + j1] = (double)x[j1];
                if (two) z[o + j2] = (double)x[j2];
            }
        }
        for (int j = Wx.i0, r = Wx.r0; r < nrhs && !pair; Wx.next(j, r)) {
            const T *x = xv + r * nx;
            if (!first) {
                T acc = T(0);
#pragma unroll 4
                for (int k = j; k < nx; ++k) acc = fma(LQ[k + j * nux], x[k], acc);
                v.wv[j + r * nx] = acc;
            }
            const long long o = r * a.kkt + (long long)(xq - 1) * w + nu + j;
            if (zacc) atomicAdd(zacc + o, (double)x[j]); else z[o] = (double)x[j];
        }
        sweep_sync<TEAM>(ctx);
        // phase 2: u = -L^{R-T} v (stored inverse) ;  lambda^{s-1} = L^Q w + p + A^{cl T} mu
        for (int i = Wu.i0, r = Wu.r0; r < nrhs; Wu.next(i, r)) {
            const T *vv = v.hh + r * nux;
            T acc = Ds[i] * vv[i];
#pragma unroll 4
            for (int k = i + 1; k < nu; ++k) acc = fma(Ls[i + k * nux], vv[k], acc);
            v.rho[i + r * nu] = -acc;
            const long long o = r * a.kkt + (long long)s * w + i;
            if (zacc) atomicAdd(zacc + o, (double)(-acc)); else z[o] = (double)(-acc);
        }
        if (!first) {
            const int sp = (s - 1 + N) % N;
            for (int ip = Wp.i0, r = Wp.r0; r < nrhs && pair; Wp.next(ip, r)) {
                const int i1 = ip, i2 = nx - 1 - ip;
                const bool two = i2 != i1;
                const T *wr = v.wv + r * nx, *mr = mu + r * nx;
                T l1, l2;
                dot2(LQ + i1, nux, wr, i1 + 1, nb[r * nv + nu + i1], LQ + i2, nux, wr, two ? i2 + 1 : 0,
                     nb[r * nv + nu + i2], l1, l2);
                if (c >= 1) {
#pragma unroll 4
                    for (int k = 0; k < nx; ++k) {
                        l1 = fma(K.F[k + i1 * nx], mr[k], l1);
                        l2 = fma(K.F[k + i2 * nx], mr[k], l2);
                    }
                }
                const long long o = r * a.kkt + (long long)sp * w + nu + nx;
                if (zacc) {
                    atomicAdd(zacc + o + i1, (double)l1);
                    if (two) atomicAdd(zacc + o + i2, (double)l2);
                } else {
                    z[o + i1] = (double)l1;
                    if (two) z[o + i2] = (double)l2;
                }
            }
            for (int i = Wx.i0, r = Wx.r0; r < nrhs && !pair; Wx.next(i, r)) {
                const T *wr = v.wv + r * nx, *mr = mu + r * nx;
                T acc = nb[r * nv + nu + i];
#pragma unroll 4
                for (int j = 0; j <= i; ++j) acc = fma(LQ[i + j * nux], wr[j], acc);
                if (c >= 1) {
#pragma unroll 4
                    for (int k = 0; k < nx; ++k) acc = fma(K.F[k + i * nx], mr[k], acc);
                }
                const long long o = r * a.kkt + (long long)sp * w + nu + nx + i;
                if (zacc) atomicAdd(zacc + o, (double)acc); else z[o] = (double)acc;
            }
        }
        sweep_sync<TEAM>(ctx);
        if (t > 0) {
            // phase 3: x^{s+1} = A_s x + B_s u + c_s
            for (int i = Wx.i0, r = Wx.r0; r < nrhs; Wx.next(i, r)) {
                const T *x = xv + r * nx, *u = v.rho + r * nu;
                T acc = -nb[r * nv + nux + i];
#pragma unroll 4
                for (int k = 0; k < nu; ++k) acc = fma(K.BA[i + k * nx], u[k], acc);
#pragma unroll 4
                for (int k = 0; k < nx; ++k) acc = fma(K.BA[i + (nu + k) * nx], x[k], acc);
                xn[i + r * nx] = acc;
            }
            T *tmp = xv; xv = xn; xn = tmp;
            if (D == 0) {
                sweep_sync<TEAM>(ctx);   // the single package is free again
                fetch(u + 1);
            }
        }
    }
    sweep_sync<TEAM>(ctx);   // shared memory is reused by the next work item
}

template <typename T, int TEAM, int NXC, int NUC>
__global__ void __launch_bounds__(TEAM) k_solve_forward(SolveArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
        const Item wi = a.items[item];
        if (a.skip && a.skip[wi.inst]) continue;
        sweep_forward_item<T, TEAM, NXC, NUC>(a, wi, smem_raw, SweepCtx{(int)threadIdx.x, 0}, a.nbuf);
    }
}

// ---------------------------------------------------------------------------
// Float32 sweeps of the whole batch in one persistent launch per sweep: teams
// of 128, 64 or 32 threads per work item (by the shared memory its stage
// packages need), CTAs that take items from their class's counter and then
// re-form their teams for the other classes (as the one-team factor does).
// Each item gets the deepest package ring (up to 4) that fits its team's slot.
// ---------------------------------------------------------------------------
namespace {

template <bool BACKWARD, int T>
__device__ void sweep_team_loop(const SolveArgs &a, const TeamPlanDev &plan, int cls, unsigned char *arena, int *cmd) {
    constexpr int TEAMS = kTeamCtaThreads / T;
    const int tmi = (int)threadIdx.x / T;
    const SweepCtx ctx{(int)threadIdx.x - tmi * T, 1 + tmi};
    const size_t slot_bytes = (size_t)plan.arena_floats * 4 / TEAMS;
    unsigned char *slot = arena + (size_t)tmi * slot_bytes;
    for (;;) {
        if (ctx.tid == 0) cmd[tmi] = atomicAdd(plan.counter + cls, 1);
        sweep_sync<T>(ctx);
        const int idx = cmd[tmi];
        sweep_sync<T>(ctx);   // the command word is read before it is rewritten
        if (idx >= plan.n[cls]) break;
        const Item wi = plan.items[plan.off[cls] + idx];
        if (a.skip && a.skip[wi.inst]) continue;
        const Inst &in = a.inst[wi.inst];
        int nbuf = 4;
        while (nbuf > 1 && solve_smem_bytes(false, in.nx, in.nu, a.nrhs, nbuf) > slot_bytes) --nbuf;
        if constexpr (BACKWARD)
            sweep_backward_item<float, T, 0, 0>(a, wi, slot, ctx, nbuf);
        else
            sweep_forward_item<float, T, 0, 0>(a, wi, slot, ctx, nbuf);
        sweep_sync<T>(ctx);   // the slot is reused by the next item
    }
}

template <bool BACKWARD>
__global__ void __launch_bounds__(kTeamCtaThreads, kSweepCtasPerSm) k_sweep_team(SolveArgs a, TeamPlanDev plan) {
    extern __shared__ __align__(16) unsigned char smem_all[];
    __shared__ int cmd[4];
    const int first = (int)blockIdx.x < plan.g0 ? 0 : ((int)blockIdx.x < plan.g0 + plan.g1 ? 1 : 2);
    for (int step = 0; step < 3; ++step) {
        const int cls = step == 0 ? first : (first == 0 ? step : step - 1 + (step - 1 >= first ? 1 : 0));
        if (plan.n[cls] > 0) {
            if (cls == 0)
                sweep_team_loop<BACKWARD, 128>(a, plan, 0, smem_all, cmd);
            else if (cls == 1)
                sweep_team_loop<BACKWARD, 64>(a, plan, 1, smem_all, cmd);
            else
                sweep_team_loop<BACKWARD, 32>(a, plan, 2, smem_all, cmd);
        }
        __syncthreads();   // every team of the CTA has left the configuration and its slots
    }
}

}  // namespace

cudaError_t launch_sweep_team(bool backward, const SolveArgs &a, const TeamPlanDev &plan, int grid, cudaStream_t st) {
    if (grid <= 0) return cudaSuccess;
    const size_t arena = (size_t)plan.arena_floats * 4;
    auto k = backward ? k_sweep_team<true> : k_sweep_team<false>;
    cudaError_t e = ensure_smem((const void *)k, arena);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(plan.counter, 0, 3 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    k<<<grid, kTeamCtaThreads, arena, st>>>(a, plan);
    return cudaGetLastError();
}

template <typename T, int TEAM, int NXC, int NUC>
static cudaError_t launch_sweep(bool backward, size_t smem, const SolveArgs &a, cudaStream_t st) {
    auto k = backward ? k_solve_backward<T, TEAM, NXC, NUC> : k_solve_forward<T, TEAM, NXC, NUC>;
    cudaError_t e = ensure_smem((const void *)k, smem);
    if (e != cudaSuccess) return e;
    k<<<a.n_items, TEAM, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int NXC, int NUC>
static cudaError_t launch_sweep_team(bool backward, int team, size_t smem, const SolveArgs &a, cudaStream_t st) {
    if (team == 32) return launch_sweep<T, 32, NXC, NUC>(backward, smem, a, st);
    if (team == 64) return launch_sweep<T, 64, NXC, NUC>(backward, smem, a, st);
    if (team == 128) return launch_sweep<T, 128, NXC, NUC>(backward, smem, a, st);
    return launch_sweep<T, 256, NXC, NUC>(backward, smem, a, st);
}

static cudaError_t launch_sweep_any(bool backward, bool fp64, int team, int shape, size_t smem, const SolveArgs &a,
                                    cudaStream_t st) {
    if (a.n_items == 0) return cudaSuccess;
    if (fp64) return launch_sweep_team<double, 0, 0>(backward, team, smem, a, st);
    switch (shape) {   // float32 kernels compiled for the listed stage shapes (kStageShapes)
        case 1: return launch_sweep_team<float, kStageShapes[1].nx, kStageShapes[1].nu>(backward, team, smem, a, st);
        case 2: return launch_sweep_team<float, kStageShapes[2].nx, kStageShapes[2].nu>(backward, team, smem, a, st);
        case 3: return launch_sweep_team<float, kStageShapes[3].nx, kStageShapes[3].nu>(backward, team, smem, a, st);
        case 4: return launch_sweep_team<float, kStageShapes[4].nx, kStageShapes[4].nu>(backward, team, smem, a, st);
        default: return launch_sweep_team<float, 0, 0>(backward, team, smem, a, st);
    }
}

cudaError_t launch_solve_backward(bool fp64, int team, int shape, size_t smem, const SolveArgs &a, cudaStream_t st) {
    return launch_sweep_any(true, fp64, team, shape, smem, a, st);
}
cudaError_t launch_solve_forward(bool fp64, int team, int shape, size_t smem, const SolveArgs &a, cudaStream_t st) {
    return launch_sweep_any(false, fp64, team, shape, smem, a, st);
}

}  // namespace cyq
