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
// a parallel matrix-vector product.  One CTA per (instance, segment); the
// next stage's blocks are copied to shared memory (cp.async) while the
// current stage is processed (or, when two packages do not fit in shared
// memory, right after it); nrhs right-hand sides share each block.
#include "cyq_internal.cuh"

namespace cyq {

namespace {

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

template <typename T, int TEAM>
__device__ void async_copy(T *dst, const T *src, int count) {
    for (int e = threadIdx.x; e < count; e += TEAM) {
        if (sizeof(T) == 8)
            cp_async8(dst + e, src + e);
        else
            cp_async4(dst + e, src + e);
    }
}

// Per-stage package in shared memory: factor blocks of stage s and the raw
// float64 [B A] of the stage whose dynamics the sweep needs next.
template <typename T>
struct Package {
    T *L, *D, *LB, *F;   // (nu+nx)^2 (ld nu+nx), nu+nx, nx*nu, nx*nx
    double *BA;          // nx x (nu+nx), ld nx (raw [B A])
};

template <typename T>
__device__ Package<T> carve_package(unsigned char *&p, int nx, int nu) {
    const int nux = nx + nu;
    Package<T> k;
    k.BA = reinterpret_cast<double *>(p);
    p += ((size_t)nx * nux * 8 + 15) / 16 * 16;
    k.L = reinterpret_cast<T *>(p);
    k.D = k.L + nux * nux;
    k.LB = k.D + nux;
    k.F = k.LB + nx * nu;
    p += (((size_t)nux * nux + nux + (size_t)nx * nu + (size_t)nx * nx) * sizeof(T) + 15) / 16 * 16;
    return k;
}

size_t package_bytes(bool fp64, int nx, int nu) {
    const size_t nux = (size_t)nx + nu;
    const size_t el = fp64 ? 8 : 4;
    return ((size_t)nx * nux * 8 + 15) / 16 * 16 +
           ((nux * nux + nux + (size_t)nx * nu + (size_t)nx * nx) * el + 15) / 16 * 16;
}

// Issue the copies of a package: factor blocks of stage s (LB/F when needed),
// and [B A] of stage sba (skipped when sba < 0; A_0 is replaced by zero).
template <typename T, int TEAM>
__device__ void fetch_package(const Package<T> &k, const SolveArgs &a, const Inst &in, int s, bool wantLB,
                              bool wantF, int sba) {
    const int nx = in.nx, nu = in.nu, nux = nx + nu;
    const T *Lg = reinterpret_cast<const T *>(a.L) + in.oL;
    const T *LBg = reinterpret_cast<const T *>(a.LB) + in.oLB;
    const T *Fg = reinterpret_cast<const T *>(a.F) + in.oF;
    const T *DIg = reinterpret_cast<const T *>(a.DI) + in.oDI;
    async_copy<T, TEAM>(k.L, Lg + (long long)s * nux * nux, nux * nux);
    async_copy<T, TEAM>(k.D, DIg + (long long)s * nux, nux);
    if (wantLB) async_copy<T, TEAM>(k.LB, LBg + (long long)s * nx * nu, nx * nu);
    if (wantF) async_copy<T, TEAM>(k.F, Fg + (long long)s * nx * nx, nx * nx);
    if (sba >= 0) {
        async_copy<double, TEAM>(k.BA, a.data.B + in.oB + (long long)sba * nx * nu, nx * nu);
        if (sba != 0)
            async_copy<double, TEAM>(k.BA + nx * nu, a.data.A + in.oA + (long long)sba * nx * nx, nx * nx);
        else
            for (int e = threadIdx.x; e < nx * nx; e += TEAM) k.BA[nx * nu + e] = 0.0;
    }
    cp_async_commit();
}

// Vectors of one work item (T), each nrhs copies.
template <typename T>
struct Vecs {
    T *hh, *rho, *pv, *tv, *wv, *gmu, *cv, *xv;
};

template <typename T>
__device__ Vecs<T> carve_vecs(unsigned char *p, int nx, int nu, int nrhs) {
    const int nux = nx + nu;
    T *q = reinterpret_cast<T *>(p);
    Vecs<T> v;
    v.hh = q; q += nux * nrhs;
    v.rho = q; q += nu * nrhs;
    v.pv = q; q += nx * nrhs;
    v.tv = q; q += nx * nrhs;
    v.wv = q; q += nx * nrhs;
    v.gmu = q; q += nx * nrhs;
    v.cv = q; q += nx * nrhs;
    v.xv = q; q += nx * nrhs;
    return v;
}

size_t vecs_bytes(bool fp64, int nx, int nu, int nrhs) {
    return ((size_t)(nx + nu) * nrhs + (size_t)nu * nrhs + 6 * (size_t)nx * nrhs) * (fp64 ? 8 : 4);
}

}  // namespace

size_t solve_smem_bytes(bool fp64, int nx, int nu, int nrhs, int nbuf) {
    return nbuf * package_bytes(fp64, nx, nu) + vecs_bytes(fp64, nx, nu, nrhs);
}

template <typename T, int TEAM>
__global__ void __launch_bounds__(TEAM) k_solve_backward(SolveArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
        const Item wi = a.items[item];
        if (a.skip && a.skip[wi.inst]) continue;
        const Inst in = a.inst[wi.inst];
        const int N = in.N, nx = in.nx, nu = in.nu, P = in.P, c = wi.seg, nrhs = a.nrhs;
        const int nux = nx + nu, w = nu + 2 * nx;
        const int len = seg_len(c, N, P);
        unsigned char *p = smem_raw;
        Package<T> pk[2];
        pk[0] = carve_package<T>(p, nx, nu);
        pk[1] = a.nbuf == 2 ? carve_package<T>(p, nx, nu) : pk[0];
        const Vecs<T> v = carve_vecs<T>(p, nx, nu, nrhs);
        const double *b = a.b + in.oZ;
        double *z = a.z + in.oZ;

        // package t: factor blocks of stage s(t) and [B A] of stage s(t+1)
        auto fetch = [&](int t) {
            const int s = seg_stage(c, t, N, P);
            const bool last = t == len - 1;
            fetch_package<T, TEAM>(pk[t & 1], a, in, s, (t == 0) || (c >= 1), c >= 1,
                                   last ? -1 : seg_stage(c, t + 1, N, P));
        };
        fetch(0);
        {
            const int s = seg_stage(c, 0, N, P), xq = xstate(s, N);
            for (int e = threadIdx.x; e < nux * nrhs; e += TEAM) {
                const int aa = e % nux, r = e / nux;
                const double *br = b + r * a.kkt;
                v.hh[e] = aa < nu ? -(T)br[(long long)s * w + aa] : -(T)br[(long long)(xq - 1) * w + nu + (aa - nu)];
            }
            for (int e = threadIdx.x; e < nx * nrhs; e += TEAM) v.gmu[e] = T(0);
        }
        for (int t = 0; t < len; ++t) {
            const int s = seg_stage(c, t, N, P), xq = xstate(s, N);
            const bool hasG = (t == 0) || (c >= 1);
            const bool last = (t == len - 1);
            const Package<T> &K = pk[t & 1];
            cp_async_wait_all();
            team_sync();
            if (!last && a.nbuf == 2) fetch(t + 1);   // overlaps with this stage
            const T *Ls = K.L, *Ds = K.D;
            const T *LQ = Ls + nu + nu * nux, *DQ = Ds + nu;
            // rho = L^{R-1} h_u  (stored inverse: diagonal Ds, strictly lower part transposed above)
            {
                int i, r;
                rect_start(threadIdx.x, nu, i, r);
                for (; r < nrhs; rect_advance(i, r, nu, TEAM)) {
                    const T *hu = v.hh + r * nux;
                    T acc = Ds[i] * hu[i];
                    for (int k = 0; k < i; ++k) acc = fma(Ls[k + i * nux], hu[k], acc);
                    v.rho[i + r * nu] = acc;
                }
            }
            // next stage's constant terms (independent of rho)
            int s2 = 0, xq2 = 0;
            if (!last) {
                s2 = seg_stage(c, t + 1, N, P);
                xq2 = xstate(s2, N);
                for (int e = threadIdx.x; e < nx * nrhs; e += TEAM) {
                    const int i = e % nx, r = e / nx;
                    v.cv[e] = -(T)b[r * a.kkt + (long long)s2 * w + nu + nx + i];
                }
            }
            team_sync();
            // p = h_x - L^S rho ;  g -= L^B rho ; park rho, p
            {
                int i, r;
                rect_start(threadIdx.x, nx, i, r);
                for (; r < nrhs; rect_advance(i, r, nx, TEAM)) {
                    const T *ro = v.rho + r * nu;
                    T acc = v.hh[r * nux + nu + i];
                    for (int k = 0; k < nu; ++k) acc = fma(-Ls[(nu + i) + k * nux], ro[k], acc);
                    v.pv[i + r * nx] = acc;
                    z[r * a.kkt + (long long)(xq - 1) * w + nu + i] = (double)acc;
                    if (hasG) {
                        T g = v.gmu[i + r * nx];
                        for (int k = 0; k < nu; ++k) g = fma(-K.LB[i + k * nx], ro[k], g);
                        v.gmu[i + r * nx] = g;
                    }
                }
                for (int e = threadIdx.x; e < nu * nrhs; e += TEAM) {
                    const int i = e % nu, r = e / nu;
                    z[r * a.kkt + (long long)s * w + i] = (double)v.rho[e];
                }
            }
            if (!last) {
                // w = L^{Q T} c
                {
                    int j, r;
                    rect_start(threadIdx.x, nx, j, r);
                    for (; r < nrhs; rect_advance(j, r, nx, TEAM)) {
                        const T *cr = v.cv + r * nx;
                        T acc = T(0);
                        for (int k = j; k < nx; ++k) acc = fma(LQ[k + j * nux], cr[k], acc);
                        v.wv[j + r * nx] = acc;
                    }
                }
                team_sync();
                // t = L^Q w + p ;  g += A^cl c
                {
                    int i, r;
                    rect_start(threadIdx.x, nx, i, r);
                    for (; r < nrhs; rect_advance(i, r, nx, TEAM)) {
                        const T *wr = v.wv + r * nx;
                        T acc = v.pv[i + r * nx];
                        for (int j = 0; j <= i; ++j) acc = fma(LQ[i + j * nux], wr[j], acc);
                        v.tv[i + r * nx] = acc;
                        if (c >= 1) {
                            const T *cr = v.cv + r * nx;
                            T g = v.gmu[i + r * nx];
                            for (int k = 0; k < nx; ++k) g = fma(K.F[i + k * nx], cr[k], g);
                            v.gmu[i + r * nx] = g;
                        }
                    }
                }
                team_sync();
                // h^_{s2} = h_{s2} + [B A]^T t
                {
                    int aa, r;
                    rect_start(threadIdx.x, nux, aa, r);
                    for (; r < nrhs; rect_advance(aa, r, nux, TEAM)) {
                        const double *br = b + r * a.kkt;
                        const T *tr = v.tv + r * nx;
                        const double *col = K.BA + aa * nx;
                        T acc = aa < nu ? -(T)br[(long long)s2 * w + aa]
                                        : -(T)br[(long long)(xq2 - 1) * w + nu + (aa - nu)];
                        for (int k = 0; k < nx; ++k) acc = fma((T)col[k], tr[k], acc);
                        v.hh[aa + r * nux] = acc;
                    }
                }
            } else {
                team_sync();
                // y = L^{Q-1} p  (inverse stored above the diagonal of this first stage's Q block)
                {
                    int i, r;
                    rect_start(threadIdx.x, nx, i, r);
                    for (; r < nrhs; rect_advance(i, r, nx, TEAM)) {
                        const T *pr = v.pv + r * nx;
                        T acc = DQ[i] * pr[i];
                        for (int k = 0; k < i; ++k) acc = fma(LQ[k + i * nux], pr[k], acc);
                        v.wv[i + r * nx] = acc;
                    }
                }
                team_sync();
                // d_bwd = L^{Q-T} y ;  d_fwd = g - L^A y
                {
                    int i, r;
                    rect_start(threadIdx.x, nx, i, r);
                    for (; r < nrhs; rect_advance(i, r, nx, TEAM)) {
                        const T *y = v.wv + r * nx;
                        T db = DQ[i] * y[i];
                        for (int k = i + 1; k < nx; ++k) db = fma(LQ[i + k * nux], y[k], db);
                        T df = v.gmu[i + r * nx];
                        if (c >= 1)
                            for (int k = 0; k < nx; ++k) df = fma(-K.F[i + k * nx], y[k], df);
                        a.dF[r * a.nvec + in.oVec + (long long)c * nx + i] = (double)df;
                        a.dB[r * a.nvec + in.oVec + (long long)c * nx + i] = (double)db;
                    }
                }
            }
            team_sync();
            if (!last && a.nbuf == 1) fetch(t + 1);   // the single package is free again
        }
    }
}

template <typename T, int TEAM>
__global__ void __launch_bounds__(TEAM) k_solve_forward(SolveArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
        const Item wi = a.items[item];
        if (a.skip && a.skip[wi.inst]) continue;
        const Inst in = a.inst[wi.inst];
        const int N = in.N, nx = in.nx, nu = in.nu, P = in.P, c = wi.seg, nrhs = a.nrhs;
        const int nux = nx + nu, w = nu + 2 * nx;
        const int len = seg_len(c, N, P);
        unsigned char *p = smem_raw;
        Package<T> pk[2];
        pk[0] = carve_package<T>(p, nx, nu);
        pk[1] = a.nbuf == 2 ? carve_package<T>(p, nx, nu) : pk[0];
        const Vecs<T> v = carve_vecs<T>(p, nx, nu, nrhs);
        T *mu = v.gmu, *nuv = v.cv;   // coupling multipliers
        const double *b = a.b + in.oZ;
        double *z = a.z + in.oZ;
        double *zacc = a.zacc ? a.zacc + in.oZ : nullptr;

        // package for processing step t (time order: t = len-1 .. 0): factor blocks
        // of stage s(t) and [B A] of that same stage (its outgoing dynamics)
        auto fetch = [&](int t) {
            const int s = seg_stage(c, t, N, P);
            fetch_package<T, TEAM>(pk[t & 1], a, in, s, (t == 0) || (c >= 1), c >= 1, t > 0 ? s : -1);
        };
        fetch(len - 1);
        for (int e = threadIdx.x; e < nx * nrhs; e += TEAM) {
            const int i = e % nx, r = e / nx;
            const double *lr = a.lam + r * a.nvec + in.oVec;
            mu[e] = (T)lr[(long long)c * nx + i];
            nuv[e] = (T)lr[(long long)((c - 1 + P) % P) * nx + i];
        }
        for (int t = len - 1; t >= 0; --t) {
            const int s = seg_stage(c, t, N, P), xq = xstate(s, N);
            const bool hasG = (t == 0) || (c >= 1);
            const bool first = (t == len - 1);
            const Package<T> &K = pk[t & 1];
            // parked rho / p of this stage
            for (int e = threadIdx.x; e < nu * nrhs; e += TEAM) {
                const int i = e % nu, r = e / nu;
                v.rho[e] = (T)z[r * a.kkt + (long long)s * w + i];
            }
            for (int e = threadIdx.x; e < nx * nrhs; e += TEAM) {
                const int i = e % nx, r = e / nx;
                v.pv[e] = (T)z[r * a.kkt + (long long)(xq - 1) * w + nu + i];
            }
            cp_async_wait_all();
            team_sync();
            if (t > 0 && a.nbuf == 2) fetch(t - 1);   // overlaps with this stage
            const T *Ls = K.L, *Ds = K.D;
            const T *LQ = Ls + nu + nu * nux, *DQ = Ds + nu;
            if (first) {
                // x^{j1} = -L^{Q-T} (L^{Q-1}(p - nu) + L^{A T} mu)
                {
                    int i, r;
                    rect_start(threadIdx.x, nx, i, r);
                    for (; r < nrhs; rect_advance(i, r, nx, TEAM)) {
                        const T *pr = v.pv + r * nx, *nr = nuv + r * nx, *mr = mu + r * nx;
                        T acc = DQ[i] * (pr[i] - nr[i]);
                        for (int k = 0; k < i; ++k) acc = fma(LQ[k + i * nux], pr[k] - nr[k], acc);
                        if (c >= 1)
                            for (int k = 0; k < nx; ++k) acc = fma(K.F[k + i * nx], mr[k], acc);
                        v.wv[i + r * nx] = acc;
                    }
                }
                team_sync();
                {
                    int i, r;
                    rect_start(threadIdx.x, nx, i, r);
                    for (; r < nrhs; rect_advance(i, r, nx, TEAM)) {
                        const T *y = v.wv + r * nx;
                        T acc = DQ[i] * y[i];
                        for (int k = i + 1; k < nx; ++k) acc = fma(LQ[i + k * nux], y[k], acc);
                        v.xv[i + r * nx] = -acc;
                    }
                }
                team_sync();
            }
            // v = L^{S T} x + rho + L^{B T} mu  ->  hh[0..nu) ;  w = L^{Q T} x (interior stages)
            {
                int k, r;
                rect_start(threadIdx.x, nu, k, r);
                for (; r < nrhs; rect_advance(k, r, nu, TEAM)) {
                    const T *x = v.xv + r * nx, *mr = mu + r * nx;
                    T acc = v.rho[k + r * nu];
                    for (int i = 0; i < nx; ++i) acc = fma(Ls[(nu + i) + k * nux], x[i], acc);
                    if (hasG)
                        for (int i = 0; i < nx; ++i) acc = fma(K.LB[i + k * nx], mr[i], acc);
                    v.hh[k + r * nux] = acc;
                }
            }
            if (!first) {
                int j, r;
                rect_start(threadIdx.x, nx, j, r);
                for (; r < nrhs; rect_advance(j, r, nx, TEAM)) {
                    const T *x = v.xv + r * nx;
                    T acc = T(0);
                    for (int k = j; k < nx; ++k) acc = fma(LQ[k + j * nux], x[k], acc);
                    v.wv[j + r * nx] = acc;
                }
            }
            team_sync();
            // u = -L^{R-T} v  (stored inverse)
            {
                int i, r;
                rect_start(threadIdx.x, nu, i, r);
                for (; r < nrhs; rect_advance(i, r, nu, TEAM)) {
                    const T *vv = v.hh + r * nux;
                    T acc = Ds[i] * vv[i];
                    for (int k = i + 1; k < nu; ++k) acc = fma(Ls[i + k * nux], vv[k], acc);
                    v.rho[i + r * nu] = -acc;
                }
            }
            // interior multiplier lambda^{s-1} = L^Q L^{Q T} x + p + A^{cl T} mu
            if (!first) {
                const int sp = (s - 1 + N) % N;
                int i, r;
                rect_start(threadIdx.x, nx, i, r);
                for (; r < nrhs; rect_advance(i, r, nx, TEAM)) {
                    const T *wr = v.wv + r * nx, *mr = mu + r * nx;
                    T acc = v.pv[i + r * nx];
                    for (int j = 0; j <= i; ++j) acc = fma(LQ[i + j * nux], wr[j], acc);
                    if (c >= 1)
                        for (int k = 0; k < nx; ++k) acc = fma(K.F[k + i * nx], mr[k], acc);
                    const long long o = r * a.kkt + (long long)sp * w + nu + nx + i;
                    if (zacc) zacc[o] += (double)acc; else z[o] = (double)acc;
                }
            }
            team_sync();
            for (int e = threadIdx.x; e < nu * nrhs; e += TEAM) {
                const int i = e % nu, r = e / nu;
                const long long o = r * a.kkt + (long long)s * w + i;
                if (zacc) zacc[o] += (double)v.rho[e]; else z[o] = (double)v.rho[e];
            }
            for (int e = threadIdx.x; e < nx * nrhs; e += TEAM) {
                const int i = e % nx, r = e / nx;
                const long long o = r * a.kkt + (long long)(xq - 1) * w + nu + i;
                if (zacc) zacc[o] += (double)v.xv[e]; else z[o] = (double)v.xv[e];
            }
            if (t > 0) {
                // x^{s+1} = A_s x + B_s u + c_s
                int i, r;
                rect_start(threadIdx.x, nx, i, r);
                for (; r < nrhs; rect_advance(i, r, nx, TEAM)) {
                    const T *x = v.xv + r * nx, *u = v.rho + r * nu;
                    T acc = -(T)b[r * a.kkt + (long long)s * w + nu + nx + i];
                    for (int k = 0; k < nu; ++k) acc = fma((T)K.BA[i + k * nx], u[k], acc);
                    for (int k = 0; k < nx; ++k) acc = fma((T)K.BA[i + (nu + k) * nx], x[k], acc);
                    v.tv[i + r * nx] = acc;
                }
                team_sync();
                for (int e = threadIdx.x; e < nx * nrhs; e += TEAM) v.xv[e] = v.tv[e];
            }
            team_sync();
            if (t > 0 && a.nbuf == 1) fetch(t - 1);   // the single package is free again
        }
    }
}

template <typename T, int TEAM>
static cudaError_t launch_sweep(bool backward, size_t smem, const SolveArgs &a, cudaStream_t st) {
    auto k = backward ? k_solve_backward<T, TEAM> : k_solve_forward<T, TEAM>;
    cudaError_t e = ensure_smem((const void *)k, smem);
    if (e != cudaSuccess) return e;
    k<<<a.n_items, TEAM, smem, st>>>(a);
    return cudaGetLastError();
}

static cudaError_t launch_sweep_any(bool backward, bool fp64, int team, size_t smem, const SolveArgs &a,
                                    cudaStream_t st) {
    if (a.n_items == 0) return cudaSuccess;
    if (fp64) {
        if (team == 32) return launch_sweep<double, 32>(backward, smem, a, st);
        if (team == 64) return launch_sweep<double, 64>(backward, smem, a, st);
        return launch_sweep<double, 128>(backward, smem, a, st);
    }
    if (team == 32) return launch_sweep<float, 32>(backward, smem, a, st);
    if (team == 64) return launch_sweep<float, 64>(backward, smem, a, st);
    return launch_sweep<float, 128>(backward, smem, a, st);
}

cudaError_t launch_solve_backward(bool fp64, int team, size_t smem, const SolveArgs &a, cudaStream_t st) {
    return launch_sweep_any(true, fp64, team, smem, a, st);
}
cudaError_t launch_solve_forward(bool fp64, int team, size_t smem, const SolveArgs &a, cudaStream_t st) {
    return launch_sweep_any(false, fp64, team, smem, a, st);
}

}  // namespace cyq
