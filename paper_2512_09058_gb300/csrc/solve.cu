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
// One CTA per (instance, segment); nrhs right-hand sides share each factor load.
#include "cyq_internal.cuh"

namespace cyq {

namespace {

template <typename T, int TEAM>
__device__ void load_T(T *dst, const T *src, int count) {
    for (int e = threadIdx.x; e < count; e += TEAM) dst[e] = src[e];
}

template <typename T, int TEAM>
__device__ void load_BA_T(T *BA, const Data &d, const Inst &in, int s) {
    const int nx = in.nx, nu = in.nu;
    const double *B = d.B + in.oB + (long long)s * nx * nu;
    const double *A = d.A + in.oA + (long long)s * nx * nx;
    for (int e = threadIdx.x; e < nx * nu; e += TEAM) BA[e] = (T)B[e];
    for (int e = threadIdx.x; e < nx * nx; e += TEAM) BA[nx * nu + e] = (s != 0) ? (T)A[e] : T(0);
}

struct SolveSmem {
    template <typename T>
    __device__ static void carve(unsigned char *raw, int nx, int nu, int nrhs, T *&Ls, T *&Ds, T *&BA, T *&Fs,
                                 T *&LB, T *&hh, T *&rho, T *&pv, T *&tv, T *&wv, T *&gmu, T *&cv, T *&xv) {
        const int nux = nx + nu;
        T *p = reinterpret_cast<T *>(raw);
        Ls = p; p += nux * nux;
        Ds = p; p += nux;
        BA = p; p += nx * nux;
        Fs = p; p += nx * nx;
        LB = p; p += nx * nu;
        hh = p; p += nux * nrhs;
        rho = p; p += nu * nrhs;
        pv = p; p += nx * nrhs;
        tv = p; p += nx * nrhs;
        wv = p; p += nx * nrhs;
        gmu = p; p += nx * nrhs;
        cv = p; p += nx * nrhs;
        xv = p; p += nx * nrhs;
    }
};

}  // namespace

size_t solve_smem_bytes(bool fp64, int nx, int nu, int nrhs) {
    const size_t nux = (size_t)nx + nu;
    const size_t cnt = nux * nux + nux + nx * nux + (size_t)nx * nx + (size_t)nx * nu + nux * nrhs +
                       (size_t)nu * nrhs + 6 * (size_t)nx * nrhs;
    return cnt * (fp64 ? 8 : 4);
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
        T *Ls, *Ds, *BA, *Fs, *LB, *hh, *rho, *pv, *tv, *wv, *gmu, *cv, *xv;
        SolveSmem::carve<T>(smem_raw, nx, nu, nrhs, Ls, Ds, BA, Fs, LB, hh, rho, pv, tv, wv, gmu, cv, xv);
        const T *DIg = reinterpret_cast<const T *>(a.DI) + in.oDI;
        const T *DQ = Ds + nu;
        const T *Lg = reinterpret_cast<const T *>(a.L) + in.oL;
        const T *LBg = reinterpret_cast<const T *>(a.LB) + in.oLB;
        const T *Fg = reinterpret_cast<const T *>(a.F) + in.oF;
        const double *b = a.b + in.oZ;
        double *z = a.z + in.oZ;
        const T *LQ = Ls + nu + nu * nux;

        // right-hand side of the first processed stage
        {
            const int s = seg_stage(c, 0, N, P), xq = xstate(s, N);
            for (int e = threadIdx.x; e < nux * nrhs; e += TEAM) {
                const int aa = e % nux, r = e / nux;
                const double *br = b + r * a.kkt;
                hh[e] = aa < nu ? -(T)br[(long long)s * w + aa] : -(T)br[(long long)(xq - 1) * w + nu + (aa - nu)];
            }
            for (int e = threadIdx.x; e < nx * nrhs; e += TEAM) gmu[e] = T(0);
        }
        for (int t = 0; t < len; ++t) {
            const int s = seg_stage(c, t, N, P), xq = xstate(s, N);
            const bool hasG = (t == 0) || (c >= 1);
            const bool last = (t == len - 1);
            load_T<T, TEAM>(Ls, Lg + (long long)s * nux * nux, nux * nux);
            load_T<T, TEAM>(Ds, DIg + (long long)s * nux, nux);
            if (hasG) load_T<T, TEAM>(LB, LBg + (long long)s * nx * nu, nx * nu);
            if (c >= 1) load_T<T, TEAM>(Fs, Fg + (long long)s * nx * nx, nx * nx);
            team_sync();
            // rho = L^{R-1} h_u
            for (int r = threadIdx.x; r < nrhs; r += TEAM) {
                const T *hu = hh + r * nux;
                T *ro = rho + r * nu;
                for (int i = 0; i < nu; ++i) {
                    T acc = hu[i];
                    for (int k = 0; k < i; ++k) acc = fma(-Ls[i + k * nux], ro[k], acc);
                    ro[i] = acc * Ds[i];
                }
            }
            team_sync();
            // p = h_x - L^S rho ;  g -= L^B rho
            for (int e = threadIdx.x; e < nx * nrhs; e += TEAM) {
                const int i = e % nx, r = e / nx;
                const T *ro = rho + r * nu;
                T acc = hh[r * nux + nu + i];
                for (int k = 0; k < nu; ++k) acc -= Ls[(nu + i) + k * nux] * ro[k];
                pv[e] = acc;
                if (hasG) {
                    T g = T(0);
                    for (int k = 0; k < nu; ++k) g += LB[i + k * nx] * ro[k];
                    gmu[e] -= g;
                }
            }
            team_sync();
            for (int e = threadIdx.x; e < nu * nrhs; e += TEAM) {
                const int i = e % nu, r = e / nu;
                z[r * a.kkt + (long long)s * w + i] = (double)rho[e];
            }
            for (int e = threadIdx.x; e < nx * nrhs; e += TEAM) {
                const int i = e % nx, r = e / nx;
                z[r * a.kkt + (long long)(xq - 1) * w + nu + i] = (double)pv[e];
            }
            if (!last) {
                const int s2 = seg_stage(c, t + 1, N, P), xq2 = xstate(s2, N);
                load_BA_T<T, TEAM>(BA, a.data, in, s2);
                for (int e = threadIdx.x; e < nx * nrhs; e += TEAM) {
                    const int i = e % nx, r = e / nx;
                    cv[e] = -(T)b[r * a.kkt + (long long)s2 * w + nu + nx + i];
                }
                team_sync();
                // w = L^{Q T} c
                for (int e = threadIdx.x; e < nx * nrhs; e += TEAM) {
                    const int j = e % nx, r = e / nx;
                    const T *cr = cv + r * nx;
                    T acc = T(0);
                    for (int k = j; k < nx; ++k) acc += LQ[k + j * nux] * cr[k];
                    wv[e] = acc;
                }
                team_sync();
                // t = L^Q w + p ;  g += A^cl c
                for (int e = threadIdx.x; e < nx * nrhs; e += TEAM) {
                    const int i = e % nx, r = e / nx;
                    const T *wr = wv + r * nx;
                    T acc = pv[e];
                    for (int j = 0; j <= i; ++j) acc += LQ[i + j * nux] * wr[j];
                    tv[e] = acc;
                    if (c >= 1) {
                        const T *cr = cv + r * nx;
                        T g = T(0);
                        for (int k = 0; k < nx; ++k) g += Fs[i + k * nx] * cr[k];
                        gmu[e] += g;
                    }
                }
                team_sync();
                // h^_{s2} = h_{s2} + [B A]^T t
                for (int e = threadIdx.x; e < nux * nrhs; e += TEAM) {
                    const int aa = e % nux, r = e / nux;
                    const double *br = b + r * a.kkt;
                    const T *tr = tv + r * nx;
                    T acc = aa < nu ? -(T)br[(long long)s2 * w + aa]
                                    : -(T)br[(long long)(xq2 - 1) * w + nu + (aa - nu)];
                    for (int k = 0; k < nx; ++k) acc += BA[k + aa * nx] * tr[k];
                    hh[e] = acc;
                }
                team_sync();
            } else {
                // y = L^{Q-1} p ;  d_bwd = L^{Q-T} y ;  d_fwd = g - L^A y
                for (int r = threadIdx.x; r < nrhs; r += TEAM) {
                    const T *pr = pv + r * nx;
                    T *y = wv + r * nx, *db = tv + r * nx;
                    for (int i = 0; i < nx; ++i) {
                        T acc = pr[i];
                        for (int k = 0; k < i; ++k) acc = fma(-LQ[i + k * nux], y[k], acc);
                        y[i] = acc * DQ[i];
                    }
                    for (int i = nx - 1; i >= 0; --i) {
                        T acc = y[i];
                        for (int k = i + 1; k < nx; ++k) acc = fma(-LQ[k + i * nux], db[k], acc);
                        db[i] = acc * DQ[i];
                    }
                }
                team_sync();
                for (int e = threadIdx.x; e < nx * nrhs; e += TEAM) {
                    const int i = e % nx, r = e / nx;
                    T df = gmu[e];
                    if (c >= 1) {
                        const T *y = wv + r * nx;
                        for (int k = 0; k < nx; ++k) df -= Fs[i + k * nx] * y[k];
                    }
                    a.dF[r * a.nvec + in.oVec + (long long)c * nx + i] = (double)df;
                    a.dB[r * a.nvec + in.oVec + (long long)c * nx + i] = (double)tv[e];
                }
            }
            team_sync();
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
        T *Ls, *Ds, *BA, *Fs, *LB, *hh, *rho, *pv, *tv, *wv, *gmu, *cv, *xv;
        SolveSmem::carve<T>(smem_raw, nx, nu, nrhs, Ls, Ds, BA, Fs, LB, hh, rho, pv, tv, wv, gmu, cv, xv);
        const T *DIg = reinterpret_cast<const T *>(a.DI) + in.oDI;
        const T *DQ = Ds + nu;
        T *mu = gmu, *nuv = cv;   // coupling multipliers (reuse)
        const T *Lg = reinterpret_cast<const T *>(a.L) + in.oL;
        const T *LBg = reinterpret_cast<const T *>(a.LB) + in.oLB;
        const T *Fg = reinterpret_cast<const T *>(a.F) + in.oF;
        const double *b = a.b + in.oZ;
        double *z = a.z + in.oZ;
        double *zacc = a.zacc ? a.zacc + in.oZ : nullptr;
        const T *LQ = Ls + nu + nu * nux;

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
            load_T<T, TEAM>(Ls, Lg + (long long)s * nux * nux, nux * nux);
            load_T<T, TEAM>(Ds, DIg + (long long)s * nux, nux);
            if (hasG) load_T<T, TEAM>(LB, LBg + (long long)s * nx * nu, nx * nu);
            if (c >= 1) load_T<T, TEAM>(Fs, Fg + (long long)s * nx * nx, nx * nx);
            for (int e = threadIdx.x; e < nu * nrhs; e += TEAM) {
                const int i = e % nu, r = e / nu;
                rho[e] = (T)z[r * a.kkt + (long long)s * w + i];
            }
            for (int e = threadIdx.x; e < nx * nrhs; e += TEAM) {
                const int i = e % nx, r = e / nx;
                pv[e] = (T)z[r * a.kkt + (long long)(xq - 1) * w + nu + i];
            }
            team_sync();
            if (first) {
                // x^{j1} = -L^{Q-T} (L^{Q-1}(p - nu) + L^{A T} mu)
                for (int r = threadIdx.x; r < nrhs; r += TEAM) {
                    const T *pr = pv + r * nx, *nr = nuv + r * nx, *mr = mu + r * nx;
                    T *y = wv + r * nx, *x = xv + r * nx;
                    for (int i = 0; i < nx; ++i) {
                        T acc = pr[i] - nr[i];
                        for (int k = 0; k < i; ++k) acc = fma(-LQ[i + k * nux], y[k], acc);
                        y[i] = acc * DQ[i];
                    }
                    if (c >= 1)
                        for (int j = 0; j < nx; ++j) {
                            T acc = T(0);
                            for (int i = 0; i < nx; ++i) acc += Fs[i + j * nx] * mr[i];
                            y[j] += acc;
                        }
                    for (int i = nx - 1; i >= 0; --i) {
                        T acc = y[i];
                        for (int k = i + 1; k < nx; ++k) acc = fma(-LQ[k + i * nux], x[k], acc);
                        x[i] = acc * DQ[i];
                    }
                    for (int i = 0; i < nx; ++i) x[i] = -x[i];
                }
                team_sync();
            }
            // v = L^{S T} x + rho + L^{B T} mu  ->  hh[0..nu)
            for (int e = threadIdx.x; e < nu * nrhs; e += TEAM) {
                const int k = e % nu, r = e / nu;
                const T *x = xv + r * nx, *mr = mu + r * nx;
                T acc = rho[e];
                for (int i = 0; i < nx; ++i) acc += Ls[(nu + i) + k * nux] * x[i];
                if (hasG)
                    for (int i = 0; i < nx; ++i) acc += LB[i + k * nx] * mr[i];
                hh[r * nux + k] = acc;
            }
            // interior multiplier lambda^{s-1} = L^Q L^{Q T} x + p + A^{cl T} mu
            if (!first) {
                for (int e = threadIdx.x; e < nx * nrhs; e += TEAM) {
                    const int j = e % nx, r = e / nx;
                    const T *x = xv + r * nx;
                    T acc = T(0);
                    for (int k = j; k < nx; ++k) acc += LQ[k + j * nux] * x[k];
                    wv[e] = acc;
                }
            }
            team_sync();
            // u = -L^{R-T} v
            for (int r = threadIdx.x; r < nrhs; r += TEAM) {
                T *v = hh + r * nux, *u = rho + r * nu;
                for (int i = nu - 1; i >= 0; --i) {
                    T acc = v[i];
                    for (int k = i + 1; k < nu; ++k) acc = fma(-Ls[k + i * nux], u[k], acc);
                    u[i] = acc * Ds[i];
                }
                for (int i = 0; i < nu; ++i) u[i] = -u[i];
            }
            if (!first) {
                const int sp = (s - 1 + N) % N;
                for (int e = threadIdx.x; e < nx * nrhs; e += TEAM) {
                    const int i = e % nx, r = e / nx;
                    const T *wr = wv + r * nx, *mr = mu + r * nx;
                    T acc = pv[e];
                    for (int j = 0; j <= i; ++j) acc += LQ[i + j * nux] * wr[j];
                    if (c >= 1)
                        for (int k = 0; k < nx; ++k) acc += Fs[k + i * nx] * mr[k];
                    const long long o = r * a.kkt + (long long)sp * w + nu + nx + i;
                    if (zacc) zacc[o] += (double)acc; else z[o] = (double)acc;
                }
            }
            team_sync();
            for (int e = threadIdx.x; e < nu * nrhs; e += TEAM) {
                const int i = e % nu, r = e / nu;
                const long long o = r * a.kkt + (long long)s * w + i;
                if (zacc) zacc[o] += (double)rho[e]; else z[o] = (double)rho[e];
            }
            for (int e = threadIdx.x; e < nx * nrhs; e += TEAM) {
                const int i = e % nx, r = e / nx;
                const long long o = r * a.kkt + (long long)(xq - 1) * w + nu + i;
                if (zacc) zacc[o] += (double)xv[e]; else z[o] = (double)xv[e];
            }
            if (t > 0) {
                // x^{s+1} = A_s x + B_s u + c_s
                load_BA_T<T, TEAM>(BA, a.data, in, s);
                team_sync();
                for (int e = threadIdx.x; e < nx * nrhs; e += TEAM) {
                    const int i = e % nx, r = e / nx;
                    const T *x = xv + r * nx, *u = rho + r * nu;
                    T acc = -(T)b[r * a.kkt + (long long)s * w + nu + nx + i];
                    for (int k = 0; k < nu; ++k) acc += BA[i + k * nx] * u[k];
                    for (int k = 0; k < nx; ++k) acc += BA[i + (nu + k) * nx] * x[k];
                    tv[e] = acc;
                }
                team_sync();
                for (int e = threadIdx.x; e < nx * nrhs; e += TEAM) xv[e] = tv[e];
            }
            team_sync();
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
