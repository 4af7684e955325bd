// Newton system of the augmented Lagrangian inner problem (paper Sec. 5,
// eqs. ocp-al-funcs, qpalm-ocp-hessians, newton-sys-with-x0, elim-x0).
//
// At the iterate (u, x) (x^0 = x_init), stage k's constraint rows
// w = C_k x^k + D_k u^k (no D term at k = N) are active where
// w + Sigma_k^{-1} y^k lies outside [bl, bu]; with Sigma^J = Sigma on the
// active rows and 0 elsewhere, and y^ = y + Sigma (w - Pi(w + Sigma^{-1} y)),
//   R~ = R + D^T Sigma^J D + Gamma_u^{-1},  S~ = S + D^T Sigma^J C,
//   Q~ = Q + C^T Sigma^J C + Gamma_x^{-1},
//   r~ = R u + S x + r + D^T y^ + Gamma_u^{-1} (u - ubar),
//   q~ = Q x + S^T u + q + C^T y^ + Gamma_x^{-1} (x - xbar)   (no S term at N),
//   c~ = B u + A x + f - x^{k+1}.
// The Newton step (du, dx, lambda) is the solution of the KKT system of
// (Q~, R~, S~, A, B) with right-hand side built from (q~, r~, c~) and a zero
// initial state.
//
// One warp per (instance, stage): the stage's [D C] rows and the iterate are
// staged in shared memory, each lane owns rows of the constraint block, then
// entries of the Hessian blocks (sums over the active rows only, a loop that
// is uniform across the warp), then entries of the gradient vectors.
#include "cyq_internal.cuh"

namespace cyq {

namespace {

__global__ void __launch_bounds__(32) k_newton_assemble(NewtonArgs a) {
    extern __shared__ __align__(16) double sm[];
    const int ii = blockIdx.x, k = blockIdx.y, lane = threadIdx.x;
    const Inst in = a.inst[ii];
    const AlmOff ao = a.off[ii];
    const int N = in.N, nx = in.nx, nu = in.nu, ny = ao.ny;
    if (k > N) return;
    const bool hasu = k < N;
    const int nux = nx + nu;
    // shared: V = [D C] (ny x nux, column-major), z = (u; x), y^, Sigma^J
    double *V = sm, *z = V + (size_t)ny * nux, *yh = z + nux, *sJ = yh + ny;
    const double *Ck = a.C + ao.oC + (long long)k * ny * nx;
    const double *Dk = hasu ? a.D + ao.oD + (long long)k * ny * nu : nullptr;
    for (int e = lane; e < ny * nux; e += 32) {
        const int i = e % ny, c = e / ny;
        V[e] = c < nu ? (hasu ? Dk[i + c * ny] : 0.0) : Ck[i + (c - nu) * ny];
    }
    const double *xk = k == 0 ? a.x0 + in.ox0 : a.x + in.oq + (long long)k * nx;
    for (int j = lane; j < nu; j += 32) z[j] = hasu ? a.u[in.orv + (long long)k * nu + j] : 0.0;
    for (int j = lane; j < nx; j += 32) z[nu + j] = xk[j];
    __syncwarp();
    // constraint rows: active set and multiplier estimate
    const long long oy = ao.oY + (long long)k * ny;
    for (int i = lane; i < ny; i += 32) {
        double cx = 0.0, du = 0.0;
        for (int j = 0; j < nx; ++j) cx = fma(V[i + (nu + j) * ny], z[nu + j], cx);
        for (int j = 0; j < nu; ++j) du = fma(V[i + j * ny], z[j], du);
        const double w = cx + du;
        const double y = a.y[oy + i], sg = a.sig[oy + i], bl = a.bl[oy + i], bu = a.bu[oy + i];
        const double zz = w + y / sg;
        const bool act = zz < bl || zz > bu;
        const double pr = fmin(fmax(zz, bl), bu);
        const double yhat = y + sg * (w - pr);
        yh[i] = yhat;
        sJ[i] = act ? sg : 0.0;
        if (a.active) a.active[oy + i] = act ? 1 : 0;
        if (a.yhat) a.yhat[oy + i] = yhat;
    }
    __syncwarp();
    const double *gx = a.gx ? a.gx + ao.ogx : nullptr, *gu = a.gu ? a.gu + ao.ogu : nullptr;
    // Hessian blocks: entry (p, q) of [R S; S^T Q] in the (u; x) numbering
    const double *Qk = a.Q + in.oQ + (long long)k * nx * nx;
    double *Qo = a.Qo + in.oQ + (long long)k * nx * nx;
    const int nR = hasu ? nu * nu : 0, nS = hasu ? nu * nx : 0, total = nR + nS + nx * nx;
    for (int e = lane; e < total; e += 32) {
        int p, q;
        double base;
        double *dst;
        if (e < nR) {
            p = e % nu;
            q = e / nu;
            base = a.R[in.oR + (long long)k * nu * nu + e] + ((p == q && gu) ? gu[p] : 0.0);
            dst = a.Ro + in.oR + (long long)k * nu * nu + e;
        } else if (e < nR + nS) {
            const int f = e - nR;
            p = f % nu;
            q = nu + f / nu;
            base = a.S ? a.S[in.oS + (long long)k * nu * nx + f] : 0.0;
            dst = a.So + in.oS + (long long)k * nu * nx + f;
        } else {
            const int f = e - nR - nS;
            p = nu + f % nx;
            q = nu + f / nx;
            base = Qk[f] + ((p == q && gx) ? gx[p - nu] : 0.0);
            dst = Qo + f;
        }
        double acc = 0.0;
        for (int i = 0; i < ny; ++i) {
            const double s = sJ[i];
            if (s != 0.0) acc = fma(s * V[i + p * ny], V[i + q * ny], acc);
        }
        *dst = base + acc;
    }
    // gradient rows
    if (hasu) {
        const double *Rk = a.R + in.oR + (long long)k * nu * nu;
        const double *Sk = a.S ? a.S + in.oS + (long long)k * nu * nx : nullptr;
        for (int p = lane; p < nu; p += 32) {
            double g = 0.0;
            for (int j = 0; j < nu; ++j) g = fma(Rk[p + j * nu], z[j], g);
            if (Sk)
                for (int j = 0; j < nx; ++j) g = fma(Sk[p + j * nu], z[nu + j], g);
            double cy = 0.0;
            for (int i = 0; i < ny; ++i) cy = fma(V[i + p * ny], yh[i], cy);
            g = g + a.r[in.orv + (long long)k * nu + p] + cy;
            if (gu) g = fma(gu[p], z[p] - a.ubar[in.orv + (long long)k * nu + p], g);
            a.ro[in.orv + (long long)k * nu + p] = g;
        }
    }
    {
        const double *Sk = (hasu && a.S) ? a.S + in.oS + (long long)k * nu * nx : nullptr;
        for (int p = lane; p < nx; p += 32) {
            double g = 0.0;
            for (int j = 0; j < nx; ++j) g = fma(Qk[p + j * nx], z[nu + j], g);
            if (Sk)
                for (int j = 0; j < nu; ++j) g = fma(Sk[j + p * nu], z[j], g);
            double cy = 0.0;
            for (int i = 0; i < ny; ++i) cy = fma(V[i + (nu + p) * ny], yh[i], cy);
            g = g + a.q[in.oq + (long long)k * nx + p] + cy;
            if (gx) g = fma(gx[p], z[nu + p] - a.xbar[in.oq + (long long)k * nx + p], g);
            a.qo[in.oq + (long long)k * nx + p] = g;
        }
    }
    // dynamics residual c~ = B u + A x + f - x^{k+1}
    if (hasu) {
        const double *Ak = a.A + in.oA + (long long)k * nx * nx, *Bk = a.B + in.oB + (long long)k * nx * nu;
        const double *xn = a.x + in.oq + (long long)(k + 1) * nx;
        for (int p = lane; p < nx; p += 32) {
            double g = 0.0;
            for (int j = 0; j < nu; ++j) g = fma(Bk[p + j * nx], z[j], g);
            for (int j = 0; j < nx; ++j) g = fma(Ak[p + j * nx], z[nu + j], g);
            a.co[in.oc + (long long)k * nx + p] = g + a.f[in.oc + (long long)k * nx + p] - xn[p];
        }
    }
}

}  // namespace

size_t newton_smem_bytes(int ny, int nx, int nu) {
    return ((size_t)ny * (nx + nu) + (size_t)(nx + nu) + 2 * (size_t)ny) * sizeof(double);
}

cudaError_t launch_newton_assemble(const NewtonArgs &a, int batch, int max_stages, size_t smem, cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    cudaError_t e = ensure_smem((const void *)k_newton_assemble, smem);
    if (e != cudaSuccess) return e;
    k_newton_assemble<<<dim3(batch, max_stages), 32, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace cyq
