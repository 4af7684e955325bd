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
// staged in shared memory; each lane owns rows of the constraint block (active
// flag, y^, and the row scaled by Sigma^J), then entries of the lower triangle
// of the Hessian blocks (sums over the compacted list of active rows, a loop
// that is uniform across the warp), then one gradient or residual row each, all
// rows written as one dot product over (u; x; y^) so that the lanes share a loop.
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
    // shared: V = [D C] (ny x nux, column-major), W = Sigma^J V, z = (u; x), y^, zeros
    double *V = sm, *W = V + (size_t)ny * nux, *z = W + (size_t)ny * nux, *yh = z + nux, *zr = yh + ny;
    int *act = reinterpret_cast<int *>(zr + ny);   // active rows, compacted
    const double *Ck = a.C + ao.oC + (long long)k * ny * nx;
    const double *Dk = hasu ? a.D + ao.oD + (long long)k * ny * nu : nullptr;
    for (int e = lane; e < ny * nux; e += 32) {
        const int i = e % ny, c = e / ny;
        V[e] = c < nu ? (hasu ? Dk[i + c * ny] : 0.0) : Ck[i + (c - nu) * ny];
    }
    const double *xk = k == 0 ? a.x0 + in.ox0 : a.x + in.oq + (long long)k * nx;
    for (int j = lane; j < nu; j += 32) z[j] = hasu ? a.u[in.orv + (long long)k * nu + j] : 0.0;
    for (int j = lane; j < nx; j += 32) z[nu + j] = xk[j];
    for (int i = lane; i < ny; i += 32) zr[i] = 0.0;
    __syncwarp();
    // constraint rows: w = C x + D u; the row is active where w + y / Sigma leaves
    // [bl, bu], i.e. (Sigma > 0) where Sigma w + y leaves [Sigma bl, Sigma bu]; then
    // y^ = y + Sigma (w - bound), and y^ = 0 on inactive rows (Pi is the identity there)
    const long long oy = ao.oY + (long long)k * ny;
    int n_act = 0;
    for (int i0 = 0; i0 < ny; i0 += 32) {
        const int i = i0 + lane;
        bool on = false;
        if (i < ny) {
            double cx = 0.0, du = 0.0;
            for (int j = 0; j < nx; ++j) cx = fma(V[i + (nu + j) * ny], z[nu + j], cx);
            for (int j = 0; j < nu; ++j) du = fma(V[i + j * ny], z[j], du);
            const double w = cx + du;
            const double y = a.y[oy + i], sg = a.sig[oy + i], bl = a.bl[oy + i], bu = a.bu[oy + i];
            const double t = fma(sg, w, y);
            const bool lo = t < sg * bl, hi = t > sg * bu;
            on = lo || hi;
            const double yhat = lo ? fma(sg, w - bl, y) : (hi ? fma(sg, w - bu, y) : 0.0);
            yh[i] = yhat;
            for (int c = 0; c < nux; ++c) W[i + c * ny] = on ? sg * V[i + c * ny] : 0.0;
            if (a.active) a.active[oy + i] = on ? 1 : 0;
            if (a.yhat) a.yhat[oy + i] = yhat;
        }
        const unsigned m = __ballot_sync(0xffffffffu, on);
        if (on) act[n_act + __popc(m & ((1u << lane) - 1u))] = i;
        n_act += __popc(m);
    }
    __syncwarp();
    const double *gx = a.gx ? a.gx + ao.ogx : nullptr, *gu = a.gu ? a.gu + ao.ogu : nullptr;
    // Hessian blocks: lower triangle of [R S; S^T Q] in the (u; x) numbering, R and Q mirrored
    const double *Qk = a.Q + in.oQ + (long long)k * nx * nx;
    double *Qo = a.Qo + in.oQ + (long long)k * nx * nx;
    const double *Rk = hasu ? a.R + in.oR + (long long)k * nu * nu : nullptr;
    double *Ro = hasu ? a.Ro + in.oR + (long long)k * nu * nu : nullptr;
    const double *Sk = (hasu && a.S) ? a.S + in.oS + (long long)k * nu * nx : nullptr;
    double *So = hasu ? a.So + in.oS + (long long)k * nu * nx : nullptr;
    // (the last stage has no u rows: only the Q block)
    const int ntri = hasu ? nux * (nux + 1) / 2 : nx * (nx + 1) / 2, shift = hasu ? 0 : nu;
    for (int e = lane; e < ntri; e += 32) {
        int p, q;
        tri_index(e, p, q);
        p += shift;
        q += shift;
        double acc = 0.0;
        for (int j = 0; j < n_act; ++j) {
            const int i = act[j];
            acc = fma(W[i + p * ny], V[i + q * ny], acc);
        }
        if (p < nu) {
            const double v = Rk[p + q * nu] + ((p == q && gu) ? gu[p] : 0.0) + acc;
            Ro[p + q * nu] = v;
            Ro[q + p * nu] = v;
        } else if (q < nu) {
            So[q + (p - nu) * nu] = (Sk ? Sk[q + (p - nu) * nu] : 0.0) + acc;
        } else {
            const int pp = p - nu, qq = q - nu;
            const double v = Qk[pp + qq * nx] + ((pp == qq && gx) ? gx[pp] : 0.0) + acc;
            Qo[pp + qq * nx] = v;
            Qo[qq + pp * nx] = v;
        }
    }
    // gradient and residual rows as one product [coefficients] . (u; x; y^) per row:
    //   r~_p: (R row p, S row p, D column p),  q~_p: (S column p, Q row p, C column p),
    //   c~_p: (B row p, A row p, 0)
    const int nr = hasu ? nu : 0, nc = hasu ? nx : 0, nout = nr + nx + nc;
    for (int o = lane; o < nout; o += 32) {
        const double *cu, *cx, *cy;
        int su, sx, sy;
        double add;
        double *dst;
        if (o < nr) {
            const int p = o;
            cu = Rk + p;
            su = nu;
            cx = Sk ? Sk + p : zr;
            sx = Sk ? nu : 0;
            cy = V + p * ny;
            sy = 1;
            add = a.r[in.orv + (long long)k * nu + p];
            if (gu) add = fma(gu[p], z[p] - a.ubar[in.orv + (long long)k * nu + p], add);
            dst = a.ro + in.orv + (long long)k * nu + p;
        } else if (o < nr + nx) {
            const int p = o - nr;
            cu = Sk ? Sk + p * nu : zr;
            su = Sk ? 1 : 0;
            cx = Qk + p;
            sx = nx;
            cy = V + (nu + p) * ny;
            sy = 1;
            add = a.q[in.oq + (long long)k * nx + p];
            if (gx) add = fma(gx[p], z[nu + p] - a.xbar[in.oq + (long long)k * nx + p], add);
            dst = a.qo + in.oq + (long long)k * nx + p;
        } else {
            const int p = o - nr - nx;
            cu = a.B + in.oB + (long long)k * nx * nu + p;
            su = nx;
            cx = a.A + in.oA + (long long)k * nx * nx + p;
            sx = nx;
            cy = zr;
            sy = 1;
            add = a.f[in.oc + (long long)k * nx + p] - a.x[in.oq + (long long)(k + 1) * nx + p];
            dst = a.co + in.oc + (long long)k * nx + p;
        }
        double g = 0.0;
        if (hasu)
            for (int j = 0; j < nu; ++j) g = fma(cu[j * su], z[j], g);
        for (int j = 0; j < nx; ++j) g = fma(cx[j * sx], z[nu + j], g);
        for (int i = 0; i < ny; ++i) g = fma(cy[i * sy], yh[i], g);
        *dst = g + add;
    }
}

}  // namespace

size_t newton_smem_bytes(int ny, int nx, int nu) {
    return (2 * (size_t)ny * (nx + nu) + (size_t)(nx + nu) + 2 * (size_t)ny) * sizeof(double) +
           (size_t)ny * sizeof(int);
}

cudaError_t launch_newton_assemble(const NewtonArgs &a, int batch, int max_stages, size_t smem, cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    cudaError_t e = ensure_smem((const void *)k_newton_assemble, smem);
    if (e != cudaSuccess) return e;
    k_newton_assemble<<<dim3(batch, max_stages), 32, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace cyq
