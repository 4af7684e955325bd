// Allocation-free factor + solve of one OCP (float64, one segment).
//
// Some callers cannot allocate device memory while they run: real-time
// control loops that allocate only at start-up, and hosts whose device memory
// belongs to another runtime or allocator.  This entry point serves them: its
// workspace (factor, coupling block, plan records) lives in one file-scope
// __device__ array of fixed size that every GPU loading the library holds
// until the process exits.  The caller passes inputs and outputs only.
//
// The array is shared by every call on a device and keeps the last call's
// contents.  Calls that overlap on the GPU (other streams, other host threads)
// race on it; serialise them.  The first call on a device looks up the
// array's device address (cudaGetSymbolAddress, with that device current) and
// keeps it for the life of the process, so a device reset after that first
// call is not supported.  The plan records are written by a one-thread
// kernel from its arguments, so nothing is copied from host memory.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "cyq.h"
#include "cyq_internal.cuh"

using namespace cyq;

namespace {

// 1 Mi doubles = 8 MiB of workspace.
constexpr long long kScratchDoubles = 1LL << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// Workspace layout (in doubles, each region rounded up to 32 doubles):
//   Inst record | Item record | instance index | status | L | LB | F | DI | Mf | Mb | Kc | U | Y | dF | dB | lam
inline long long round32(long long x) { return (x + 31) / 32 * 32; }

long long required_doubles(int N, int nx, int nu) {
    const long long nux = nx + nu;
    long long n = 0;
    n += round32((sizeof(Inst) + 7) / 8);
    n += round32((sizeof(Item) + 7) / 8);
    n += 32;                                  // instance index (int)
    n += 32;                                  // status (int)
    n += round32((long long)N * nux * nux);   // L
    n += round32((long long)N * nx * nu);     // LB
    n += round32((long long)N * nx * nx);     // F
    n += round32((long long)N * nux);         // DI
    n += 5 * round32((long long)nx * nx);     // Mf, Mb, Kc, U, Y
    n += 3 * round32(nx);                     // dF, dB, lam
    return n;
}

// The plan of a single instance with one segment, written on the device from
// kernel arguments (no host buffer is involved), and the status word cleared.
__global__ void k_noalloc_setup(Inst *inst, Item *item, int *list, int *status, int N, int nx, int nu) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    Inst in{};
    in.N = N;
    in.nx = nx;
    in.nu = nu;
    in.P = 1;
    *inst = in;
    *item = Item{0, 0};
    *list = 0;
    *status = 0;
}

int team_for(int nx, int nu) {
    const int nux = nx + nu;
    return nux <= 24 ? 32 : (nux <= 48 ? 64 : 128);
}

cyq_status fail(cyq_status s, const std::string &msg) {
    set_last_error_message(msg);   // readable through cyq_last_error()
    return s;
}

}  // namespace

extern "C" cyq_status cyq_factor_solve_noalloc(int32_t N, int32_t nx, int32_t nu, const double *Q, const double *R,
                                               const double *S, const double *A, const double *B,
                                               const double *Sigma, const double *b, double *z,
                                               int32_t *status_out, cyq_stream stream) {
    if (N < 1 || nx < 1 || nu < 1 || !Q || !R || !A || !B || !b || !z)
        return fail(CYQ_ERR_INVALID_ARG, "cyq_factor_solve_noalloc: bad size or NULL pointer");
    const long long need = required_doubles(N, nx, nu);
    if (need > kScratchDoubles)
        return fail(CYQ_ERR_INVALID_ARG,
                    "cyq_factor_solve_noalloc: problem needs " + std::to_string(need) +
                        " doubles of workspace, the fixed limit is " + std::to_string(kScratchDoubles));
    int smem_optin = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(CYQ_ERR_NO_DEVICE, "cyq_factor_solve_noalloc: no current CUDA device");
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const bool staged = factor_smem_bytes(true, nx, nu, true, false) <= (size_t)smem_optin / 2;
    const size_t fs = factor_smem_bytes(true, nx, nu, staged, false), ss1 = solve_smem_bytes(true, nx, nu, 1, 1);
    const int nbuf = solve_smem_bytes(true, nx, nu, 1, 2) <= (size_t)smem_optin ? 2 : 1;
    const size_t ss = solve_smem_bytes(true, nx, nu, 1, nbuf);
    if (fs > (size_t)smem_optin || ss1 > (size_t)smem_optin)
        return fail(CYQ_ERR_INVALID_ARG, "cyq_factor_solve_noalloc: stage blocks too large for shared memory");

    // per-device set-up: the device address of the workspace array
    double *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess)
                return fail(CYQ_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch_ptr[dev] = static_cast<double *>(p);
        }
        base = g_scratch_ptr[dev];
    }

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const long long nux = nx + nu;
    double *p = base;
    Inst *d_inst = reinterpret_cast<Inst *>(p);  p += round32((sizeof(Inst) + 7) / 8);
    Item *d_item = reinterpret_cast<Item *>(p);  p += round32((sizeof(Item) + 7) / 8);
    int *d_list = reinterpret_cast<int *>(p);    p += 32;
    int *d_status = reinterpret_cast<int *>(p);  p += 32;
    double *L = p;   p += round32((long long)N * nux * nux);
    double *LB = p;  p += round32((long long)N * nx * nu);
    double *F = p;   p += round32((long long)N * nx * nx);
    double *DI = p;  p += round32((long long)N * nux);
    double *Mf = p;  p += round32((long long)nx * nx);
    double *Mb = p;  p += round32((long long)nx * nx);
    double *Kc = p;  p += round32((long long)nx * nx);
    double *U = p;   p += round32((long long)nx * nx);
    double *Y = p;   p += round32((long long)nx * nx);
    double *dF = p;  p += round32(nx);
    double *dB = p;  p += round32(nx);
    double *lam = p; p += round32(nx);

    // plan records of a single instance with one segment, and a cleared status word
    cudaError_t e;
    k_noalloc_setup<<<1, 32, 0, st>>>(d_inst, d_item, d_list, d_status, N, nx, nu);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return fail(CYQ_ERR_CUDA, std::string("cyq_factor_solve_noalloc: ") + cudaGetErrorString(e));

    const int team = team_for(nx, nu);
    FactorArgs fa{};
    fa.inst = d_inst;
    fa.items = d_item;
    fa.n_items = 1;
    fa.data = Data{Q, R, S, A, B, Sigma};
    fa.L = L; fa.LB = LB; fa.F = F; fa.DI = DI;
    fa.Mf = Mf; fa.Mb = Mb; fa.Kc = Kc; fa.U = U; fa.Y = Y;
    fa.status = d_status;
    fa.stage_in_smem = staged;
    fa.need_G2 = false;
    fa.skip = nullptr;
    if ((e = launch_factor_segments(true, team, 0, fs, fa, st)) != cudaSuccess)
        return fail(CYQ_ERR_CUDA, std::string("cyq_factor_solve_noalloc: ") + cudaGetErrorString(e));

    SolveArgs sa{};
    sa.inst = d_inst;
    sa.items = d_item;
    sa.n_items = 1;
    sa.data = fa.data;
    sa.L = L; sa.LB = LB; sa.F = F; sa.DI = DI;
    sa.Mf = Mf; sa.Kc = Kc; sa.U = U; sa.Y = Y;
    sa.b = b;
    sa.z = z;
    sa.kkt = (long long)N * (nu + 2 * nx);
    sa.nrhs = 1;
    sa.dF = dF; sa.dB = dB; sa.lam = lam;
    sa.nvec = nx;
    sa.skip = nullptr;
    sa.nbuf = nbuf;
    if ((e = launch_solve_backward(true, team, 0, ss, sa, st)) != cudaSuccess ||
        (e = launch_cr_solve(1, d_list, 128, (size_t)2 * nx * sizeof(double), sa, st)) != cudaSuccess ||
        (e = launch_solve_forward(true, team, 0, ss, sa, st)) != cudaSuccess)
        return fail(CYQ_ERR_CUDA, std::string("cyq_factor_solve_noalloc: ") + cudaGetErrorString(e));
    if (status_out &&
        (e = cudaMemcpyAsync(status_out, d_status, sizeof(int), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return fail(CYQ_ERR_CUDA, std::string("cyq_factor_solve_noalloc: ") + cudaGetErrorString(e));
    return CYQ_OK;
}
