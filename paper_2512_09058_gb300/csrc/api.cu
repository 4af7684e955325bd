// Host side of the cyq C ABI: planning (segments, teams, chunks), workspace
// allocation and the launch sequences of factor, solve, refinement and
// adjoint.  See include/cyq.h for the contract of every entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "cyq.h"
#include "cyq_internal.cuh"

using namespace cyq;

namespace {

thread_local std::string g_last_error;

// Streaming multiprocessors of a device (queried once per device).
int sm_count(int dev) {
    static std::mutex mu;
    static std::map<int, int> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    cache[dev] = n;
    return n;
}

struct Group {
    int cls = 0;
    int team = 32;
    bool need_G2 = false;                      // some item propagates A^cl (P > 1)
    bool staged[2] = {true, true};             // factor stages copied to shared memory, [float, double]
    size_t smem_factor[2] = {0, 0};
    int solve_nbuf[2] = {2, 2};                // solve stage packages in shared memory, [float, double]
    int team_factor[2] = {0, 0};               // tuned threads per item of the stage factor (0: heuristic)
    int team_solve[2] = {0, 0};                // tuned threads per item of the sweeps, for team_solve_nrhs
    int team_solve_nrhs = 0;
    int shape = -1;                            // kStageShapes index shared by all items (0: mixed / other)
    int max_nx = 0, max_nu = 0;
    std::vector<Item> items;
    Item *d_items = nullptr;
    // float32 factor: the items not covered by the persistent team launch
    std::vector<Item> items_rest;
    Item *d_items_rest = nullptr;
    bool rest_set = false;                     // items_rest replaces items in float32 factor launches
    bool warp_on = true;                       // (mirrors the handle's factor path)
};

struct FactorSet {
    void *L = nullptr, *LB = nullptr, *F = nullptr, *DI = nullptr;
    void *BA = nullptr;   // float32 [B A] copies (float32 sets only)
    float *Hf = nullptr;  // float32 stage matrices of the persistent team factor (float32 sets only)
    bool fp64 = true;
};

struct DevicePtrs {
    std::vector<void *> all;
    long long bytes = 0;
    template <typename T> cudaError_t alloc(T **p, size_t count) {
        *p = nullptr;
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
        if (e == cudaSuccess) {
            all.push_back((void *)*p);
            bytes += (long long)(count * sizeof(T));
        }
        return e;
    }
    void free_all() {
        for (void *p : all) cudaFree(p);
        all.clear();
        bytes = 0;
    }
};

}  // namespace

struct cyq_handle_s {
    // recompute mode: the batch is planned as consecutive chunks of instances (sub-handles)
    // that share one stage-factor window; every solve re-factors each chunk before its sweeps
    std::vector<cyq_handle_s *> subs;
    std::vector<int> sub_first;   // first instance of each chunk
    long long z_lo = 0, z_n = 0;  // elements of the KKT vector this handle's instances cover
    int device = 0;
    int batch = 0;
    int precision = CYQ_FP64;
    int max_nrhs = 1, it_max = 10, esc_max = 3;
    double tol = 1e-10;
    std::vector<Inst> inst;
    std::vector<Group> groups;
    std::vector<int> cr_list;     // instances with P > 1
    std::vector<CrJob> cr_jobs;
    CrPlan cr_plan;
    int cr_team = 128;
    std::vector<Chunk> chunks;
    long long kkt = 0, nL = 0, nLB = 0, nF = 0, nDI = 0, nblk = 0, nvec = 0;
    size_t crs_smem1 = 0;
    int max_nx = 0;
    int smem_optin = 0;
    int sms = 1;                  // streaming multiprocessors of the device
    // device
    DevicePtrs mem;
    Inst *d_inst = nullptr;
    int *d_cr_list = nullptr, *d_all_list = nullptr;
    // coupling solve: level-parallel over instances with P > 1 when they are few and have
    // many segments (cr_levels), single-CTA per instance otherwise / for P = 1 (p1_list)
    bool cr_levels = false;
    bool esc_possible = true;     // every size class has a float64 plan (float32 mode escalation)
    bool early_esc = false;       // float32 mode: predicted escalation after two corrections
    bool certify = false;         // stop only when the worst-case evaluation bound allows (k_certify)
    std::vector<int> p1_list;
    int *d_p1_list = nullptr;
    Chunk *d_chunks = nullptr;
    FactorSet fac;                // factor in the handle's precision
    FactorSet fac64;              // float64 factor for precision escalation (float32 mode only)
    // float32 mode: the escalation's float64 factor and corrections on a plan of its own with
    // more segments per long instance (the same instances, data, r, dz and status words), so
    // the float64 critical path of a long instance spreads over several SMs; null: fac64
    cyq_handle_s *esc_h = nullptr;
    FactorSet fac32;              // float32 copy of the float64 factor (float64 mode with float32 corrections)
    double *Mf = nullptr, *Mb = nullptr, *Kc = nullptr, *U = nullptr, *Y = nullptr;
    double *dF = nullptr, *dB = nullptr, *lam = nullptr;
    int *status = nullptr;
    double *r = nullptr, *dz = nullptr, *rr = nullptr, *bb = nullptr, *rel = nullptr;
    // certified stop: || |b| + |K||z| ||^2 accumulators and the certified value of the last stop
    double *aa = nullptr, *cert = nullptr;
    int *done = nullptr, *steps = nullptr;
    int *comp = nullptr;          // instances whose residual rows are evaluated compensated
    // early float64 escalation: residuals after the first solve, the instances to factor
    // now, and the side stream (with its fork / join events) that factors them
    double *rel0 = nullptr;
    int *esc = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    Data data{};
    bool factored = false;
    long long launches = 0;
    int last_nrhs = 0;
    // float32 factor, one team per item: items by class (longest first), the plan, the queue heads
    std::vector<Item> warp_items;
    TeamPlanDev team_plan;
    Item *d_warp_items = nullptr;
    int *d_warp_counter = nullptr;
    // float32 sweeps in one persistent launch each (all float32 items, by class)
    std::vector<Item> sweep_items;
    TeamPlanDev sweep_plan;
    Item *d_sweep_items = nullptr;
    int *d_sweep_counter = nullptr;
    int sweep_grid = 0;
    std::vector<IngestChunk> ingest_chunks;
    IngestChunk *d_ingest_chunks = nullptr;
    long long nHf = 0;            // floats of the ingested stage matrices
    size_t warp_arena = 0;
    int warp_grid = 0;
    bool warp_on = true;          // float32 factor path: one team per item in one launch (else per-class kernels)
    bool sweep_on = true;         // float32 sweeps: one persistent launch per sweep (else per-class kernels)
    // Newton-system assembly: constraint rows per instance and the offsets they imply
    std::vector<int> alm_ny;
    std::vector<AlmOff> alm_off;
    AlmOff *d_alm_off = nullptr;
    size_t alm_smem = 0;
};

namespace {

cyq_status fail_cuda(cudaError_t e, const char *where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return CYQ_ERR_CUDA;
}

#define CYQ_CUDA(call)                                           \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return fail_cuda(e_, #call);      \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (dev >= 0 && dev != prev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Update columns a stage of cyq_update_factor can carry (at least nx).
constexpr int kUpdateColumns = 32;

// Records per residual work item: small enough that the last refinement steps,
// with few instances left, still spread over many SMs (8 for one right-hand
// side: uneven batch step 192.5 ms with 32, 188.0 with 16, 184.3 with 8, 184.6
// with 4, where the full-batch residual itself slows from 8.4 to 8.9 ms; 32
// where several right-hand sides share every matrix load and the CTAs already
// carry more work).
constexpr int kResidChunk1 = 8, kResidChunkN = 32;
// Stages per warp of the float32 ingest and of the L^{R-1} pass: short runs keep many
// warps in flight on the memory-bound ingest and balance the uneven instances.
constexpr int kIngestChunk = 4;

int choose_team(int nx, int nu) {
    const int nux = nx + nu;
    if (nux <= 24) return 32;
    if (nux <= 48) return 64;
    return 128;
}

// Solve sweeps: enough threads for one pass over the (row, right-hand side)
// pairs of a stage block, up to 256.
int solve_team(int nux, int nrhs) {
    const int need = nux * nrhs;
    if (need <= 32) return 32;
    if (need <= 64) return 64;
    if (need <= 128) return 128;
    return 256;
}

int factor_team_of(const Group &g, bool fp64) {
    const int t = g.team_factor[fp64 ? 1 : 0];
    return t ? t : g.team;
}

int sweep_team_of(const Group &g, bool fp64, int nrhs) {
    const int t = g.team_solve[fp64 ? 1 : 0];
    return (t && g.team_solve_nrhs == nrhs) ? t : solve_team(g.max_nx + g.max_nu, nrhs);
}

// Size class of an instance: work items are launched per class so that the
// shared-memory carve-out and the team size match the blocks they hold.
int size_class(int nx, int nu) {
    static const int bounds[] = {8, 16, 24, 32, 48, 64, 80, 96, 128, 160, 192, 256};
    const int nux = nx + nu;
    for (int i = 0; i < (int)(sizeof(bounds) / sizeof(bounds[0])); ++i)
        if (nux <= bounds[i]) return i;
    return 99;
}

// Segments per instance: enough (instance, segment) work items to occupy the
// GPU when the batch is small, at least 8 stages per segment, a power of two.
int auto_segments(int batch, int N, int sms) {
    const int target = 2 * sms;
    if (batch >= target) return 1;
    const int want = (target + batch - 1) / batch;
    int P = 1;
    while (P < want) P <<= 1;
    while (P > 1 && N / P < 8) P >>= 1;
    return P;
}

cudaStream_t to_stream(cyq_stream s) { return reinterpret_cast<cudaStream_t>(s); }

SolveArgs solve_args(cyq_handle h, const FactorSet &fs, const Group &g, const double *b, double *z, int nrhs,
                     const int *skip, double *zacc = nullptr) {
    SolveArgs a{};
    a.inst = h->d_inst;
    a.items = g.d_items;
    a.n_items = (int)g.items.size();
    a.data = h->data;
    a.L = fs.L;
    a.LB = fs.LB;
    a.F = fs.F;
    a.DI = fs.DI;
    a.Mf = h->Mf;
    a.Kc = h->Kc;
    a.U = h->U;
    a.Y = h->Y;
    a.b = b;
    a.z = z;
    a.kkt = h->kkt;
    a.nrhs = nrhs;
    a.dF = h->dF;
    a.dB = h->dB;
    a.lam = h->lam;
    a.nvec = h->nvec;
    a.skip = skip;
    a.zacc = zacc;
    a.BA = fs.fp64 ? nullptr : fs.BA;
    a.nbuf = g.solve_nbuf[fs.fp64 ? 1 : 0];
    return a;
}

// One sweep (backward or forward) over the work items of one size class.
cudaError_t launch_group_sweep(cyq_handle h, const FactorSet &fs, const Group &g, bool backward, const double *b,
                               double *z, int nrhs, const int *skip, double *zacc, cudaStream_t st) {
    SolveArgs a = solve_args(h, fs, g, b, z, nrhs, skip, zacc);
    const size_t smem = solve_smem_bytes(fs.fp64, g.max_nx, g.max_nu, nrhs, a.nbuf);
    const int team = sweep_team_of(g, fs.fp64, nrhs);
    const int shape = g.shape > 0 ? g.shape : 0;
    return backward ? launch_solve_backward(fs.fp64, team, shape, smem, a, st)
                    : launch_solve_forward(fs.fp64, team, shape, smem, a, st);
}

// One solve with a stored factor (float64 or float32 arithmetic).  With
// zacc, the solution is added into zacc and z only holds sweep intermediates.
cyq_status run_solve(cyq_handle h, const FactorSet &fs, const double *b, double *z, int nrhs, const int *skip,
                     cudaStream_t st, double *zacc = nullptr) {
    // float32 sweeps: one persistent launch per sweep for the whole batch
    const bool team = !fs.fp64 && h->sweep_on && !h->sweep_items.empty();
    TeamPlanDev plan = h->sweep_plan;
    plan.items = h->d_sweep_items;
    plan.counter = h->d_sweep_counter;
    if (team) {
        SolveArgs a = solve_args(h, fs, h->groups[0], b, z, nrhs, skip, zacc);
        CYQ_CUDA(launch_sweep_team(true, a, plan, h->sweep_grid, st));
        ++h->launches;
    } else {
        for (const Group &g : h->groups) {
            CYQ_CUDA(launch_group_sweep(h, fs, g, true, b, z, nrhs, skip, zacc, st));
            ++h->launches;
        }
    }
    {
        SolveArgs a = solve_args(h, fs, h->groups[0], b, z, nrhs, skip, zacc);
        size_t smem = ((size_t)h->crs_smem1) * (nrhs + 1);
        if (h->cr_levels) {
            if (!h->p1_list.empty()) {
                CYQ_CUDA(launch_cr_solve((int)h->p1_list.size(), h->d_p1_list, 128, smem, a, st));
                ++h->launches;
            }
            CYQ_CUDA(launch_cr_solve_levels(h->cr_plan, h->max_nx, a, st, &h->launches));
        } else {
            CYQ_CUDA(launch_cr_solve(h->batch, h->d_all_list, 128, smem, a, st));
            ++h->launches;
        }
    }
    if (team) {
        SolveArgs a = solve_args(h, fs, h->groups[0], b, z, nrhs, skip, zacc);
        CYQ_CUDA(launch_sweep_team(false, a, plan, h->sweep_grid, st));
        ++h->launches;
    } else {
        for (const Group &g : h->groups) {
            CYQ_CUDA(launch_group_sweep(h, fs, g, false, b, z, nrhs, skip, zacc, st));
            ++h->launches;
        }
    }
    return CYQ_OK;
}

// Factor all instances (or those whose skip flag is zero) into a factor set,
// including the cyclic reduction of the coupling blocks (always float64).
FactorArgs factor_args(cyq_handle h, const FactorSet &fs, const int *skip) {
    FactorArgs a{};
    a.inst = h->d_inst;
    a.data = h->data;
    a.L = fs.L;
    a.LB = fs.LB;
    a.F = fs.F;
    a.DI = fs.DI;
    a.BAf = fs.fp64 ? nullptr : fs.BA;
    if (fs.fp64 && &fs == &h->fac && h->precision == CYQ_FP64_IR32) {
        // the float64 factorization also writes the float32 copy used by the corrections
        a.Lc = static_cast<float *>(h->fac32.L);
        a.LBc = static_cast<float *>(h->fac32.LB);
        a.Fc = static_cast<float *>(h->fac32.F);
        a.DIc = static_cast<float *>(h->fac32.DI);
        a.BAf = h->fac32.BA;
    }
    a.Mf = h->Mf;
    a.Mb = h->Mb;
    a.Kc = h->Kc;
    a.U = h->U;
    a.Y = h->Y;
    a.status = h->status;
    a.skip = skip;
    a.Hf = fs.Hf;
    return a;
}

// The stage factor over the work items of one size class.
cudaError_t launch_group_factor(const FactorSet &fs, const Group &g, FactorArgs a, cudaStream_t st) {
    const int pi = fs.fp64 ? 1 : 0;
    const bool rest = !fs.fp64 && g.rest_set && g.warp_on;
    a.items = rest ? g.d_items_rest : g.d_items;
    a.n_items = (int)(rest ? g.items_rest.size() : g.items.size());
    if (a.n_items == 0) return cudaSuccess;
    a.stage_in_smem = g.staged[pi];
    a.need_G2 = g.need_G2;
    return launch_factor_segments(fs.fp64, factor_team_of(g, fs.fp64), g.shape > 0 ? g.shape : 0, g.smem_factor[pi], a,
                                  st);
}

cyq_status run_factor(cyq_handle h, const FactorSet &fs, const int *skip, cudaStream_t st) {
    FactorArgs a = factor_args(h, fs, skip);
    if (!fs.fp64 && !h->warp_items.empty() && h->warp_on) {
        // every segment without A^cl of the batch in one persistent launch
        IngestArgs g{};
        g.inst = h->d_inst;
        g.chunks = h->d_ingest_chunks;
        g.n_chunks = (int)h->ingest_chunks.size();
        g.data = h->data;
        g.Hf = fs.Hf;
        g.BAf = static_cast<float *>(fs.BA);
        CYQ_CUDA(launch_ingest_f32(g, st));
        ++h->launches;
        TeamPlanDev plan = h->team_plan;
        plan.items = h->d_warp_items;
        plan.counter = h->d_warp_counter;
        CYQ_CUDA(launch_factor_team(a, plan, h->warp_grid, st));
        CYQ_CUDA(launch_inv_R_f32(g, static_cast<float *>(fs.L), static_cast<const float *>(fs.DI), st));
        h->launches += 2;
    }
    for (const Group &g : h->groups) {
        if (!fs.fp64 && g.rest_set && g.warp_on && g.items_rest.empty()) continue;
        CYQ_CUDA(launch_group_factor(fs, g, a, st));
        ++h->launches;
    }
    if (!h->cr_list.empty()) CYQ_CUDA(launch_cr_factor_levels(h->cr_plan, h->cr_team, h->max_nx, a, st, &h->launches));
    return CYQ_OK;
}

ResidArgs resid_args(cyq_handle h, const double *b, const double *z, double *r, const int *skip,
                     bool need_bb = true) {
    ResidArgs a{};
    a.need_bb = need_bb;
    a.max_nx = h->max_nx;
    a.inst = h->d_inst;
    a.chunks = h->d_chunks;
    a.n_chunks = (int)h->chunks.size();
    a.data = h->data;
    a.b = b;
    a.z = z;
    a.r = r;
    a.rr = h->rr;
    a.bb = h->bb;
    a.skip = skip;
    a.kkt = h->kkt;
    a.batch = h->batch;
    return a;
}

// The float64 factorization of the instances with skip[i] == 0 for the precision
// escalation (a failed float32 pivot is cleared first): on the escalation plan
// (more segments per long instance) or fac64.
cyq_status run_escalation_factor(cyq_handle h, const int *skip, cudaStream_t st) {
    CYQ_CUDA(launch_clear_not_pd(h->batch, skip, h->status, st));
    ++h->launches;
    if (!h->esc_h) return run_factor(h, h->fac64, skip, st);
    cyq_handle e = h->esc_h;
    e->data = h->data;
    const long long l0 = e->launches;
    const cyq_status s = run_factor(e, e->fac, skip, st);
    h->launches += e->launches - l0;
    return s;
}

// Solve + float64 iterative refinement on all right-hand sides at once:
//   z = K~^{-1} b;  repeat: r = b - K z (float64), stop per instance once
//   every ||r|| / ||b|| plus twice the rounding bound of its evaluation is
//   <= tol (certified stop, k_certify), else z += K~^{-1} r
// where K~ is the stored factor (float32 or float64).  All decisions are taken
// on the device (per-instance flags), so the sequence can be graph-captured.
cyq_status run_refined_solve(cyq_handle h, const double *b, double *z, int nrhs, cudaStream_t st) {
    const int B = h->batch;
    CYQ_CUDA(cudaMemsetAsync(h->done, 0, sizeof(int) * B, st));
    CYQ_CUDA(cudaMemsetAsync(h->comp, 0, sizeof(int) * B, st));
    CYQ_CUDA(cudaMemsetAsync(h->steps, 0, sizeof(int) * B, st));
    CYQ_CUDA(cudaMemsetAsync(h->rr, 0, sizeof(double) * B * h->max_nrhs, st));
    CYQ_CUDA(cudaMemsetAsync(h->bb, 0, sizeof(double) * B * h->max_nrhs, st));
    CYQ_CUDA(cudaMemsetAsync(h->aa, 0, sizeof(double) * B * h->max_nrhs, st));
    CYQ_CUDA(cudaMemsetAsync(h->cert, 0, sizeof(double) * B * h->max_nrhs, st));
    cyq_status s = run_solve(h, h->fac, b, z, nrhs, nullptr, st);
    if (s != CYQ_OK) return s;
    // corrections: with the handle's factor, or with its float32 copy (CYQ_FP64_IR32)
    const FactorSet &corr = h->precision == CYQ_FP64_IR32 ? h->fac32 : h->fac;
    int step = 0;
    // residual of every instance still refining; with certify, the ones at or below tol
    // (done = 3) evaluate || |b| + |K||z| || and stop only if the certified value is at or
    // below tol too
    auto evaluate = [&](bool first) -> cudaError_t {
        cudaError_t e;
        ResidArgs ra = resid_args(h, b, z, h->r, h->done, first);
        ra.comp = h->comp;
        if ((e = launch_residual(ra, nrhs, st)) ||
            (e = launch_resid_finalize(B, nrhs, h->rr, h->bb, h->rel, h->done, h->tol, h->steps, step, true,
                                       h->certify ? 3 : 1, h->comp, st)))
            return e;
        h->launches += 3;
        if (!h->certify) return cudaSuccess;
        ResidArgs sa = resid_args(h, b, z, nullptr, h->done, false);
        sa.rr = h->aa;
        sa.run_if = 3;
        if ((e = launch_residual_scale(sa, nrhs, st)) ||
            (e = launch_certify(h->d_inst, B, nrhs, h->aa, h->bb, h->rel, h->cert, h->done, h->tol, st)))
            return e;
        h->launches += 2;
        return cudaSuccess;
    };
    // float32 mode: after kPredict corrections, the instances whose residual contracts too
    // slowly to reach tol in the remaining ones are parked, and their float64 factorization
    // starts on the side stream while the float32 corrections of the others continue
    constexpr int kPredict = 2;
    const bool early = h->early_esc && !h->fac.fp64 && h->esc_max > 0 && h->esc_possible && h->side &&
                       h->it_max > kPredict + 1;
    bool forked = false;
    for (int it = 0; it <= h->it_max; ++it, ++step) {
        // ||b||^2 once (first residual); later steps reuse it
        CYQ_CUDA(evaluate(it == 0));
        if (it == h->it_max) break;
        if (early && it == 0)
            CYQ_CUDA(cudaMemcpyAsync(h->rel0, h->rel, sizeof(double) * B * nrhs, cudaMemcpyDeviceToDevice, st));
        if (early && it == kPredict) {
            CYQ_CUDA(launch_predict_escalation(B, nrhs, h->rel0, h->rel, h->done, h->esc, h->tol, kPredict,
                                               h->it_max - kPredict, st));
            CYQ_CUDA(cudaEventRecord(h->ev_fork, st));
            CYQ_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
            s = run_escalation_factor(h, h->esc, h->side);
            if (s != CYQ_OK) return s;
            CYQ_CUDA(cudaEventRecord(h->ev_join, h->side));
            h->launches += 1;
            forked = true;
        }
        // correction: z += K~^{-1} r for the instances still above tol
        s = run_solve(h, corr, h->r, h->dz, nrhs, h->done, st, z);
        if (s != CYQ_OK) return s;
    }
    if (forked) CYQ_CUDA(cudaStreamWaitEvent(st, h->ev_join, 0));
    if (!corr.fp64 && h->esc_max > 0 && h->esc_possible) {
        // precision escalation: instances the float32 corrections could not bring to
        // tol continue with float64 corrections (float32 mode: after a float64 factorization;
        // the parked instances have theirs already, the others still above tol get it now)
        const bool refactor = !h->fac.fp64;
        if (refactor) {
            s = run_escalation_factor(h, h->done, st);
            if (s != CYQ_OK) return s;
        }
        if (forked) {
            CYQ_CUDA(launch_unpark(B, h->done, st));
            ++h->launches;
        }
        cyq_handle ph = refactor && h->esc_h ? h->esc_h : h;   // the plan of the float64 factor
        const FactorSet &f64 = refactor ? (h->esc_h ? h->esc_h->fac : h->fac64) : h->fac;
        for (int it = 0; it < h->esc_max; ++it) {
            ++step;
            const long long l0 = ph->launches;
            s = run_solve(ph, f64, h->r, h->dz, nrhs, h->done, st, z);
            if (s != CYQ_OK) return s;
            if (ph != h) h->launches += ph->launches - l0;
            CYQ_CUDA(evaluate(false));
        }
    }
    CYQ_CUDA(launch_mark_not_converged(B, h->done, h->status, st));
    ++h->launches;
    h->last_nrhs = nrhs;
    return CYQ_OK;
}

}  // namespace

extern "C" {

const char *cyq_status_string(cyq_status s) {
    switch (s) {
        case CYQ_OK: return "ok";
        case CYQ_ERR_INVALID_ARG: return "invalid argument";
        case CYQ_ERR_NOT_PD: return "matrix not positive definite";
        case CYQ_ERR_NOT_CONVERGED: return "refinement did not converge";
        case CYQ_ERR_CUDA: return "CUDA error";
        case CYQ_ERR_TIMEOUT: return "device wait timed out";
        case CYQ_ERR_NO_FACTOR: return "no factorization";
        case CYQ_ERR_UNIMPLEMENTED: return "unimplemented";
        case CYQ_ERR_NO_DEVICE: return "no CUDA device";
        case CYQ_ERR_UPDATE_RANK: return "update rank above the workspace";
    }
    return "unknown status";
}

const char *cyq_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace {

// Options of a chunk of a recompute-mode handle: the offsets of its first
// instance in the whole batch's data and vectors, the whole batch's KKT size,
// shared refinement vectors, and no stage-factor allocation of its own.
struct CreateOpts {
    bool chunk = false;
    Inst base{};
    long long kkt_full = 0;
    double *r = nullptr, *dz = nullptr;   // shared refinement vectors (chunks, escalation plan)
    int *status = nullptr;                // shared status words (escalation plan)
};

// Segments of an instance in the float64 escalation plan: halved stage runs of at
// least 12 stages, at most 16 segments.
int escalation_segments(int N) {
    int P = 1;
    while (P < 16 && N / (2 * P) >= 12) P *= 2;
    return P;
}

cyq_status create_impl(const cyq_desc *desc, const CreateOpts &o, cyq_handle *out) {
    if (!desc || !out) return CYQ_ERR_INVALID_ARG;
    *out = nullptr;
    if (desc->batch < 1 || !desc->N || !desc->nx || !desc->nu) return CYQ_ERR_INVALID_ARG;
    if (desc->precision != CYQ_FP64 && desc->precision != CYQ_FP32_REFINE && desc->precision != CYQ_FP64_IR32)
        return CYQ_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        g_last_error = "no CUDA device";
        return CYQ_ERR_NO_DEVICE;
    }
    int dev = desc->device;
    if (dev < 0) cudaGetDevice(&dev);
    if (dev >= ndev) return CYQ_ERR_INVALID_ARG;
    DeviceGuard guard(dev);
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int sms = sm_count(dev);

    cyq_handle h = new cyq_handle_s();
    h->sms = sms;
    h->device = dev;
    h->batch = desc->batch;
    h->precision = desc->precision;
    h->max_nrhs = desc->max_nrhs > 0 ? desc->max_nrhs : 1;
    h->it_max = desc->it_max >= 0 ? desc->it_max : 10;
    h->esc_max = desc->esc_max >= 0 ? desc->esc_max : 3;
    h->tol = desc->tol > 0 ? desc->tol : 1e-10;
    h->early_esc = desc->early_escalation != 0;
    h->certify = desc->certify != 0;
    h->smem_optin = smem_optin;
    // float64 factorization (CYQ_FP64, CYQ_FP64_IR32); float32 plans for the sweeps unless CYQ_FP64
    const bool fp64 = h->precision != CYQ_FP32_REFINE;
    const bool float_sweeps = h->precision != CYQ_FP64;

    long long oQ = 0, oR = 0, oS = 0, oA = 0, oB = 0, oSig = 0, oZ = 0, oL = 0, oLB = 0, oF = 0, oDI = 0, oBA = 0, oBlk = 0,
              oVec = 0, oq = 0, orv = 0, oc = 0, ox0 = 0, oNs = 0, oNn = 0;
    std::vector<Item> all_items;
    int item = 0;
    for (int i = 0; i < desc->batch; ++i) {
        const int N = desc->N[i], nx = desc->nx[i], nu = desc->nu[i];
        if (N < 1 || nx < 1 || nu < 1) { delete h; return CYQ_ERR_INVALID_ARG; }
        int P = desc->P_per_instance ? desc->P_per_instance[i] : desc->P;
        if (P <= 0) P = auto_segments(desc->batch, N, sms);
        if (P > N) P = N;
        Inst in{};
        in.N = N; in.nx = nx; in.nu = nu; in.P = P; in.item0 = item;
        in.oQ = oQ; in.oR = oR; in.oS = oS; in.oA = oA; in.oB = oB; in.oSig = oSig; in.oZ = oZ;
        in.oL = oL; in.oLB = oLB; in.oF = oF; in.oDI = oDI; in.oBA = oBA; in.oBlk = oBlk; in.oVec = oVec;
        in.oq = oq; in.orv = orv; in.oc = oc; in.ox0 = ox0;
        in.oN = oNs; in.oNn = oNn;
        if (o.chunk) {   // data and vectors of the whole batch
            in.oQ += o.base.oQ; in.oR += o.base.oR; in.oS += o.base.oS; in.oA += o.base.oA; in.oB += o.base.oB;
            in.oSig += o.base.oSig; in.oZ += o.base.oZ;
            in.oq += o.base.oq; in.orv += o.base.orv; in.oc += o.base.oc; in.ox0 += o.base.ox0;
        }
        const long long nux = nx + nu;
        oQ += (long long)(N + 1) * nx * nx; oR += (long long)N * nu * nu; oS += (long long)N * nu * nx;
        oA += (long long)N * nx * nx; oB += (long long)N * nx * nu; oSig += (long long)(N + 1) * (nu + nx);
        oZ += (long long)N * (nu + 2 * nx);
        oL += (long long)N * nux * nux; oLB += (long long)N * nx * nu; oF += (long long)N * nx * nx;
        oDI += (long long)N * nux;
        oBA += (long long)N * nx * nux;
        oBlk += (long long)P * nx * nx; oVec += (long long)P * nx;
        oq += (long long)(N + 1) * nx; orv += (long long)N * nu; oc += (long long)N * nx; ox0 += nx;
        oNs += N; oNn += (long long)N * nux;
        h->inst.push_back(in);
        if (P > 1) h->cr_list.push_back(i);
        else h->p1_list.push_back(i);
        // work items and their team class
        const int team = choose_team(nx, nu);
        const int cls = size_class(nx, nu);
        Group *g = nullptr;
        for (Group &gg : h->groups)
            if (gg.cls == cls) g = &gg;
        if (!g) {
            h->groups.emplace_back();
            g = &h->groups.back();
            g->cls = cls;
            g->team = team;
        }
        g->team = std::max(g->team, team);
        {
            const int sh = stage_shape_index(nx, nu);
            g->shape = g->shape < 0 ? sh : (g->shape == sh ? sh : 0);
        }
        g->max_nx = std::max(g->max_nx, nx);
        g->max_nu = std::max(g->max_nu, nu);
        for (int c = 0; c < P; ++c) g->items.push_back(Item{i, c});
        item += P;
        // residual chunks of up to kResidChunk1 / kResidChunkN records
        const int rchunk = h->max_nrhs > 1 ? kResidChunkN : kResidChunk1;
        for (int k0 = 0; k0 < N; k0 += rchunk) h->chunks.push_back(Chunk{i, k0, std::min(N, k0 + rchunk)});
        h->max_nx = std::max(h->max_nx, nx);
        h->crs_smem1 = std::max(h->crs_smem1, (size_t)P * nx * sizeof(double));
    }
    // longest items first inside a class (work ~ segment length x (nx+nu)^3)
    for (Group &g : h->groups) {
        auto cost = [&](const Item &it) {
            const Inst &in = h->inst[it.inst];
            const double nux = in.nx + in.nu;
            return (double)seg_len(it.seg, in.N, in.P) * nux * nux * nux;
        };
        std::stable_sort(g.items.begin(), g.items.end(),
                         [&](const Item &x, const Item &y) { return cost(x) > cost(y); });
    }
    for (Group &g : h->groups) {
        for (const Item &it : g.items) g.need_G2 |= it.seg >= 1;
        for (int pi = 0; pi < 2; ++pi) {
            const bool f64 = pi == 1;
            if (!f64 && !float_sweeps) continue;   // float32 plans only where float32 sweeps run
            // stage the raw blocks in shared memory while two CTAs still fit on an SM
            g.staged[pi] = factor_smem_bytes(f64, g.max_nx, g.max_nu, true, g.need_G2) <= (size_t)smem_optin / 2;
            g.smem_factor[pi] = factor_smem_bytes(f64, g.max_nx, g.max_nu, g.staged[pi], g.need_G2);
            // solve: a ring of up to 4 stage packages (prefetch depth 3) within the shared
            // memory one CTA may take while all of the class's items stay resident
            {
                const long long per_sm = std::max<long long>(1, ((long long)g.items.size() + sms - 1) / sms);
                const size_t budget = std::max<size_t>(48 * 1024, (size_t)228 * 1024 / per_sm);
                int nb = 1;
                for (int cand = 4; cand >= 2; --cand) {
                    const size_t need = solve_smem_bytes(f64, g.max_nx, g.max_nu, h->max_nrhs, cand);
                    if (need <= (size_t)smem_optin && need <= budget) {
                        nb = cand;
                        break;
                    }
                }
                g.solve_nbuf[pi] = nb;
            }
            const bool fits = g.smem_factor[pi] <= (size_t)smem_optin &&
                              solve_smem_bytes(f64, g.max_nx, g.max_nu, h->max_nrhs, g.solve_nbuf[pi]) <=
                                  (size_t)smem_optin;
            if (!fits && f64 && h->precision == CYQ_FP32_REFINE) {
                h->esc_possible = false;   // float32 mode: only the float64 escalation needs this plan
                continue;
            }
            if (!fits) {
                delete h;
                g_last_error = "stage blocks too large for shared memory";
                return CYQ_ERR_INVALID_ARG;
            }
        }
    }
    if (h->crs_smem1 * (h->max_nrhs + 1) > (size_t)smem_optin) { delete h; return CYQ_ERR_INVALID_ARG; }
    if (float_sweeps) {
        // float32 sweeps: every item by the smallest shared memory its packages need
        // (one package, no prefetch), longest first, in the arena classes of the one-team
        // factor; used only when every item fits
        int smem_sm = 0;
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        const size_t part = (size_t)smem_sm / kSweepCtasPerSm;
        const size_t arena = std::min<size_t>((size_t)smem_optin, part > 1536 ? (part - 1536) / 64 * 64 : 0);
        const int arena_floats = (int)(arena / 64 * 16);
        const size_t slot2 = (size_t)(arena_floats / 4) * 4, slot1 = (size_t)(arena_floats / 2) * 4,
                     slot0 = (size_t)arena_floats * 4;
        struct Cand { Item it; double cost; int cls; };
        std::vector<Cand> cand;
        bool all = true;
        for (const Group &g : h->groups)
            for (const Item &it : g.items) {
                const Inst &in = h->inst[it.inst];
                const size_t b = solve_smem_bytes(false, in.nx, in.nu, h->max_nrhs, 1);
                if (b > slot0) all = false;
                const double nux = in.nx + in.nu;
                cand.push_back(Cand{it, seg_len(it.seg, in.N, in.P) * (nux * nux + in.nx * nux),
                                    b <= slot2 ? 2 : (b <= slot1 ? 1 : 0)});
            }
        if (all) {
            std::stable_sort(cand.begin(), cand.end(), [](const Cand &x, const Cand &y) { return x.cost > y.cost; });
            TeamPlanDev &tp = h->sweep_plan;
            double work[3] = {0.0, 0.0, 0.0};
            int off = 0;
            for (int k = 0; k < 3; ++k) {
                tp.off[k] = off;
                for (const Cand &c : cand)
                    if (c.cls == k) {
                        h->sweep_items.push_back(c.it);
                        work[k] += c.cost;
                        ++off;
                    }
                tp.n[k] = off - tp.off[k];
            }
            tp.arena_floats = arena_floats;
            const int grid = kSweepCtasPerSm * sms;
            const double wsum = work[0] + work[1] + work[2];
            int gg[3] = {0, 0, 0};
            for (int k = 0; k < 2; ++k) {
                if (tp.n[k] == 0) continue;
                const int teams = k == 0 ? 1 : 2;
                gg[k] = std::max(1, (int)std::lround(grid * work[k] / std::max(wsum, 1.0)));
                gg[k] = std::min(gg[k], (tp.n[k] + teams - 1) / teams);
            }
            gg[2] = tp.n[2] > 0 ? std::max(1, grid - gg[0] - gg[1]) : 0;
            tp.g0 = gg[0];
            tp.g1 = gg[1];
            h->sweep_grid = gg[0] + gg[1] + gg[2];
        }
    }
    if (h->precision == CYQ_FP32_REFINE) {
        // float32 factor: segments without A^cl (segment 0) whose padded blocks fit
        // three rows per lane go to the one-team-per-item launch, longest first,
        // packed into CTA arenas (kFactorCtasPerSm CTAs per SM)
        int smem_sm = 0;
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        // each CTA takes its arena, its static shared memory and the 1 KB the system
        // reserves per CTA
        const size_t part = (size_t)smem_sm / kFactorCtasPerSm;
        const size_t arena = std::min<size_t>((size_t)smem_optin, part > 1536 ? (part - 1536) / 64 * 64 : 0);
        struct Cand { Item it; double cost; size_t bytes; int np; };
        std::vector<Cand> cand;
        for (Group &g : h->groups) {
            g.rest_set = true;
            g.items_rest.clear();
            for (const Item &it : g.items) {
                const Inst &in = h->inst[it.inst];
                const int nup = (in.nu + 3) & ~3, nxp = (in.nx + 3) & ~3;
                const size_t bytes = warp_slot_bytes(in.nx, in.nu);
                if (it.seg == 0 && nup + nxp <= kWarpMaxNp && nxp <= kWarpMaxNxp && nup <= 32 && bytes <= arena) {
                    const double np = nup + nxp;
                    const double per = np * np * np / 6.0 + 0.5 * np * np * nxp + 0.5 * np * nxp * nxp;
                    cand.push_back(Cand{it, seg_len(it.seg, in.N, in.P) * per, bytes, nup + nxp});
                } else {
                    g.items_rest.push_back(it);
                }
            }
        }
        std::stable_sort(cand.begin(), cand.end(), [](const Cand &x, const Cand &y) { return x.cost > y.cost; });
        // classes by the slot an item needs: four per CTA arena (teams of 32), two (64), one (128)
        const int arena_floats = (int)(arena / 64 * 16);   // every team slot a multiple of 16 bytes
        const size_t slot2 = (size_t)(arena_floats / 4) / 4 * 16, slot1 = (size_t)(arena_floats / 2) / 4 * 16;
        std::vector<Item> cls[3];
        double work[3] = {0.0, 0.0, 0.0};
        for (const Cand &c : cand) {
            int k = c.bytes <= slot2 ? 2 : (c.bytes <= slot1 ? 1 : 0);
            while (k > 0 && c.np > kTeamRows[k]) --k;   // the class's team must cover every row
            cls[k].push_back(c.it);
            work[k] += c.cost;
        }
        TeamPlanDev &tp = h->team_plan;
        int off = 0;
        for (int k = 0; k < 3; ++k) {
            tp.off[k] = off;
            tp.n[k] = (int)cls[k].size();
            off += tp.n[k];
            for (const Item &it : cls[k]) h->warp_items.push_back(it);
        }
        tp.arena_floats = arena_floats;
        // CTAs per configuration in proportion to the class's work (every CTA has four warps);
        // teams that run out of items continue with the smaller classes
        const int grid = kFactorCtasPerSm * sms;
        const double wsum = work[0] + work[1] + work[2];
        int g[3] = {0, 0, 0};
        for (int k = 0; k < 2; ++k) {
            if (tp.n[k] == 0) continue;
            const int teams = k == 0 ? 1 : 2;
            g[k] = std::max(1, (int)std::lround(grid * work[k] / std::max(wsum, 1.0)));
            g[k] = std::min(g[k], (tp.n[k] + teams - 1) / teams);
        }
        g[2] = tp.n[2] > 0 ? std::max(1, grid - g[0] - g[1]) : 0;
        tp.g0 = g[0];
        tp.g1 = g[1];
        // float32 stage matrices of the covered segments (stage s of instance i at oHf + s np^2)
        long long oHf = 0;
        for (const Item &it : h->warp_items) {
            Inst &in = h->inst[it.inst];
            in.oHf = oHf;
            oHf += (long long)in.N * (long long)warp_stage_floats(in.nx, in.nu);
            const int len = seg_len(it.seg, in.N, in.P);
            for (int t0 = 0; t0 < len; t0 += kIngestChunk)
                h->ingest_chunks.push_back(IngestChunk{it.inst, t0, std::min(len, t0 + kIngestChunk)});
        }
        h->nHf = oHf;
        h->warp_arena = arena;
        h->warp_grid = g[0] + g[1] + g[2];
    }
    // level-parallel cyclic-reduction jobs
    {
        int maxP = 1;
        for (int i : h->cr_list) maxP = std::max(maxP, h->inst[i].P);
        int levels = 0;
        while ((1 << levels) < maxP) ++levels;
        CrPlan &cp = h->cr_plan;
        cp.levels = levels;
        for (int l = 0; l < levels; ++l) {
            const int st = 1 << l;
            cp.elim_off[l] = (int)h->cr_jobs.size();
            for (int i : h->cr_list)
                for (int k = st; k < h->inst[i].P; k += 2 * st) h->cr_jobs.push_back(CrJob{i, k});
        }
        cp.elim_off[levels] = (int)h->cr_jobs.size();
        for (int l = 0; l < levels; ++l) {
            const int st = 1 << l;
            cp.upd_off[l] = (int)h->cr_jobs.size();
            for (int i : h->cr_list)
                for (int k = 0; k < h->inst[i].P; k += 2 * st) h->cr_jobs.push_back(CrJob{i, k});
        }
        cp.upd_off[levels] = (int)h->cr_jobs.size();
        cp.n_inst = (int)h->cr_list.size();
        h->cr_team = h->max_nx <= 8 ? 32 : 128;
        if ((size_t)4 * h->max_nx * h->max_nx * 8 > (size_t)smem_optin) {
            delete h;
            g_last_error = "state dimension too large for the coupling blocks";
            return CYQ_ERR_INVALID_ARG;
        }
    }
    h->kkt = o.chunk ? o.kkt_full : oZ; h->nL = oL; h->nLB = oLB; h->nF = oF; h->nDI = oDI; h->nblk = oBlk; h->nvec = oVec;
    h->z_lo = o.chunk ? o.base.oZ : 0;
    h->z_n = oZ;

    auto fail = [&](cudaError_t e, const char *what) {
        cyq_status s = fail_cuda(e, what);
        h->mem.free_all();
        delete h;
        return s;
    };
#define ALLOC(ptr, count)                                      \
    do {                                                       \
        cudaError_t e_ = h->mem.alloc(&(ptr), (count));        \
        if (e_ != cudaSuccess) return fail(e_, "cudaMalloc");  \
    } while (0)
    ALLOC(h->d_inst, h->inst.size());
    ALLOC(h->d_chunks, h->chunks.size());
    ALLOC(h->d_cr_list, h->cr_list.size());
    {
        CrJob *pj;
        ALLOC(pj, h->cr_jobs.size());
        h->cr_plan.jobs = pj;
    }
    ALLOC(h->d_all_list, (size_t)h->batch);
    ALLOC(h->d_p1_list, h->p1_list.size());
    {
        int maxP = 0;
        for (int i : h->cr_list) maxP = std::max(maxP, h->inst[i].P);
        h->cr_levels = !h->cr_list.empty() && (int)h->cr_list.size() < 2 * sms && maxP >= 8;
    }
    for (Group &g : h->groups) ALLOC(g.d_items, g.items.size());
    for (Group &g : h->groups)
        if (g.rest_set) ALLOC(g.d_items_rest, g.items_rest.size());
    if (!h->sweep_items.empty()) {
        ALLOC(h->d_sweep_items, h->sweep_items.size());
        ALLOC(h->d_sweep_counter, 3);
    }
    if (!h->warp_items.empty()) {
        ALLOC(h->d_warp_items, h->warp_items.size());
        ALLOC(h->d_warp_counter, 3);
        ALLOC(h->d_ingest_chunks, h->ingest_chunks.size());
        if (!o.chunk) ALLOC(h->fac.Hf, (size_t)h->nHf);
    }
    // float32 mode: a float64 escalation plan of its own where some instance gets more
    // segments there (then no fac64 here; created at the end, fac64 again if that fails)
    bool want_esc = false;
    if (h->precision == CYQ_FP32_REFINE && !o.chunk && h->esc_max > 0)
        for (const Inst &in : h->inst) want_esc |= escalation_segments(in.N) > in.P;
    // fac (the handle's factor) and, in float32 mode, fac64 (escalation), in float64
    // mode with float32 corrections, fac32 (float32 copy)
    for (int pass = 0; pass < (float_sweeps ? 2 : 1); ++pass) {
        FactorSet &fs = pass == 0 ? h->fac : (fp64 ? h->fac32 : h->fac64);
        fs.fp64 = pass == 0 ? fp64 : !fp64;
        const size_t el = fs.fp64 ? sizeof(double) : sizeof(float);
        if (o.chunk) continue;   // the chunk's stage factors live in the shared window
        if (want_esc && &fs == &h->fac64) continue;
        char *p;
        ALLOC(p, (size_t)oL * el); fs.L = p;
        ALLOC(p, (size_t)oLB * el); fs.LB = p;
        ALLOC(p, (size_t)oF * el); fs.F = p;
        ALLOC(p, (size_t)oDI * el); fs.DI = p;
        if (!fs.fp64) { ALLOC(p, (size_t)oBA * el); fs.BA = p; }
    }
    ALLOC(h->Mf, (size_t)oBlk);
    ALLOC(h->Mb, (size_t)oBlk);
    ALLOC(h->Kc, (size_t)oBlk);
    ALLOC(h->U, (size_t)oBlk);
    ALLOC(h->Y, (size_t)oBlk);
    ALLOC(h->dF, (size_t)oVec * h->max_nrhs);
    ALLOC(h->dB, (size_t)oVec * h->max_nrhs);
    ALLOC(h->lam, (size_t)oVec * h->max_nrhs);
    if (o.status) h->status = o.status;
    else ALLOC(h->status, (size_t)h->batch);
    if (o.r) {
        h->r = o.r;
        h->dz = o.dz;
    } else {
        ALLOC(h->r, (size_t)oZ * h->max_nrhs);
        ALLOC(h->dz, (size_t)oZ * h->max_nrhs);
    }
    ALLOC(h->rr, (size_t)h->batch * h->max_nrhs);
    ALLOC(h->bb, (size_t)h->batch * h->max_nrhs);
    ALLOC(h->rel, (size_t)h->batch * h->max_nrhs);
    ALLOC(h->aa, (size_t)h->batch * h->max_nrhs);
    ALLOC(h->cert, (size_t)h->batch * h->max_nrhs);
    ALLOC(h->done, (size_t)h->batch);
    ALLOC(h->comp, (size_t)h->batch);
    ALLOC(h->steps, (size_t)h->batch);
    if (h->precision == CYQ_FP32_REFINE) {
        ALLOC(h->rel0, (size_t)h->batch * h->max_nrhs);
        ALLOC(h->esc, (size_t)h->batch);
    }
#undef ALLOC
    {
        // default paths (cyq_autotune times both): the persistent launches where the batch has
        // several size classes or stage blocks wider than the compiled register kernels
        int max_nux = 0;
        for (const Inst &in : h->inst) max_nux = std::max(max_nux, in.nx + in.nu);
        const bool persistent = h->groups.size() > 1 || max_nux > 24;
        h->warp_on = h->sweep_on = persistent;
        for (Group &g : h->groups) g.warp_on = persistent;
    }
    std::vector<int> all(h->batch);
    for (int i = 0; i < h->batch; ++i) all[i] = i;
    cudaError_t e;
    if ((e = cudaMemcpy(h->d_inst, h->inst.data(), sizeof(Inst) * h->inst.size(), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(h->d_chunks, h->chunks.data(), sizeof(Chunk) * h->chunks.size(), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(h->d_all_list, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice)) ||
        (!h->p1_list.empty() && (e = cudaMemcpy(h->d_p1_list, h->p1_list.data(), sizeof(int) * h->p1_list.size(),
                                                cudaMemcpyHostToDevice))) ||
        (e = cudaMemset(h->status, 0, sizeof(int) * h->batch)) ||
        (e = cudaMemset(h->rr, 0, sizeof(double) * h->batch * h->max_nrhs)) ||
        (e = cudaMemset(h->bb, 0, sizeof(double) * h->batch * h->max_nrhs)) ||
        (e = cudaMemset(h->rel, 0, sizeof(double) * h->batch * h->max_nrhs)) ||
        (e = cudaMemset(h->aa, 0, sizeof(double) * h->batch * h->max_nrhs)) ||
        (e = cudaMemset(h->cert, 0, sizeof(double) * h->batch * h->max_nrhs)) ||
        (e = cudaMemset(h->steps, 0, sizeof(int) * h->batch)))
        return fail(e, "cudaMemcpy");
    if (!h->cr_list.empty() &&
        ((e = cudaMemcpy(h->d_cr_list, h->cr_list.data(), sizeof(int) * h->cr_list.size(), cudaMemcpyHostToDevice)) ||
         (e = cudaMemcpy((void *)h->cr_plan.jobs, h->cr_jobs.data(), sizeof(CrJob) * h->cr_jobs.size(),
                         cudaMemcpyHostToDevice))))
        return fail(e, "cudaMemcpy");
    h->cr_plan.inst_list = h->d_cr_list;
    for (Group &g : h->groups)
        if ((e = cudaMemcpy(g.d_items, g.items.data(), sizeof(Item) * g.items.size(), cudaMemcpyHostToDevice)))
            return fail(e, "cudaMemcpy");
    if (h->precision == CYQ_FP32_REFINE &&
        ((e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking)) ||
         (e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming)) ||
         (e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming))))
        return fail(e, "cudaStreamCreate");
    for (Group &g : h->groups)
        if (g.rest_set && !g.items_rest.empty() &&
            (e = cudaMemcpy(g.d_items_rest, g.items_rest.data(), sizeof(Item) * g.items_rest.size(),
                            cudaMemcpyHostToDevice)))
            return fail(e, "cudaMemcpy");
    if (!h->sweep_items.empty() &&
        (e = cudaMemcpy(h->d_sweep_items, h->sweep_items.data(), sizeof(Item) * h->sweep_items.size(),
                        cudaMemcpyHostToDevice)))
        return fail(e, "cudaMemcpy");
    if (!h->warp_items.empty() &&
        ((e = cudaMemcpy(h->d_warp_items, h->warp_items.data(), sizeof(Item) * h->warp_items.size(),
                         cudaMemcpyHostToDevice)) ||
         (e = cudaMemcpy(h->d_ingest_chunks, h->ingest_chunks.data(), sizeof(IngestChunk) * h->ingest_chunks.size(),
                         cudaMemcpyHostToDevice))))
        return fail(e, "cudaMemcpy");
    if (want_esc) {
        // more segments only where the float64 stage blocks with the A^cl propagation still
        // fit in shared memory: the widest instances first lose them until the plan is made
        cyq_handle eh = nullptr;
        std::vector<int32_t> Pe(h->batch);
        for (int cap = 128; cap >= 16 && !eh; cap -= 16) {
            bool any = false;
            for (int i = 0; i < h->batch; ++i) {
                const Inst &in = h->inst[i];
                Pe[i] = in.nx + in.nu <= cap ? std::max(in.P, escalation_segments(in.N)) : in.P;
                any |= Pe[i] > in.P;
            }
            if (!any) break;
            cyq_desc d = *desc;
            d.precision = CYQ_FP64;
            d.P = 0;
            d.P_per_instance = Pe.data();
            d.it_max = 0;
            d.esc_max = 0;
            d.recompute_factors = 0;
            d.early_escalation = 0;
            d.certify = 0;
            CreateOpts eo;
            eo.r = h->r;
            eo.dz = h->dz;
            eo.status = h->status;
            if (create_impl(&d, eo, &eh) != CYQ_OK) eh = nullptr;
        }
        if (eh) {
            h->esc_h = eh;
            h->esc_possible = true;
        } else {   // the escalation on the handle's own plan
            FactorSet &fs = h->fac64;
            char *p[4] = {nullptr, nullptr, nullptr, nullptr};
            const long long n[4] = {oL, oLB, oF, oDI};
            for (int k = 0; k < 4; ++k)
                if ((e = h->mem.alloc(&p[k], (size_t)n[k] * 8)) != cudaSuccess) return fail(e, "cudaMalloc");
            fs.L = p[0];
            fs.LB = p[1];
            fs.F = p[2];
            fs.DI = p[3];
        }
    }
    *out = h;
    return CYQ_OK;
}

}  // namespace

extern "C" {

cyq_status cyq_create(const cyq_desc *desc, cyq_handle *out) {
    if (!desc || !out) return CYQ_ERR_INVALID_ARG;
    if (!desc->recompute_factors) return create_impl(desc, CreateOpts{}, out);
    *out = nullptr;
    if (desc->batch < 1 || !desc->N || !desc->nx || !desc->nu) return CYQ_ERR_INVALID_ARG;
    const int B = desc->batch;
    const int K = std::max(1, std::min(B, desc->recompute_chunks > 0 ? desc->recompute_chunks : 4));
    // chunks of consecutive instances with about equal stage-factor storage
    std::vector<long long> fsz(B);
    long long tot = 0;
    for (int i = 0; i < B; ++i) {
        if (desc->N[i] < 1 || desc->nx[i] < 1 || desc->nu[i] < 1) return CYQ_ERR_INVALID_ARG;
        const long long nux = desc->nx[i] + desc->nu[i];
        fsz[i] = (long long)desc->N[i] * (nux * nux + nux + desc->nx[i] * nux);
        tot += fsz[i];
    }
    std::vector<int> first;
    long long acc = 0;
    for (int i = 0; i < B; ++i) {
        if (first.empty() || (acc * K >= tot * (long long)first.size() && (int)first.size() < K)) first.push_back(i);
        acc += fsz[i];
    }
    cyq_handle h = new cyq_handle_s();
    h->batch = B;
    h->precision = desc->precision;
    h->max_nrhs = desc->max_nrhs > 0 ? desc->max_nrhs : 1;
    h->it_max = desc->it_max >= 0 ? desc->it_max : 10;
    h->device = desc->device;
    if (h->device < 0) cudaGetDevice(&h->device);
    DeviceGuard guard(h->device);
    // offsets of every instance in the whole batch (the layout of include/cyq.h)
    std::vector<Inst> base(B);
    {
        Inst c{};
        for (int i = 0; i < B; ++i) {
            base[i] = c;
            const long long N = desc->N[i], nx = desc->nx[i], nu = desc->nu[i];
            c.oQ += (N + 1) * nx * nx; c.oR += N * nu * nu; c.oS += N * nu * nx; c.oA += N * nx * nx;
            c.oB += N * nx * nu; c.oSig += (N + 1) * (nu + nx); c.oZ += N * (nu + 2 * nx);
            c.oq += (N + 1) * nx; c.orv += N * nu; c.oc += N * nx; c.ox0 += nx;
        }
        h->kkt = c.oZ;
    }
    h->z_n = h->kkt;
    auto fail = [&](cyq_status st) {
        for (cyq_handle sh : h->subs) cyq_destroy(sh);
        h->mem.free_all();
        delete h;
        return st;
    };
    if (h->mem.alloc(&h->r, (size_t)h->kkt * h->max_nrhs) != cudaSuccess ||
        h->mem.alloc(&h->dz, (size_t)h->kkt * h->max_nrhs) != cudaSuccess)
        return fail(fail_cuda(cudaGetLastError(), "cudaMalloc"));
    for (size_t k = 0; k < first.size(); ++k) {
        const int i0 = first[k], i1 = k + 1 < first.size() ? first[k + 1] : B;
        cyq_desc d = *desc;
        d.batch = i1 - i0;
        d.N = desc->N + i0;
        d.nx = desc->nx + i0;
        d.nu = desc->nu + i0;
        d.P_per_instance = desc->P_per_instance ? desc->P_per_instance + i0 : nullptr;
        d.recompute_factors = 0;
        CreateOpts o;
        o.chunk = true;
        o.base = base[i0];
        o.kkt_full = h->kkt;
        o.r = h->r;
        o.dz = h->dz;
        cyq_handle sh = nullptr;
        const cyq_status st = create_impl(&d, o, &sh);
        if (st != CYQ_OK) return fail(st);
        h->subs.push_back(sh);
        h->sub_first.push_back(i0);
    }
    // the shared window: the largest chunk's stage factors of each factor set
    FactorSet *sets[3] = {&h->fac, &h->fac64, &h->fac32};
    for (int si = 0; si < 3; ++si) {
        long long nL = 0, nLB = 0, nF = 0, nDI = 0, nBA = 0, nHf = 0;
        bool used = false, fp64 = true;
        for (cyq_handle sh : h->subs) {
            FactorSet *ss[3] = {&sh->fac, &sh->fac64, &sh->fac32};
            const bool present = si == 0 || (si == 1 && sh->precision == CYQ_FP32_REFINE) ||
                                 (si == 2 && sh->precision == CYQ_FP64_IR32);
            if (!present) continue;
            used = true;
            fp64 = ss[si]->fp64;
            nL = std::max(nL, sh->nL); nLB = std::max(nLB, sh->nLB); nF = std::max(nF, sh->nF);
            nDI = std::max(nDI, sh->nDI);
            long long ba = 0;
            for (const Inst &in : sh->inst) ba += (long long)in.N * in.nx * (in.nx + in.nu);
            nBA = std::max(nBA, ba);
            if (si == 0) nHf = std::max(nHf, sh->nHf);
        }
        if (!used) continue;
        FactorSet &fs = *sets[si];
        fs.fp64 = fp64;
        const size_t el = fp64 ? 8 : 4;
        char *p;
        if (h->mem.alloc(&p, (size_t)nL * el) != cudaSuccess) return fail(fail_cuda(cudaGetLastError(), "cudaMalloc"));
        fs.L = p;
        if (h->mem.alloc(&p, (size_t)nLB * el) != cudaSuccess) return fail(fail_cuda(cudaGetLastError(), "cudaMalloc"));
        fs.LB = p;
        if (h->mem.alloc(&p, (size_t)nF * el) != cudaSuccess) return fail(fail_cuda(cudaGetLastError(), "cudaMalloc"));
        fs.F = p;
        if (h->mem.alloc(&p, (size_t)nDI * el) != cudaSuccess) return fail(fail_cuda(cudaGetLastError(), "cudaMalloc"));
        fs.DI = p;
        if (!fp64) {
            if (h->mem.alloc(&p, (size_t)nBA * el) != cudaSuccess)
                return fail(fail_cuda(cudaGetLastError(), "cudaMalloc"));
            fs.BA = p;
        }
        if (si == 0 && nHf > 0) {
            if (h->mem.alloc(&fs.Hf, (size_t)nHf) != cudaSuccess) return fail(fail_cuda(cudaGetLastError(), "cudaMalloc"));
        }
        for (cyq_handle sh : h->subs) {
            FactorSet *ss[3] = {&sh->fac, &sh->fac64, &sh->fac32};
            const bool present = si == 0 || (si == 1 && sh->precision == CYQ_FP32_REFINE) ||
                                 (si == 2 && sh->precision == CYQ_FP64_IR32);
            if (!present) continue;
            ss[si]->L = fs.L; ss[si]->LB = fs.LB; ss[si]->F = fs.F; ss[si]->DI = fs.DI; ss[si]->BA = fs.BA;
            if (si == 0) ss[si]->Hf = fs.Hf;
        }
    }
    *out = h;
    return CYQ_OK;
}

void cyq_destroy(cyq_handle h) {
    if (!h) return;
    DeviceGuard guard(h->device);
    cudaDeviceSynchronize();
    for (cyq_handle sh : h->subs) cyq_destroy(sh);
    if (h->esc_h) cyq_destroy(h->esc_h);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    h->mem.free_all();
    delete h;
}

int64_t cyq_kkt_size(cyq_handle h) { return h ? h->kkt : -1; }

cyq_status cyq_get_stage_factor(cyq_handle h, int32_t instance, int32_t stage, double *L_out) {
    if (!h || !L_out || instance < 0 || instance >= h->batch) return CYQ_ERR_INVALID_ARG;
    if (!h->subs.empty()) return CYQ_ERR_UNIMPLEMENTED;   // not offered for recompute-mode handles
    if (!h->factored) return CYQ_ERR_NO_FACTOR;
    const Inst &in = h->inst[instance];
    if (stage < 0 || stage >= in.N) return CYQ_ERR_INVALID_ARG;
    DeviceGuard guard(h->device);
    const size_t nux = (size_t)in.nx + in.nu, n = nux * nux;
    const long long off = in.oL + (long long)stage * (long long)n;
    CYQ_CUDA(cudaDeviceSynchronize());
    if (h->fac.fp64) {
        CYQ_CUDA(cudaMemcpy(L_out, static_cast<const double *>(h->fac.L) + off, n * sizeof(double),
                            cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> tmp(n);
        CYQ_CUDA(cudaMemcpy(tmp.data(), static_cast<const float *>(h->fac.L) + off, n * sizeof(float),
                            cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; ++i) L_out[i] = tmp[i];
    }
    return CYQ_OK;
}

cyq_status cyq_get_segments(cyq_handle h, int32_t *P_out) {
    if (!h || !P_out) return CYQ_ERR_INVALID_ARG;
    if (!h->subs.empty()) {
        for (size_t k = 0; k < h->subs.size(); ++k) cyq_get_segments(h->subs[k], P_out + h->sub_first[k]);
        return CYQ_OK;
    }
    for (int i = 0; i < h->batch; ++i) P_out[i] = h->inst[i].P;
    return CYQ_OK;
}

cyq_status cyq_segment_stages(int32_t N, int32_t P, int32_t c, int32_t *stages, int32_t *len) {
    if (N < 1 || P < 1 || P > N || c < 0 || c >= P || !len) return CYQ_ERR_INVALID_ARG;
    *len = seg_len(c, N, P);
    if (stages)
        for (int t = 0; t < *len; ++t) stages[t] = seg_stage(c, t, N, P);
    return CYQ_OK;
}

int64_t cyq_last_launch_count(cyq_handle h) { return h ? h->launches : -1; }

cyq_status cyq_factor(cyq_handle h, const double *Q, const double *R, const double *S, const double *A,
                      const double *B, const double *Sigma, cyq_stream stream) {
    if (!h || !Q || !R || !A || !B) return CYQ_ERR_INVALID_ARG;
    if (!h->subs.empty()) {
        // every chunk in turn through the shared window: statuses and coupling factors remain
        h->launches = 0;
        for (cyq_handle sh : h->subs) {
            const cyq_status st = cyq_factor(sh, Q, R, S, A, B, Sigma, stream);
            if (st != CYQ_OK) return st;
            h->launches += sh->launches;
        }
        h->data = Data{Q, R, S, A, B, Sigma};
        h->factored = true;
        return CYQ_OK;
    }
    DeviceGuard guard(h->device);
    cudaStream_t st = to_stream(stream);
    h->launches = 0;
    h->data = Data{Q, R, S, A, B, Sigma};
    CYQ_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int) * h->batch, st));
    cyq_status s = run_factor(h, h->fac, nullptr, st);
    if (s != CYQ_OK) return s;
    h->factored = true;
    return CYQ_OK;
}

cyq_status cyq_solve(cyq_handle h, const double *b, double *z, int32_t nrhs, cyq_stream stream) {
    if (!h || !b || !z || nrhs < 1 || nrhs > h->max_nrhs) return CYQ_ERR_INVALID_ARG;
    if (!h->factored) return CYQ_ERR_NO_FACTOR;
    if (!h->subs.empty()) {
        // recompute mode: each chunk's stage factors again, then its solve
        h->launches = 0;
        for (cyq_handle sh : h->subs) {
            DeviceGuard guard(sh->device);
            cyq_status st = run_factor(sh, sh->fac, nullptr, to_stream(stream));
            if (st != CYQ_OK) return st;
            h->launches += sh->launches;
            st = cyq_solve(sh, b, z, nrhs, stream);
            if (st != CYQ_OK) return st;
            h->launches += sh->launches;
        }
        return CYQ_OK;
    }
    DeviceGuard guard(h->device);
    cudaStream_t st = to_stream(stream);
    h->launches = 0;
    if (h->it_max == 0) {
        h->last_nrhs = 0;
        return run_solve(h, h->fac, b, z, nrhs, nullptr, st);
    }
    return run_refined_solve(h, b, z, nrhs, st);
}

cyq_status cyq_apply_factor(cyq_handle h, const double *r, double *dz, int32_t nrhs, cyq_stream stream) {
    if (!h || !r || !dz || nrhs < 1 || nrhs > h->max_nrhs) return CYQ_ERR_INVALID_ARG;
    if (!h->subs.empty()) return CYQ_ERR_UNIMPLEMENTED;   // not offered for recompute-mode handles
    if (!h->factored) return CYQ_ERR_NO_FACTOR;
    DeviceGuard guard(h->device);
    h->launches = 0;
    // the factor the refinement corrections use: the float32 copy in CYQ_FP64_IR32 mode
    const FactorSet &fs = h->precision == CYQ_FP64_IR32 ? h->fac32 : h->fac;
    return run_solve(h, fs, r, dz, nrhs, nullptr, to_stream(stream));
}

cyq_status cyq_update_factor(cyq_handle h, const double *Q, const double *R, const double *S, const double *w,
                             const double *delta, int32_t m_max, cyq_stream stream) {
    if (!h || !Q || !R || !w || !delta || m_max < 1) return CYQ_ERR_INVALID_ARG;
    if (!h->subs.empty()) return CYQ_ERR_UNIMPLEMENTED;   // not offered for recompute-mode handles
    if (!h->factored) return CYQ_ERR_NO_FACTOR;
    if (!h->cr_list.empty()) {
        set_last_error_message("cyq_update_factor: instances with more than one segment are not supported");
        return CYQ_ERR_UNIMPLEMENTED;
    }
    DeviceGuard guard(h->device);
    cudaStream_t st = to_stream(stream);
    int max_nu = 0;
    for (const Inst &in : h->inst) max_nu = std::max(max_nu, in.nu);
    UpdateArgs u{};
    u.inst = h->d_inst;
    u.inst_list = h->d_all_list;
    u.n_inst = h->batch;
    u.data = h->data;
    u.L = h->fac.L;
    u.LB = h->fac.LB;
    u.DI = h->fac.DI;
    if (h->precision == CYQ_FP64_IR32) {
        u.Lc = static_cast<float *>(h->fac32.L);
        u.LBc = static_cast<float *>(h->fac32.LB);
        u.DIc = static_cast<float *>(h->fac32.DI);
    }
    u.Mf = h->Mf;
    u.Mb = h->Mb;
    u.w = w;
    u.delta = delta;
    u.m_max = m_max;
    u.mcap = std::max(h->max_nx, kUpdateColumns);
    u.max_nx = h->max_nx;
    u.max_nu = max_nu;
    u.status = h->status;
    const size_t smem = h->fac.fp64 ? update_smem_bytes<double>(h->max_nx, max_nu, u.mcap)
                                    : update_smem_bytes<float>(h->max_nx, max_nu, u.mcap);
    if (smem > (size_t)h->smem_optin) {
        set_last_error_message("cyq_update_factor: stage blocks too large for the update workspace");
        return CYQ_ERR_INVALID_ARG;
    }
    CYQ_CUDA(launch_update_factor(h->fac.fp64, u, st));
    h->launches = 1;
    // the residual and the refinement read the updated matrices from now on
    h->data.Q = Q;
    h->data.R = R;
    h->data.S = S;
    return CYQ_OK;
}

cyq_status cyq_build_rhs(cyq_handle h, const double *q, const double *r, const double *c, const double *x_init,
                         double *b, cyq_stream stream) {
    if (!h || !q || !r || !c || !x_init || !b) return CYQ_ERR_INVALID_ARG;
    if (!h->factored) return CYQ_ERR_NO_FACTOR;
    DeviceGuard guard(h->device);
    if (!h->subs.empty()) {
        for (cyq_handle sh : h->subs) {
            const cyq_status st = cyq_build_rhs(sh, q, r, c, x_init, b, stream);
            if (st != CYQ_OK) return st;
        }
        return CYQ_OK;
    }
    CYQ_CUDA(launch_build_rhs(h->d_inst, h->batch, h->data, q, r, c, x_init, b, h->z_lo, h->z_n, to_stream(stream)));
    return CYQ_OK;
}

cyq_status cyq_set_pcr_tail(cyq_handle h, int32_t levels) {
    if (!h || levels < 0) return CYQ_ERR_INVALID_ARG;
    if (!h->subs.empty()) return CYQ_ERR_UNIMPLEMENTED;   // not offered for recompute-mode handles
    if (h->cr_list.empty()) return CYQ_OK;   // no instance has more than one segment
    DeviceGuard guard(h->device);
    CYQ_CUDA(cudaDeviceSynchronize());   // the old plan may still be in use
    int maxP = 1;
    for (int i : h->cr_list) maxP = std::max(maxP, h->inst[i].P);
    int total = 0;
    while ((1 << total) < maxP) ++total;
    const int T = std::min<int>(levels, total), L0 = total - T, s0 = 1 << L0;
    std::vector<CrJob> jobs;
    CrPlan cp = h->cr_plan;
    cp.levels = L0;
    for (int l = 0; l < L0; ++l) {
        const int st = 1 << l;
        cp.elim_off[l] = (int)jobs.size();
        for (int i : h->cr_list)
            for (int k = st; k < h->inst[i].P; k += 2 * st) jobs.push_back(CrJob{i, k});
    }
    cp.elim_off[L0] = (int)jobs.size();
    for (int l = 0; l < L0; ++l) {
        const int st = 1 << l;
        cp.upd_off[l] = (int)jobs.size();
        for (int i : h->cr_list)
            for (int k = 0; k < h->inst[i].P; k += 2 * st) jobs.push_back(CrJob{i, k});
    }
    cp.upd_off[L0] = (int)jobs.size();
    cp.tail = T;
    cp.s0 = s0;
    std::vector<long long> oT(h->batch, 0), oV(h->batch, 0);
    long long nT = 0, nV = 0;
    for (int i : h->cr_list) {
        const int v = (h->inst[i].P + s0 - 1) / s0, nx = h->inst[i].nx;
        oT[i] = nT;
        oV[i] = nV;
        nT += (long long)v * T * nx * nx;
        nV += (long long)v * nx;
    }
    for (int t = 0; t < T; ++t) {
        cp.pcr_off[t] = (int)jobs.size();
        for (int i : h->cr_list) {
            const int v = (h->inst[i].P + s0 - 1) / s0;
            if (v > (1 << t))
                for (int j = 0; j < v; ++j) jobs.push_back(CrJob{i, j});
        }
    }
    cp.pcr_off[T] = (int)jobs.size();
    if (T > 0)
        for (int i : h->cr_list) {
            const int v = (h->inst[i].P + s0 - 1) / s0;
            for (int j = 0; j < v; ++j) jobs.push_back(CrJob{i, j});
        }
    cp.pcr_base_end = (int)jobs.size();
    // new device buffers (the previous plan's stay allocated until cyq_destroy)
    CrJob *dj = nullptr;
    CYQ_CUDA(h->mem.alloc(&dj, jobs.size()));
    CYQ_CUDA(cudaMemcpy(dj, jobs.data(), sizeof(CrJob) * jobs.size(), cudaMemcpyHostToDevice));
    cp.jobs = dj;
    if (T > 0) {
        long long *doT = nullptr, *doV = nullptr;
        CYQ_CUDA(h->mem.alloc(&doT, (size_t)h->batch));
        CYQ_CUDA(h->mem.alloc(&doV, (size_t)h->batch));
        CYQ_CUDA(cudaMemcpy(doT, oT.data(), sizeof(long long) * h->batch, cudaMemcpyHostToDevice));
        CYQ_CUDA(cudaMemcpy(doV, oV.data(), sizeof(long long) * h->batch, cudaMemcpyHostToDevice));
        cp.oT_dev = doT;
        cp.oV_dev = doV;
        CYQ_CUDA(h->mem.alloc(&cp.Lt, (size_t)nT));
        CYQ_CUDA(h->mem.alloc(&cp.At, (size_t)nT));
        CYQ_CUDA(h->mem.alloc(&cp.Bt, (size_t)nT));
        CYQ_CUDA(h->mem.alloc(&cp.bt, (size_t)nV * h->max_nrhs));
        cp.nvt = nV;
    }
    h->cr_jobs = jobs;
    h->cr_plan = cp;
    // the parallel tail runs on the level-parallel coupling solve
    h->cr_levels = T > 0 || ((int)h->cr_list.size() < 2 * h->sms && maxP >= 8);
    h->factored = false;
    return CYQ_OK;
}

cyq_status cyq_set_factor_path(cyq_handle h, int32_t one_warp_per_item) {
    if (!h || one_warp_per_item < 0 || one_warp_per_item > 1) return CYQ_ERR_INVALID_ARG;
    for (cyq_handle sh : h->subs) cyq_set_factor_path(sh, one_warp_per_item);
    h->warp_on = one_warp_per_item == 1;
    h->sweep_on = h->warp_on;
    for (Group &g : h->groups) g.warp_on = h->warp_on;
    h->factored = false;
    return CYQ_OK;
}

cyq_status cyq_set_sweep_path(cyq_handle h, int32_t persistent) {
    if (!h || persistent < 0 || persistent > 1) return CYQ_ERR_INVALID_ARG;
    if (!h->subs.empty()) {
        for (cyq_handle sh : h->subs) {
            const cyq_status st = cyq_set_sweep_path(sh, persistent);
            if (st != CYQ_OK) return st;
        }
        return CYQ_OK;
    }
    if (persistent == 1 && h->sweep_items.empty()) return CYQ_ERR_INVALID_ARG;
    h->sweep_on = persistent == 1;
    return CYQ_OK;
}

cyq_status cyq_get_sweep_path(cyq_handle h, int32_t *persistent, int64_t *items) {
    if (!h) return CYQ_ERR_INVALID_ARG;
    if (!h->subs.empty()) return cyq_get_sweep_path(h->subs[0], persistent, items);
    if (persistent) *persistent = h->sweep_on && !h->sweep_items.empty() ? 1 : 0;
    if (items) *items = (int64_t)h->sweep_items.size();
    return CYQ_OK;
}

cyq_status cyq_get_factor_path(cyq_handle h, int32_t *one_warp_per_item, int64_t *warp_items) {
    if (!h) return CYQ_ERR_INVALID_ARG;
    if (!h->subs.empty()) {
        int64_t n = 0;
        for (cyq_handle sh : h->subs) n += (int64_t)sh->warp_items.size();
        if (one_warp_per_item) *one_warp_per_item = h->subs[0]->warp_on ? 1 : 0;
        if (warp_items) *warp_items = n;
        return CYQ_OK;
    }
    if (one_warp_per_item) *one_warp_per_item = h->warp_on ? 1 : 0;
    if (warp_items) *warp_items = (int64_t)h->warp_items.size();
    return CYQ_OK;
}

cyq_status cyq_get_pcr_tail(cyq_handle h, int32_t *levels) {
    if (!h || !levels) return CYQ_ERR_INVALID_ARG;
    *levels = h->cr_plan.tail;
    return CYQ_OK;
}

cyq_status cyq_assemble_newton(cyq_handle h, const cyq_newton_in *in, const cyq_newton_out *out,
                               cyq_stream stream) {
    if (!h || !in || !out || !in->ny) return CYQ_ERR_INVALID_ARG;
    if (!h->subs.empty()) return CYQ_ERR_UNIMPLEMENTED;   // not offered for recompute-mode handles
    if (!in->Q || !in->R || !in->A || !in->B || !in->q || !in->r || !in->c || !in->x_init || !in->u || !in->x ||
        !in->C || !in->D || !in->bl || !in->bu || !in->y || !in->sigma)
        return CYQ_ERR_INVALID_ARG;
    if ((in->gx && !in->xbar) || (in->gu && !in->ubar)) return CYQ_ERR_INVALID_ARG;
    if (!out->Q || !out->R || !out->S || !out->q || !out->r || !out->c) return CYQ_ERR_INVALID_ARG;
    DeviceGuard guard(h->device);
    cudaStream_t st = to_stream(stream);
    const std::vector<int> ny(in->ny, in->ny + h->batch);
    int max_stages = 0;
    for (int i = 0; i < h->batch; ++i) {
        if (ny[i] < 1) return CYQ_ERR_INVALID_ARG;
        max_stages = std::max(max_stages, h->inst[i].N + 1);
    }
    if (max_stages > 65535) return CYQ_ERR_INVALID_ARG;
    if (ny != h->alm_ny) {
        // offsets of the constraint arrays, uploaded once per distinct ny
        std::vector<AlmOff> off(h->batch);
        long long oC = 0, oD = 0, oY = 0, ogx = 0, ogu = 0;
        size_t smem = 0;
        for (int i = 0; i < h->batch; ++i) {
            const Inst &n = h->inst[i];
            off[i] = AlmOff{oC, oD, oY, ogx, ogu, ny[i], 0};
            oC += (long long)(n.N + 1) * ny[i] * n.nx;
            oD += (long long)n.N * ny[i] * n.nu;
            oY += (long long)(n.N + 1) * ny[i];
            ogx += n.nx;
            ogu += n.nu;
            smem = std::max(smem, newton_smem_bytes(ny[i], n.nx, n.nu));
        }
        if (smem > (size_t)h->smem_optin) {
            g_last_error = "constraint rows of a stage too large for shared memory";
            return CYQ_ERR_INVALID_ARG;
        }
        if (!h->d_alm_off) CYQ_CUDA(h->mem.alloc(&h->d_alm_off, (size_t)h->batch));
        CYQ_CUDA(cudaStreamSynchronize(st));   // the previous table may still be read
        h->alm_off = off;
        CYQ_CUDA(cudaMemcpy(h->d_alm_off, h->alm_off.data(), sizeof(AlmOff) * h->batch, cudaMemcpyHostToDevice));
        h->alm_ny = ny;
        h->alm_smem = smem;
    }
    NewtonArgs a{};
    a.inst = h->d_inst;
    a.off = h->d_alm_off;
    a.Q = in->Q; a.R = in->R; a.S = in->S; a.A = in->A; a.B = in->B;
    a.q = in->q; a.r = in->r; a.f = in->c; a.x0 = in->x_init; a.u = in->u; a.x = in->x;
    a.C = in->C; a.D = in->D; a.bl = in->bl; a.bu = in->bu; a.y = in->y; a.sig = in->sigma;
    a.gx = in->gx; a.gu = in->gu; a.xbar = in->xbar; a.ubar = in->ubar;
    a.Qo = out->Q; a.Ro = out->R; a.So = out->S; a.qo = out->q; a.ro = out->r; a.co = out->c;
    a.active = out->active; a.yhat = out->yhat;
    CYQ_CUDA(launch_newton_assemble(a, h->batch, max_stages, h->alm_smem, st));
    ++h->launches;
    return CYQ_OK;
}

namespace {

cyq_status residual_impl(cyq_handle h, const double *b, const double *z, double *res, double *rel,
                         cyq_stream stream, bool compensated) {
    if (!h || !b || !z) return CYQ_ERR_INVALID_ARG;
    if (!h->factored) return CYQ_ERR_NO_FACTOR;
    if (!h->subs.empty()) {
        for (size_t k = 0; k < h->subs.size(); ++k) {
            const cyq_status st = residual_impl(h->subs[k], b, z, res, rel ? rel + h->sub_first[k] : nullptr, stream,
                                                compensated);
            if (st != CYQ_OK) return st;
        }
        return CYQ_OK;
    }
    DeviceGuard guard(h->device);
    cudaStream_t st = to_stream(stream);
    CYQ_CUDA(cudaMemsetAsync(h->rr, 0, sizeof(double) * h->batch, st));
    CYQ_CUDA(cudaMemsetAsync(h->bb, 0, sizeof(double) * h->batch, st));
    ResidArgs ra = resid_args(h, b, z, res, nullptr);
    if (compensated) {   // every instance's rows compensated (the refinement resets these flags)
        CYQ_CUDA(launch_fill_int(h->batch, h->comp, 1, st));
        ra.comp = h->comp;
    }
    CYQ_CUDA(launch_residual(ra, 1, st));
    CYQ_CUDA(launch_resid_finalize(h->batch, 1, h->rr, h->bb, rel ? rel : h->rel, nullptr, 0.0, nullptr, 0, false, 1,
                                   nullptr, st));
    return CYQ_OK;
}

}  // namespace

cyq_status cyq_residual(cyq_handle h, const double *b, const double *z, double *res, double *rel,
                        cyq_stream stream) {
    return residual_impl(h, b, z, res, rel, stream, false);
}

cyq_status cyq_residual_compensated(cyq_handle h, const double *b, const double *z, double *res, double *rel,
                                    cyq_stream stream) {
    return residual_impl(h, b, z, res, rel, stream, true);
}

cyq_status cyq_solve_adjoint(cyq_handle h, const double *x_init, const double *z, const double *dL_dz, double *w,
                             double *dQ, double *dq, double *dR, double *dr, double *dS, double *dA, double *dB,
                             double *dc, double *dx_init, double *dSigma, cyq_stream stream) {
    if (!h || !x_init || !z || !dL_dz) return CYQ_ERR_INVALID_ARG;
    if (!h->factored) return CYQ_ERR_NO_FACTOR;
    if (!h->subs.empty()) {
        // recompute mode: each chunk's stage factors again, just before its adjoint solve
        if (!w && h->it_max > 0) return CYQ_ERR_INVALID_ARG;
        h->launches = 0;
        for (cyq_handle sh : h->subs) {
            DeviceGuard guard(sh->device);
            cyq_status s2 = run_factor(sh, sh->fac, nullptr, to_stream(stream));
            if (s2 != CYQ_OK) return s2;
            h->launches += sh->launches;
            s2 = cyq_solve_adjoint(sh, x_init, z, dL_dz, w, dQ, dq, dR, dr, dS, dA, dB, dc, dx_init, dSigma, stream);
            if (s2 != CYQ_OK) return s2;
            h->launches += sh->launches;
        }
        return CYQ_OK;
    }
    DeviceGuard guard(h->device);
    cudaStream_t st = to_stream(stream);
    double *wbuf = w ? w : h->dz;
    if (!w && h->it_max > 0) return CYQ_ERR_INVALID_ARG;   // dz is the refinement workspace
    cyq_status s = cyq_solve(h, dL_dz, wbuf, 1, stream);
    if (s != CYQ_OK) return s;
    GradArgs g{};
    g.inst = h->d_inst;
    g.chunks = h->d_chunks;
    g.x0 = x_init;
    g.z = z;
    g.w = wbuf;
    g.dQ = dQ; g.dq = dq; g.dR = dR; g.dr = dr; g.dS = dS; g.dA = dA; g.dB = dB; g.dc = dc; g.dSig = dSigma;
    CYQ_CUDA(launch_adjoint(g, (int)h->chunks.size(), h->batch, h->data, dx_init, st));
    return CYQ_OK;
}

cyq_status cyq_pivot_eval(const double *d, double *l, double *il, const float *df, float *lf, float *ilf,
                          int64_t n, cyq_stream stream) {
    if (n < 0 || (d && (!l || !il)) || (df && (!lf || !ilf))) return CYQ_ERR_INVALID_ARG;
    CYQ_CUDA(launch_pivot_eval(d, l, il, df, lf, ilf, (long long)n, to_stream(stream)));
    return CYQ_OK;
}

cyq_status cyq_get_instance_status(cyq_handle h, int32_t *host_status, cyq_stream stream) {
    if (!h || !host_status) return CYQ_ERR_INVALID_ARG;
    if (!h->subs.empty()) {
        cyq_status first = CYQ_OK;
        for (size_t k = 0; k < h->subs.size(); ++k) {
            const cyq_status st = cyq_get_instance_status(h->subs[k], host_status + h->sub_first[k], stream);
            if (st == CYQ_ERR_CUDA || st == CYQ_ERR_INVALID_ARG) return st;
            if (first == CYQ_OK) first = st;
        }
        return first;
    }
    DeviceGuard guard(h->device);
    cudaStream_t st = to_stream(stream);
    CYQ_CUDA(cudaStreamSynchronize(st));
    CYQ_CUDA(cudaMemcpy(host_status, h->status, sizeof(int) * h->batch, cudaMemcpyDeviceToHost));
    for (int i = 0; i < h->batch; ++i)
        if (host_status[i] != 0) return (cyq_status)host_status[i];
    return CYQ_OK;
}

cyq_status cyq_get_escalation_segments(cyq_handle h, int32_t *host_P) {
    if (!h || !host_P) return CYQ_ERR_INVALID_ARG;
    if (!h->subs.empty()) {
        for (size_t k = 0; k < h->subs.size(); ++k) {
            const cyq_status st = cyq_get_escalation_segments(h->subs[k], host_P + h->sub_first[k]);
            if (st != CYQ_OK) return st;
        }
        return CYQ_OK;
    }
    for (int i = 0; i < h->batch; ++i) host_P[i] = h->esc_h ? h->esc_h->inst[i].P : 0;
    return CYQ_OK;
}

int64_t cyq_workspace_bytes(cyq_handle h) {
    if (!h) return -1;
    long long b = h->mem.bytes;
    for (cyq_handle sh : h->subs) b += cyq_workspace_bytes(sh);
    if (h->esc_h) b += cyq_workspace_bytes(h->esc_h);
    return b;
}

cyq_status cyq_get_stats(cyq_handle h, cyq_stats *out, cyq_stream stream) {
    if (!h || !out) return CYQ_ERR_INVALID_ARG;
    if (!h->subs.empty()) {
        cyq_stats t{};
        t.max_rel_residual = -1.0;
        t.max_certified = -1.0;
        t.P_min = 1 << 30;
        for (cyq_handle sh : h->subs) {
            cyq_stats c{};
            const cyq_status st = cyq_get_stats(sh, &c, stream);
            if (st != CYQ_OK) return st;
            t.refine_steps = std::max(t.refine_steps, c.refine_steps);
            t.max_rel_residual = std::max(t.max_rel_residual, c.max_rel_residual);
            t.max_certified = std::max(t.max_certified, c.max_certified);
            t.P_min = std::min(t.P_min, c.P_min);
            t.P_max = std::max(t.P_max, c.P_max);
            t.work_items += c.work_items;
        }
        *out = t;
        return CYQ_OK;
    }
    DeviceGuard guard(h->device);
    CYQ_CUDA(cudaStreamSynchronize(to_stream(stream)));
    const int nr = std::max(h->last_nrhs, 1);
    std::vector<double> rel((size_t)h->batch * nr), cert((size_t)h->batch * nr);
    std::vector<int> steps(h->batch);
    CYQ_CUDA(cudaMemcpy(rel.data(), h->rel, sizeof(double) * rel.size(), cudaMemcpyDeviceToHost));
    CYQ_CUDA(cudaMemcpy(cert.data(), h->cert, sizeof(double) * cert.size(), cudaMemcpyDeviceToHost));
    CYQ_CUDA(cudaMemcpy(steps.data(), h->steps, sizeof(int) * h->batch, cudaMemcpyDeviceToHost));
    out->refine_steps = 0;
    out->max_rel_residual = h->last_nrhs > 0 ? 0.0 : -1.0;
    for (int i = 0; i < h->batch; ++i) out->refine_steps = std::max(out->refine_steps, steps[i]);
    out->max_certified = h->last_nrhs > 0 && h->certify ? 0.0 : -1.0;
    if (h->last_nrhs > 0) {
        for (double v : rel) out->max_rel_residual = std::max(out->max_rel_residual, v);
        if (h->certify)
            for (double v : cert) out->max_certified = std::max(out->max_certified, v);
    }
    out->P_min = 1 << 30;
    out->P_max = 0;
    for (const Inst &in : h->inst) {
        out->P_min = std::min(out->P_min, in.P);
        out->P_max = std::max(out->P_max, in.P);
    }
    long long items = 0;
    for (const Group &g : h->groups) items += (long long)g.items.size();
    out->work_items = items;
    return CYQ_OK;
}

// ---------------------------------------------------------------------------
// Autotuning (host-timed with CUDA events on the caller's stream)
// ---------------------------------------------------------------------------

}  // extern "C"

namespace {

// Mean time in ms of `reps` calls of fn (each returns a cudaError_t) on st.
template <typename F>
cyq_status time_ms(cudaStream_t st, int reps, F &&fn, float *ms) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return fail_cuda(cudaGetLastError(), "cudaEventCreate");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail_cuda(cudaGetLastError(), "cudaEventCreate");
    }
    cudaError_t e = cudaEventRecord(e0, st);
    for (int i = 0; i < reps && e == cudaSuccess; ++i) e = fn();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail_cuda(e, "autotune");
    *ms = t / reps;
    return CYQ_OK;
}

}  // namespace

extern "C" {

cyq_status cyq_autotune(cyq_handle h, const double *Q, const double *R, const double *S, const double *A,
                        const double *B, const double *Sigma, const double *b, double *z, int32_t nrhs,
                        int32_t reps, cyq_stream stream) {
    if (!h || !b || !z || nrhs < 1 || nrhs > h->max_nrhs) return CYQ_ERR_INVALID_ARG;
    if (!h->subs.empty()) {
        // each chunk tunes its own launch shapes (leaves every chunk factored in turn)
        for (cyq_handle sh : h->subs) {
            const cyq_status st = cyq_autotune(sh, Q, R, S, A, B, Sigma, b, z, nrhs, reps, stream);
            if (st != CYQ_OK) return st;
        }
        h->data = Data{Q, R, S, A, B, Sigma};
        h->factored = true;
        return CYQ_OK;
    }
    if (reps < 1) reps = 3;
    cyq_status s = cyq_factor(h, Q, R, S, A, B, Sigma, stream);   // binds the data
    if (s != CYQ_OK) return s;
    DeviceGuard guard(h->device);
    cudaStream_t st = to_stream(stream);
    const FactorSet &fs = h->fac;
    const int pi = fs.fp64 ? 1 : 0;
    // a plain solve fills the coupling multipliers that the forward sweep reads
    s = run_solve(h, fs, b, z, nrhs, nullptr, st);
    if (s != CYQ_OK) return s;
    const FactorArgs fa = factor_args(h, fs, nullptr);
    static const int cand_factor[] = {16, 32, 64, 128};   // 16: two items per warp
    static const int cand_sweep[] = {32, 64, 128, 256};
    // the float32 correction sweeps of CYQ_FP64_IR32 (their plans exist once the handle is factored)
    const bool tune32 = h->precision == CYQ_FP64_IR32;
    for (Group &g : h->groups) {
        float best = 3.0e38f;
        int pick = 0;
        for (int t : cand_factor) {
            if (t < 32 && (size_t)(32 / t) * ((g.smem_factor[pi] + 15) / 16 * 16) > (size_t)h->smem_optin) continue;
            g.team_factor[pi] = t;
            float ms = 0.0f;
            s = time_ms(st, reps, [&] { return launch_group_factor(fs, g, fa, st); }, &ms);
            if (s != CYQ_OK) { g.team_factor[pi] = 0; return s; }
            if (ms < best) { best = ms; pick = t; }
        }
        g.team_factor[pi] = pick;
        best = 3.0e38f;
        pick = 0;
        g.team_solve_nrhs = nrhs;
        for (int t : cand_sweep) {
            g.team_solve[pi] = t;
            float ms = 0.0f;
            s = time_ms(st, reps, [&] {
                cudaError_t e = launch_group_sweep(h, fs, g, true, b, z, nrhs, nullptr, nullptr, st);
                return e != cudaSuccess ? e : launch_group_sweep(h, fs, g, false, b, z, nrhs, nullptr, nullptr, st);
            }, &ms);
            if (s != CYQ_OK) { g.team_solve[pi] = 0; return s; }
            if (ms < best) { best = ms; pick = t; }
        }
        g.team_solve[pi] = pick;
        if (tune32) {
            best = 3.0e38f;
            pick = 0;
            for (int t : cand_sweep) {
                g.team_solve[0] = t;
                float ms = 0.0f;
                s = time_ms(st, reps, [&] {
                    cudaError_t e = launch_group_sweep(h, h->fac32, g, true, b, z, nrhs, nullptr, nullptr, st);
                    return e != cudaSuccess ? e
                                            : launch_group_sweep(h, h->fac32, g, false, b, z, nrhs, nullptr, nullptr, st);
                }, &ms);
                if (s != CYQ_OK) { g.team_solve[0] = 0; return s; }
                if (ms < best) { best = ms; pick = t; }
            }
            g.team_solve[0] = pick;
        }
    }
    // float32 factor and sweeps: the persistent launches against the per-class ones
    if (!fs.fp64 && !h->warp_items.empty()) {
        float best = 3.0e38f;
        bool pick = true;
        for (int on = 1; on >= 0; --on) {
            h->warp_on = on == 1;
            for (Group &g : h->groups) g.warp_on = h->warp_on;
            float ms = 0.0f;
            s = time_ms(st, reps, [&] { return run_factor(h, fs, nullptr, st) == CYQ_OK ? cudaSuccess : cudaErrorUnknown; },
                        &ms);
            if (s != CYQ_OK) return s;
            if (ms < best) { best = ms; pick = h->warp_on; }
        }
        h->warp_on = pick;
        for (Group &g : h->groups) g.warp_on = pick;
    }
    s = run_factor(h, fs, nullptr, st);   // (refreshes the float32 copy of CYQ_FP64_IR32 too)
    if (s != CYQ_OK) return s;
    const FactorSet &fs32 = h->precision == CYQ_FP64_IR32 ? h->fac32 : fs;
    if (!fs32.fp64 && !h->sweep_items.empty()) {
        float best = 3.0e38f;
        bool pick = true;
        for (int on = 1; on >= 0; --on) {
            h->sweep_on = on == 1;
            float ms = 0.0f;
            s = time_ms(st, reps, [&] { return run_solve(h, fs32, b, z, nrhs, nullptr, st) == CYQ_OK ? cudaSuccess
                                                                                                 : cudaErrorUnknown; },
                        &ms);
            if (s != CYQ_OK) return s;
            if (ms < best) { best = ms; pick = h->sweep_on; }
        }
        h->sweep_on = pick;
    }
    // the timed launches left the factor intact (same data); refresh it as a whole
    s = run_factor(h, fs, nullptr, st);
    if (s != CYQ_OK) return s;
    CYQ_CUDA(cudaStreamSynchronize(st));
    return CYQ_OK;
}

cyq_status cyq_get_launch_shapes(cyq_handle h, int32_t *n_groups, int32_t *factor_team, int32_t *sweep_team,
                                 int32_t nrhs) {
    if (!h || !n_groups) return CYQ_ERR_INVALID_ARG;
    if (!h->subs.empty()) return cyq_get_launch_shapes(h->subs[0], n_groups, factor_team, sweep_team, nrhs);
    *n_groups = (int32_t)h->groups.size();
    const bool f64 = h->fac.fp64;
    for (size_t i = 0; i < h->groups.size(); ++i) {
        if (factor_team) factor_team[i] = factor_team_of(h->groups[i], f64);
        if (sweep_team) sweep_team[i] = sweep_team_of(h->groups[i], f64, nrhs > 0 ? nrhs : 1);
    }
    return CYQ_OK;
}

cyq_status cyq_set_launch_shapes(cyq_handle h, const int32_t *factor_team, const int32_t *sweep_team, int32_t nrhs) {
    if (!h) return CYQ_ERR_INVALID_ARG;
    if (!h->subs.empty()) return CYQ_ERR_UNIMPLEMENTED;   // not offered for recompute-mode handles
    const int pi = h->fac.fp64 ? 1 : 0;
    for (size_t i = 0; i < h->groups.size(); ++i) {
        const int f = factor_team ? factor_team[i] : 0, w = sweep_team ? sweep_team[i] : 0;
        if (!(f == 0 || f == 16 || f == 32 || f == 64 || f == 128)) return CYQ_ERR_INVALID_ARG;
        if (f == 16 && 2 * ((h->groups[i].smem_factor[pi] + 15) / 16 * 16) > (size_t)h->smem_optin)
            return CYQ_ERR_INVALID_ARG;
        if (!(w == 0 || w == 32 || w == 64 || w == 128 || w == 256)) return CYQ_ERR_INVALID_ARG;
    }
    if (sweep_team && nrhs < 1) return CYQ_ERR_INVALID_ARG;
    for (size_t i = 0; i < h->groups.size(); ++i) {
        Group &g = h->groups[i];
        if (factor_team) g.team_factor[pi] = factor_team[i];
        if (sweep_team) {
            g.team_solve[pi] = sweep_team[i];
            g.team_solve_nrhs = nrhs;
        }
    }
    return CYQ_OK;
}

cyq_status cyq_tune_segments(const cyq_desc *desc, const double *Q, const double *R, const double *S,
                             const double *A, const double *B, const double *Sigma, const double *b, double *z,
                             int32_t nrhs, int32_t reps, cyq_stream stream, int32_t *P_out) {
    if (!desc || !P_out || desc->batch < 1 || !desc->N || !b || !z || nrhs < 1) return CYQ_ERR_INVALID_ARG;
    if (reps < 1) reps = 2;
    const int batch = desc->batch;
    int dev = desc->device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return CYQ_ERR_NO_DEVICE;
    const int sms = sm_count(dev);
    std::vector<int> base(batch);
    for (int i = 0; i < batch; ++i) {
        const int N = desc->N[i];
        if (N < 1) return CYQ_ERR_INVALID_ARG;
        int P = desc->P_per_instance ? desc->P_per_instance[i] : desc->P;
        if (P <= 0) P = auto_segments(batch, N, sms);
        base[i] = std::min(P, N);
    }
    cudaStream_t st = to_stream(stream);
    std::vector<std::vector<int>> tried;
    std::vector<int> best_P = base;
    float best = 3.0e38f;
    int best_fail = batch + 1;      // instances not solved to the tolerance (or not factored)
    std::vector<int32_t> status(batch);
    for (int shift = -2; shift <= 2; ++shift) {
        std::vector<int> P(batch);
        for (int i = 0; i < batch; ++i) {
            long long p = shift >= 0 ? (long long)base[i] << shift : base[i] >> -shift;
            P[i] = (int)std::max(1LL, std::min<long long>(p, desc->N[i]));
        }
        if (std::find(tried.begin(), tried.end(), P) != tried.end()) continue;
        tried.push_back(P);
        cyq_desc d = *desc;
        d.P = 0;
        d.P_per_instance = P.data();
        if (d.max_nrhs < nrhs) d.max_nrhs = nrhs;
        cyq_handle h = nullptr;
        if (cyq_create(&d, &h) != CYQ_OK) {
            if (shift == 0) return CYQ_ERR_INVALID_ARG;
            continue;   // e.g. the workspace of this candidate does not fit
        }
        // warm-up, then factor + solve timed together
        cyq_status s = cyq_factor(h, Q, R, S, A, B, Sigma, stream);
        if (s == CYQ_OK) s = cyq_solve(h, b, z, nrhs, stream);
        float ms = 0.0f;
        if (s == CYQ_OK)
            s = time_ms(st, reps, [&] {
                cyq_status q = cyq_factor(h, Q, R, S, A, B, Sigma, stream);
                if (q == CYQ_OK) q = cyq_solve(h, b, z, nrhs, stream);
                return q == CYQ_OK ? cudaSuccess : cudaErrorUnknown;
            }, &ms);
        // a candidate that leaves more instances uncertified (e.g. one whose float64
        // escalation plan does not fit) loses to any that certifies more of them
        int fail = 0;
        if (s == CYQ_OK) {
            const cyq_status g = cyq_get_instance_status(h, status.data(), stream);
            if (g != CYQ_OK && g != CYQ_ERR_NOT_CONVERGED && g != CYQ_ERR_NOT_PD) s = g;
            for (int i = 0; i < batch; ++i) fail += status[i] != CYQ_OK;
        }
        cyq_destroy(h);
        if (s != CYQ_OK) return s;
        if (fail < best_fail || (fail == best_fail && ms < best)) {
            best = ms;
            best_fail = fail;
            best_P = P;
        }
    }
    for (int i = 0; i < batch; ++i) P_out[i] = best_P[i];
    return CYQ_OK;
}

}  // extern "C"

void cyq::set_last_error_message(const char *msg) { g_last_error = msg ? msg : ""; }

cudaError_t cyq::ensure_smem(const void *kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> set;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    size_t &cur = set[std::make_pair(dev, kernel)];
    if (bytes <= cur) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}
