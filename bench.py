#!/usr/bin/env python3
"""KKT factor+solve benchmark on one node.

Workload (default): the uneven batch, 4096 independent linear-quadratic OCPs
with N uniform in [16, 256], nx in {4..64}, nu in {2..32} (551,381 stages,
20 GB of float64 data), stage cross terms S and diagonal regularisation Sigma
log-uniform in [1e-6, 1e6]; one factorization + one right-hand side per OCP.
One step = factor all OCPs + solve, with the inputs resident in device
memory (far larger than the 129 MB L2).  ``--workload`` selects the other
workloads (single OCP, 1024 OCPs of N = 64 with 4 right-hand sides, long
horizon, adjoint, mass-spring MPC, Newton step); each has its own list of
methods, and the headline is the first of them that solves every instance
to the tolerance.

Methods (each timed over the same K steps):
  fp64_refine  float64 factor + solve, float64 residual and refinement until
               ||b - Kz|| / ||b|| <= 5e-11 for every OCP and right-hand side
               (the metric's gate 1e-10 with a factor-2 margin)
  fp64         plain float64 factor + solve (no residual computed)
  fp32_refine  float32 factor + solve, float64 residual + refinement to 5e-11,
               float64 factor for the instances float32 cannot bring there
  fp64_ir32    float64 factor + solve; corrections by float32 sweeps with a
               float32 copy of the factor, float64 residual to 5e-11

Prints ONE JSON line on rank 0.  ``--impl reference`` times the CPU oracle
(plain FP64 C Riccati recursion) on the host instead.  Under torchrun every
rank solves its own batch (weak scaling, no data-path collective).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2512_09058_gb300 import inputs, shard  # noqa: E402

METRIC = "KKT factor+solve/sec and ns/stage at rel. residual ≤1e-10; % of roofline"
UNIT = "OCP factor+solve/s"
# pipe peaks per SM and clock: 2 FP64 FMA (measured on this GPU: one warp instruction per
# 64 cycles on each of the four sub-partitions' FP64 units) and 128 FP32 lanes
FP64_FMA_PER_CLK_SM = 2
FP32_FMA_PER_CLK_SM = 128
HBM_FALLBACK_GBS = 6800.0
WORKLOAD = "uneven4096"
# method -> (factor precision, refinement step budget).  Float64 refinement
# converges in one or two steps (a few more where the compensated residual rows
# take over near the target); float32 needs ~5-8 at cond(K) ~ 1e11.
METHODS = {"fp64": ("fp64", 0), "fp64_refine": ("fp64", 5), "fp32_refine": ("fp32_refine", 8),
           "fp64_ir32": ("fp64_ir32", 3), "fp64_refine_recompute": ("fp64", 5)}
# methods that keep the stage factors of one chunk of instances at a time and factor
# every chunk again in each solve and adjoint: method -> chunks
RECOMPUTE = {"fp64_refine_recompute": 4}
# refinement target: the metric's gate 1e-10 with a factor-2 margin, so that
# another float64 evaluation of the returned solution's residual (the oracle's;
# they differ by up to a few percent near the gate) is within the gate too.  The
# worst-case evaluation bound (cyq_desc.certify) lies above 1e-10 for many
# instances of these workloads and cannot serve as the stop criterion
REFINE_TOL = 5e-11
# DRAM bytes (read + write) per launch of a part of the step, from ncu captures
# of its current kernels (dram__bytes_read.sum + dram__bytes_write.sum), keyed by
# workload, factor precision and the part's kernels; absent where no capture of
# the current kernels exists.  Uneven batch: captured on its first 512 instances
# (71,441 stages) and scaled by stages to the whole batch (551,381): every stage's
# data, tile and factor moves once per launch, so the traffic grows in proportion.
_UNEVEN_SCALE = 551381.0 / 71441.0
NCU_TRAFFIC = {("batch1024_n64_nx12_nu4", "fp64_ir32", "k_factor_pairs<12, 4>"): 217.1e6 + 219.5e6,
               ("uneven4096", "fp32_refine", "k_ingest_f32 + k_factor_team + k_inv_R_f32"):
                   (3727e6 + 2272e6 + 296.9e6) * _UNEVEN_SCALE,
               ("uneven4096", "fp32_refine", "k_sweep_team<true> + k_cr_solve + k_sweep_team<false> (1 rhs)"):
                   (1563e6 + 1592e6) * _UNEVEN_SCALE}
# workload -> methods (headline: the first one that certifies every instance),
# CUDA-graph replay, adjoint in the step, segment counts tuned by timing
# (cyq_tune_segments); launch shapes are always tuned by timing (cyq_autotune)
# before the timed region
WORKLOADS = {
    "batch1024_n64_nx12_nu4": dict(methods=["fp64_ir32", "fp64_refine", "fp64", "fp32_refine"], graph=True,
                                   adjoint=False, tune_segments=True),
    "single_n32_nx8_nu4": dict(methods=["fp64", "fp64_refine"], graph=True, adjoint=False, tune_segments=True),
    "long_n4096_nx32_nu16": dict(methods=["fp32_refine", "fp64", "fp64_refine"], graph=True, adjoint=False,
                                 tune_segments=True),
    "uneven4096": dict(methods=["fp32_refine", "fp64_refine"], graph=True, adjoint=False, tune_segments=True,
                       steps=40),
    "adjoint512_n128_nx24_nu8": dict(methods=["fp64_refine", "fp64_refine_recompute"], graph=True, adjoint=True,
                                     tune_segments=True),
    "massspring150_M18_N96": dict(methods=["fp32_refine", "fp64_refine", "fp64_ir32"], graph=True, adjoint=False,
                                  tune_segments=True),
    # step = Newton-system assembly + factor + solve of the augmented Lagrangian inner problem
    "newton1024_n64_nx12_nu4_ny16": dict(methods=["fp32_refine", "fp64_refine", "fp64_ir32"], graph=True,
                                         adjoint=False, tune_segments=True, newton=True),
}


# Fixed segment count / launch shapes (--segments, --launch-shapes) in place of
# the timing tuners, e.g. to reproduce a tuned configuration under a profiler,
# whose serialised launches distort the tuners' timings.
FIXED = {"P": 0, "shapes": None, "pcr_tail": 0, "early_esc": False, "it_max": -1}


def method_budget(method):
    """(factor precision, refinement step budget) of a method (--it-max overrides the budget)."""
    precision, it_max = METHODS[method]
    if FIXED["it_max"] >= 0 and it_max > 0:
        it_max = FIXED["it_max"]
    return precision, it_max


def tuned_solver(torch, cyq, batch, data, b, method, tune_segments, P=None):
    """A solver for `method` with timed-autotuned segment counts (when asked, or
    the given P) and launch shapes; returns (solver, P).  Untimed setup."""
    precision, it_max = method_budget(method)
    nrhs = len(batch.rhs)
    if P is None and FIXED["P"] > 0:
        P = np.minimum(np.asarray(batch.N), FIXED["P"]).astype(np.int32)
    if P is None and tune_segments:
        P = cyq.tune_segments(batch.N, batch.nx, batch.nu, data, b, nrhs=nrhs, reps=2, precision=precision,
                              it_max=it_max, tol=REFINE_TOL)
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision=precision, max_nrhs=nrhs, it_max=it_max,
                   tol=REFINE_TOL, P_per_instance=P, early_escalation=FIXED["early_esc"],
                   recompute_chunks=RECOMPUTE.get(method, 0))
    if FIXED["pcr_tail"] > 0:
        s.set_pcr_tail(FIXED["pcr_tail"])
    if FIXED["shapes"] is not None:
        n = len(s.launch_shapes(nrhs=nrhs)["factor"])
        s.set_launch_shapes(factor=[FIXED["shapes"][0]] * n, sweep=[FIXED["shapes"][1]] * n, nrhs=nrhs)
    else:
        s.autotune(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"], b, nrhs=nrhs, reps=3)
    return s, P


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=0,
                   help="timed steps (default: the workload's, about a minute of timed work)")
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="cyq", choices=["cyq", "reference"])
    p.add_argument("--workload", default=WORKLOAD, choices=sorted(inputs.CONFIGS))
    p.add_argument("--methods", default="", help="comma list; default: the workload's methods")
    p.add_argument("--instances", type=int, default=0,
                   help="use only the first K instances of the workload (small profiling cases)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--segments", type=int, default=0, help="segments per OCP instead of the segment tuner")
    p.add_argument("--graph", type=int, default=-1, help="1 / 0: force CUDA-graph replay on / off")
    p.add_argument("--pcr-tail", type=int, default=0,
                   help="levels of the coupling solve done by parallel cyclic reduction (0: plain)")
    p.add_argument("--update-sweep", action="store_true",
                   help="also time factorization updates against refactorization (one-segment workloads)")
    p.add_argument("--it-max", type=int, default=-1,
                   help="refinement step budget of the refined methods instead of theirs")
    p.add_argument("--early-escalation", action="store_true",
                   help="float32 refinement: predicted float64 escalation after two corrections")
    p.add_argument("--launch-shapes", default="",
                   help="F,S: threads per item of the factor and of the sweeps instead of the launch tuner")
    return p.parse_args()


def factor_kernel_name(batch, r, f64):
    """The stage-factor kernels the timed factorization launched (the roofline's kernel)."""
    nx, nu = set(np.asarray(batch.nx).tolist()), set(np.asarray(batch.nu).tolist())
    one_seg = int(r["segments"].max()) == 1
    if f64 and one_seg and set(r["shapes"]["factor"]) == {16} and len(nx) == 1 and len(nu) == 1 \
            and (nx.pop(), nu.pop()) in ((12, 4), (8, 4)):
        return "k_factor_pairs<%d, %d>" % (int(batch.nx[0]), int(batch.nu[0]))
    path = r.get("path") or {}
    if not f64 and path.get("one_warp_per_item") and path.get("warp_items", 0) > 0:
        return "k_ingest_f32 + k_factor_team + k_inv_R_f32%s" % (
            "" if one_seg else " (+ k_factor_segments<float> for segments >= 1, cyclic reduction)")
    return "k_factor_segments<%s>%s" % ("double" if f64 else "float", "" if one_seg else " (+ cyclic reduction)")


def riccati_fma_per_stage(nx, nu):
    """Serial factorized Riccati, FMA = 1 (paper Sec. 4.5): 1/2 nux nx^2 + 1/2 nux^2 nx + 1/6 nux^3."""
    nux = nx + nu
    return 0.5 * nux * nx * nx + 0.5 * nux * nux * nx + nux ** 3 / 6.0


def _seg_len(c, N, P):
    b = lambda k: (k * N) // P
    return N - b(P - 1) if c == 0 else b(c) - b(c - 1)


def factor_fma(N, nx, nu, P):
    """Algorithmic FMAs (FMA = 1, leading terms as in paper Sec. 4.5) of the
    factorization as scheduled: P segments of the modified Riccati recursion
    (Alg. fact-mod-riccati), the Schur blocks (compute-schur) and the cyclic
    reduction of the P coupling blocks."""
    nux = nx + nu
    total = 0.0
    for c in range(P):
        L = _seg_len(c, N, P)
        prop = c >= 1
        for t in range(L):
            total += nux ** 3 / 6.0                                        # potrf
            if t == 0 or prop:
                total += 0.5 * nx * nu * nu + nx * nx * nu + 0.5 * nx * nx * nu   # trsm L^B, gemm A^cl, syrk M_fwd
            if t < L - 1:
                total += 0.5 * nux * nx * nx + 0.5 * nux * nux * nx          # trmm V, syrk H + V V^T
                if prop:
                    total += nux * nx * nx                                     # gemm [B^ A^] = A^cl [B A]
        if prop:
            total += 1.5 * nx ** 3                                             # trsm L^A, syrk L^A L^A^T, trmm K
        total += nx ** 3 / 3.0                                                 # trtri, lauum (M_bwd)
    n3 = float(nx) ** 3
    if P == 1:
        total += n3 / 6.0
    else:
        s = 1
        while s < P:
            for k in range(s, P, 2 * s):
                total += n3 / 6.0 + 0.5 * n3 + (0.5 * n3 if k + s < P else 0.0)
            for i in range(0, P, 2 * s):
                total += (0.5 * n3 if i - s >= 0 else 0.0) + (0.5 * n3 if i + s < P else 0.0) \
                    + (n3 if i - 2 * s >= 0 else 0.0)
            s *= 2
        total += n3 / 6.0
    return total


def device_peaks(torch, clk):
    """Pipe peaks (GFLOP/s) from the device's SM count and the SM clock sampled
    under load (its maximum), and the HBM peak: the measured copy bandwidth in
    MEASURED_PEAKS.json when the file is there, else the fallback figure."""
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count
    measured = {}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            measured = json.load(f)
    mhz = (clk or {}).get("sm_max_mhz") or measured.get("sm_max_mhz") or 2070.0
    ghz = float(mhz) / 1e3
    hbm = measured.get("hbm_gbs")
    return dict(sms=sms, ghz=ghz, fp64=sms * FP64_FMA_PER_CLK_SM * 2 * ghz, fp32=sms * FP32_FMA_PER_CLK_SM * 2 * ghz,
                hbm=float(hbm) if hbm else HBM_FALLBACK_GBS,
                hbm_source="of measured (MEASURED_PEAKS.json hbm_gbs)" if hbm else "of fallback",
                pipe_source="derived: %d SMs x %%d FMA/clk x 2 x %.3f GHz" % (sms, ghz))


def data_bytes(batch):
    """Float64 bytes of the stage data (Q, R, S, A, B, Sigma) that a pass over the batch reads."""
    b = batch.Q.nbytes + batch.R.nbytes + batch.S.nbytes + batch.A.nbytes + batch.B.nbytes
    return b + (batch.Sigma.nbytes if batch.Sigma is not None else 0)


def factor_store_elems(batch):
    """Elements of the stored stage factor per batch: L ((nu+nx)^2), 1/diag (nu+nx),
    [B A] (nx (nu+nx)) per stage."""
    N, nx, nu = (np.asarray(v, np.int64) for v in (batch.N, batch.nx, batch.nu))
    nux = nx + nu
    return int((N * (nux * nux + nux + nx * nux)).sum())


def residual_fma(batch):
    """FMAs of one float64 residual (rows of eq. opt-cond-ocp-eq) per right-hand
    side, as the kernel runs them: per stage k, R u, B^T lambda, B u and Q x;
    A x and S x for k > 0; A^T lambda and S^T u for k < N - 1; Sigma as its own
    term of the u and x rows; the identity couplings of x and lambda are not
    products.  S terms only where S is given, Sigma terms where Sigma is."""
    N, nx, nu = (np.asarray(v, np.int64) for v in (batch.N, batch.nx, batch.nu))
    f = N * (nu * nu + 2 * nx * nu + nx * nx) + 2 * (N - 1) * nx * nx
    if batch.S is not None:
        f = f + 2 * (N - 1) * nx * nu
    if batch.Sigma is not None:
        f = f + N * (nu + nx)
    return int(f.sum())


def roofline_of(name, flops, bytes_alg, ms, pipe_peak, hbm_peak, pipe_name, peaks, traffic=None):
    """The roofline entry of one kernel (or phase): its bound is the larger of the
    time at the pipe peak and the time at the HBM peak for its algorithmic work."""
    t_alu = flops / (pipe_peak * 1e9)
    t_hbm = bytes_alg / (hbm_peak * 1e9)
    sec = ms / 1e3
    if t_hbm >= t_alu:
        ach = bytes_alg / sec / 1e9
        out = {"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
               "frac": ach / hbm_peak, "peak_source": peaks["hbm_source"]}
    else:
        ach = flops / sec / 1e9
        out = {"kernel": name, "bound": "alu", "achieved": ach, "peak": pipe_peak, "unit": "GFLOP/s",
               "frac": ach / pipe_peak,
               "peak_source": peaks["pipe_source"] % (FP64_FMA_PER_CLK_SM if pipe_name == "fp64" else
                                                     FP32_FMA_PER_CLK_SM) + " (%s pipe)" % pipe_name}
    out.update({"traffic": traffic, "algorithmic_bytes": bytes_alg, "algorithmic_flops": flops, "ms": ms,
                "t_at_hbm_peak_ms": t_hbm * 1e3, "t_at_pipe_peak_ms": t_alu * 1e3})
    return out


def batch_factor_fma(batch, segments):
    cache = {}
    tot = 0.0
    for N, nx, nu, P in zip(batch.N, batch.nx, batch.nu, segments):
        key = (int(N), int(nx), int(nu), int(P))
        if key not in cache:
            cache[key] = factor_fma(*key)
        tot += cache[key]
    return tot


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.path = None
        self.idx = device_index

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        loaded = [r for r in rows if r["power"] > 0.3 * max(x["power"] for x in rows)] or rows
        reasons = set()
        for r in loaded:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in loaded), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(loaded),
                "power_w_max": max(r["power"] for r in rows)}


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and the cpu_baseline)
# ---------------------------------------------------------------------------
def time_oracle(batch, nrhs, budget_s=2.0, max_instances=None):
    """Oracle (FP64 C, textbook Riccati; one factorization shared by the nrhs
    right-hand sides) over the batch's instances in order, until ``budget_s``
    seconds of CPU work or ``max_instances`` instances.  Returns (OCP/s, count, s)."""
    import oracle   # CPU-baseline / reference leg only
    insts = batch.instances if max_instances is None else batch.instances[:max_instances]
    done, el = 0, 0.0
    t0 = time.perf_counter()
    for x in insts:
        b = np.stack([oracle.build_rhs(x, *x.rhs[j]) for j in range(nrhs)])
        t = time.perf_counter()
        oracle.riccati_solve(x, b)
        el += time.perf_counter() - t
        done += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    return done / el, done, el


def _oracle_proc(name, indices, nrhs, q_in, q_out):
    """One host core, pinned to its instances: regenerates them from the seeded
    generator (untimed, at most 64 of them, all before the first timed step) and,
    for every budget it receives, solves them in turn, cycling, until that many
    seconds of solving; answers (count, seconds)."""
    import oracle   # CPU-baseline / reference leg only
    cache = []
    pos = 0
    while True:
        budget = q_in.get()
        if budget is None:
            return
        if budget < 0:   # generate every instance first, so that no step times a neighbour's generation
            for k in range(len(cache), len(indices)):
                x = inputs.make_batch(name, [indices[k]]).instances[0]
                cache.append((x, np.stack([oracle.build_rhs(x, *x.rhs[j]) for j in range(nrhs)])))
            q_out.put((0, 0.0))
            continue
        done, el = 0, 0.0
        while el < budget:
            k = pos % len(indices)
            if k >= len(cache):
                x = inputs.make_batch(name, [indices[k]]).instances[0]
                cache.append((x, np.stack([oracle.build_rhs(x, *x.rhs[j]) for j in range(nrhs)])))
            x, b = cache[k]
            t = time.perf_counter()
            oracle.riccati_solve(x, b)
            el += time.perf_counter() - t
            done += 1
            pos += 1
        q_out.put((done, el))


class OraclePool:
    """The oracle on every host core at once: one spawned process per core, each
    on its own instances of the workload (round-robin over the batch), kept for
    every step so that each process generates its instances only once."""

    def __init__(self, name, n_instances, nrhs, workers=None):
        import multiprocessing
        ctx = multiprocessing.get_context("spawn")
        workers = workers or os.cpu_count() or 1
        self.procs, self.qin, self.qout = [], [], []
        # one thread per process: the oracle is single-threaded, and library threads of the
        # generator would compete with the other processes' timed solves
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            for w in range(min(workers, n_instances)):
                qi, qo = ctx.Queue(), ctx.Queue()
                idx = list(range(w, n_instances, workers))[:64]
                p = ctx.Process(target=_oracle_proc, args=(name, idx, nrhs, qi, qo), daemon=True)
                p.start()
                self.procs.append(p)
                self.qin.append(qi)
                self.qout.append(qo)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        for q in self.qin:   # every instance generated before any timed step
            q.put(-1.0)
        for q in self.qout:
            q.get()

    def step(self, budget_s):
        """(OCP/s summed over the concurrent processes, instances solved, cores)."""
        for q in self.qin:
            q.put(budget_s)
        res = [q.get() for q in self.qout]
        return sum(d / e for d, e in res if e > 0), sum(d for d, _ in res), len(res)

    def close(self):
        for q in self.qin:
            q.put(None)
        for p in self.procs:
            p.join(timeout=30)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def time_oracle_all_cores(name, n_instances, nrhs, budget_s=2.0, workers=None):
    """One measurement of the oracle on every host core at once (OraclePool)."""
    with OraclePool(name, n_instances, nrhs, workers) as pool:
        return pool.step(budget_s)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def _loss_grad(torch, batch, z):
    """dL/dz of L = sum of squared states and inputs (multiplier entries zero)."""
    g = 2.0 * z
    off = 0
    for x in batch.instances:
        w = x.nu + 2 * x.nx
        g[off:off + x.kkt_size].view(x.N, w)[:, x.nu + x.nx:] = 0.0
        off += x.kkt_size
    return g


L2_BYTES = 129e6


def newton_setup(torch, cyq, batch, data, rhs_dev, indices, cfg):
    """Newton workload: the constraint data and iterate on the device, the assembled
    blocks (which the timing tuners factor) and the Newton system's right-hand side."""
    alms = inputs.config_alm(cfg, batch.instances, indices)
    cat = inputs.concat_alm(alms)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    alm = {k: t(getattr(cat, k)) for k in ("C", "D", "bl", "bu", "y", "gx", "gu", "xbar", "ubar")}
    alm["sigma"], alm["ny"] = t(cat.sig), cat.ny
    q, r, c, x0 = rhs_dev[0]
    ctx = dict(data=data, q=q, r=r, c=c, x0=x0, u=t(cat.u), x=t(cat.x), alm=alm, zero=torch.zeros_like(x0))
    s0 = cyq.Solver(batch.N, batch.nx, batch.nu, it_max=0)
    ctx["out"] = s0.assemble_newton(data, q, r, c, x0, ctx["u"], ctx["x"], alm)
    out = ctx["out"]
    ndata = dict(Q=out["Q"], R=out["R"], S=out["S"], A=data["A"], B=data["B"], Sigma=None)
    s0.factor(ndata["Q"], ndata["R"], ndata["S"], ndata["A"], ndata["B"], None)
    b = s0.build_rhs(out["q"], out["r"], out["c"], ctx["zero"])
    torch.cuda.synchronize()
    s0.close()
    return ctx, ndata, b


def run_method(torch, cyq, batch, data, b, x0, method, steps, warmup, dist, graph=False, adjoint=False,
               flush=None, tune_segments=False, newton=None):
    """Time `steps` factor+solve steps.  With `flush` (a device buffer larger than
    L2), the buffer is rewritten between steps, outside the per-step events, and
    the step time is the sum of the per-step event intervals.  With `newton`
    (newton_setup's context) the factor part starts with the Newton-system
    assembly and the solve part with building its right-hand side."""
    precision, it_max = method_budget(method)
    nrhs = len(batch.rhs)
    s, P = tuned_solver(torch, cyq, batch, data, b, method, tune_segments)
    shapes = s.launch_shapes(nrhs=nrhs)
    path = s.factor_path()
    z = torch.empty_like(b)
    mask = _loss_grad(torch, batch, torch.ones_like(b[:s.kkt_size])) / 2.0 if adjoint else None

    def factor():
        if newton is not None:
            n = newton
            s.assemble_newton(n["data"], n["q"], n["r"], n["c"], n["x0"], n["u"], n["x"], n["alm"], out=n["out"])
        s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])

    def solve():
        if newton is not None:
            o = newton["out"]
            s.build_rhs(o["q"], o["r"], o["c"], newton["zero"], b=b)
        s.solve(b, z, nrhs=nrhs)
        if adjoint:
            g = 2.0 * z[:s.kkt_size] * mask
            s.solve_adjoint(x0, z[:s.kkt_size], g)

    factor()
    launches_factor = s.launch_count() + (1 if newton is not None else 0)   # + the assembly
    solve()
    launches_solve = s.launch_count() + (1 if newton is not None else 0)     # + building b
    launches_solve += (1 + 2 * 3 + 1 if adjoint else 0)   # adjoint: solve + grads
    for _ in range(warmup):
        factor()
        solve()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    g_factor = g_solve = None
    if graph:
        # one step captured as two graphs (factor, solve): every launch and memset of
        # the library is stream-ordered, so the whole refinement loop replays
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            factor()
            solve()
        stream.wait_stream(side)
        torch.cuda.synchronize()
        g_factor, g_solve = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_factor):
            factor()
        with torch.cuda.graph(g_solve):
            solve()
        for _ in range(max(1, warmup)):
            g_factor.replay()
            g_solve.replay()
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t_start.record(stream)
    for i in range(steps):
        if flush is not None:
            flush.zero_()
        ev[i][0].record(stream)
        if graph:
            g_factor.replay()
        else:
            factor()
        ev[i][1].record(stream)
        if graph:
            g_solve.replay()
        else:
            solve()
        ev[i][2].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    total_ms = t_start.elapsed_time(t_end)
    if flush is not None:
        total_ms = sum(e[0].elapsed_time(e[2]) for e in ev)
    total_ms = shard.reduce_time_ms(total_ms, dist, device="cuda")
    if dist is not None:
        dist.barrier()
    factor_ms = [e[0].elapsed_time(e[1]) for e in ev]
    solve_ms = [e[1].elapsed_time(e[2]) for e in ev]
    # the residual and the correction (one substitution with the stored factor, both sweeps
    # and the coupling solve) timed on their own with CUDA events, for their rooflines
    kk = s.kkt_size
    dz = torch.empty_like(b)
    reps = max(3, min(steps, 10))
    phase = {}
    parts = [("residual", lambda: s.residual(b[:kk], z[:kk]))]
    if method not in RECOMPUTE:   # (the recompute mode keeps no factor to apply on its own)
        parts.append(("correction", lambda: s.apply_factor(b, dz, nrhs=nrhs)))
    for name, fn in parts:
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            if flush is not None:
                flush.zero_()
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        phase[name] = e0.elapsed_time(e1) / reps
    if flush is not None:   # the flushes inside the loop above are not the phases' time
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(reps):
            flush.zero_()
        f1.record(stream)
        torch.cuda.synchronize()
        for k in phase:
            phase[k] = max(0.0, phase[k] - f0.elapsed_time(f1) / reps)
    phase.setdefault("correction", None)
    status = s.instance_status()
    st = s.stats()
    if it_max == 0:   # plain solve: measure the residual it reached (outside the timed region)
        worst = 0.0
        for j in range(nrhs):
            kk = s.kkt_size
            rel = s.residual(b[j * kk:(j + 1) * kk], z[j * kk:(j + 1) * kk])
            worst = max(worst, float(rel.max().item()))
        st["max_rel_residual"] = worst
    segments = s.segments
    esc_seg = s.escalation_segments() if precision == "fp32_refine" else None
    wbytes = s.workspace_bytes
    s.close()
    return dict(total_ms=total_ms, factor_ms=float(np.mean(factor_ms)), solve_ms=float(np.mean(solve_ms)),
                status_ok=bool((status == 0).all()), stats=st, segments=segments,
                launches_per_step=launches_factor + launches_solve, P=P, shapes=shapes, phase=phase,
                path=path, workspace_bytes=wbytes,
                escalation_segments=None if esc_seg is None else [int(esc_seg.min()), int(esc_seg.max())])


def run_e2e(torch, cyq, batch, method, steps, warmup, data, b, P=None, adjoint=False):
    """Same metric through the public API with host buffers: every step copies
    the data and (q, r, c, x_init) from pinned host memory, builds the KKT
    right-hand sides, factors, solves and copies z back to pinned memory.  The
    solver is tuned like the device-resident one (same segment counts)."""
    precision, it_max = method_budget(method)
    nrhs = len(batch.rhs)
    s, _ = tuned_solver(torch, cyq, batch, data, b, method, False, P=P)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    host = {k: pin(getattr(batch, k)) for k in ("Q", "R", "S", "A", "B")}
    host["Sigma"] = pin(batch.Sigma) if batch.Sigma is not None else None
    host_rhs = [[pin(x) for x in r] for r in batch.rhs]
    dev = {k: (torch.empty_like(v, device="cuda") if v is not None else None) for k, v in host.items()}
    dev_rhs = [[torch.empty_like(x, device="cuda") for x in r] for r in host_rhs]
    kk = s.kkt_size
    b = torch.empty(nrhs * kk, dtype=torch.float64, device="cuda")
    z = torch.empty_like(b)
    nout = nrhs * kk
    mask = _loss_grad(torch, batch, torch.ones(kk, dtype=torch.float64, device="cuda")) / 2.0 if adjoint else None
    out_host = torch.empty(nout + (int(batch.A.size) if adjoint else 0), dtype=torch.float64).pin_memory()
    h2d = sum(v.numel() * 8 for v in host.values() if v is not None) + sum(x.numel() * 8 for r in host_rhs for x in r)
    d2h = out_host.numel() * 8

    def step():
        for k, v in host.items():
            if v is not None:
                dev[k].copy_(v, non_blocking=True)
        for hr, dr in zip(host_rhs, dev_rhs):
            for h, d in zip(hr, dr):
                d.copy_(h, non_blocking=True)
        s.factor(dev["Q"], dev["R"], dev["S"], dev["A"], dev["B"], dev["Sigma"])
        for j in range(nrhs):
            s.build_rhs(*dev_rhs[j], b=b[j * kk:(j + 1) * kk])
        s.solve(b, z, nrhs=nrhs)
        out_host[:nout].copy_(z, non_blocking=True)
        if adjoint:
            gr = s.solve_adjoint(dev_rhs[0][3], z[:kk], 2.0 * z[:kk] * mask, want=("w", "dA"))
            out_host[nout:].copy_(gr["dA"], non_blocking=True)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    s.close()
    return ms / steps, h2d, d2h


def update_crossover(torch, cyq, batch, data, b, precision="fp64", m_list=(1, 2, 4, 8, 16, 32), reps=10, seed=7):
    """Factorization update (cyq_update_factor) against refactorization (cyq_factor)
    of the modified data, on the batch with one segment per OCP.  For m changed
    rows per instance, at m distinct random stages (stage 0: rows of the input
    part only), the update adds the rows (delta > 0) and a downdate of the same rows
    restores the factor, so the timed pairs repeat on the same matrices; the
    update time is half a pair.  Also one changed row at every stage.  Returns
    the times in ms and whether the update matched the refactorization."""
    g = np.random.default_rng(seed)
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision=precision, P=1, it_max=0)
    s.autotune(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"], b, nrhs=1, reps=2)
    stream = torch.cuda.current_stream()
    out = []
    # (changes at every stage carry a rank that grows with the horizon: beyond the update
    # workspace the call reports CYQ_ERR_UPDATE_RANK and a refactorization is the way)
    cases = [("total", m) for m in m_list] + [("per_stage", 1)]
    for kind, m in cases:
        W, D, mods = [], [], []
        mm = m if kind == "per_stage" else 1   # rows per stage
        for x in batch.instances:
            n = x.nu + x.nx
            w = np.zeros((x.N, mm, n))
            d = np.zeros((x.N, mm))
            stages = np.arange(x.N) if kind == "per_stage" else g.choice(x.N, size=min(m, x.N), replace=False)
            for st in stages:
                for r in range(mm):
                    w[st, r] = g.standard_normal(n) / np.sqrt(n)
                    if st == 0:
                        w[st, r, x.nu:] = 0.0
                    d[st, r] = 10.0 ** g.uniform(-1, 1)
            W.append(w)
            D.append(d)
            R, S, Q = x.R.copy(), x.S.copy(), x.Q.copy()
            nu, nx, N = x.nu, x.nx, x.N
            for st in stages:
                for r in range(mm):
                    wu, wx = w[st, r, :nu], w[st, r, nu:]
                    R[st * nu * nu:(st + 1) * nu * nu] += (d[st, r] * np.outer(wu, wu)).flatten(order="F")
                    xq = st if st > 0 else N
                    Q[xq * nx * nx:(xq + 1) * nx * nx] += (d[st, r] * np.outer(wx, wx)).flatten(order="F")
                    if st > 0:
                        S[st * nu * nx:(st + 1) * nu * nx] += (d[st, r] * np.outer(wu, wx)).flatten(order="F")
            mods.append((Q, R, S))
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        wd = t(np.concatenate([w.reshape(-1) for w in W]))
        dp = t(np.concatenate([d.reshape(-1) for d in D]))
        dm = -dp
        mQ, mR, mS = (t(np.concatenate([mm[k] for mm in mods])) for k in range(3))
        # correctness of one update against the refactorization (solve of the same b)
        s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
        s.update_factor(mQ, mR, mS, wd, dp, mm)
        z1 = s.solve(b[:s.kkt_size])
        st_upd = s.instance_status()
        s.factor(mQ, mR, mS, data["A"], data["B"], data["Sigma"])
        z2 = s.solve(b[:s.kkt_size])
        torch.cuda.synchronize()
        ok = bool((st_upd == 0).all())
        rank_exceeded = int((st_upd == 9).sum())
        err = float(torch.linalg.norm(z1 - z2) / torch.linalg.norm(z2)) if ok else None
        # timings (CUDA events on the current stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            s.update_factor(mQ, mR, mS, wd, dp, mm)
            s.update_factor(data["Q"], data["R"], data["S"], wd, dm, mm)
        e1.record(stream)
        torch.cuda.synchronize()
        upd = e0.elapsed_time(e1) / (2 * reps)
        e0.record(stream)
        for _ in range(reps):
            s.factor(mQ, mR, mS, data["A"], data["B"], data["Sigma"])
        e1.record(stream)
        torch.cuda.synchronize()
        ref = e0.elapsed_time(e1) / reps
        out.append({"rows": ("%d per stage" % m) if kind == "per_stage" else m, "update_ms": upd, "refactor_ms": ref,
                    "update_ok": ok, "instances_rank_exceeded": rank_exceeded, "rel_diff_vs_refactor": err})
    s.close()
    return out


def main():
    args = parse()
    FIXED["P"] = args.segments
    FIXED["pcr_tail"] = args.pcr_tail
    FIXED["early_esc"] = args.early_escalation
    FIXED["it_max"] = args.it_max
    if args.launch_shapes:
        FIXED["shapes"] = tuple(int(v) for v in args.launch_shapes.split(","))
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    cfg = inputs.CONFIGS[args.workload]
    prof = dict(WORKLOADS[args.workload])
    if args.steps <= 0:
        args.steps = prof.get("steps", 200)
    if args.graph >= 0:
        prof["graph"] = bool(args.graph)
    nominal = lambda key: cfg[key] if not isinstance(cfg[key], tuple) else "U%s" % (cfg[key],)

    if args.impl == "reference":
        if rank != 0:
            return 0
        if "alm" in cfg:
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the LQ KKT workloads; "
                              "the Newton-step workload has no oracle timing"}))
            return 0
        n = cfg["batch"]
        nrhs = int(cfg["nrhs"])
        dims = inputs.config_dims(cfg, batch=n)
        rates, samples = [], []
        cores = 1
        with OraclePool(args.workload, n, nrhs) as pool:   # every step: its processes keep their instances
            for _ in range(args.warmup):
                pool.step(0.25)
            for _ in range(args.steps):
                r, d, cores = pool.step(1.0)
                rates.append(r)
                samples.append(d)
        value = float(np.mean(rates))
        per_stage = float(np.mean(dims[0]))
        ms = n / value * 1e3
        sample = ("per step, every host core solves its own OCPs of the workload (round-robin over the batch, "
                  "at most 64 per core, cycled) for ~1 s "
                  "of solving (%d OCPs x %d rhs per step on average over %d cores)"
                  % (int(np.mean(samples)), nrhs, cores))
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "ns_per_stage": 1e9 / (value * per_stage),
            "config": {"workload": args.workload, "global_batch": n, "stages_per_ocp": nominal("N"),
                       "nx": nominal("nx"), "nu": nominal("nu"), "nrhs": nrhs,
                       "method": "cpu oracle (textbook Riccati, FP64)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return 0

    import torch
    from paper_2512_09058_gb300 import build, cyq
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    torch.cuda.set_device(local_rank)
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    cyq.load()

    # every rank solves its own batch of the workload (weak scaling)
    n = cfg["batch"]
    if args.instances:
        n = min(n, args.instances)
    batch = inputs.make_batch(args.workload, shard.shard_indices(n, rank))
    nrhs = len(batch.rhs)
    stages = int(batch.N.sum())
    # KKT right-hand sides of the original problem, built on the device by the library
    data, rhs_dev = cyq.to_device(batch)
    s0 = cyq.Solver(batch.N, batch.nx, batch.nu, max_nrhs=nrhs, it_max=0)
    s0.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    b = torch.empty(nrhs * s0.kkt_size, dtype=torch.float64, device="cuda")
    for j in range(nrhs):
        s0.build_rhs(*rhs_dev[j], b=b[j * s0.kkt_size:(j + 1) * s0.kkt_size])
    torch.cuda.synchronize()
    s0.close()
    x0 = rhs_dev[0][3]
    newton = None
    if prof.get("newton"):
        # the Newton system's blocks replace the OCP data in the timing tuners and the residual
        newton, data, b = newton_setup(torch, cyq, batch, data, rhs_dev, shard.shard_indices(n, rank), cfg)

    methods = [m for m in (args.methods.split(",") if args.methods else prof["methods"]) if m]
    sbytes = (batch.Q.nbytes + batch.R.nbytes + batch.S.nbytes + batch.A.nbytes + batch.B.nbytes
              + (batch.Sigma.nbytes if batch.Sigma is not None else 0))
    flush = torch.empty(int(2 * L2_BYTES) // 4, dtype=torch.float32, device="cuda") if sbytes < L2_BYTES else None
    clocks = ClockSampler(local_rank)
    clocks.start()
    results = {m: run_method(torch, cyq, batch, data, b, x0, m, args.steps, args.warmup, dist,
                             graph=prof["graph"], adjoint=prof["adjoint"], flush=flush,
                             tune_segments=prof["tune_segments"], newton=newton) for m in methods}
    clk = clocks.stop()
    # headline: the first listed method that solved every instance to the tolerance
    head = next((m for m in methods if results[m]["status_ok"]), methods[0])
    R = results[head]
    ms = R["total_ms"] / args.steps
    value = shard.job_throughput(batch.size, world, ms)

    e2e = None
    if not args.no_e2e and newton is None:
        e2e_ms, h2d, d2h = run_e2e(torch, cyq, batch, head, max(3, args.steps // 4), args.warmup, data, b,
                                   P=R["P"], adjoint=prof["adjoint"])
        e2e_ms = shard.reduce_time_ms(e2e_ms, dist, device="cuda")
        e2e = {"value": world * batch.size / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and newton is None:
        rate1, done1, el1 = time_oracle(batch, nrhs, budget_s=3.0)
        rate, done, cores = time_oracle_all_cores(args.workload, batch.size, nrhs, budget_s=2.0)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "every host core (one spawned process each) solves its own OCPs of the workload, "
                         "round-robin over the batch (at most 64 per core, cycled), for ~2 s of solving: %d OCPs x %d "
                         "rhs in total; rates summed over the concurrent processes" % (done, nrhs),
               "value_1core": rate1,
               "sample_1core": "first %d OCPs of the workload x %d rhs (%.1f s of one host core)" % (done1, nrhs, el1)}

    peaks = device_peaks(torch, clk)
    dbytes = data_bytes(batch)
    felems = factor_store_elems(batch)

    def phase_rooflines(m, r):
        """Rooflines of the factor phase, the residual and the correction of method m."""
        prec = METHODS[m][0]
        f64 = prec in ("fp64", "fp64_ir32")   # the stage factor runs in float64
        el = 8 if prec == "fp64" else (12 if prec == "fp64_ir32" else 4)   # bytes of the stored factor per element
        fl = 2.0 * batch_factor_fma(batch, r["segments"])
        kname = factor_kernel_name(batch, r, f64)
        tkey = (args.workload, prec, kname)
        fac = roofline_of(kname, fl, dbytes + el * felems, r["factor_ms"], peaks["fp64" if f64 else "fp32"],
                          peaks["hbm"], "fp64" if f64 else "fp32", peaks, NCU_TRAFFIC.get(tkey))
        kk8 = 8.0 * batch.kkt_size
        rname = "k_residual (1 rhs) + k_resid_finalize"   # the phase is timed on one right-hand side
        res = roofline_of(rname, 2.0 * residual_fma(batch), dbytes + 3 * kk8,
                          r["phase"]["residual"], peaks["fp64"], peaks["hbm"], "fp64", peaks,
                          NCU_TRAFFIC.get((args.workload, prec, rname)))
        cel = 8 if prec == "fp64" else 4   # the correction's factor
        nux = np.asarray(batch.nx, np.int64) + np.asarray(batch.nu, np.int64)
        cfl = 2.0 * nrhs * float((np.asarray(batch.N, np.int64) * (2 * nux * nux + 2 * np.asarray(batch.nx) * nux)).sum())
        team = cel == 4 and (r.get("path") or {}).get("sweep_persistent", False)
        cname = ("k_sweep_team<true> + k_cr_solve + k_sweep_team<false> (%d rhs)" if team else
                 "k_solve_backward + k_cr_solve + k_solve_forward (%d rhs)") % nrhs
        cor = roofline_of(cname, cfl, 2.0 * cel * felems + nrhs * 4 * kk8, r["phase"]["correction"],
                          peaks["fp64" if cel == 8 else "fp32"], peaks["hbm"], "fp64" if cel == 8 else "fp32", peaks,
                          NCU_TRAFFIC.get((args.workload, prec, cname)))
        return {"factor": fac, "residual": res, "correction": cor}

    variants = {}
    for m, r in results.items():
        msm = r["total_ms"] / args.steps
        rl = phase_rooflines(m, r) if r["phase"]["correction"] is not None else None
        variants[m] = {"value": world * batch.size / (msm / 1e3), "ms_per_step": msm,
                       "factor_ms": r["factor_ms"], "solve_ms": r["solve_ms"],
                       "residual_ms": r["phase"]["residual"], "correction_ms": r["phase"]["correction"],
                       "ns_per_stage": msm * 1e6 / stages,
                       "max_rel_residual": r["stats"]["max_rel_residual"],
                       "max_certified": r["stats"]["max_certified"],
                       "refine_steps": r["stats"]["refine_steps"], "status_ok": r["status_ok"],
                       "segments_per_ocp": [int(r["segments"].min()), int(r["segments"].max())],
                       "segments_tuned": r["P"] is not None,
                       "threads_per_item": r["shapes"], "factor_path": r["path"],
                       "workspace_bytes": r["workspace_bytes"],
                       "escalation_segments_per_ocp": r["escalation_segments"]}
        if rl is not None:
            variants[m]["factor_gflops"] = rl["factor"]["algorithmic_flops"] / (r["factor_ms"] / 1e3) / 1e9
            variants[m]["rooflines"] = {k: {kk: v[kk] for kk in ("bound", "achieved", "unit", "frac", "ms")}
                                        for k, v in rl.items()}
    # recompute mode against the stored-factor form of the same method: device memory saved,
    # time added per step
    recompute = None
    for m in results:
        if m in RECOMPUTE and m.replace("_recompute", "") in results:
            a, c = results[m.replace("_recompute", "")], results[m]
            recompute = {"method": m, "chunks": RECOMPUTE[m], "workspace_bytes_stored": a["workspace_bytes"],
                         "workspace_bytes_recompute": c["workspace_bytes"],
                         "saved_bytes": a["workspace_bytes"] - c["workspace_bytes"],
                         "ms_per_step_stored": a["total_ms"] / args.steps,
                         "ms_per_step_recompute": c["total_ms"] / args.steps,
                         "time_added_ms": (c["total_ms"] - a["total_ms"]) / args.steps}
    rl = phase_rooflines(head, R)
    # the dominant part of the step: the factor phase against the residual and the correction
    # times the number of refinement steps (an upper bound of their share: later steps skip the
    # instances already at the tolerance)
    nsteps = max(1, R["stats"]["refine_steps"] + 1)
    share = {"factor": R["factor_ms"], "residual": R["phase"]["residual"] * nsteps,
             "correction": R["phase"]["correction"] * nsteps}
    dominant = max(share, key=share.get)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp64_ir32": "f64+f32", "fp32_refine": "f32+f64"}[METHODS[head][0]], "data": "synthetic",
        "ns_per_stage": ms * 1e6 / stages,
        "config": {"workload": args.workload, "global_batch": world * batch.size,
                   "stages_per_ocp": nominal("N"), "nx": nominal("nx"), "nu": nominal("nu"), "nrhs": nrhs,
                   "method": head, "cuda_graph": prof["graph"], "adjoint": prof["adjoint"],
                   "pcr_tail_levels": args.pcr_tail,
                   "parallelism": "dp%d" % world,
                   "l2": ("inputs larger than L2 (%.0f MB float64 data per GPU)" % (sbytes / 1e6))
                   if flush is None else "L2 flushed between steps (%.1f MB float64 data per GPU < L2)" % (sbytes / 1e6)},
        "max_rel_residual": R["stats"]["max_rel_residual"],
        "max_certified": R["stats"]["max_certified"],
        "refine_steps": R["stats"]["refine_steps"],
        "status_ok": R["status_ok"],
        "roofline": dict(rl[dominant], part=dominant),
        "rooflines": rl,
        "peaks": {k: peaks[k] for k in ("sms", "ghz", "fp64", "fp32", "hbm", "hbm_source")},
        "variants": variants,
        "recompute": recompute,
        "gpu_launches": R["launches_per_step"] * args.steps,
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    if args.update_sweep and rank == 0:
        out["update_crossover"] = update_crossover(torch, cyq, batch, data, b)
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
