#!/usr/bin/env python3
"""KKT factor+solve benchmark on one node.

Workload (default): 1024 independent linear-quadratic OCPs, N = 64 stages,
nx = 12, nu = 4, stage cross terms S and diagonal regularisation Sigma
log-uniform in [1e-6, 1e6]; one factorization + 4 right-hand sides per OCP.
One step = factor all OCPs + solve the 4 right-hand sides, with the inputs
resident in device memory (218 MB of float64 data, larger than the 129 MB L2).

Methods (each timed over the same K steps):
  fp64_refine  float64 factor + solve, float64 residual and refinement until
               ||b - Kz|| / ||b|| <= 1e-10 for every OCP and right-hand side
               (the headline: float64 arithmetic, certified at the metric's gate)
  fp64         plain float64 factor + solve (no residual computed)
  fp32_refine  float32 factor + solve, float64 residual + refinement to 1e-10

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

from paper_2512_09058_gb300 import inputs  # noqa: E402

METRIC = "KKT factor+solve/sec and ns/stage at rel. residual ≤1e-10; % of roofline"
UNIT = "OCP factor+solve/s"
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07   # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz = 1258.6
WORKLOAD = "batch1024_n64_nx12_nu4"
# method -> (factor precision, refinement step budget).  Float64 refinement
# converges in one step here; float32 needs ~5 at cond(K) ~ 1e11.
METHODS = {"fp64": ("fp64", 0), "fp64_refine": ("fp64", 3), "fp32_refine": ("fp32_refine", 8)}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="cyq", choices=["cyq", "reference"])
    p.add_argument("--workload", default=WORKLOAD, choices=sorted(inputs.CONFIGS))
    p.add_argument("--methods", default="fp64_refine,fp64,fp32_refine")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    return p.parse_args()


def riccati_fma_per_stage(nx, nu):
    """Serial factorized Riccati, FMA = 1 (paper Sec. 4.5): 1/2 nux nx^2 + 1/2 nux^2 nx + 1/6 nux^3."""
    nux = nx + nu
    return 0.5 * nux * nx * nx + 0.5 * nux * nux * nx + nux ** 3 / 6.0


def solve_fma_per_stage(nx, nu):
    """Segment solve sweeps per right-hand side (backward + forward, P = 1):
    nu^2 + 2 nx nu + 2 nx^2 + 2 nux nx."""
    return nu * nu + 2 * nx * nu + 2 * nx * nx + 2 * (nx + nu) * nx


def residual_fma_per_stage(nx, nu):
    """Float64 residual rows per right-hand side: R, S (twice), B (twice), Q, A (twice)."""
    return nu * nu + 2 * nu * nx + 2 * nx * nu + nx * nx + 2 * nx * nx


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
def time_oracle(batch, nrhs, min_seconds=2.0, max_instances=None):
    import oracle   # CPU-baseline / reference leg only
    insts = batch.instances if max_instances is None else batch.instances[:max_instances]
    bs = [np.stack([oracle.build_rhs(x, *x.rhs[j]) for j in range(nrhs)]) for x in insts]
    done, t0 = 0, time.perf_counter()
    while True:
        for x, b in zip(insts, bs):
            oracle.riccati_solve(x, b)
        done += len(insts)
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    return done / el, done, el


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_method(torch, cyq, batch, data, b, method, steps, warmup, rank, world, dist):
    precision, it_max = METHODS[method]
    nrhs = len(batch.rhs)
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision=precision, max_nrhs=nrhs, it_max=it_max)
    z = torch.empty_like(b)
    stream = torch.cuda.current_stream()

    def step():
        s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
        s.solve(b, z, nrhs=nrhs)

    s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
    launches_factor = s.launch_count()
    s.solve(b, z, nrhs=nrhs)
    launches_solve = s.launch_count()
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t_start.record(stream)
    for i in range(steps):
        ev[i][0].record(stream)
        s.factor(data["Q"], data["R"], data["S"], data["A"], data["B"], data["Sigma"])
        ev[i][1].record(stream)
        s.solve(b, z, nrhs=nrhs)
        ev[i][2].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    total_ms = t_start.elapsed_time(t_end)
    if dist is not None:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    factor_ms = [e[0].elapsed_time(e[1]) for e in ev]
    solve_ms = [e[1].elapsed_time(e[2]) for e in ev]
    status = s.instance_status()
    st = s.stats()
    if it_max == 0:   # plain solve: measure the residual it reached (outside the timed region)
        worst = 0.0
        for j in range(nrhs):
            kk = s.kkt_size
            rel = s.residual(b[j * kk:(j + 1) * kk], z[j * kk:(j + 1) * kk])
            worst = max(worst, float(rel.max().item()))
        st["max_rel_residual"] = worst
    s.close()
    return dict(total_ms=total_ms, factor_ms=float(np.mean(factor_ms)), solve_ms=float(np.mean(solve_ms)),
                status_ok=bool((status == 0).all()), stats=st,
                launches_per_step=launches_factor + launches_solve)


def run_e2e(torch, cyq, batch, method, steps, warmup):
    """Same metric through the public API with host buffers: every step copies
    the data and (q, r, c, x_init) from pinned host memory, builds the KKT
    right-hand sides, factors, solves and copies z back to pinned memory."""
    precision, it_max = METHODS[method]
    nrhs = len(batch.rhs)
    s = cyq.Solver(batch.N, batch.nx, batch.nu, precision=precision, max_nrhs=nrhs, it_max=it_max)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    host = {k: pin(getattr(batch, k)) for k in ("Q", "R", "S", "A", "B")}
    host["Sigma"] = pin(batch.Sigma) if batch.Sigma is not None else None
    host_rhs = [[pin(x) for x in r] for r in batch.rhs]
    dev = {k: (torch.empty_like(v, device="cuda") if v is not None else None) for k, v in host.items()}
    dev_rhs = [[torch.empty_like(x, device="cuda") for x in r] for r in host_rhs]
    kk = s.kkt_size
    b = torch.empty(nrhs * kk, dtype=torch.float64, device="cuda")
    z = torch.empty_like(b)
    z_host = torch.empty(nrhs * kk, dtype=torch.float64).pin_memory()
    h2d = sum(v.numel() * 8 for v in host.values() if v is not None) + sum(x.numel() * 8 for r in host_rhs for x in r)
    d2h = z_host.numel() * 8

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
        z_host.copy_(z, non_blocking=True)

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


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    cfg = inputs.CONFIGS[args.workload]

    if args.impl == "reference":
        if rank != 0:
            return 0
        batch = inputs.make_batch(args.workload)
        nrhs = len(batch.rhs)
        stages = int(batch.N.sum())
        for _ in range(args.warmup):
            time_oracle(batch, nrhs, min_seconds=0.0, max_instances=16)
        rate, done, el = time_oracle(batch, nrhs, min_seconds=0.0)   # one pass per step
        t_steps = []
        for _ in range(args.steps):
            r, d, e = time_oracle(batch, nrhs, min_seconds=0.0)
            t_steps.append(e)
        ms = 1e3 * float(np.mean(t_steps))
        value = batch.size / (ms / 1e3)
        sample = "the full workload (%d OCPs x %d rhs) per step, one host core" % (batch.size, nrhs)
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "ns_per_stage": ms * 1e6 / stages,
            "config": {"workload": args.workload, "global_batch": batch.size, "stages_per_ocp": int(cfg["N"]),
                       "nx": cfg["nx"], "nu": cfg["nu"], "nrhs": nrhs, "method": "cpu oracle (textbook Riccati, FP64)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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
    batch = inputs.make_batch(args.workload, range(rank * n, (rank + 1) * n)) if world > 1 else \
        inputs.make_batch(args.workload)
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

    methods = [m for m in args.methods.split(",") if m]
    clocks = ClockSampler(local_rank)
    clocks.start()
    results = {m: run_method(torch, cyq, batch, data, b, m, args.steps, args.warmup, rank, world, dist)
               for m in methods}
    clk = clocks.stop()
    head = methods[0]
    R = results[head]
    ms = R["total_ms"] / args.steps
    value = world * batch.size / (ms / 1e3)

    e2e = None
    if not args.no_e2e:
        e2e_ms, h2d, d2h = run_e2e(torch, cyq, batch, head, max(3, args.steps // 4), args.warmup)
        if dist is not None:
            t = torch.tensor([e2e_ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_ms = float(t.item())
        e2e = {"value": world * batch.size / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, done, el = time_oracle(batch, nrhs, min_seconds=2.0)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "whole %d-OCP workload x %d rhs, repeated for %.1f s (%d OCPs), one host core"
                         % (batch.size, nrhs, el, done)}

    nx, nu = int(cfg["nx"]), int(cfg["nu"])
    fl_factor = 2.0 * riccati_fma_per_stage(nx, nu) * stages
    achieved = fl_factor / (R["factor_ms"] / 1e3) / 1e9
    variants = {}
    for m, r in results.items():
        msm = r["total_ms"] / args.steps
        variants[m] = {"value": world * batch.size / (msm / 1e3), "ms_per_step": msm,
                       "factor_ms": r["factor_ms"], "solve_ms": r["solve_ms"],
                       "ns_per_stage": msm * 1e6 / stages,
                       "max_rel_residual": r["stats"]["max_rel_residual"],
                       "refine_steps": r["stats"]["refine_steps"], "status_ok": r["status_ok"],
                       "factor_gflops": (fl_factor / (r["factor_ms"] / 1e3) / 1e9)}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "ns_per_stage": ms * 1e6 / stages,
        "config": {"workload": args.workload, "global_batch": world * batch.size, "stages_per_ocp": int(cfg["N"]),
                   "nx": nx, "nu": nu, "nrhs": nrhs, "method": head, "parallelism": "dp%d" % world,
                   "l2": "inputs larger than L2 (%.0f MB float64 data per GPU)"
                         % ((batch.Q.nbytes + batch.R.nbytes + batch.S.nbytes + batch.A.nbytes + batch.B.nbytes
                             + (batch.Sigma.nbytes if batch.Sigma is not None else 0)) / 1e6)},
        "max_rel_residual": R["stats"]["max_rel_residual"],
        "refine_steps": R["stats"]["refine_steps"],
        "roofline": {"kernel": "k_factor_segments<double,32>", "bound": "alu", "achieved": achieved,
                     "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s", "frac": achieved / FP64_PEAK_GFLOPS,
                     "traffic": None,
                     "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz (recipe's 1.25 TF nominal)"},
        "variants": variants,
        "gpu_launches": R["launches_per_step"] * args.steps,
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
