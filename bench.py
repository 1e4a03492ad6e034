#!/usr/bin/env python
"""Throughput of the staggered RBF-FD Navier-Stokes fractional step on GB300.

Workload: lid-driven cavity at Re = 10^4 on a jittered 1000 x 1000 P-lattice
(1,000,000 pressure nodes, ~3,000,000 velocity nodes), (n, m, q) = (28, 7, 3),
dt = 2e-4, from rest.  A step is one full fractional step (convection,
Crank-Nicolson viscous solves, divergence, pressure Poisson solve, pressure,
correction) through rbffd_step.  The headline is the FP64 path (FP64 weights,
vectors and Krylov recurrences, FP32 multigrid preconditioner, solves to 1e-10
relative residual); the MIXED path (FP32 SpMVs and inner Krylov iterations,
FP64 refinement to the same residual) is timed beside it on the same box.

The timed steps follow --spinup steps from rest (a developed start) and
--warmup steps.  Prints one JSON line.  `--impl reference` times the CPU
oracle instead; `--profile-step` and `--profile-ops` are profiler captures.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NS time steps/s at 1M nodes (mixed vs FP64 GPU); stencil SpMV % HBM peak"
UNIT = "steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=1000, help="P-lattice side (n x n P-nodes)")
    ap.add_argument("--re", type=float, default=1.0e4)
    ap.add_argument("--dt", type=float, default=2e-4)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--max-iter", type=int, default=400000)
    ap.add_argument("--spinup", type=int, default=200,
                    help="untimed steps from rest before the warm-up steps (a developed "
                         "start; the pressure iteration count of the first steps is not typical)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variants", action="store_true",
                    help="also time the exactly projecting step beside the paper's")
    ap.add_argument("--inner-tol", type=float, default=1e-2,
                    help="relative tolerance of the FP32 inner solves (MIXED)")
    ap.add_argument("--only", choices=["both", "mixed", "fp64"], default="both")
    ap.add_argument("--profile-ops", action="store_true",
                    help="profiler capture of the operator kernels: the V->V operators of an "
                         "n x n cavity, then between cudaProfilerStart/Stop three "
                         "rbffd_apply_op launches of D_x with FP64 and three with FP32 weights "
                         "and one rbffd_build_weights of --weights-sample V-nodes; prints the "
                         "launch sizes")
    ap.add_argument("--weights-sample", type=int, default=200000)
    ap.add_argument("--ensemble", type=int, default=64,
                    help="members of the batched ensemble timed beside the headline (0: none)")
    ap.add_argument("--ens-n", type=int, default=316,
                    help="P-lattice side of the ensemble's cavities (316: 100k P-nodes)")
    ap.add_argument("--ens-dt", type=float, default=2.5e-4,
                    help="time step of the ensemble (stable for Re 100 to 5000 at 316^2)")
    ap.add_argument("--ens-steps", type=int, default=10)
    ap.add_argument("--profile-ensemble", action="store_true",
                    help="profiler capture: the batched ensemble (--ensemble members on an "
                         "--ens-n cavity) after --warmup steps, then one ensemble step between "
                         "cudaProfilerStart/Stop; prints its statistics")
    ap.add_argument("--wake", type=int, default=0,
                    help="the cylinder wake of Section 5.2 instead of the benchmark: this many "
                         "steps (dt 0.005, Re --wake-re) from the impulsive start on the "
                         "paper-sized layout, drag and lift every 10 steps; prints a summary "
                         "(and writes the history to --wake-out)")
    ap.add_argument("--wake-re", type=float, default=100.0)
    ap.add_argument("--wake-out", default="")
    ap.add_argument("--profile-step", action="store_true",
                    help="profiler capture: set up, take --warmup steps, then one step between "
                         "cudaProfilerStart/Stop (for ncu --profile-from-start off); prints its "
                         "statistics instead of the benchmark line")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers
def replica_seed(rank: int) -> int:
    """Seed of the cavity a rank simulates: replicas of the workload, one per GPU."""
    return 2 + rank


def max_over_ranks(x: float, world: int, device="cuda") -> float:
    """The largest value over all ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(steps: int, world: int, ms_max: float) -> float:
    """Steps per second of the whole job: every rank's steps over the slowest rank's time."""
    return steps * world / (ms_max * 1e-3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append([time.time()] + parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self, windows=()):
        """Samples taken inside the (start, end) wall-clock windows (all if none)."""
        rows = [r[1:] for r in self.rows
                if not windows or any(a <= r[0] <= b for a, b in windows)]
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# The source text that defines the pressure-solve SpMV: the tile-staging
# helpers and the kernel itself (step.cu, between these markers).  Its hash
# keys the committed DRAM-traffic capture, so that a change to the kernel, and
# only to the kernel, retires the counters.
SPMV_SOURCE_MARKERS = {
    # the pressure SpMV: the tile-staging helpers and k_spmv_pc
    "k_spmv_pc": (
        ("// ------------------------------------------------ staged ELL tiles (bulk copies)",
         "// ----------------------------------------------------------- Krylov kernels"),
        ("// Preconditioned-solve SpMVs with the operand",
         "// x += alpha (zp + kap_p) + omega (zs + kap_s)"),
    ),
    # the viscous SpMV (direct loads): the row gather and k_spmv_p
    "k_spmv_p": (
        ("// sum_s w[s][i] * x[idx[s][i]] for one or two vectors sharing the stencil,",
         "// ------------------------------------------------ staged ELL tiles (bulk copies)"),
        ("// v = A p ; reduce (rh, v).", "// s = r - alpha v ; reduce (s, s) and sum(s)"),
    ),
}


def spmv_source_sha(kernel_key: str = "k_spmv_pc") -> str:
    """Fingerprint of the source of the kernel a traffic record belongs to."""
    family = "k_spmv_pc" if kernel_key.startswith("k_spmv_pc") else "k_spmv_p"
    src = open(os.path.join(ROOT, "paper_2206_06495_gb300", "csrc", "step.cu")).read()
    h = hashlib.sha256()
    for a, b in SPMV_SOURCE_MARKERS[family]:
        i = src.index(a)
        h.update(src[i:src.index(b, i)].encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_key: str, rows: int):
    """DRAM bytes per launch of a kernel from the committed ncu summary, scaled
    to `rows`, or None when the kernel's source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        sha = spmv_source_sha(kernel_key)
        for line in open(path):
            line = line.split("#")[0].split()
            if len(line) >= 4 and line[0] == kernel_key and line[3] == sha:
                return float(line[1]) / float(line[2]) * rows
    except (OSError, ValueError):
        pass
    return None


# ----------------------------------------------------------- CPU baseline
# The CPU oracle as it stands, timed on this machine's host cores in a child
# process (BLAS threads pinned to one): fractional steps of a 150 x 150 cavity
# sample (the largest whose set-up, with the sparse LU of the paper, ends in
# well under a minute), the stencil-weight build of the benchmark's own V->V
# family on a sample of its nodes (one thread, and all cores through a spawn
# pool over independent stencils), and 10 CSR SpMVs of D^(V,V)_x over all of
# its rows.  Nothing here is extrapolated except the step rate, which is also
# given per node and scaled to the benchmark's node count by node count.
ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import rbffd_oracle as O
from paper_2206_06495_gb300 import nodesets as ns

out = {{}}
nd = ns.jittered_cavity({n}, 2)
t0 = time.time()
fs = O.FractionalStep(nd, Re={re}, dt={dt})
out["setup_s"] = time.time() - t0
st = fs.initial_state()
gu, gv = O.lid_bc(nd)
for _ in range({warm}):
    st = fs.step(st, gu, gv)
t0 = time.time()
for _ in range({steps}):
    st = fs.step(st, gu, gv)
out.update(M=nd.M, N=nd.N, step_s=(time.time() - t0) / {steps})
if {full}:
    big = ns.jittered_cavity({n_full}, 2)
    t0 = time.time()
    iv = O.knn(big.vx, big.vy, big.vx, big.vy, 28)
    out["knn_s"] = time.time() - t0
    out["knn_n"] = big.N
    ns_w = min({n_weights}, big.N)
    ops = (O.OP_DX, O.OP_DY, O.OP_LAP)
    t0 = time.time()
    O.build_weights(big.vx[:ns_w], big.vy[:ns_w], big.vx, big.vy, 28, 7, 3, ops, idx=iv[:ns_w])
    out["weights_s"] = time.time() - t0
    out["weights_n"] = ns_w
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    per = 8192
    n_all = min(big.N, cores * 4 * per)
    jobs = [(np.stack([big.vx[i:i + per], big.vy[i:i + per]], -1),
             np.stack([big.vx[iv[i:i + per]], big.vy[iv[i:i + per]]], -1), 7, 3, ops)
            for i in range(0, n_all, per)]
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.starmap(O.stencil_weights, jobs[:cores])  # workers warm
        t0 = time.time()
        pool.starmap(O.stencil_weights, jobs)
        out["weights_all_s"] = time.time() - t0
    out.update(weights_all_n=n_all, cores=cores)
    w = np.random.default_rng(0).standard_normal((big.N, 28))
    D = O.csr(iv, w, big.N)
    f = np.random.default_rng(1).standard_normal(big.N)
    D @ f
    t0 = time.time()
    for _ in range(10):
        D @ f
    out.update(spmv_s=(time.time() - t0) / 10, spmv_rows=big.N)
print(json.dumps(out))
"""


def host_cpu():
    """Host core count and CPU model name."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.startswith("Model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return os.cpu_count() or 1, model or "unknown"


def oracle_sample(n=150, steps=5, warm=1, re=1e4, dt=2e-4, full=False, n_full=1000,
                  n_weights=50000):
    """Run the oracle snippet in a child process with one BLAS thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1")
    code = ORACLE_SNIPPET.format(root=ROOT, n=n, re=re, dt=dt, warm=warm, steps=steps,
                                 full=bool(full), n_full=n_full, n_weights=n_weights)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         timeout=1500)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline_record(M_target, n_full, re, dt, n=150, steps=5, warm=1):
    r = oracle_sample(n=n, steps=steps, warm=warm, re=re, dt=dt, full=True, n_full=n_full)
    cores, model = host_cpu()
    scaled = (1.0 / r["step_s"]) * (r["M"] / M_target)
    return {"value": scaled, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"oracle fractional steps (sparse-LU solves, as the paper) on a {n}x{n} "
                       f"P-lattice cavity sample (M={r['M']}, N={r['N']}), Re={re:g}, dt={dt:g}: "
                       f"{steps} timed after {warm} warm-up, {r['step_s'] * 1e3:.1f} ms/step "
                       f"measured, one thread; value = that rate scaled to M={M_target} by "
                       f"node count"),
            "host": {"nproc": cores, "cpu_model": model},
            "measured": {
                "steps": {"M": r["M"], "N": r["N"], "steps_per_s": 1.0 / r["step_s"],
                          "node_steps_per_s": r["M"] / r["step_s"], "threads": 1,
                          "setup_s": r["setup_s"]},
                "weights": {"family": f"V->V D_x, D_y, Lap (28, 7, 3) of the {n_full}x{n_full} "
                                      f"cavity",
                            "knn_stencils_per_s": r["knn_n"] / r["knn_s"],
                            "stencils_per_s_1thread": r["weights_n"] / r["weights_s"],
                            "sample_1thread": r["weights_n"],
                            "stencils_per_s_all_cores": r["weights_all_n"] / r["weights_all_s"],
                            "sample_all_cores": r["weights_all_n"], "cores": r["cores"]},
                "spmv": {"rows": r["spmv_rows"], "ms": r["spmv_s"] * 1e3,
                         "achieved_gbs_352B_per_row": r["spmv_rows"] * 352 / r["spmv_s"] / 1e9,
                         "threads": 1, "kind": "scipy CSR D^(V,V)_x @ f, 10 timed"}}}


# ----------------------------------------------------------------- GPU arm
def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2206_06495_gb300 import build
    from paper_2206_06495_gb300 import nodesets as ns
    build.build()
    from paper_2206_06495_gb300 import rbffd as R

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    ctx = R.Context(28, 7, 3)
    nd = ns.jittered_cavity(args.n, replica_seed(rank))
    t_setup = time.time()
    flows = {}
    for name, prec in (("mixed", R.PREC_MIXED), ("fp64", R.PREC_FP64)):
        if args.only not in ("both", name):
            continue
        if not flows:
            base = R.flow_from_nodes(ctx, nd, Re=args.re, dt=args.dt, precision=prec,
                                     tol=args.tol, inner_tol=args.inner_tol,
                                     max_iter=args.max_iter)
            flows[name] = base
        else:
            b0 = next(iter(flows.values()))
            flows[name] = R.Flow(N=b0.N, M=b0.M, tensors=b0.tensors, Re=args.re, dt=args.dt,
                                 precision=prec, tol=args.tol, inner_tol=args.inner_tol,
                                 max_iter=args.max_iter)
    torch.cuda.synchronize()
    t_setup = time.time() - t_setup
    gu_h = np.zeros(nd.N)
    gu_h[nd.v_wall == ns.WALL_TOP] = 1.0
    gu = torch.as_tensor(gu_h, device="cuda")
    gv = torch.zeros(nd.N, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    res = {}
    sampler = ClockSampler(local) if rank == 0 else None
    failed = {}
    windows = []
    if sampler:
        # nvidia-smi's start-up stalls the driver for a moment: start it before
        # the warm-up steps and let it deliver its first sample
        sampler.start()
        t_wait = time.time()
        while not sampler.rows and time.time() - t_wait < 5.0:
            time.sleep(0.05)
    def spun_up(c, flow):
        """A state after --spinup + --warmup steps from rest in context c."""
        st = R.State.zeros(flow)
        flow.profile = 0
        for _ in range(args.spinup + args.warmup):
            R.step(c, flow, st, gu, gv, 1)
        return st

    for name, flow in flows.items():
        try:
            st = spun_up(ctx, flow)
        except R.RbffdError as e:
            failed[name] = str(e)[:300]
            continue
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        agg = {"poisson_iters": 0, "helm_iters": 0, "launches": 0, "spmv_ms": 0.0,
               "spmv_launches": 0, "refinements": 0}
        iters = []
        w0 = time.time()
        e0.record(stream)
        try:
            for _ in range(args.steps):
                s = R.step(ctx, flow, st, gu, gv, 1)
                iters.append(s["poisson_iters"])
                for k in agg:
                    agg[k] += s[k]
        except R.RbffdError as e:
            failed[name] = str(e)[:300]
            continue
        e1.record(stream)
        barrier()
        windows.append((w0, time.time()))
        ms = max_over_ranks(e0.elapsed_time(e1), world)
        res[name] = {"ms": ms, "agg": agg, "relres": s["poisson_relres"]}
        # per-launch CUDA events around every pressure-solve SpMV need eager
        # launches (the timed steps replay CUDA graphs): one more step, profiled
        flow.profile = 1
        s = R.step(ctx, flow, st, gu, gv, 1)
        flow.profile = 0
        res[name]["spmv_ms"], res[name]["spmv_launches"] = s["spmv_ms"], s["spmv_launches"]
        res[name]["spmv_batch_ms"] = s["spmv_batch_ms"]
        res[name]["spmv_batch_launches"] = s["spmv_batch_launches"]
        res[name]["vspmv_batch_ms"] = s["vspmv_batch_ms"]
        res[name]["vspmv_batch_launches"] = s["vspmv_batch_launches"]
        res[name]["state"] = st
        # End to end, on the same steps: a second context takes the same steps
        # from rest (the path is deterministic, so it reaches the same state
        # with the same solver history), then the timed steps are taken again
        # with the step's boundary data copied in from pinned host memory and
        # the velocity copied out, every step.
        ctx2 = R.Context(28, 7, 3)
        st2 = spun_up(ctx2, flow)
        gu_p = torch.empty(nd.N, dtype=torch.float64, pin_memory=True)
        gv_p = torch.empty(nd.N, dtype=torch.float64, pin_memory=True)
        gu_p.copy_(torch.as_tensor(gu_h))
        gv_p.zero_()
        u_p = torch.empty(nd.N, dtype=torch.float64, pin_memory=True)
        v_p = torch.empty(nd.N, dtype=torch.float64, pin_memory=True)
        gu_d = torch.empty_like(gu)
        gv_d = torch.empty_like(gv)
        barrier()
        e2e_iters = []
        w0 = time.time()
        e0.record(stream)
        for _ in range(args.steps):
            gu_d.copy_(gu_p, non_blocking=True)
            gv_d.copy_(gv_p, non_blocking=True)
            e2e_iters.append(R.step(ctx2, flow, st2, gu_d, gv_d, 1)["poisson_iters"])
            u_p.copy_(st2.u, non_blocking=True)
            v_p.copy_(st2.v, non_blocking=True)
        e1.record(stream)
        barrier()
        windows.append((w0, time.time()))
        res[name]["e2e_ms"] = max_over_ranks(e0.elapsed_time(e1), world)
        res[name]["e2e_same_steps"] = e2e_iters == iters
        res[name]["iters"] = iters
        res[name]["e2e_iters"] = e2e_iters
        ctx2.close()
        del st2
        torch.cuda.empty_cache()
    # The exactly projecting step (composed pressure operator D^(P,V) G0,
    # discretely divergence-free velocity) on the same workload, timed the
    # same way (spin-up, warm-up, device-resident steps); reported beside the
    # paper's step, not as the headline.
    variants = {}
    if args.variants and flows:
        b0 = next(iter(flows.values()))
        for name, prec in (("mixed", R.PREC_MIXED), ("fp64", R.PREC_FP64)):
            if args.only not in ("both", name):
                continue
            fl = R.Flow(N=b0.N, M=b0.M, tensors=b0.tensors, Re=args.re, dt=args.dt,
                        precision=prec, tol=args.tol, inner_tol=args.inner_tol,
                        max_iter=args.max_iter, projection=R.PROJ_EXACT)
            stv = None
            try:
                stv = spun_up(ctx, fl)
                barrier()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                it, flux = [], []
                w0 = time.time()
                e0.record(stream)
                for _ in range(args.steps):
                    sv = R.step(ctx, fl, stv, gu, gv, 1)
                    it.append(sv["poisson_iters"])
                    flux.append(sv["wall_flux"])
                e1.record(stream)
                barrier()
                windows.append((w0, time.time()))
                msv = max_over_ranks(e0.elapsed_time(e1), world)
                variants[name] = {"steps_per_s": args.steps / (msv * 1e-3),
                                  "ms_per_step": msv / args.steps,
                                  "poisson_iters_per_step": sum(it) / args.steps,
                                  "wall_flux_max": max(abs(x) for x in flux)}
            except R.RbffdError as e:
                variants[name] = {"error": str(e)[:300]}
            del stv
            torch.cuda.empty_cache()
    if sampler:
        sampler.stop()

    # stencil SpMV on its own: D^(V,V)_x over all V-nodes, FP64 and FP32 weights
    spmv = {}
    t = flows[next(iter(flows))].tensors
    idx, wx = t["vv_idx"], t["vv_dx"]
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    for wname, w in (("fp64", wx), ("fp32", wx.float())):
        x = torch.randn(nd.N, dtype=torch.float64 if wname == "fp64" else torch.float32,
                        device="cuda")
        y = torch.empty_like(x)
        for _ in range(3):
            R.apply_op(ctx, idx, w, nd.N, nd.N, x, y)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20
        a.record(stream)
        for _ in range(reps):
            R.apply_op(ctx, idx, w, nd.N, nd.N, x, y)
        b.record(stream)
        torch.cuda.synchronize()
        per = a.elapsed_time(b) / reps * 1e-3
        k = 28
        wb = 8 if wname == "fp64" else 4
        bytes_row = k * 4 + k * wb + 2 * wb  # idx, weights, y written, x read once
        gbs = nd.N * bytes_row / per / 1e9
        thr, bps = R.apply_op_shape(ctx, idx, w, nd.N, nd.N, x.dtype)
        spmv[wname] = {"rows": nd.N, "bytes_per_row": bytes_row, "us": per * 1e6,
                       "achieved_gbs": gbs, "frac": gbs / hbm,
                       "launch": {"threads": thr, "blocks_per_sm": bps, "picked_by": "autotuner"}}

    # batched weight build: V->V stencils (3 operators) of this node set, and the
    # measured FP64 FMA peak it is held against
    fp64_peak = R.probe_fma(ctx, R.F64, 8192)
    fp32_peak = R.probe_fma(ctx, R.F32, 8192)
    vx, vy = flows[next(iter(flows))].tensors["vx"], flows[next(iter(flows))].tensors["vy"]
    R.build_weights(ctx, vx[:4096].contiguous(), vy[:4096].contiguous(), vx, vy,
                    R.OP_DX | R.OP_DY | R.OP_LAP)  # warm
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    R.build_weights(ctx, vx, vy, vx, vy, R.OP_DX | R.OP_DY | R.OP_LAP)
    b.record(stream)
    torch.cuda.synchronize()
    wsec = a.elapsed_time(b) * 1e-3
    S, nrhs = 28 + 10, 3
    flops_sys = (2.0 / 3.0) * S ** 3 + 2.0 * nrhs * S * S
    weights = {"stencils": nd.N, "system": S, "operators": nrhs, "seconds": wsec,
               "stencils_per_s": nd.N / wsec, "bound": "alu",
               "achieved_gflops": nd.N * flops_sys / wsec / 1e9,
               "fp64_peak_gflops": fp64_peak, "fp32_peak_gflops": fp32_peak,
               "frac": nd.N * flops_sys / wsec / 1e9 / fp64_peak if fp64_peak else None,
               "flops_per_system": flops_sys, "note": "k-NN search included in the time"}
    # The (n, m, q) parameter study (Section 4) on a 200,000-stencil sample of
    # this node set's V->V family: weights of D_x and the Laplacian plus their
    # per-node relative errors on the test function, per triple, then the
    # condition numbers of the chosen triple's local systems.
    from paper_2206_06495_gb300.sweep import parameter_sweep
    ns_s = min(200000, nd.N)
    sx, sy = vx[:ns_s].contiguous(), vy[:ns_s].contiguous()
    triples = [(28, 3, 3), (28, 5, 3), (28, 7, 3), (28, 9, 3), (28, 7, 1), (28, 7, 2),
               (28, 7, 4), (21, 7, 3), (35, 7, 3)]
    parameter_sweep(sx[:4096].contiguous(), sy[:4096].contiguous(), vx, vy, triples[:1])
    torch.cuda.synchronize()
    t0 = time.time()
    rows = parameter_sweep(sx, sy, vx, vy, triples)
    torch.cuda.synchronize()
    sweep_s = time.time() - t0
    cctx = R.Context(28, 7, 3)
    cidx, _, _ = R.build_weights(cctx, sx, sy, vx, vy, R.OP_DX)
    R.stencil_condition(cctx, sx[:4096].contiguous(), sy[:4096].contiguous(), vx, vy,
                        cidx[:, :4096].contiguous())
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    cond = R.stencil_condition(cctx, sx, sy, vx, vy, cidx)
    b.record(stream)
    torch.cuda.synchronize()
    cond_ms = a.elapsed_time(b)
    sweep = {"stencils_per_triple": ns_s, "triples": len(triples), "seconds": sweep_s,
             "stencil_triples_per_s": ns_s * len(triples) / sweep_s,
             "timing": "wall clock around the whole sweep (context creation, k-NN, weights "
                       "and error kernels per triple), after one warm-up triple",
             "E": {f"{r['n']},{r['m']},{r['q']}": {"dx": float(r["E_dx"]),
                                                    "lap": float(r["E_lap"])} for r in rows},
             "cond_28_7_3": {"ms": cond_ms, "stencils_per_s": ns_s / (cond_ms * 1e-3),
                             "median": float(cond.median()), "max": float(cond.max())}}
    cctx.close()
    ensemble = ensemble_record(R, args, hbm, peak_kind) if args.ensemble > 0 else None
    if rank != 0:
        return None
    if not res:
        return {"metric": METRIC, "value": None, "unit": UNIT, "error": failed}
    # the headline is the FP64 path (the faster one since the pressure and
    # viscous solves start from extrapolated guesses); MIXED is timed beside it
    head = "fp64" if "fp64" in res else "mixed"
    r = res[head]
    value = whole_job_rate(args.steps, world, r["ms"])
    e2e = whole_job_rate(args.steps, world, r["e2e_ms"])
    agg = r["agg"]
    # roofline of the pressure solve's SpMV (k_spmv_pc): the algorithmic bytes
    # of a k = 28 stencil SpMV row (k column indices, k weights, the operand
    # read once, the output written: 232 B in FP32, 352 B in FP64); the
    # kernel also streams three fused per-row vectors (the dot-product
    # partner, the row sum A 1 and the rank-one column), listed apart
    k = 28
    if head == "mixed":
        bytes_row, fused, key = 8 * k + 2 * 4, 3 * 4, "k_spmv_pc_fp32"  # FP32 inner solves
    else:
        bytes_row, fused, key = 12 * k + 2 * 8, 3 * 8, "k_spmv_pc_fp64"
    # launch duration: back-to-back launches after each profiled pressure solve
    # (primary), and in the solve itself between graph-node events (which add
    # their own gaps)
    per_launch_ms = r["spmv_batch_ms"] / max(r["spmv_batch_launches"], 1)
    in_step_ms = r["spmv_ms"] / max(r["spmv_launches"], 1)
    achieved = (nd.M * bytes_row / (per_launch_ms * 1e-3) / 1e9
                if r["spmv_batch_launches"] > 0 and per_launch_ms > 0 else None)
    in_step = (nd.M * bytes_row / (in_step_ms * 1e-3) / 1e9
               if r["spmv_launches"] > 0 and in_step_ms > 0 else None)
    traffic = profiled_traffic(key, nd.M)
    pres_roof = {"kernel": key, "bound": "hbm", "achieved": achieved, "peak": hbm,
                 "unit": "GB/s", "frac": achieved / hbm if achieved else None,
                 "traffic": traffic,
                 "bytes_per_row": bytes_row, "fused_bytes_per_row": fused,
                 "frac_with_fused": ((achieved * (bytes_row + fused) / bytes_row) / hbm
                                     if achieved else None),
                 "rows": nd.M, "peak_kind": peak_kind,
                 "launches_timed": r["spmv_batch_launches"],
                 "us_per_launch": per_launch_ms * 1e3,
                 "timing": "CUDA events around 20 back-to-back launches of this kernel on "
                           "the operator and vectors of each pressure solve of one "
                           "profiled step right after the timed steps",
                 "in_step": {"us_per_launch": in_step_ms * 1e3, "achieved": in_step,
                             "frac": in_step / hbm if in_step else None,
                             "launches_timed": r["spmv_launches"],
                             "timing": "external event-record graph nodes around every "
                                       "launch inside the profiled step's solves"}}
    roofline = pres_roof
    if head == "fp64":
        roofline = viscous_roofline(r, nd.N, k, hbm, peak_kind, fp64_peak, pres_roof) or pres_roof
    iters_ok = r.get("e2e_same_steps")
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if head == "mixed" else "f64",
        "data": "synthetic",
        "config": workload_config(args, nd.M, nd.N, head, world),
        "gpu_launches": agg["launches"],
        "poisson_iters_per_step": agg["poisson_iters"] / args.steps,
        "helm_iters_per_step": agg["helm_iters"] / args.steps,
        "setup_s": t_setup,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 2 * nd.N * 8,
                "d2h_bytes_per_step": 2 * nd.N * 8,
                "same_steps": iters_ok,
                "how": "a second context takes the same spin-up and warm-up steps from rest "
                       "(deterministic path: same state and solver history), then the timed "
                       "steps again through rbffd_step with wall data copied in from pinned "
                       "host memory and u, v copied out every step; same_steps: equal "
                       "pressure iteration counts step by step"},
        "roofline": roofline,
        "spmv": spmv,
        "weights": weights,
        "sweep": sweep,
        "ensemble": ensemble,
        "clocks": sampler.summary(windows) if sampler else None,
        "failed": failed,
    }
    if "mixed" in res and "fp64" in res:
        # the mixed-precision fields against the FP64 path after the same steps
        a, b = res["mixed"]["state"], res["fp64"]["state"]

        def rel(x, y):
            return float((x - y).abs().max() / y.abs().max().clamp_min(1e-300))
        out["mixed_vs_fp64"] = {
            "steps": args.spinup + args.warmup + args.steps + 1,
            "u_max_abs": float((a.u - b.u).abs().max()), "v_max_abs": float((a.v - b.v).abs().max()),
            "u_rel": rel(a.u, b.u), "v_rel": rel(a.v, b.v),
            "p_rel": rel(a.p, b.p), "pt_rel": rel(a.pt, b.pt)}
    if variants:
        out["exact_projection"] = dict(
            variants, note="projection = RBFFD_PROJ_EXACT: pressure operator D^(P,V) G0 "
                           "(composed, read directly with its runtime width), velocity "
                           "discretely divergence-free at every P-node; same workload, "
                           "spin-up and timing as the headline")
    for name in res:
        rr = res[name]
        out[name] = {"steps_per_s": args.steps / (rr["ms"] * 1e-3),
                     "ms_per_step": rr["ms"] / args.steps,
                     "poisson_iters_per_step": rr["agg"]["poisson_iters"] / args.steps,
                     "refinements_per_step": rr["agg"]["refinements"] / args.steps,
                     "e2e_steps_per_s": args.steps / (rr["e2e_ms"] * 1e-3),
                     "e2e_same_steps": rr["e2e_same_steps"],
                     "poisson_iters": rr["iters"]}
    if world == 1 and not args.no_cpu_baseline:
        try:
            out["cpu_baseline"] = cpu_baseline_record(nd.M, args.n, args.re, args.dt)
        except Exception as e:  # reported, never fatal
            out["cpu_baseline"] = {"error": str(e)[:300]}
    return out


def ensemble_record(R, args, hbm, peak_kind):
    """E independent cavities (Re ~ U[100, 5000], lid speed 1 + 0.05 N(0, 1),
    seeded) on one node set, stepped together by rbffd_ensemble_step, against
    the same members stepped one at a time by rbffd_step (the first four
    members, each with its own step plan, scaled to E).  The batched pressure
    SpMV (every operator row read once for all E members) goes on the
    roofline: algorithmic bytes per launch = M (28 * 4 + 28 * 4) for the
    operator + M E (4 + 4) for the operand read once and the output."""
    import numpy as np
    import torch

    from paper_2206_06495_gb300 import nodesets as ns
    E, dt, steps = args.ensemble, args.ens_dt, args.ens_steps
    nd = ns.jittered_cavity(args.ens_n, 4)
    rng = np.random.default_rng(4)
    Re = [float(r) for r in rng.uniform(100.0, 5000.0, E)]
    lid = 1.0 + 0.05 * rng.standard_normal(E)
    ctx = R.Context(28, 7, 3)
    try:
        flow = R.flow_from_nodes(ctx, nd, Re=1.0, dt=dt, precision=R.PREC_MIXED, tol=args.tol,
                                 inner_tol=args.inner_tol, max_iter=args.max_iter)
        top = nd.v_wall == ns.WALL_TOP
        gu_h = np.zeros((nd.N, E))
        gu_h[top, :] = lid[None, :]
        gu = torch.as_tensor(gu_h.ravel(), device="cuda")
        gv = torch.zeros_like(gu)
        st = R.ensemble_zeros(flow, E)
        R.ensemble_step(ctx, flow, Re, st, gu, gv, max(args.warmup, 3))
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s = R.ensemble_step(ctx, flow, Re, st, gu, gv, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        flow.profile = 1
        sp = R.ensemble_step(ctx, flow, Re, st, gu, gv, 1)
        flow.profile = 0
        per_ms = sp["spmv_batch_ms"] / max(sp["spmv_batch_launches"], 1)
        k = 28
        bytes_launch = nd.M * (k * 4 + k * 4) + nd.M * E * (4 + 4)
        achieved = bytes_launch / (per_ms * 1e-3) / 1e9 if per_ms > 0 else None
        # the same members one at a time, in the ensemble's precision (MIXED)
        # and in FP64 (the faster single-flow path)
        nm = min(4, E)
        g1 = torch.zeros(nd.N, dtype=torch.float64, device="cuda")
        topd = torch.as_tensor(top, device="cuda")
        seq = {}
        for pname, prec in (("mixed", R.PREC_MIXED), ("fp64", R.PREC_FP64)):
            seq_ms, seq_iters = 0.0, 0
            for e in range(nm):
                fl1 = R.Flow(N=flow.N, M=flow.M, tensors=flow.tensors, Re=Re[e], dt=dt,
                             precision=prec, tol=args.tol, inner_tol=args.inner_tol,
                             max_iter=args.max_iter)
                s1 = R.State.zeros(fl1)
                g1.zero_()
                g1[topd] = float(lid[e])
                g2 = torch.zeros_like(g1)
                R.step(ctx, fl1, s1, g1, g2, max(args.warmup, 3))
                torch.cuda.synchronize()
                e0.record(stream)
                r1 = R.step(ctx, fl1, s1, g1, g2, steps)
                e1.record(stream)
                torch.cuda.synchronize()
                seq_ms += e0.elapsed_time(e1)
                seq_iters += r1["poisson_iters"]
            seq[pname] = (nm * steps / (seq_ms * 1e-3), seq_iters / (nm * steps))
        seq_rate = seq["mixed"][0]
        seq_iters_step = seq["mixed"][1]
        rate = E * steps / (ms * 1e-3)
        return {"members": E, "M": nd.M, "N": nd.N, "dt": dt, "steps": steps,
                "re_range": [min(Re), max(Re)],
                "member_steps_per_s": rate, "ms_per_step": ms / steps,
                "poisson_iters_per_step": s["poisson_iters"] / steps,
                "poisson_sweeps_per_step": s["refinements"] / steps,
                "helm_iters_per_step": s["helm_iters"] / steps,
                "launches_per_step": s["launches"] / steps,
                "sequential_steps_per_s": seq_rate,
                "sequential_poisson_iters_per_step": seq_iters_step,
                "speedup_vs_sequential": rate / seq_rate,
                "sequential_fp64_steps_per_s": seq["fp64"][0],
                "sequential_fp64_poisson_iters_per_step": seq["fp64"][1],
                "speedup_vs_best_sequential": rate / max(seq_rate, seq["fp64"][0]),
                "spmm_roofline": {"kernel": "e_spmv_v (batched pressure SpMV)", "bound": "hbm",
                                  "bytes_per_member_row": (k * 8) / E + 8,
                                  "us_per_launch": per_ms * 1e3, "achieved": achieved,
                                  "peak": hbm, "unit": "GB/s", "peak_kind": peak_kind,
                                  "frac": achieved / hbm if achieved else None},
                "how": "CUDA events around the timed steps after warm-up; the same flows one "
                       "at a time through rbffd_step (first four members, each with its own "
                       "step plan) give the sequential rates, in MIXED (the ensemble's "
                       "precision) and in FP64; MIXED precision, solves to "
                       f"{args.tol:g}; the SpMV timed alone in 20 back-to-back launches"}
    except R.RbffdError as e:
        return {"members": E, "error": str(e)[:300]}
    finally:
        ctx.close()


def viscous_roofline(r, rows, k, hbm, hbm_kind, fp64_peak_gflops, pressure):
    """Roofline of the viscous SpMV (k_spmv_p: two right sides, FP64, direct
    loads), the largest kernel of the FP64 step (its launch list is in
    profiles/step_launches_fp64_cavity1m.md), from the profiled step's 20
    back-to-back launches per viscous solve.  It is bound by the FP64 pipe:
    per row k FMAs and one dot-product FMA per right side, 4 (k + 1) flops,
    against the FP64 FMA rate rbffd_probe_fma measures in the same run.  Its
    HBM side: k indices and k weights once for both right sides, each operand
    read once and each output written (368 B at k = 28), plus the fused
    dot-product partner of each right side.  None without the timing."""
    if not r.get("vspmv_batch_launches") or not r.get("vspmv_batch_ms") or not fp64_peak_gflops:
        return None
    v_ms = r["vspmv_batch_ms"] / r["vspmv_batch_launches"]
    vrow, vfused = 12 * k + 2 * (8 + 8), 2 * 8
    gbs = rows * vrow / (v_ms * 1e-3) / 1e9
    flops_row = 4 * (k + 1)
    tflops = rows * flops_row / (v_ms * 1e-3) / 1e12
    peak = fp64_peak_gflops / 1e3
    return {"kernel": "k_spmv_p_fp64_2rhs", "bound": "alu", "achieved": tflops, "peak": peak,
            "unit": "TFLOP/s", "frac": tflops / peak,
            "peak_kind": "FP64 FMA throughput measured by rbffd_probe_fma in this run "
                         "(nominal 1.25 TFLOP/s)",
            "flops_per_row": flops_row,
            "traffic": profiled_traffic("k_spmv_p_fp64_2rhs", rows),
            "hbm": {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                    "bytes_per_row": vrow, "fused_bytes_per_row": vfused,
                    "frac_with_fused": gbs * (vrow + vfused) / vrow / hbm,
                    "peak_kind": hbm_kind},
            "rows": rows, "launches_timed": r["vspmv_batch_launches"],
            "us_per_launch": v_ms * 1e3,
            "timing": "CUDA events around 20 back-to-back launches of this kernel on the "
                      "operator and vectors of each viscous solve of one profiled step right "
                      "after the timed steps",
            "pressure_spmv": pressure}


def workload_config(args, M, N, precision, world):
    """The benchmark's `config`, shared by both arms."""
    return {"workload": f"lid-driven cavity Re={args.re:g}, jittered {args.n}x{args.n} "
                        f"P-lattice (M={M}, N={N}), (n,m,q)=(28,7,3), "
                        f"dt={args.dt:g}, timed after {args.spinup} spin-up and "
                        f"{args.warmup} warm-up steps from rest, pressure/viscous solves "
                        f"to {args.tol:g} relative residual (the FP64 path's viscous "
                        f"solves to 1e-3 of it, not below 1e-13)",
            "precision": precision, "parallelism": f"replicas{world}",
            "spinup_steps": args.spinup,
            "l2": "working set (operators ~7 GB) exceeds L2; no flush needed"}


def run_reference(args):
    """The CPU oracle as it stands, on a 150 x 150 sample of the workload, one
    thread: --warmup untimed and --steps timed fractional steps."""
    rank, world, local = dist_env()
    if rank != 0:
        return None
    n_sample = 150
    t0 = time.time()
    r = oracle_sample(n=n_sample, steps=args.steps, warm=args.warmup, re=args.re, dt=args.dt)
    from paper_2206_06495_gb300 import nodesets as ns
    full = ns.jittered_cavity(args.n, replica_seed(0))
    M_target = full.M
    value = (1.0 / r["step_s"]) * (r["M"] / M_target)
    cores, model = host_cpu()
    sample = (f"CPU oracle fractional steps (sparse-LU solves) on a {n_sample}x{n_sample} "
              f"P-lattice cavity sample (M={r['M']}, N={r['N']}), {args.steps} timed after "
              f"{args.warmup} warm-up, one thread, {r['step_s'] * 1e3:.1f} ms/step measured; "
              f"value = that rate scaled to M={M_target} by node count")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            # the sample's own measured time per step (the timed region is
            # steps * ms_per_step); value is per step of the full workload
            "ms_per_step": r["step_s"] * 1e3,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, full.M, full.N, "fp64", world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample, "host": {"nproc": cores, "cpu_model": model}},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "setup_s": r["setup_s"], "wall_s": time.time() - t0}


def profile_step(args):
    """One fractional step of the benchmark workload between cudaProfilerStart
    and cudaProfilerStop, after --warmup steps (plan, graphs and caches warm)."""
    import numpy as np
    import torch

    from paper_2206_06495_gb300 import build
    from paper_2206_06495_gb300 import nodesets as ns
    build.build()
    from paper_2206_06495_gb300 import rbffd as R

    prec = R.PREC_FP64 if args.only == "fp64" else R.PREC_MIXED
    ctx = R.Context(28, 7, 3)
    nd = ns.jittered_cavity(args.n, 2)
    flow = R.flow_from_nodes(ctx, nd, Re=args.re, dt=args.dt, precision=prec, tol=args.tol,
                             inner_tol=5e-3, max_iter=args.max_iter)
    gu_h = np.zeros(nd.N)
    gu_h[nd.v_wall == ns.WALL_TOP] = 1.0
    gu = torch.as_tensor(gu_h, device="cuda")
    gv = torch.zeros_like(gu)
    st = R.State.zeros(flow)
    for _ in range(args.warmup):
        R.step(ctx, flow, st, gu, gv, 1)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    s = R.step(ctx, flow, st, gu, gv, 1)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    return {"profile_step": "mixed" if prec == R.PREC_MIXED else "fp64", "M": nd.M, "N": nd.N,
            "stats": s}


def profile_ensemble(args):
    """One batched ensemble step between cudaProfilerStart and cudaProfilerStop
    (for ncu --profile-from-start off), after --warmup steps: the members,
    Reynolds numbers, wall data and time step of bench.py's ensemble record."""
    import numpy as np
    import torch

    from paper_2206_06495_gb300 import build
    from paper_2206_06495_gb300 import nodesets as ns
    build.build()
    from paper_2206_06495_gb300 import rbffd as R

    E = args.ensemble
    nd = ns.jittered_cavity(args.ens_n, 4)
    rng = np.random.default_rng(4)
    Re = [float(r) for r in rng.uniform(100.0, 5000.0, E)]
    lid = 1.0 + 0.05 * rng.standard_normal(E)
    ctx = R.Context(28, 7, 3)
    flow = R.flow_from_nodes(ctx, nd, Re=1.0, dt=args.ens_dt, precision=R.PREC_MIXED,
                             tol=args.tol, inner_tol=args.inner_tol, max_iter=args.max_iter)
    gu_h = np.zeros((nd.N, E))
    gu_h[nd.v_wall == ns.WALL_TOP, :] = lid[None, :]
    gu = torch.as_tensor(gu_h.ravel(), device="cuda")
    gv = torch.zeros_like(gu)
    st = R.ensemble_zeros(flow, E)
    R.ensemble_step(ctx, flow, Re, st, gu, gv, max(args.warmup, 1))
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    s = R.ensemble_step(ctx, flow, Re, st, gu, gv, 1)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    return {"profile_ensemble": E, "M": nd.M, "N": nd.N, "dt": args.ens_dt, "stats": s}


def wake_run(args):
    """The cylinder wake (Section 5.2) on the paper-sized layout: --wake steps
    of dt 0.005 from the impulsive start (u = 1 off the cylinder), MIXED
    precision, solves to 1e-10; C_D and C_L every 10 steps.  The summary gives
    the cost per step and, over the last quarter of the run, the mean drag,
    the lift amplitude and the Strouhal number of the lift."""
    import numpy as np
    import torch

    from paper_2206_06495_gb300 import build
    from paper_2206_06495_gb300 import nodesets as ns
    build.build()
    from paper_2206_06495_gb300 import rbffd as R
    from paper_2206_06495_gb300 import wake

    nd = ns.cylinder_wake()
    ctx = R.Context(28, 7, 3)
    flow = wake.wake_flow(ctx, nd, Re=args.wake_re, dt=0.005, precision=R.PREC_MIXED,
                          tol=1e-10, inner_tol=1e-2)
    gu, gv = wake.wake_data(nd)
    st = R.State.zeros(flow)
    cyl = torch.as_tensor(nd.v_wall == ns.WALL_CYLINDER, device="cuda")
    st.u.copy_(torch.where(cyl, torch.zeros_like(gu), torch.ones_like(gu)))
    rows, _ = wake.surface_rows(nd)
    hist, iters = [], 0
    t0 = time.time()
    for j in range(0, args.wake, 10):
        s = R.step(ctx, flow, st, gu, gv, min(10, args.wake - j))
        iters += s["poisson_iters"]
        cd, cl = wake.forces(ctx, flow, st, nd, rows)
        hist.append((min(j + 10, args.wake) * 0.005, cd, cl))
    wall = time.time() - t0
    h = np.array(hist)
    if args.wake_out:
        np.savetxt(args.wake_out, h, header="t C_D C_L")
    tail = h[h[:, 0] >= 0.75 * h[-1, 0]]
    try:
        st_num = wake.strouhal(tail[:, 0], tail[:, 2])
    except ValueError:
        st_num = None
    return {"wake": {"Re": args.wake_re, "M": nd.M, "N": nd.N, "steps": args.wake,
                     "t_end": float(h[-1, 0]), "ms_per_step": 1e3 * wall / args.wake,
                     "poisson_iters_per_step": iters / args.wake,
                     "window": [float(tail[0, 0]), float(tail[-1, 0])],
                     "C_D_mean": float(tail[:, 1].mean()),
                     "C_L_amplitude": float(0.5 * (tail[:, 2].max() - tail[:, 2].min())),
                     "St": st_num,
                     "C_D_at": {f"{t:g}": float(h[np.argmin(np.abs(h[:, 0] - t)), 1])
                                for t in (5, 10, 20, 40, 60, 80, 100) if t <= h[-1, 0]}}}


def profile_ops(args):
    """Operator kernels of the benchmark's node family between
    cudaProfilerStart/Stop (for ncu --profile-from-start off)."""
    import numpy as np
    import torch

    from paper_2206_06495_gb300 import build
    from paper_2206_06495_gb300 import nodesets as ns
    build.build()
    from paper_2206_06495_gb300 import rbffd as R

    ctx = R.Context(28, 7, 3)
    nd = ns.jittered_cavity(args.n, 2)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")  # noqa: E731
    vx, vy = d(nd.vx), d(nd.vy)
    idx, w, _ = R.build_weights(ctx, vx, vy, vx, vy, R.OP_DX | R.OP_DY | R.OP_LAP)
    wx64, wx32 = w[0].contiguous(), w[0].float().contiguous()
    f = torch.randn(nd.N, dtype=torch.float64, device="cuda")
    f32 = f.float()
    y64, y32 = torch.empty_like(f), torch.empty_like(f32)
    ns_w = min(args.weights_sample, nd.N)
    sx, sy = vx[:ns_w].contiguous(), vy[:ns_w].contiguous()
    for _ in range(2):  # autotune and warm both shapes
        R.apply_op(ctx, idx, wx64, nd.N, nd.N, f, y64)
        R.apply_op(ctx, idx, wx32, nd.N, nd.N, f32, y32)
    R.build_weights(ctx, sx, sy, vx, vy, R.OP_DX | R.OP_DY | R.OP_LAP)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    for _ in range(3):
        R.apply_op(ctx, idx, wx64, nd.N, nd.N, f, y64)
    for _ in range(3):
        R.apply_op(ctx, idx, wx32, nd.N, nd.N, f32, y32)
    R.build_weights(ctx, sx, sy, vx, vy, R.OP_DX | R.OP_DY | R.OP_LAP)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    return {"profile_ops": True, "rows": nd.N, "weights_stencils": ns_w,
            "spmv_fp64_shape": R.apply_op_shape(ctx, idx, wx64, nd.N, nd.N, f.dtype),
            "spmv_fp32_shape": R.apply_op_shape(ctx, idx, wx32, nd.N, nd.N, f32.dtype)}


def main():
    args = parse()
    if args.profile_ops:
        print(json.dumps(profile_ops(args)))
        return
    if args.profile_step:
        print(json.dumps(profile_step(args)))
        return
    if args.profile_ensemble:
        print(json.dumps(profile_ensemble(args)))
        return
    if args.wake:
        print(json.dumps(wake_run(args)))
        return
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
