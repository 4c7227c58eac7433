"""Benchmark of the direct PP N-body hot path on GB300.

Workload (one "step"): one KDK leapfrog step (Eq. 5-7: the O(N^2) force and
potential sum of Eq. 1-2 plus the fused O(N) update) and the Eq. 8-10
diagnostics, on the exponential-disk + Plummer-halo model at N = 2^20
(eps = 0.02, dt = 5e-4, seed 20180113), in binary64 (the headline `value`)
and in the mixed FP32-pair / FP64-accumulate mode (reported beside it).
Ginteractions/s counts N^2 pair evaluations per force evaluation (the self
pair included in the count; 20 flop per interaction where flops are quoted).

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Multi-GPU runs (torchrun) are independent replicas: each rank steps its own
copy of the workload; value = all ranks' interactions / slowest rank's time.
--impl reference times the FP64 CPU oracle on the host cores instead, on a
bounded sample of particles of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Ginteractions/s at N=2^20, FP64 vs mixed at stated force error; p99 step latency"
UNIT = "Ginteractions/s"
FLOP_PER_INTERACTION = 20
N_FULL = 2 ** 20
EPS, DT = 0.02, 5e-4
# Work each force kernel issues on the pipe that bounds it, per interaction
# (counted from the kernels' source, confirmed by ncu instruction counts):
# FP64 pipe instructions of the binary64 paths: 9 one-sided (3 DADD, 3 DFMA for
# |d|^2 + eps^2, 3 DFMA for the acceleration sums; the potential sum is an
# integer add); 12 per pair evaluated once for both particles (both potential
# sums integer adds), i.e. 6 per interaction.
FP64_INSTR_PER_INTERACTION = {False: 9, True: 6}
# FP32 FMA-pipe lane operations: mixed 13 (3 differences, 3 FMAs for
# |d|^2 + eps^2, m y, y^2, m y^3, 3 FMAs and 1 add into the sums; two j per
# packed instruction); F64E float-float 162 one-sided, 112 per interaction
# when each pair is evaluated once (ncu: 111.8 packed FMA-pipe instructions
# per pair evaluation).
MIXED_LANEOPS_PER_INTERACTION = 13
F64E_LANEOPS_PER_INTERACTION = {False: 162, True: 112}


# DRAM traffic of one FP64 force launch at N = 2^20 (dram__bytes_read.sum +
# dram__bytes_write.sum from one full-size ncu capture; see the k_force_f64 DRAM
# profile summary).  It is reported only while the kernel's source is the one
# that was captured: `src_sha` hashes rsqrt_recip_sig, mul_sig, body_f64 and
# k_force_f64.
TRAFFIC = {"k_force_f64": {"bytes": 47.05e6 + 62.96e6, "n": 2 ** 20, "src_sha": "01dc06074becbf43"},
           # each pair once, blocks of 384: per force evaluation 1 one-sided launch on the
           # 2731 diagonal blocks + 1365 block diagonals in launches of 8 (pair kernel and
           # combine); bytes of the first launch of each kernel in one full-size capture,
           # the pair and combine launches scaled by 1365 / 8
           "k_force_f64_sym": {"bytes": 34.00e6 + 1365 / 8 * (679.80e6 + 589.80e6), "n": 2 ** 20,
                               "src_sha": "39fcfb6aac42cd11"}}


def _kernel_src_sha(names):
    import hashlib
    src = open(os.path.join(ROOT, "paper_1803_01190_gb300", "csrc", "force.cu")).read()
    parts = []
    for start in names:
        i = src.index(start)
        j = src.index("{", i)
        depth = 0
        for k in range(j, len(src)):
            depth += src[k] == "{"
            depth -= src[k] == "}"
            if depth == 0:
                parts.append(src[i:k + 1])
                break
    return hashlib.sha256("\n".join(parts).encode()).hexdigest()[:16]


def traffic_f64(n, sym=False):
    if sym:
        t = TRAFFIC["k_force_f64_sym"]
        sha = _kernel_src_sha(["__device__ __forceinline__ void rsqrt_recip_sig(",
                               "__device__ __forceinline__ uint64_t mul_sig(",
                               "__device__ __forceinline__ uint64_t add_pos_bits(",
                               "__device__ __forceinline__ void acc_pos(",
                               "__device__ __forceinline__ void scale_pair(",
                               "__device__ __forceinline__ void body_f64_sym(",
                               "__global__ void __launch_bounds__(BT) k_force_f64_sym(",
                               "__global__ void k_sym_combine("])
        return t["bytes"] if (sha == t["src_sha"] and n == t["n"]) else None
    t = TRAFFIC["k_force_f64"]
    sha = _kernel_src_sha(["__device__ __forceinline__ void rsqrt_recip_sig(",
                           "__device__ __forceinline__ uint64_t mul_sig(",
                           "__device__ __forceinline__ void body_f64(",
                           "__global__ void __launch_bounds__(BT) k_force_f64("])
    return t["bytes"] if (sha == t["src_sha"] and n == t["n"]) else None


def workload_desc(n):
    seed = 20180113 if n >= 2 ** 20 else 20180112   # nbody_ics.workload("disk_halo", n)
    return (f"exponential disk (Rd=1, Rmax=5, h=0.05, Q=1.2) + live Plummer halo (a=3), 1:1, "
            f"N={n}, eps={EPS}, KDK dt={DT}, seed {seed}")


# ------------------------------------------------------------------ helpers
class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def max_over_ranks(value, device="cpu"):
    """Largest `value` over all ranks of the default process group (identity
    without one): the slowest replica sets the whole job's time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def sample_rows(n, k, seed=7):
    return np.sort(np.random.default_rng(seed).choice(n, k, replace=False))


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import nbody_ics
    import oracle
    w = nbody_ics.workload("disk_halo", n=N_FULL)
    cores = oracle.max_threads()
    rows_per_step = args.ref_rows
    steps = []
    for k in range(args.warmup + args.steps):
        rows = sample_rows(N_FULL, rows_per_step, seed=100 + k)
        t0 = time.perf_counter()
        oracle.accel(w["pos"], w["mass"], EPS, 1.0, rows=rows, threads=cores)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            steps.append(dt)
    inter = rows_per_step * N_FULL
    value = inter / statistics.mean(steps) / 1e9
    sample = (f"{rows_per_step} sampled i-particles x all {N_FULL} j per step "
              f"(FP64 oracle, Neumaier sums, OpenMP)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(steps) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(N_FULL), "mode": "fp64", "sample_rows": rows_per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def time_mode(nb, torch, w, mode, args, flush, clocks=None):
    """W warm-up + K timed KDK steps (with diagnostics) of one simulation.
    Returns per-step ms, force-kernel ms per launch, launches, diag, sim."""
    n = len(w["mass"])
    sim = nb.Simulation(n, mode=mode, eps=EPS)
    sim.set_state(w["pos"], w["vel"], w["mass"])
    stream = torch.cuda.current_stream()
    diag0 = sim.diagnostics()           # a(t0) and E0
    for _ in range(args.warmup):
        sim.step(DT, 1)
        sim.diagnostics()
    torch.cuda.synchronize()
    if args.world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sim.profile(True)
    sim.profile_read()
    l0 = sim.launch_count
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if clocks:
        clocks.start()
    diags = []
    for k in range(args.steps):
        flush.zero_()                   # evict L2 (buffer larger than L2) between timed steps
        ev[k][0].record(stream)
        sim.step(DT, 1)
        diags.append(sim.diagnostics())
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    launches = sim.launch_count - l0
    fms, fl = sim.profile_read()
    sim.profile(False)
    per_step = [a.elapsed_time(b) for a, b in ev]
    return dict(per_step=per_step, force_ms=fms / max(fl, 1), force_launches=fl,
                launches=launches, diag0=diag0, diags=diags, sim=sim, clocks=clk)


def e2e_mode(nb, torch, w, mode, steps, warmup):
    """The Eq. 1-2 force call through the C ABI with pinned host buffers: the
    H2D copy of positions and masses and the D2H copy of accelerations and
    potentials are inside the timed region."""
    import ctypes
    n = len(w["mass"])
    pos = torch.tensor(w["pos"]).pin_memory()
    mass = torch.tensor(w["mass"]).pin_memory()
    acc = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    pot = torch.empty((n,), dtype=torch.float64).pin_memory()
    sim = nb.Simulation(n, mode=mode, eps=EPS)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    call = lambda: nb.check(nb.lib.nbody_accel(sim._h, ptr(pos), ptr(mass), ptr(acc), ptr(pot), 0),  # noqa: E731
                            "nbody_accel")
    for _ in range(warmup):
        call()
    ts = []
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        call()                          # synchronising: outputs are on the host when it returns
        ts.append(time.perf_counter() - t0)
    sim.close()
    return dict(sec=statistics.mean(ts), h2d=pos.numel() * 8 + mass.numel() * 8,
                d2h=acc.numel() * 8 + pot.numel() * 8)


def run_serving(args, fp64_kernel="fp64"):
    """Serving workload: Poisson arrivals (200/s) of independent Plummer or
    disk + halo simulations, N log-uniform in [2^10, 2^16], FP64 or MIXED
    50/50, 100 KDK steps each, through the continuous-batching server for a
    bounded wall-clock window.  Offered load (~1e13 interactions/s) exceeds
    one GPU, so the queue grows; reported: per-mode tick (= per-step)
    latency p50/p99, aggregate throughput, admitted/completed/queued."""
    from paper_1803_01190_gb300 import serve
    reqs = serve.poisson_requests(int(200 * args.serve_seconds) + 1, rate=200.0, seed=20180115,
                                  nsteps=100, dt=DT)
    srv = serve.Server(capacity={"fp64": 2 ** 20, "mixed": 2 ** 22},
                       max_sims={"fp64": 16, "mixed": 64}, autotune=True, keep_state=False,
                       fp64_kernel=fp64_kernel)
    out = srv.run(reqs, duration=args.serve_seconds)
    srv.close()
    out.pop("done")
    out["workload"] = ("Poisson 200 req/s; N log-uniform [2^10, 2^16]; Plummer (eps 0.01) or disk+halo "
                       "(eps 0.02) 50/50; FP64 or mixed 50/50; 100 KDK steps dt=5e-4; seed 20180115")
    out["pools"] = {"fp64": {"capacity": 2 ** 20, "max_sims": 16, "kernel": fp64_kernel},
                    "mixed": {"capacity": 2 ** 22, "max_sims": 64, "kernel": "mixed"}}
    return out


def run_gpu(args):
    import torch
    world, rank, local = dist_setup(args)
    args.world = world
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    import nbody_ics
    import paper_1803_01190_gb300 as nb
    n = args.n
    w = nbody_ics.workload("disk_halo", n=n)
    flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2
    clocks = ClockSampler(local)
    inter = float(n) * n
    # pipe issue rates of this GPU, measured in this run: the roofline denominators
    pipes = nb.measure_pipes()

    fp64 = time_mode(nb, torch, w, "fp64", args, flush, clocks=clocks)
    mixed = time_mode(nb, torch, w, "mixed", args, flush)
    f64e = time_mode(nb, torch, w, "f64e", args, flush)

    def agg(per_step):
        return max_over_ranks(statistics.mean(per_step), device="cuda")

    ms64 = agg(fp64["per_step"])
    msmx = agg(mixed["per_step"])
    msfe = agg(f64e["per_step"])
    value = world * inter / (ms64 * 1e-3) / 1e9
    value_mx = world * inter / (msmx * 1e-3) / 1e9

    # end to end through the C ABI with host buffers
    e2e64 = e2e_mode(nb, torch, w, "fp64", steps=args.e2e_steps, warmup=args.e2e_warmup)
    e2emx = e2e_mode(nb, torch, w, "mixed", steps=max(args.steps, 3), warmup=args.warmup)
    serving = run_serving(args) if args.serve_seconds > 0 else None
    serving_f64e = run_serving(args, fp64_kernel="f64e") if args.serve_seconds > 0 else None

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
        return

    # CPU baseline and force error: the oracle on sampled particles of the
    # current (post-step) state of both runs
    import oracle
    cores = oracle.max_threads()
    p64, _, _, _ = fp64["sim"].get_state()
    a64, pot64 = fp64["sim"].get_accel()
    pmx, _, _, _ = mixed["sim"].get_state()
    amx, _ = mixed["sim"].get_accel()
    rows = sample_rows(n, args.ref_rows)
    t0 = time.perf_counter()
    ao64, po64, smag = oracle.accel(p64, w["mass"], EPS, 1.0, rows=rows, threads=cores)
    cpu_s = time.perf_counter() - t0
    aomx, _, _ = oracle.accel(pmx, w["mass"], EPS, 1.0, rows=rows, threads=cores)
    pfe, _, _, _ = f64e["sim"].get_state()
    afe, _ = f64e["sim"].get_accel()
    aofe, _, smag_fe = oracle.accel(pfe, w["mass"], EPS, 1.0, rows=rows, threads=cores)
    cpu_value = len(rows) * n / cpu_s / 1e9
    t0 = time.perf_counter()
    oracle.plain_accel(p64, w["mass"], EPS, 1.0, rows=rows, threads=cores)
    plain_s = time.perf_counter() - t0

    def errs(a, ao):
        e = np.linalg.norm(a[rows] - ao, axis=1) / np.linalg.norm(ao, axis=1)
        return {"rms": float(np.sqrt((e ** 2).mean())), "max": float(e.max())}

    U = 2.0 ** -53
    gate = np.linalg.norm(a64[rows] - ao64, axis=1) <= (
        1e-12 * np.linalg.norm(ao64, axis=1) + 4 * U * np.sqrt(n) * smag)

    def drift(d0, ds):
        E0, P0, L0 = d0["E"], d0["P"], d0["L"][2]
        return {"dE_over_E0": max(abs(d["E"] / E0 - 1) for d in ds),
                "dP_abs": max(float(np.linalg.norm(d["P"] - P0)) for d in ds),
                "dLz_over_Lz0": max(abs(d["L"][2] / L0 - 1) for d in ds)}

    fms = fp64["force_ms"]
    sym = fp64["sim"].get_symmetric()[1]
    achieved_tf = inter * FLOP_PER_INTERACTION / (fms * 1e-3) / 1e12
    per = sorted(fp64["per_step"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms64, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(n), "n": n, "mode": "fp64", "scheme": "kdk",
                   "l2": "flushed between timed steps (256 MB device write)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "launch": {**fp64["sim"].get_launch(), "each_pair_once": sym}},
        "p50_step_ms": float(np.percentile(per, 50)), "p99_step_ms": float(np.percentile(per, 99)),
        "roofline": roofline_fp64(n, sym, fms, ms64, pipes),
        "gpu_launches": fp64["launches"] * world,
        "clocks": fp64["clocks"],
        "e2e": {"value": world * inter / e2e64["sec"] / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": e2e64["h2d"], "d2h_bytes_per_step": e2e64["d2h"],
                "call": "nbody_accel (host pinned buffers), FP64", "steps": args.e2e_steps},
        "cpu_baseline": {"value": cpu_value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{len(rows)} sampled i-particles x all {n} j of the FP64 "
                                   f"state after the timed steps ({cpu_s:.1f} s)",
                         "plain_loop": {"value": len(rows) * n / plain_s / 1e9, "unit": UNIT,
                                        "cores": cores, "kind": "plain binary64 OpenMP simd loop, "
                                        "no compensation, -O3 (the CPU throughput figure)",
                                        "sample": f"the same {len(rows)} i-particles ({plain_s:.1f} s)"}},
        "pipes": pipes,
        "force_error_vs_oracle": {"fp64": {**errs(a64, ao64), "gate_1e-12_pass": bool(gate.all())},
                                  "f64e": {**errs(afe, aofe), "gate_1e-12_pass_fraction": float(np.mean(
                                      np.linalg.norm(afe[rows] - aofe, axis=1) <= 1e-12 * np.linalg.norm(aofe, axis=1)
                                      + 4 * U * np.sqrt(n) * smag_fe))},
                                  "mixed": errs(amx, aomx), "rows": len(rows)},
        "f64e": {"value": world * inter / (msfe * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": msfe,
                 "speedup_vs_fp64": (world * inter / (msfe * 1e-3) / 1e9) / value,
                 "force_ms_per_launch": f64e["force_ms"],
                 "note": "binary64-class float-float arithmetic on the FP32 pipes (about 48 bits)",
                 "roofline": roofline_fp32_pipe(
                     "k_force_f64e_sym" if f64e["sim"].get_symmetric()[1] else "k_force_f64e",
                     F64E_LANEOPS_PER_INTERACTION[f64e["sim"].get_symmetric()[1]], n, f64e["force_ms"],
                     pipes),
                 "gpu_launches": f64e["launches"] * world, "launch": f64e["sim"].get_launch()},
        "mixed": {"value": value_mx, "unit": UNIT, "ms_per_step": msmx,
                  "speedup_vs_fp64": value_mx / value,
                  "p50_step_ms": float(np.percentile(mixed["per_step"], 50)),
                  "p99_step_ms": float(np.percentile(mixed["per_step"], 99)),
                  "force_ms_per_launch": mixed["force_ms"],
                  "roofline": roofline_fp32_pipe("k_force_mixed", MIXED_LANEOPS_PER_INTERACTION, n,
                                                 mixed["force_ms"], pipes),
                  "order": mixed["sim"].get_order(),
                  "e2e": {"value": world * inter / e2emx["sec"] / 1e9, "unit": UNIT},
                  "gpu_launches": mixed["launches"] * world,
                  "launch": mixed["sim"].get_launch()},
        "drift_over_timed_steps": {"fp64": drift(fp64["diag0"], fp64["diags"]),
                                   "f64e": drift(f64e["diag0"], f64e["diags"]),
                                   "mixed": drift(mixed["diag0"], mixed["diags"])},
        "serving": serving,
        "serving_fp64_requests_on_f64e": serving_f64e,
        "paper_context": {
            "note": "the paper's Table 1, one Tesla K80, its own disk model (not this workload): "
                    "seconds per KDK step at N = 1024K, as N^2 interactions per second",
            "dp_k80_ginteractions_per_s": 1048576.0 ** 2 / 60.0 / 1e9,
            "sp_k80_ginteractions_per_s": 1048576.0 ** 2 / 27.4 / 1e9},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()


def roofline_fp64(n, sym, force_ms, step_ms, pipes):
    """The binary64 force path is bound by the FP64 pipe: achieved = its FP64
    instructions per interaction x N^2 / the force evaluation's CUDA-event
    time; peak = the DFMA issue rate measured in the same run."""
    inter = float(n) * n
    ipi = FP64_INSTR_PER_INTERACTION[sym]
    achieved = inter * ipi / (force_ms * 1e-3) / 1e9
    conv = inter * FLOP_PER_INTERACTION / (force_ms * 1e-3) / 1e12
    return {"bound": "alu", "pipe": "fp64", "kernel": "k_force_f64_sym" if sym else "k_force_f64",
            "achieved": achieved, "peak": pipes["dfma_ginstr_s"], "unit": "G FP64-pipe instr/s",
            "frac": achieved / pipes["dfma_ginstr_s"],
            "peak_source": (f"measured in this run: nbody_measure_pipes DFMA issue rate "
                            f"({pipes['dfma_per_clk_sm']:.3f}/clk/SM x {pipes['sms']:.0f} SMs at "
                            f"{pipes['sm_mhz']:.0f} MHz)"),
            "instr_per_interaction": ipi,
            "traffic": traffic_f64(n, sym),
            "traffic_note": ("DRAM bytes per force evaluation from one full-size ncu capture: mostly the "
                             "per-diagonal row/column slices of the each-pair-once schedule, O(N^2/384), far "
                             "above the O(N) algorithmic bytes but ~0.3% of HBM bandwidth over the evaluation"
                             if sym else
                             "DRAM bytes per force evaluation from one full-size ncu capture; the O(N) "
                             "algorithmic bytes (32 B in + partial sums out per particle) mostly stay in L2"),
            "convention_20flop": {"achieved": conv, "peak": 2 * pipes["dfma_ginstr_s"] / 1e3,
                                  "unit": "TFLOP/s", "frac": conv / (2 * pipes["dfma_ginstr_s"] / 1e3),
                                  "note": "20 flop/interaction x N^2 against 2 flop per measured DFMA; "
                                          + ("each pair is evaluated once for both particles, so this "
                                             "can exceed 1" if sym else "")},
            "force_ms_per_launch": force_ms, "force_ms_note": "one force evaluation (all its launches)",
            "force_share_of_step": force_ms / step_ms}


def roofline_fp32_pipe(kernel, laneops, n, force_ms, pipes):
    """Kernels on the binary32 FMA pipes (mixed, F64E): achieved = FMA-pipe lane
    operations per interaction x N^2 / force time; peak = the packed FFMA2
    lane-operation rate measured in the same run."""
    inter = float(n) * n
    achieved = inter * laneops / (force_ms * 1e-3) / 1e9
    conv = inter * FLOP_PER_INTERACTION / (force_ms * 1e-3) / 1e12
    return {"bound": "alu", "pipe": "fp32 fma", "kernel": kernel, "achieved": achieved,
            "peak": pipes["ffma2_glane_s"], "unit": "G FMA-pipe lane-ops/s",
            "frac": achieved / pipes["ffma2_glane_s"], "laneops_per_interaction": laneops,
            "peak_source": (f"measured in this run: nbody_measure_pipes packed FFMA2 lane-op rate "
                            f"({pipes['ffma2_lane_per_clk_sm']:.1f}/clk/SM at {pipes['sm_mhz']:.0f} MHz)"),
            "convention_20flop_tflops": conv, "force_ms_per_launch": force_ms}


def run_peaks(args):
    """The measured pipe rates alone (nbody_measure_pipes), as one JSON line."""
    import torch
    import paper_1803_01190_gb300 as nb
    torch.cuda.set_device(0)
    print(json.dumps({"pipes": nb.measure_pipes(), "gpu": torch.cuda.get_device_name(0)}), flush=True)


def profile_force(args):
    """One force evaluation (Eq. 1-2) of the benchmark workload in one mode and
    nothing else: the command the ncu captures of a single force launch run."""
    import torch
    import nbody_ics
    import paper_1803_01190_gb300 as nb
    w = nbody_ics.workload("disk_halo", n=args.n)
    with nb.Simulation(args.n, mode=args.profile_force, eps=EPS) as sim:
        if args.symmetric != -1:
            sim.set_symmetric(args.symmetric)
        if args.order != "default":
            sim.set_order(args.order)
        sim.accel(w["pos"], w["mass"])
        torch.cuda.synchronize()
    print(json.dumps({"profile_force": args.profile_force, "n": args.n}))


def run_drift(args):
    """Conservation over a long run on the disk + halo model, in the terms of the
    paper's Table 2: max over the run of |E - E0| / |E0|, |P - P0| (absolute)
    and |Lz - Lz0| / |Lz0|, sampled every --drift-every steps (Eq. 8-10 reduced
    on the GPU in binary64 from the mode's own state)."""
    import torch
    import nbody_ics
    import paper_1803_01190_gb300 as nb
    w = nbody_ics.workload("disk_halo", n=args.n)
    dt = args.drift_dt
    out = {"drift": args.drift, "scheme": args.drift_scheme, "n": args.n, "eps": EPS, "dt": dt,
           "steps": args.drift_steps, "every": args.drift_every, "workload": workload_desc(args.n),
           "force_evaluations": args.drift_steps * {"kdk": 1, "fr4": 3, "rk4": 4}[args.drift_scheme]}
    with nb.Simulation(args.n, mode=args.drift, eps=EPS) as sim:
        if args.order != "default":
            sim.set_order(args.order)
        out["order"] = sim.get_order()
        sim.set_state(w["pos"], w["vel"], w["mass"])
        d0 = sim.diagnostics()
        curve = []
        t0 = time.perf_counter()
        done = 0
        log = open(args.drift_out, "w") if args.drift_out else None
        while done < args.drift_steps:
            k = min(args.drift_every, args.drift_steps - done)
            sim.step(dt, k, scheme=args.drift_scheme)
            done += k
            d = sim.diagnostics()
            curve.append([done, d["E"] / d0["E"] - 1, float(np.linalg.norm(d["P"] - d0["P"])),
                          d["L"][2] / d0["L"][2] - 1])
            if log:   # the curve so far survives an interrupted run
                log.write(json.dumps({"step": done, "wall_s": time.perf_counter() - t0,
                                      "dE_over_E0": curve[-1][1], "dP_abs": curve[-1][2],
                                      "dLz_over_Lz0": curve[-1][3]}) + "\n")
                log.flush()
        if log:
            log.close()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    c = np.array(curve)
    out.update({"E0": d0["E"], "P0": d0["P"].tolist(), "Lz0": d0["L"][2],
                "max_dE_over_E0": float(np.abs(c[:, 1]).max()), "max_dP_abs": float(c[:, 2].max()),
                "max_dLz_over_Lz0": float(np.abs(c[:, 3]).max()), "wall_s": wall,
                "ms_per_step": wall / args.drift_steps * 1e3, "curve": curve})
    print(json.dumps(out), flush=True)


def run_evolution(args):
    """The paper's SP-against-DP evolution diagnostics as data (Figs. 6-7): the
    same disk + halo initial state integrated in each mode of --evolution; every
    --evolution-every steps the deviation of the total momentum |P - P0| and of
    the centre of mass |R_cm - R_cm0| (whole system and disk), and the disk's
    surface density on a 128 x 128 grid over [-6, 6]^2 (mass per unit area of
    the disk particles projected on the z = 0 plane).  Maps and curves go to
    --evolution-out (npz); the JSON line summarises them against the first mode
    listed (the reference).  A mode written with a trailing "~" starts from the
    same state with one coordinate moved by one ulp: N-body dynamics is chaotic,
    so this control shows how far any rounding difference alone carries."""
    import torch
    import nbody_ics
    import paper_1803_01190_gb300 as nb
    modes = args.evolution.split(",")
    w = nbody_ics.workload("disk_halo", n=args.n)
    nd = args.n // 2                   # disk particles come first
    edges = np.linspace(-6.0, 6.0, args.evolution_grid + 1)
    area = (edges[1] - edges[0]) ** 2
    data, summary = {}, {}
    for mode in modes:
        times, com, com_disk, dP, maps = [], [], [], [], []
        pos0 = w["pos"].copy()
        if mode.endswith("~"):
            pos0[0, 0] = np.nextafter(pos0[0, 0], np.inf)
        with nb.Simulation(args.n, mode=mode.rstrip("~"), eps=EPS) as sim:
            sim.set_state(pos0, w["vel"], w["mass"])
            P0 = sim.diagnostics()["P"]
            done = 0
            t0 = time.perf_counter()
            while True:
                pos, vel, t, _ = sim.get_state()
                m = w["mass"]
                times.append(t)
                com.append((m[:, None] * pos).sum(0) / m.sum())
                com_disk.append((m[:nd, None] * pos[:nd]).sum(0) / m[:nd].sum())
                dP.append(float(np.linalg.norm(sim.diagnostics()["P"] - P0)))
                if args.evolution_counts:   # particles per cell (equal masses: sigma = counts m / area)
                    h, _, _ = np.histogram2d(pos[:nd, 0], pos[:nd, 1], bins=[edges, edges])
                    maps.append(h.astype(np.uint16))
                else:
                    h, _, _ = np.histogram2d(pos[:nd, 0], pos[:nd, 1], bins=[edges, edges],
                                             weights=m[:nd])
                    maps.append(h / area)
                if done >= args.evolution_steps:
                    break
                k = min(args.evolution_every, args.evolution_steps - done)
                sim.step(DT, k)
                done += k
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        com, com_disk, maps = np.array(com), np.array(com_disk), np.array(maps)
        data.update({f"{mode}_t": np.array(times), f"{mode}_com": com, f"{mode}_com_disk": com_disk,
                     f"{mode}_dP": np.array(dP),
                     f"{mode}_counts" if args.evolution_counts else f"{mode}_sigma": maps})
        summary[mode] = {"wall_s": wall,
                         "max_dP_abs": float(max(dP)),
                         "max_dRcm": float(np.linalg.norm(com - com[0], axis=1).max()),
                         "max_dRcm_disk": float(np.linalg.norm(com_disk - com_disk[0], axis=1).max())}
    ref = modes[0]
    key = "counts" if args.evolution_counts else "sigma"
    for mode in modes[1:]:
        a, b = data[f"{ref}_{key}"].astype(float), data[f"{mode}_{key}"].astype(float)
        summary[mode]["sigma_L1_diff_vs_" + ref] = [
            float(np.abs(a[k] - b[k]).sum() / a[k].sum()) for k in range(len(a))]
        summary[mode]["sigma_max_abs_diff_vs_" + ref] = [float(np.abs(a[k] - b[k]).max())
                                                         for k in range(len(a))]
    summary["times"] = data[f"{ref}_t"].tolist()
    if args.evolution_out:
        np.savez_compressed(args.evolution_out, edges=edges, particle_mass=w["mass"][0], **data)
    print(json.dumps({"evolution": modes, "n": args.n, "eps": EPS, "dt": DT,
                      "steps": args.evolution_steps, "every": args.evolution_every,
                      "workload": workload_desc(args.n), "out": args.evolution_out,
                      "summary": summary}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_FULL)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--e2e-warmup", type=int, default=1,
                    help="untimed FP64 end-to-end calls before the timed one (the kernel is warm already)")
    ap.add_argument("--ref-rows", type=int, default=1024)
    ap.add_argument("--serve-seconds", type=float, default=30.0)
    ap.add_argument("--drift", choices=["fp64", "f64e", "mixed", "fp32"], default=None,
                    help="long conservation run of the workload in this mode (Table 2 quantities)")
    ap.add_argument("--drift-steps", type=int, default=10000)
    ap.add_argument("--drift-scheme", choices=["kdk", "fr4", "rk4"], default="kdk")
    ap.add_argument("--evolution", default=None,
                    help="comma-separated modes, the first the reference: SP-against-DP evolution data")
    ap.add_argument("--evolution-steps", type=int, default=20000)
    ap.add_argument("--evolution-every", type=int, default=2000)
    ap.add_argument("--evolution-out", default=None, help="npz file for the maps and curves")
    ap.add_argument("--evolution-grid", type=int, default=128, help="surface-density cells per side")
    ap.add_argument("--evolution-counts", action="store_true",
                    help="store particles per cell (uint16) instead of surface densities")
    ap.add_argument("--drift-dt", type=float, default=DT)
    ap.add_argument("--drift-every", type=int, default=100)
    ap.add_argument("--drift-out", default=None,
                    help="--drift: also write each sample of the curve to this file as it is taken")
    ap.add_argument("--symmetric", type=int, choices=[-1, 0, 1], default=-1,
                    help="--profile-force: each-pair-once path -1 automatic, 0 off, 1 on")
    ap.add_argument("--profile-force", choices=["fp64", "f64e", "mixed", "fp32"], default=None,
                    help="run one force evaluation of the workload in this mode and exit")
    ap.add_argument("--order", choices=["default", "input", "spatial"], default="default",
                    help="--profile-force / --drift: particle order of the force sum")
    ap.add_argument("--peaks", action="store_true", help="print the measured pipe rates and exit")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.peaks:
        run_peaks(args)
    elif args.drift:
        run_drift(args)
    elif args.evolution:
        run_evolution(args)
    elif args.profile_force:
        profile_force(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
