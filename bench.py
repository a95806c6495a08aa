#!/usr/bin/env python
"""ChebFD benchmark: fused-filter SpMMV throughput on the 64x64x32
topological-insulator lattice (N = 524288, complex128, n_s = 128, n_b = 32,
n_p = 1000, SELL-C-sigma C = 32).

One step = one full ChebFD filter application (n_s / n_b blocks of n_p fused
steps).  Prints one JSON line.  --impl reference times the CPU oracle on a
bounded sample of the same workload.  Under torchrun every rank filters its
own disorder realisation (independent problems, no data-path collective).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1803_02156_gb300 import model, workloads  # noqa: E402

METRIC = "fused filter SpMMV GB/s"
UNIT = "GB/s"
WORKLOAD = workloads.MEDIUM
BOUNDS = (-8.6, 8.6)          # contains the Gershgorin interval [-8.5, 8.5] of the gamma = 1 lattice
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07e9 / 1e9   # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
HBM_FALLBACK_GBS = 6800.0


def measured_hbm_gbs():
    """Measured HBM copy bandwidth of this GPU pool (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return HBM_FALLBACK_GBS, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n-b", type=int, default=WORKLOAD.n_b)
    ap.add_argument("--n-p", type=int, default=WORKLOAD.n_p)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=0)
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg (profiling runs)")
    ap.add_argument("--prec", default="c128", choices=["c128", "c64"], help="filter arithmetic")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# --------------------------------------------------------------- clocks --

class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait(timeout=10)

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ reference --

def cpu_oracle_sample(w, n_b, sample_steps, seed):
    """Time the CPU oracle's filter on one n_b block of the workload for a bounded
    number of steps; returns (GB/s by the traffic model, seconds, threads, steps)."""
    import oracle
    from paper_1803_02156_gb300 import inputs
    H = oracle.topi_csr(*w.lattice, t=w.t, m=w.m, gamma=w.gamma, seed=seed, periodic=w.periodic)
    X = inputs.gaussian_block(H.N, n_b, seed=w.x_seed)
    t0 = time.perf_counter()
    oracle.chebfd_filter(H, BOUNDS[0], BOUNDS[1], -0.3, 0.3, sample_steps, X, n_b)
    dt = time.perf_counter() - t0
    byts = sample_steps * model.step_bytes(H.N, H.nnz, n_b, "c128")
    return byts / dt / 1e9, dt, oracle.lib().orc_num_threads(), sample_steps


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = WORKLOAD
    steps = a.cpu_sample_steps or 150
    vals = []
    for _ in range(a.warmup if a.warmup < 1 else 1):
        cpu_oracle_sample(w, a.n_b, 2, w.seed)
    t_all = 0.0
    cores = 1
    for _ in range(a.steps):
        v, dt, cores, _ = cpu_oracle_sample(w, a.n_b, steps, w.seed)
        vals.append(v)
        t_all += dt
    value = statistics.median(vals)
    sample = "%d fused steps of one n_b=%d block of %s (CPU oracle, fp64), per bench step" % (steps, a.n_b, w.name)
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(1e3 * t_all / max(a.steps, 1), 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
           "data": "synthetic", "config": {"workload": w.name, "n_s": w.n_s, "n_b": a.n_b, "n_p": steps,
                                           "lattice": list(w.lattice)},
           "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------- ours --

def run_gpu(a):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1803_02156_gb300 import binding as b, inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    w = WORKLOAD
    n_b, n_p, n_s = a.n_b, a.n_p, w.n_s
    seed = w.seed + rank
    prec = a.prec
    cdt = torch.complex128 if prec == "c128" else torch.complex64
    H = b.cfd_build_matrix(b.topi_params(*w.lattice, t=w.t, m=w.m, gamma=w.gamma, seed=seed,
                                         periodic=w.periodic), w.sell_C, w.sell_sigma, prec)
    N, nnz = H.N, H.nnz
    lam_l, lam_r = -0.3, 0.3
    X0 = torch.from_numpy(inputs.gaussian_block(N, n_s, seed=w.x_seed)).to(cdt).cuda()
    X = X0.clone()
    ws = b.cfd_filter_workspace(N, n_s, n_b, n_p, prec, prec)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step(Xd):
        b.cfd_filter(H, BOUNDS[0], BOUNDS[1], lam_l, lam_r, n_p, Xd, n_b, work=work)

    for _ in range(a.warmup):
        X.copy_(X0)
        step(X)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(a.steps):
            step(X)
        ev1.record(stream)
        torch.cuda.synchronize()
    t = ev0.elapsed_time(ev1) / 1e3
    if world > 1:
        tt = torch.tensor([t], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
        dist.barrier()
    clocks = clk.summary()

    n_blocks = n_s // n_b
    step_bytes = model.step_bytes(N, nnz, n_b, prec)
    filt_bytes = n_blocks * n_p * step_bytes
    filt_flops = n_blocks * n_p * model.step_flops(N, nnz, n_b)
    value = world * a.steps * filt_bytes / t / 1e9
    gflops = world * a.steps * filt_flops / t / 1e9
    launches_per_step = 1 + n_blocks * n_p      # weights + one fused kernel per recurrence step
    t_launch = t / (a.steps * n_blocks * n_p)
    fma_flops = model.step_fma_flops(N, nnz, n_b)
    achieved = fma_flops / t_launch / 1e9

    e2e = None
    if not a.no_e2e:
        Xh = X0.cpu().pin_memory()
        Xo = torch.empty_like(Xh).pin_memory()
        for _ in range(1):
            X.copy_(Xh, non_blocking=True)
            step(X)
            Xo.copy_(X, non_blocking=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            X.copy_(Xh, non_blocking=True)
            step(X)
            Xo.copy_(X, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        te = e0.elapsed_time(e1) / 1e3
        if world > 1:
            tt = torch.tensor([te], device="cuda", dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            te = float(tt.item())
        nbytes = N * n_s * (16 if prec == "c128" else 8)
        e2e = {"value": round(world * a.steps * filt_bytes / te / 1e9, 3), "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}

    hbm, hbm_src = measured_hbm_gbs()
    gbs_launch = step_bytes / t_launch / 1e9
    if prec == "c128":
        roof = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(FP64_PEAK_GFLOPS, 1),
                "unit": "GFLOP/s", "frac": round(achieved / FP64_PEAK_GFLOPS, 4), "traffic": None,
                "peak_source": "nominal FP64 FMA rate (152 SMs x 2/clk x 2.07 GHz)",
                "kernel": "k_cheb_step<double,%d,%d,GENERAL>" % (n_b, 1 if n_b <= 32 else 2),
                "avg_launch_ms": round(1e3 * t_launch, 4),
                "hbm_gbs": round(gbs_launch, 1), "hbm_frac": round(gbs_launch / hbm, 4)}
    else:
        roof = {"bound": "hbm", "achieved": round(gbs_launch, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(gbs_launch / hbm, 4), "traffic": None, "peak_source": hbm_src,
                "kernel": "k_cheb_step<float,%d,2,GENERAL>" % n_b, "avg_launch_ms": round(1e3 * t_launch, 4)}
    if rank == 0:
        cpu = None
        if world == 1 and not a.no_cpu:
            v, dt, cores, sst = cpu_oracle_sample(w, n_b, a.cpu_sample_steps or 150, seed)
            cpu = {"value": round(v, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": "%d fused steps of one n_b=%d block of %s, fp64 C oracle, %.1f s" % (sst, n_b, w.name, dt)}
        out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": round(1e3 * t / a.steps, 3), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
               "config": {"workload": w.name, "lattice": list(w.lattice), "N": N, "nnz": nnz, "n_s": n_s,
                          "n_b": n_b, "n_p": n_p, "sell_C": w.sell_C, "sell_sigma": w.sell_sigma,
                          "l2": "inputs larger than L2 (X 1.07 GB, work blocks 0.54 GB)",
                          "parallelism": "replicas" if world > 1 else "single"},
               "gflops": round(gflops, 2),
               "roofline": roof,
               "clocks": clocks, "gpu_launches": a.steps * launches_per_step,
               "cpu_baseline": cpu, "e2e": e2e}
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)


if __name__ == "__main__":
    main()
