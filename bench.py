#!/usr/bin/env python
"""ChebFD benchmark: the fused block polynomial filter on the 200x200x100
topological-insulator lattice (N = 16,000,000, complex128, n_s = 256 in
subspace blocks of n_b = 32, SELL-C-sigma C = 32), and time to eigenpairs,
fp64 against the mixed-precision policy, on the 128x128x64 lattice.

One step = one subspace block of n_b = 32 vectors filtered with n_p = 100
fused steps (with moments), through cfd_filter; step k filters block
k mod 8 of the N x 256 search space in place.  The metric is the filter's
minimum-traffic bytes per second (nnz (s + 4) + 5 N n_b s bytes per fused
step).  Prints one JSON line, which also carries the time-to-eigenpairs
comparison (run once after the timed region).  --impl reference times the CPU
oracle on a bounded sample of the same workload.  Under torchrun every rank
works on its own disorder realisation (independent problems, no data-path
collective).  --mode iteration is the whole ChebFD iteration (filter, SVQB,
Rayleigh-Ritz) on the 64x64x32 lattice.
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
WORKLOAD = workloads.MEDIUM          # --mode iteration
LARGE = workloads.LARGE              # the default filter workload
TTE_WORKLOAD = workloads.MIXED       # time to eigenpairs, fp64 vs mixed
LARGE_WINDOW = (-0.3, 0.3)           # search interval of the large instance (does not change the filter's work)
BOUNDS = (-8.6, 8.6)          # contains the Gershgorin interval [-8.5, 8.5] of the gamma = 1 lattice
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07e9 / 1e9   # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
HBM_FALLBACK_GBS = 6800.0
PROFILES = os.path.join(ROOT, "profiles")


def source_digest(paths):
    """First 16 hex digits of the SHA-256 of the concatenated source files."""
    import hashlib
    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, n_b, N):
    """DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
    `kernel` at block width n_b, scaled to N rows, from the committed ncu
    summaries: a line 'traffic-record: kernel=K n_b=B N=R bytes=T
    sources=a,b digest=D' in profiles/*.md.  The record counts only while the
    digest of its source files equals the digest of those files now (a kernel
    changed since the capture gives None).  The per-launch traffic of the step
    is per row (matrix row + n_b block entries), so it scales with N."""
    import glob
    for path in sorted(glob.glob(os.path.join(PROFILES, "*.md"))):
        with open(path) as f:
            for line in f:
                line = line.strip().strip("`")
                if not line.startswith("traffic-record:"):
                    continue
                kv = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
                if kv.get("kernel") != kernel or int(kv.get("n_b", -1)) != n_b:
                    continue
                try:
                    if source_digest(kv["sources"].split(",")) != kv["digest"]:
                        continue
                except (OSError, KeyError):
                    continue
                return float(kv["bytes"]) * N / float(kv["N"]), os.path.relpath(path, ROOT)
    return None, None


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
    ap.add_argument("--n-b", type=int, default=None, help="subspace block width (default: the workload's)")
    ap.add_argument("--n-p", type=int, default=None, help="filter degree (default: the workload's)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=0, help="steps of the end-to-end leg (0: --steps)")
    ap.add_argument("--cpu-sample-steps", type=int, default=0)
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg (profiling runs)")
    ap.add_argument("--no-single-core", action="store_true",
                    help="reference arm: skip the extra one-thread oracle sample")
    ap.add_argument("--no-tte", action="store_true",
                    help="filter mode: skip the time-to-eigenpairs comparison after the timed region")
    ap.add_argument("--tte", action="store_true", help="iteration mode: also time cfd_solve, fp64 vs mixed")
    ap.add_argument("--tte-workload", default=None, choices=sorted(workloads.ALL),
                    help="the workload whose time to eigenpairs is measured (default: the 128x128x64 one)")
    ap.add_argument("--mode", default="filter",
                    choices=["filter", "iteration", "batch", "fusion", "host", "sweep", "tte", "peaks", "dense", "kernel",
                             "dist"],
                    help="filter: n_b = 32 blocks of the 200x200x100 lattice at n_p = 100, plus time to "
                         "eigenpairs (default); iteration: the 64x64x32 ChebFD iteration (filter, SVQB, "
                         "Rayleigh-Ritz); batch: 64 uneven realisations, batched vs looped; fusion: fused step "
                         "vs separate SpMMV + BLAS-1 calls; host: search space in host memory vs in HBM, against "
                         "n_p; sweep: fused-filter throughput per configuration; tte: time to eigenpairs, fp64 "
                         "vs mixed policy, on --tte-workload; peaks: measured FMA rates of the fp64 and fp32 "
                         "pipes; kernel: filter calls on one n_b block of the 64x64x32 lattice (profiling case); "
                         "dist: the 200x200x100 lattice split into z-slabs, one per rank, halos over NCCL")
    ap.add_argument("--dist-mode", type=int, default=0, help="dist mode: 0 vector (Algorithm 3), 1 pipelined (4)")
    ap.add_argument("--host-lattice", default="64x64x32", help="host mode: lattice Nx x Ny x Nz")
    ap.add_argument("--host-n-s", type=int, default=128, help="host mode: search space width")
    ap.add_argument("--host-n-ps", default="2,5,10,20,50,100", help="host mode: filter degrees (comma list)")
    ap.add_argument("--host-layout", default="blocked", choices=["blocked", "rowmajor"],
                    help="host mode: search space block after block (one contiguous copy per block) or row-major")
    ap.add_argument("--realisations", type=int, default=workloads.BATCH_COUNT)
    ap.add_argument("--prec", default="c128", choices=["c128", "c64"], help="filter arithmetic")
    ap.add_argument("--gather", type=int, default=0, help="kernel mode: cfd_filter_opts.gather")
    ap.add_argument("--vpt", type=int, default=0, help="kernel mode: vectors per thread (0: default)")
    ap.add_argument("--no-moments", action="store_true", help="kernel mode: filter without moments")
    ap.add_argument("--dense-n", type=int, default=4194304, help="dense mode: rows of the N x 256 block")
    ap.add_argument("--footprint", type=int, default=0,
                    help="cfd_filter_opts.footprint: 0 footprint-staged general steps where they apply, -1 never")
    ap.add_argument("--arith", default="dw", choices=["native", "dw"],
                    help="complex128 filter: double-word arithmetic on the fp32 pipe (cfd_filter_opts.arith = 1, "
                         "the default) or native fp64 arithmetic")
    ap.add_argument("--tte-policies", default="fp64,mixed_dw",
                    help="time to eigenpairs: comma list of fp64, fp64_dw, mixed, mixed_dw (the first is the "
                         "reference the others' speedups and eigenvalue differences are taken against)")
    ap.add_argument("--storage", default="packed", choices=["packed", "complex"],
                    help="matrix values as real-or-imaginary scalars (exact for Topi) or complex pairs")
    a = ap.parse_args()
    w = LARGE if a.mode in ("filter", "dist") else WORKLOAD
    a.n_b = a.n_b or w.n_b
    a.n_p = a.n_p or w.n_p
    return a


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(seconds, device="cpu"):
    """Slowest rank's time (every rank gets the same value); identity on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(base_seed, rank):
    """Disorder seed of the realisation rank `rank` works on (independent replicas)."""
    return base_seed + rank


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

_ORACLE_CACHE = {}


def host_block(N, n_b, seed):
    """Complex Gaussian N x n_b start block for the oracle's timing samples,
    drawn on the host with numpy's seeded generator (values do not change the
    oracle's work; large blocks are too slow to draw with SplitMix64 in numpy)."""
    import numpy as np
    z = np.random.default_rng(seed).standard_normal((N, n_b, 2))
    return (z[..., 0] + 1j * z[..., 1]) * (0.5 ** 0.5)


def cpu_oracle_sample(w, n_b, sample_steps, seed):
    """Time the CPU oracle's filter on one n_b block of the workload for a bounded
    number of steps; returns (GB/s by the traffic model, seconds, threads, steps).
    The CSR and the block are built once per process (untimed)."""
    import oracle
    key = (w.name, seed, n_b)
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE.clear()
        H = oracle.topi_csr(*w.lattice, t=w.t, m=w.m, gamma=w.gamma, seed=seed, periodic=w.periodic)
        _ORACLE_CACHE[key] = (H, host_block(H.N, n_b, w.x_seed))
    H, X = _ORACLE_CACHE[key]
    t0 = time.perf_counter()
    oracle.chebfd_filter(H, BOUNDS[0], BOUNDS[1], -0.3, 0.3, sample_steps, X, n_b)
    dt = time.perf_counter() - t0
    byts = sample_steps * model.step_bytes(H.N, H.nnz, n_b, "c128")
    return byts / dt / 1e9, dt, oracle.lib().orc_num_threads(), sample_steps


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    large = a.mode == "filter"
    w = LARGE if large else WORKLOAD
    # per bench step: a bounded sample of fused steps of one n_b block (a few
    # seconds of the C oracle on all host cores)
    steps = a.cpu_sample_steps or (4 if large else 150)
    vals = []
    cpu_oracle_sample(w, a.n_b, 2, w.seed)      # untimed: builds the CSR and the block, warms the caches
    t_all = 0.0
    cores = 1
    for _ in range(a.steps):
        v, dt, cores, _ = cpu_oracle_sample(w, a.n_b, steps, w.seed)
        vals.append(v)
        t_all += dt
    value = statistics.median(vals)
    sample = "%d fused steps of one n_b=%d block of %s (CPU oracle, fp64), per bench step" % (steps, a.n_b, w.name)
    single = None
    if not a.no_single_core and cores > 1:
        # the same oracle on one thread, in a child process (OpenMP reads the
        # thread count at start-up), on a shorter sample
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--impl", "reference", "--steps", "1",
                            "--warmup", "0", "--cpu-sample-steps", "1" if large else "10", "--no-single-core",
                            "--mode", a.mode],
                           env=dict(os.environ, OMP_NUM_THREADS="1"), capture_output=True, text=True)
        try:
            single = {"value": json.loads(r.stdout.strip().splitlines()[-1])["value"], "unit": UNIT, "cores": 1,
                      "sample": "%d fused step(s) of one n_b=%d block" % (1 if large else 10, a.n_b)}
        except (ValueError, IndexError, KeyError):
            single = None
    cfg = {"workload": w.name, "lattice": list(w.lattice), "N": w.N, "nnz": w.nnz, "n_s": w.n_s, "n_b": a.n_b,
           "n_p": a.n_p, "oracle_steps_per_sample": steps}
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(1e3 * t_all / max(a.steps, 1), 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
           "data": "synthetic", "config": cfg,
           "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample, "single_core": single},
           "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------- ours --

def setup_problem(b, w, seed, storage, H=None, with_kpm=False):
    """Matrix, spectral bounds and the KPM window holding about n_t states
    (untimed setup).  with_kpm: also an independent KPM count of that window
    from 32 other random vectors (the window's count is n_t by construction
    for the 16 vectors that chose it)."""
    import torch
    from paper_1803_02156_gb300 import inputs
    p = b.topi_params(*w.lattice, t=w.t, m=w.m, gamma=w.gamma, seed=seed, periodic=w.periodic)
    suffix = "p" if storage == "packed" else ""
    if H is None:
        H = b.cfd_build_matrix(p, w.sell_C, w.sell_sigma, "c128" + suffix)
    lmin, lmax = b.cfd_spectral_bounds(H, 40, seed=w.lanczos_seed)
    # KPM estimate of the window from 16 random vectors and 2 n_p moments
    # (stochastic error about sqrt(n_t / 16) states)
    R = torch.from_numpy(inputs.gaussian_block(H.N, 16, seed=w.x_seed + 100)).cuda()
    mu = b.cfd_filter(H, lmin, lmax, lmin, lmax, w.n_p, R, 16, moments=True).cpu().numpy()
    lam_l, lam_r = b.cfd_kpm_window(mu, H.N, lmin, lmax, 0.0, float(w.n_t))
    del R
    if not with_kpm:
        return p, H, lmin, lmax, lam_l, lam_r
    R = inputs.gaussian_block_device(H.N, 32, seed=w.x_seed + 200)
    mu = b.cfd_kpm_moments(H, lmin, lmax, w.n_p, R, 32).cpu().numpy()
    del R
    return p, H, lmin, lmax, lam_l, lam_r, b.cfd_kpm_count(mu, H.N, lmin, lmax, lam_l, lam_r)


def fp64_peak(b):
    """FP64 FMA peak: (nominal GFLOP/s from the unit count and the maximum
    clock, measured GFLOP/s of the library's FMA probe or None)."""
    try:
        meas = b.cfd_probe_fma("c128", 1 << 15) / 1e9
    except Exception:            # the probe is optional for the roofline
        meas = None
    return FP64_PEAK_GFLOPS, meas


def run_filter(a):
    """Default: n_b = 32 subspace blocks of the 200x200x100 lattice filtered at
    n_p = 100 (Algorithm 1 on one block of Algorithm 2), one block per step."""
    import torch
    import torch.distributed as dist
    from paper_1803_02156_gb300 import binding as b, inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    w = LARGE
    n_b, n_p, n_s = a.n_b, a.n_p, w.n_s
    n_blocks = n_s // n_b
    seed = replica_seed(w.seed, rank)
    prec = a.prec
    suffix = "p" if a.storage == "packed" else ""
    p = b.topi_params(*w.lattice, t=w.t, m=w.m, gamma=w.gamma, seed=seed, periodic=w.periodic)
    H = b.cfd_build_matrix(p, w.sell_C, w.sell_sigma, "c128" + suffix)
    lmin, lmax = b.cfd_spectral_bounds(H, 40, seed=w.lanczos_seed)
    lam_l, lam_r = LARGE_WINDOW
    if prec != "c128":
        del H
        torch.cuda.empty_cache()
        H = b.cfd_build_matrix(p, w.sell_C, w.sell_sigma, prec + suffix)
    N, nnz = H.N, H.nnz
    # the N x n_s search space (65.5 GB), drawn on the device from a seeded generator
    X = inputs.gaussian_block_device(N, n_s, seed=w.x_seed + rank)
    work = torch.empty(b.cfd_filter_workspace(N, n_s, n_b, n_p, H.prec, b.CFD_C128), dtype=torch.uint8,
                       device="cuda")
    mu = torch.empty(n_b, 2 * n_p, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    L = b.lib()
    blocks = [b.block_of(X[:, k * n_b:(k + 1) * n_b]) for k in range(n_blocks)]

    dw = prec == "c128" and a.arith == "dw"
    opts = b.cfd_filter_opts(0, 0, 0, 0, 0, 0, 1 if dw else 0, 0, a.footprint)
    # the footprint-staged steps apply to complex-float and double-word filters
    # of C = 32, sigma = 1 packed matrices at n_b = 32
    fp_on = (a.footprint >= 0 and n_b == 32 and w.sell_C == 32 and w.sell_sigma == 1 and a.storage == "packed"
             and (dw or prec == "c64"))

    def filt(blk, npp=n_p):
        b._check(L.cfd_filter_ex(H.ref(), lmin, lmax, lam_l, lam_r, npp, blk, n_b, b._ptr(work), work.numel(),
                                 b._ptr(mu), b.ctypes.byref(opts), b._stream()))

    for k in range(a.warmup):
        filt(blocks[k % n_blocks])
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
    n0 = b.cfd_launch_count()
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        ev[0].record(stream)
        for k in range(a.steps):
            filt(blocks[k % n_blocks])
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
    launches = b.cfd_launch_count() - n0
    t = ev[0].elapsed_time(ev[-1]) / 1e3
    t = max_over_ranks(t, "cuda")
    if world > 1:
        dist.barrier()
    clocks = clk.summary()
    b.cfd_workspace_status(work)         # a recorded device-side error voids the run

    # per-launch time of the general fused step: a step's time less that of
    # the same call with n_p = 3 (weights, prepared values, steps 1 and 2, one
    # general step, moments), over its n_p - 3 remaining general steps; CUDA
    # events on the launch stream
    t_steps = sorted(ev[k].elapsed_time(ev[k + 1]) / 1e3 for k in range(a.steps))
    t_med = t_steps[len(t_steps) // 2]

    mu3 = torch.empty(n_b, 6, dtype=torch.float64, device="cuda")

    def fixed_part(o):
        cal = []
        for k in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b._check(L.cfd_filter_ex(H.ref(), lmin, lmax, lam_l, lam_r, 3, blocks[k % n_blocks], n_b, b._ptr(work),
                                     work.numel(), b._ptr(mu3), b.ctypes.byref(o), b._stream()))
            e1.record(stream)
            torch.cuda.synchronize()
            cal.append(e0.elapsed_time(e1) / 1e3)
        return sorted(cal)[1]
    t_fixed = fixed_part(opts)
    t_launch = (t_med - t_fixed) / (n_p - 3)

    step_bytes = model.step_bytes(N, nnz, n_b, prec)
    value = world * a.steps * n_p * step_bytes / t / 1e9
    gflops = world * a.steps * n_p * model.step_flops(N, nnz, n_b) / t / 1e9
    gbs_launch = step_bytes / t_launch / 1e9
    hbm, hbm_src = measured_hbm_gbs()
    if dw:
        kname = "k_cheb_step_fp_dw" if fp_on else "k_cheb_step_dw"
        traffic, tsrc = profiled_traffic(kname, n_b, N)
        roof = {"bound": "hbm", "achieved": round(gbs_launch, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(gbs_launch / hbm, 4), "traffic": traffic, "traffic_source": tsrc,
                "peak_source": hbm_src,
                "kernel": ("k_cheb_step_fp<double-word,%d,2,moments,2 stages,16+1 warps>" % n_b if fp_on else
                           "k_cheb_step_dw<%d,%d,moments,chunk height 32>" % (n_b, 2 if n_b >= 16 else 1)),
                "algorithmic": "nnz (16 + 4) + 5 N n_b 16 bytes per launch",
                "avg_launch_ms": round(1e3 * t_launch, 4)}
    elif prec == "c128":
        nominal, measured = fp64_peak(b)
        fma = model.step_fma_flops(N, nnz, n_b, packed=(a.storage == "packed"), prepared=True)
        achieved = fma / t_launch / 1e9
        kname = "k_cheb_step_staged_c128"
        traffic, tsrc = profiled_traffic(kname, n_b, N)
        roof = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(nominal, 1), "unit": "GFLOP/s",
                "frac": round(achieved / nominal, 4), "traffic": traffic, "traffic_source": tsrc,
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
                "measured_peak": round(measured, 1) if measured else None,
                "frac_of_measured_peak": round(achieved / measured, 4) if measured else None,
                "kernel": "k_cheb_step_staged<double,%d,%d,moments,%s>" % (n_b, 2 if n_b >= 16 else 1, a.storage),
                "algorithmic": "(4 nnz + 12 N) n_b FMA-pipe flops per launch",
                "avg_launch_ms": round(1e3 * t_launch, 4), "hbm_gbs": round(gbs_launch, 1),
                "hbm_frac": round(gbs_launch / hbm, 4), "hbm_peak": hbm}
    else:
        kname = "k_cheb_step_fp_c64" if fp_on else "k_cheb_step_staged_c64"
        traffic, tsrc = profiled_traffic(kname, n_b, N)
        roof = {"bound": "hbm", "achieved": round(gbs_launch, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(gbs_launch / hbm, 4), "traffic": traffic, "traffic_source": tsrc,
                "peak_source": hbm_src,
                "kernel": ("k_cheb_step_fp<complex float,%d,4,moments,4 stages,2x8+1 warps>" % n_b if fp_on else
                           "k_cheb_step_staged<float,%d,2,moments,%s>" % (n_b, a.storage)),
                "algorithmic": "nnz (8 + 4) + 5 N n_b 8 bytes per launch",
                "avg_launch_ms": round(1e3 * t_launch, 4)}
    roof["avg_launch_note"] = ("(median step - median n_p=3 call) / (n_p - 3), CUDA events on the launch stream; "
                               "n_p=3 call %.2f ms" % (1e3 * t_fixed))

    native = None
    if dw:
        # the same block step with the native fp64 arithmetic, and the
        # double-word result's distance from it (filtered block, moments)
        onat = b.cfd_filter_opts(0, 0, 0, 0, 0, 0, 0, 0)
        X0 = X[:, :n_b].contiguous()
        Xd, Xn = X0.clone(), X0.clone()
        mu_n = torch.empty_like(mu)
        bn = b.block_of(Xn)
        tn = []
        for k in range(3):
            Xn.copy_(X0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b._check(L.cfd_filter_ex(H.ref(), lmin, lmax, lam_l, lam_r, n_p, bn, n_b, b._ptr(work), work.numel(),
                                     b._ptr(mu_n), b.ctypes.byref(onat), b._stream()))
            e1.record(stream)
            torch.cuda.synchronize()
            if k:
                tn.append(e0.elapsed_time(e1) / 1e3)
        filt(b.block_of(Xd))
        torch.cuda.synchronize()
        err_x = float(torch.linalg.norm(Xd - Xn) / torch.linalg.norm(Xn))
        err_mu = float(torch.max(torch.abs(mu - mu_n)) / torch.max(torch.abs(mu_n)))
        nominal, measured = fp64_peak(b)
        t_nat = statistics.median(tn)
        fma = model.step_fma_flops(N, nnz, n_b, packed=(a.storage == "packed"), prepared=True)
        tl_nat = (t_nat - fixed_part(onat)) / (n_p - 3)
        native = {"ms_per_step": round(1e3 * t_nat, 3), "gbs": round(n_p * step_bytes / t_nat / 1e9, 1),
                  "avg_launch_ms": round(1e3 * tl_nat, 4),
                  "fp64_pipe_gflops": round(fma / tl_nat / 1e9, 1), "fp64_peak_gflops": round(nominal, 1),
                  "fp64_peak_measured_gflops": round(measured, 1) if measured else None,
                  "speedup_dw": round(t_nat / t_med, 3),
                  "dw_vs_native_rel_frobenius": err_x, "dw_vs_native_moments_rel": err_mu}
        del X0, Xd, Xn

    e2e = None
    if not a.no_e2e:
        # through the C ABI with the search space in host memory: the library's
        # host-memory filter (cfd_filter_host_blocked) takes a page-locked
        # block-after-block array of kb blocks, brings block k + 1 in and
        # writes block k - 1 back while block k is filtered, and the moments
        # are read back; every step moves one n_b block in and out
        import numpy as np
        ke = a.e2e_steps or a.steps
        kb = min(ke, 4)
        Xn = np.empty((kb, N, n_b), dtype=np.complex128)
        rc = torch.cuda.cudart().cudaHostRegister(Xn.ctypes.data, Xn.nbytes, 0)
        if int(rc) != 0:
            raise RuntimeError("cudaHostRegister of %d bytes failed (%s)" % (Xn.nbytes, rc))
        Xh = torch.from_numpy(Xn)
        for k in range(kb):
            Xh[k].copy_(X[:, (k % n_blocks) * n_b:(k % n_blocks + 1) * n_b])
        hw = b.cfd_filter_host_workspace(N, kb * n_b, n_b, n_p, H.prec, b.CFD_C128)
        del work
        work = torch.empty(hw, dtype=torch.uint8, device="cuda")
        muh_dev = torch.empty(kb * n_b, 2 * n_p, dtype=torch.float64, device="cuda")
        muh = torch.empty(kb * n_b, 2 * n_p, dtype=torch.float64).pin_memory()
        hopts = b.cfd_filter_opts(0, 0, 0, 0, 0, 0, 1 if dw else 0, 0)    # the host filter takes arith only

        def host_call(nblk):
            blk = b.cfd_block(Xh.data_ptr(), N, n_b, nblk * n_b, b.CFD_C128)
            b._check(L.cfd_filter_host_blocked(H.ref(), lmin, lmax, lam_l, lam_r, n_p, blk, n_b, b._ptr(work),
                                               work.numel(), b._ptr(muh_dev), b.ctypes.byref(hopts), b._stream()))
            muh[:nblk * n_b].copy_(muh_dev[:nblk * n_b], non_blocking=True)
        host_call(1)                       # warm-up: one block
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        done = 0
        while done < ke:
            nb_ = min(kb, ke - done)
            host_call(nb_)
            done += nb_
        e1.record(stream)
        torch.cuda.synchronize()
        te = max_over_ranks(e0.elapsed_time(e1) / 1e3, "cuda")
        e2e = {"value": round(world * ke * n_p * step_bytes / te / 1e9, 3), "unit": UNIT,
               "h2d_bytes_per_step": N * n_b * 16, "d2h_bytes_per_step": N * n_b * 16 + n_b * 2 * n_p * 8,
               "steps": ke, "api": "cfd_filter_host_blocked, %d blocks per call, page-locked host memory" % kb}
        torch.cuda.cudart().cudaHostUnregister(Xn.ctypes.data)
        del Xh, Xn
    del X, work
    torch.cuda.empty_cache()

    tte = None
    if not a.no_tte and rank == 0:
        tw = workloads.ALL[a.tte_workload] if a.tte_workload else TTE_WORKLOAD
        tp, tH, tlmin, tlmax, tl, tr, kpm = setup_problem(b, tw, tw.seed, a.storage, with_kpm=True)
        tte = time_to_eigenpairs(b, tw, tp, tH, tlmin, tlmax, tl, tr, a.storage, tuple(a.tte_policies.split(",")))
        tte["workload"] = tw.name
        tte["kpm_count_in_window"] = round(kpm, 2)
        del tH
        torch.cuda.empty_cache()

    if rank == 0:
        cpu = None
        if world == 1 and not a.no_cpu:
            v, dt, cores, sst = cpu_oracle_sample(w, n_b, a.cpu_sample_steps or 4, seed)
            cpu = {"value": round(v, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": "%d fused steps of one n_b=%d block of %s, fp64 C oracle, %.1f s" % (
                       sst, n_b, w.name, dt)}
        out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": round(1e3 * t / a.steps, 3), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32x2" if dw else prec, "data": "synthetic",
               "config": {"workload": w.name, "lattice": list(w.lattice), "N": N, "nnz": nnz, "n_s": n_s,
                          "n_b": n_b, "n_p": n_p, "window": list(LARGE_WINDOW),
                          "bounds": [round(lmin, 6), round(lmax, 6)], "sell_C": w.sell_C,
                          "sell_sigma": w.sell_sigma, "matrix_values": a.storage,
                          "step": "one n_b block filtered with n_p fused steps and moments (block k mod %d)"
                                  % n_blocks,
                          "filter_precision": ("fp64 storage, double-word (2 x fp32) arithmetic" if dw else "fp64")
                                              if prec == "c128" else "fp32 filter on fp64 block (mixed)",
                          "l2": "inputs larger than L2 (X %.1f GB, work blocks %.1f GB)" % (
                              N * n_s * 16 / 1e9, 2 * N * n_b * (16 if prec == "c128" else 8) / 1e9),
                          "parallelism": "replicas" if world > 1 else "single"},
               "gflops": round(gflops, 2), "roofline": roof, "clocks": clocks, "gpu_launches": launches,
               "cpu_baseline": cpu, "e2e": e2e}
        if native is not None:
            out["native_fp64"] = native
        if tte is not None:
            out["time_to_eigenpairs"] = tte
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_iteration(a):
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
    seed = replica_seed(w.seed, rank)
    prec = a.prec
    suffix = "p" if a.storage == "packed" else ""
    p, H, lmin, lmax, lam_l, lam_r = setup_problem(b, w, seed, a.storage)
    Hf = H if prec == "c128" else b.cfd_build_matrix(p, w.sell_C, w.sell_sigma, "c64" + suffix)
    N, nnz = H.N, H.nnz
    X0 = torch.from_numpy(inputs.gaussian_block(N, n_s, seed=w.x_seed)).cuda()
    X = X0.clone()
    fws = b.cfd_filter_workspace(N, n_s, n_b, n_p, Hf.prec, b.CFD_C128)
    work = torch.empty(max(fws, b.lib().cfd_orthogonalize_workspace(N, n_s),
                           b.lib().cfd_rayleigh_ritz_workspace(N, n_s)), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    mu = torch.empty(n_s, 2 * n_p, dtype=torch.float64, device="cuda")
    ev = torch.empty(n_s, dtype=torch.float64, device="cuda")
    rs = torch.empty(n_s, dtype=torch.float64, device="cuda")
    L = b.lib()
    import ctypes

    def step(Xd, evs):
        """One ChebFD iteration: filter (with moments), SVQB, Rayleigh-Ritz."""
        blk = b.block_of(Xd)
        evs[0].record(stream)
        b._check(L.cfd_filter(Hf.ref(), lmin, lmax, lam_l, lam_r, n_p, blk, n_b, b._ptr(work), work.numel(),
                              b._ptr(mu), b._stream()))
        evs[1].record(stream)
        b._check(L.cfd_orthogonalize(blk, 0.0, None, b._ptr(work), work.numel(), b._stream()))
        evs[2].record(stream)
        b._check(L.cfd_rayleigh_ritz(H.ref(), blk, b._ptr(ev), b._ptr(rs), b._ptr(work), work.numel(),
                                     b._stream()))
        evs[3].record(stream)

    def mk():
        return [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    for _ in range(a.warmup):
        step(X, mk())
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    evlist = [mk() for _ in range(a.steps)]
    n0 = b.cfd_launch_count()
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        for k in range(a.steps):
            step(X, evlist[k])
        torch.cuda.synchronize()
    launches = b.cfd_launch_count() - n0
    t = evlist[0][0].elapsed_time(evlist[-1][3]) / 1e3
    phase = [sum(e[i].elapsed_time(e[i + 1]) for e in evlist) / 1e3 for i in range(3)]
    t = max_over_ranks(t, "cuda")
    if world > 1:
        dist.barrier()
    clocks = clk.summary()

    n_blocks = n_s // n_b
    fprec = prec
    step_bytes = model.step_bytes(N, nnz, n_b, fprec)
    filt_bytes = n_blocks * n_p * step_bytes
    filt_flops = n_blocks * n_p * model.step_flops(N, nnz, n_b)
    value = world * a.steps * filt_bytes / t / 1e9
    t_launch = phase[0] / (a.steps * n_blocks * n_p)
    gbs_launch = step_bytes / t_launch / 1e9
    hbm, hbm_src = measured_hbm_gbs()
    if prec == "c128":
        fma = model.step_fma_flops(N, nnz, n_b, packed=(a.storage == "packed"), prepared=True)
        achieved = fma / t_launch / 1e9
        roof = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(FP64_PEAK_GFLOPS, 1),
                "unit": "GFLOP/s", "frac": round(achieved / FP64_PEAK_GFLOPS, 4),
                "traffic": profiled_traffic("k_cheb_step_staged_c128", n_b, N)[0],
                "peak_source": "nominal FP64 FMA rate (152 SMs x 2/clk x 2.07 GHz)",
                "kernel": "k_cheb_step_staged<double,%d,%d,moments,%s>" % (n_b, 2 if n_b >= 16 else 1, a.storage),
                "avg_launch_ms": round(1e3 * t_launch, 4), "hbm_gbs": round(gbs_launch, 1),
                "hbm_frac": round(gbs_launch / hbm, 4)}
    else:
        roof = {"bound": "hbm", "achieved": round(gbs_launch, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(gbs_launch / hbm, 4), "traffic": profiled_traffic("k_cheb_step_staged_c64", n_b, N)[0],
                "peak_source": hbm_src,
                "kernel": "k_cheb_step_staged<float,%d,2,moments,%s%s>" % (
                    n_b, a.storage, ",chunk height 32" if a.storage == "packed" else ""),
                "avg_launch_ms": round(1e3 * t_launch, 4)}

    e2e = None
    if not a.no_e2e:
        Xh = X0.cpu().pin_memory()
        Xo = torch.empty_like(Xh).pin_memory()
        evh = torch.empty(n_s, dtype=torch.float64).pin_memory()
        X.copy_(Xh, non_blocking=True)
        step(X, mk())
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            X.copy_(Xh, non_blocking=True)
            step(X, mk())
            Xo.copy_(X, non_blocking=True)
            evh.copy_(ev, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        te = max_over_ranks(e0.elapsed_time(e1) / 1e3, "cuda")
        nbytes = N * n_s * 16
        e2e = {"value": round(world * a.steps * filt_bytes / te / 1e9, 3), "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + n_s * 8}

    tte = time_to_eigenpairs(b, w, p, H, lmin, lmax, lam_l, lam_r, a.storage,
                             tuple(a.tte_policies.split(","))) if (a.tte and rank == 0) else None

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
                          "n_b": n_b, "n_p": n_p, "n_t": w.n_t, "window": [round(lam_l, 6), round(lam_r, 6)],
                          "bounds": [round(lmin, 6), round(lmax, 6)], "sell_C": w.sell_C,
                          "sell_sigma": w.sell_sigma, "matrix_values": a.storage,
                          "step": "filter (moments) + SVQB x2 + Rayleigh-Ritz",
                          "filter_precision": ("fp64 storage, double-word (2 x fp32) arithmetic" if dw else "fp64")
                                              if prec == "c128" else "fp32 filter on fp64 block (mixed)",
                          "l2": "inputs larger than L2 (X 1.07 GB, work blocks 0.54 GB)",
                          "parallelism": "replicas" if world > 1 else "single"},
               "gflops": round(world * a.steps * filt_flops / t / 1e9, 2),
               "filter_only": {"value": round(a.steps * filt_bytes / phase[0] / 1e9, 3), "unit": UNIT,
                               "gflops": round(a.steps * filt_flops / phase[0] / 1e9, 2)},
               "phase_ms_per_step": {"filter": round(1e3 * phase[0] / a.steps, 2),
                                     "orthogonalize": round(1e3 * phase[1] / a.steps, 2),
                                     "rayleigh_ritz": round(1e3 * phase[2] / a.steps, 2)},
               "roofline": roof, "clocks": clocks, "gpu_launches": launches,
               "cpu_baseline": cpu, "e2e": e2e}
        if tte is not None:
            out["time_to_eigenpairs"] = tte
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


POLICIES = {"fp64": ("CFD_POLICY_FP64", False), "fp64_dw": ("CFD_POLICY_FP64_DW", False),
            "mixed": ("CFD_POLICY_MIXED", True), "mixed_dw": ("CFD_POLICY_MIXED_DW", True)}


def time_to_eigenpairs(b, w, p, H, lmin, lmax, lam_l, lam_r, storage, policies=("fp64", "mixed_dw")):
    """Wall time of cfd_solve to n_t eigenpairs at residual <= 1e-10 from a random
    start block for each policy (fp64: native fp64 filter; fp64_dw: double-word
    filter; mixed: fp32 filter, then fp64; mixed_dw: fp32 filter, then
    double-word), with the workload's n_p and n_b.  The first policy is the
    reference of the speedups and eigenvalue differences."""
    import numpy as np
    import torch
    suffix = "p" if storage == "packed" else ""
    Hl = b.cfd_build_matrix(p, w.sell_C, w.sell_sigma, "c64" + suffix) if any(
        POLICIES[q][1] for q in policies) else None
    out = {}
    res = {}
    for name in policies:
        pol = getattr(b, POLICIES[name][0])
        hl = Hl if POLICIES[name][1] else None
        X = torch.empty(H.N, w.n_s, dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        th, rs, r = b.cfd_solve(H, X, lam_l, lam_r, w.n_p, w.n_b, H_low=hl, policy=pol, lmin=lmin, lmax=lmax,
                                tol=1e-10, n_t=w.n_t, max_iter=30, seed=w.x_seed, raise_noconv=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        conv = (th >= lam_l) & (th <= lam_r) & (rs <= 1e-10)
        res[name] = np.sort(th[conv])
        out[name] = {"seconds": round(dt, 3), "iters": r.iters, "iters_fp32": r.iters_low, "n_conv": int(r.n_conv),
                     "stop": "n_t reached" if r.n_conv >= w.n_t else "converged count stable",
                     "max_resid": float(rs[conv].max()) if conv.any() else None,
                     "t_filter": round(r.t_filter, 3), "t_orth": round(r.t_orth, 3), "t_rr": round(r.t_rr, 3)}
        del X
        torch.cuda.empty_cache()
    # each run may converge a pair or two the other has not reached yet (the
    # levels come in degenerate pairs): match every reference eigenvalue with
    # the nearest one of the other run and compare the pairs both found
    ref = policies[0]
    for name in policies[1:]:
        a, m = res[ref], res[name]
        if len(a) and len(m):
            d = np.abs(a[:, None] - m[None, :]).min(axis=1)
            both = d < 1e-8
            out[name]["common_pairs"] = int(both.sum())
            out[name]["max_eval_diff_vs_" + ref] = float(d[both].max()) if both.any() else None
        else:
            out[name]["common_pairs"] = 0
            out[name]["max_eval_diff_vs_" + ref] = None
        out[name]["speedup_vs_" + ref] = round(out[ref]["seconds"] / out[name]["seconds"], 3)
    out["reference_policy"] = ref
    out["tol"] = 1e-10
    out["n_t"] = w.n_t
    out["n_s"] = w.n_s
    out["n_p"] = w.n_p
    out["window"] = [round(lam_l, 6), round(lam_r, 6)]
    del Hl
    return out


def run_batch(a):
    """Batched workload: R realisations of uneven lattices (Nx, Ny in 16..48,
    Nz in 8..24), n_s = 64, n_p = 500, complex64 filter with fp64 SVQB and
    Rayleigh-Ritz (mixed policy).  Times (1) one filter application of all
    realisations: batched persistent launch vs looping cfd_filter; (2) time to
    n_t = 32 eigenpairs per realisation at 1e-10: cfd_solve_batched vs looping
    cfd_solve."""
    import numpy as np
    import torch
    from paper_1803_02156_gb300 import binding as b, inputs
    torch.cuda.set_device(0)
    w = workloads.BATCH
    R = a.realisations
    lat = inputs.batched_lattices(R)
    params = [b.topi_params(nx, ny, nz, t=w.t, m=w.m, gamma=w.gamma, seed=sd, periodic=w.periodic)
              for (nx, ny, nz, sd) in lat]
    n_s, n_p, n_b, n_t = w.n_s, w.n_p, w.n_b, w.n_t
    singles, wins = [], []
    for p in params:                         # per-realisation bounds and KPM window (untimed setup)
        H = b.cfd_build_matrix(p, 32, 1, "c128p")
        Hl = b.cfd_build_matrix(p, 32, 1, "c64p")
        lmin, lmax = b.cfd_spectral_bounds(H, 40)
        Rv = torch.from_numpy(inputs.gaussian_block(H.N, 16, seed=w.x_seed + 100)).cuda()
        mu = b.cfd_filter(H, lmin, lmax, lmin, lmax, n_p, Rv, 16, moments=True).cpu().numpy()
        lo, hi = b.cfd_kpm_window(mu, H.N, lmin, lmax, 0.0, float(n_t))
        singles.append((H, Hl))
        wins.append([lmin, lmax, lo, hi])
    wins = np.array(wins)
    B = b.cfd_build_batch(params, 32, 1, "c128p")
    Bl = b.cfd_build_batch(params, 32, 1, "c64p")
    Ntot = B.N
    rows = int(sum(4 * p.Nx * p.Ny * p.Nz for p in params))
    wdev = torch.from_numpy(wins).cuda()
    X = torch.from_numpy(inputs.gaussian_block(Ntot, n_s, seed=w.x_seed)).cuda()
    end = b.batch_row_end(B)
    for r in range(R):
        X[end[r]:B.row_off[r + 1]] = 0
    Xs = [X[B.row_off[r]:end[r]].clone() for r in range(R)]

    def timed(f, reps):
        f()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            f()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    def batched_filter():
        b.cfd_filter_batched(Bl, wdev, n_p, X, n_b)

    def persistent_filter():
        b.cfd_filter_batched(Bl, wdev, n_p, X, n_b, persistent=1)

    def looped_filter():
        for r in range(R):
            b.cfd_filter(singles[r][1], *wins[r], n_p, Xs[r], n_b)

    tb = timed(batched_filter, a.steps)
    tp = timed(persistent_filter, 1)
    tl = timed(looped_filter, a.steps)
    byts = sum(model.filter_bytes(s[0].N, s[0].nnz, n_s, n_b, n_p, "c64") for s in singles)

    # time to eigenpairs (mixed policy), batched vs looped
    Xb = torch.empty(Ntot, n_s, dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev, rs, res = b.cfd_solve_batched(B, Xb, wins, [n_t] * R, n_p, n_b, B_low=Bl, policy=b.CFD_POLICY_MIXED,
                                      max_iter=30, raise_noconv=False)
    torch.cuda.synchronize()
    tsb = time.perf_counter() - t0
    conv_b = [int(x.n_conv) for x in res]
    t0 = time.perf_counter()
    conv_l, diffs, common = [], [], []
    for r in range(R):
        Y = torch.empty(singles[r][0].N, n_s, dtype=torch.complex128, device="cuda")
        th, rr, rres = b.cfd_solve(singles[r][0], Y, wins[r][2], wins[r][3], n_p, n_b, H_low=singles[r][1],
                                   policy=b.CFD_POLICY_MIXED, lmin=wins[r][0], lmax=wins[r][1], n_t=n_t,
                                   max_iter=30, raise_noconv=False)
        conv_l.append(int(rres.n_conv))
        cl = np.sort(th[(th >= wins[r][2]) & (th <= wins[r][3]) & (rr <= 1e-10)])
        cb = np.sort(ev[r][(ev[r] >= wins[r][2]) & (ev[r] <= wins[r][3]) & (rs[r] <= 1e-10)])
        # each run may converge a few pairs beyond n_t the other did not reach:
        # compare every looped eigenvalue with the nearest batched one
        if len(cl) and len(cb):
            d = np.abs(cl[:, None] - cb[None, :]).min(axis=1)
            common.append(int((d < 1e-8).sum()))
            diffs.append(float(d[d < 1e-8].max()) if (d < 1e-8).any() else None)
    torch.cuda.synchronize()
    tsl = time.perf_counter() - t0
    out = {"metric": "batched ChebFD: filter GB/s and time to eigenpairs, batched vs looped", "unit": "GB/s",
           "value": round(byts / tb / 1e9, 3), "n_gpus": 1, "steps": a.steps, "dtype": "c64 filter / fp64 RR",
           "data": "synthetic", "higher_is_better": True,
           "config": {"workload": w.name, "realisations": R, "rows_total": rows, "rows_padded": Ntot,
                      "n_s": n_s, "n_p": n_p, "n_b": n_b, "n_t": n_t,
                      "lattices": [list(l[:3]) for l in lat]},
           "filter": {"batched_s": round(tb, 4), "looped_s": round(tl, 4), "speedup": round(tl / tb, 3),
                      "persistent_s": round(tp, 4),
                      "batched_gbs": round(byts / tb / 1e9, 1), "looped_gbs": round(byts / tl / 1e9, 1)},
           "time_to_eigenpairs": {"batched_s": round(tsb, 3), "looped_s": round(tsl, 3),
                                  "speedup": round(tsl / tsb, 3), "iters_batched": max(x.iters for x in res),
                                  "batched_phase_s": {"filter": round(res[0].t_filter, 3),
                                                      "orthogonalize": round(res[0].t_orth, 3),
                                                      "rayleigh_ritz": round(res[0].t_rr, 3)},
                                  "converged_batched": conv_b, "converged_looped": conv_l,
                                  "common_pairs": common,
                                  "max_eval_diff_common": max(x for x in diffs if x is not None) if any(
                                      x is not None for x in diffs) else None, "tol": 1e-10}}
    print(json.dumps(out))


def run_fusion(a):
    """Fusion ablation on the 64x64x32 lattice (Sect. 4, Fig. 2): one n_b = 32
    block of n_p steps (with moments) through the fused step and through the
    chain of separate SpMMV and BLAS-1 kernels, complex128 and complex64
    (packed values; complex64 fused with and without TMA staging).  Reports
    ms per step, model GB/s of the fused step, and the chain's own traffic."""
    import torch
    from paper_1803_02156_gb300 import binding as b, inputs
    torch.cuda.set_device(0)
    w = WORKLOAD
    n_b, n_p = a.n_b, min(a.n_p, 200)
    p = b.topi_params(*w.lattice, t=w.t, m=w.m, gamma=w.gamma, seed=w.seed, periodic=w.periodic)
    X0 = None
    res = {}
    for prec in ("c128", "c64"):
        H = b.cfd_build_matrix(p, w.sell_C, w.sell_sigma, prec + "p")
        N, nnz = H.N, H.nnz
        if X0 is None:
            X0 = torch.from_numpy(inputs.gaussian_block(N, n_b, seed=w.x_seed)).cuda()
        X = X0.to(torch.complex128 if prec == "c128" else torch.complex64)
        ws = max(b.cfd_filter_unfused_workspace(N, n_b, n_b, n_p, prec, prec),
                 b.cfd_filter_workspace(N, n_b, n_b, n_p, prec, prec))
        work = torch.empty(ws, dtype=torch.uint8, device="cuda")
        arms = {"fused": lambda: b.cfd_filter(H, *BOUNDS, -0.3, 0.3, n_p, X, n_b, moments=True, work=work),
                "unfused": lambda: b.cfd_filter_unfused(H, *BOUNDS, -0.3, 0.3, n_p, X, n_b, moments=True,
                                                        work=work)}
        if prec == "c64":
            arms["fused_unstaged"] = lambda: b.cfd_filter_ex(H, *BOUNDS, -0.3, 0.3, n_p, X, n_b, moments=True,
                                                             work=work, staged=-1)
        out = {}
        for name, f in arms.items():
            for _ in range(max(a.warmup, 1)):
                X.copy_(X0)
                f()
            ts = []
            for _ in range(max(a.steps, 1)):
                X.copy_(X0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                f()
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) / 1e3 / n_p)
            t = statistics.median(ts)
            out[name] = {"ms_per_step": round(t * 1e3, 4),
                         "model_gbs": round(model.step_bytes(N, nnz, n_b, prec) / t / 1e9, 1)}
        out["unfused"]["own_traffic_gbs"] = round(model.unfused_step_bytes(N, nnz, n_b, prec) / (
            out["unfused"]["ms_per_step"] * 1e-3) / 1e9, 1)
        out["fusion_speedup"] = round(out["unfused"]["ms_per_step"] / out["fused"]["ms_per_step"], 3)
        res[prec] = out
        del work, H
    print(json.dumps({"metric": "fused vs unfused ChebFD step", "unit": "ms/step", "n_gpus": 1,
                      "steps": a.steps, "warmup": a.warmup, "data": "synthetic",
                      "config": {"workload": "topi-64x64x32", "n_b": n_b, "n_p": n_p, "storage": "packed"},
                      "results": res}))


def run_host(a):
    """Search space in host memory (Sect. 5's larger-than-fast-memory case):
    the filter with X resident in HBM (cfd_filter_ex) against X in page-locked
    host memory streamed block by block over the chip-to-chip link
    (cfd_filter_host_ex), complex128 packed, --arith, for several n_p.  The
    host penalty is (t_host - t_device) / t_device.  The start block is drawn
    on the device (seeded) and copied into one page-locked host buffer; both
    are refilled from the seed before every run, so no second copy of X is
    held anywhere (the N x 512 block of the 200x200x100 lattice is 131 GB)."""
    import torch
    from paper_1803_02156_gb300 import binding as b, inputs
    torch.cuda.set_device(0)
    w = WORKLOAD
    L = tuple(int(v) for v in a.host_lattice.split("x"))
    n_s, n_b = a.host_n_s, a.n_b
    arith = 1 if a.arith == "dw" else 0
    p = b.topi_params(*L, t=w.t, m=w.m, gamma=w.gamma, seed=w.seed, periodic=w.periodic)
    H = b.cfd_build_matrix(p, w.sell_C, w.sell_sigma, "c128p")
    N, nnz = H.N, H.nnz
    n_ps = [int(v) for v in a.host_n_ps.split(",")]
    ws = max(b.cfd_filter_host_workspace(N, n_s, n_b, max(n_ps), "c128", "c128"),
             b.cfd_filter_workspace(N, n_s, n_b, max(n_ps), "c128", "c128"))
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    dev = torch.empty(N, n_s, dtype=torch.complex128, device="cuda")
    # page-locked by registering exactly the array's bytes (torch's pinned
    # allocator would round a 131 GB request up to a power of two)
    import numpy as np
    blocked = a.host_layout == "blocked"
    nblk = n_s // n_b
    Xn = np.empty((nblk, N, n_b) if blocked else (N, n_s), dtype=np.complex128)
    rc = torch.cuda.cudart().cudaHostRegister(Xn.ctypes.data, Xn.nbytes, 0)
    if int(rc) != 0:
        raise RuntimeError("cudaHostRegister of %d bytes failed (%s)" % (Xn.nbytes, rc))
    Xh = torch.from_numpy(Xn)
    stream = torch.cuda.current_stream()
    o = b.cfd_filter_opts(0, 0, 0, 0, 0, 0, arith, 0)

    def reset():
        inputs.fill_gaussian_device(dev, w.x_seed)
        if blocked:
            for k in range(nblk):
                Xh[k].copy_(dev[:, k * n_b:(k + 1) * n_b])
        else:
            Xh.copy_(dev)
        torch.cuda.synchronize()

    def timed(f):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        f()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    rows = []
    for n_p in n_ps:
        def run_dev():
            b._check(b.lib().cfd_filter_ex(H.ref(), BOUNDS[0], BOUNDS[1], -0.3, 0.3, n_p, b.block_of(dev), n_b,
                                           b._ptr(work), work.numel(), b._ptr(None), b.ctypes.byref(o),
                                           b._stream(stream)))

        def run_host_():
            if blocked:
                blk = b.cfd_block(Xh.data_ptr(), N, n_b, n_s, b.CFD_C128)
                b._check(b.lib().cfd_filter_host_blocked(H.ref(), BOUNDS[0], BOUNDS[1], -0.3, 0.3, n_p, blk, n_b,
                                                         b._ptr(work), work.numel(), b._ptr(None), b.ctypes.byref(o),
                                                         b._stream(stream)))
            else:
                b._check(b.lib().cfd_filter_host_ex(H.ref(), BOUNDS[0], BOUNDS[1], -0.3, 0.3, n_p, b.block_of(Xh),
                                                    n_b, b._ptr(work), work.numel(), b._ptr(None),
                                                    b.ctypes.byref(o), b._stream(stream)))
        res = {"device": [], "host": []}
        for r in range(a.warmup + a.steps):
            reset()
            td = timed(run_dev)
            th = timed(run_host_)
            if r >= a.warmup:
                res["device"].append(td)
                res["host"].append(th)
        # the host filter's result equals the device filter's (sampled rows)
        idx = torch.linspace(0, N - 1, 4096, dtype=torch.int64)
        hrows = torch.cat([Xh[k][idx] for k in range(nblk)], dim=1) if blocked else Xh[idx]
        same = bool(torch.equal(hrows, dev[idx.cuda()].cpu()))
        td, th = statistics.median(res["device"]), statistics.median(res["host"])
        moved = 2 * N * n_s * 16
        rows.append({"n_p": n_p, "device_s": round(td, 5), "host_s": round(th, 5),
                     "penalty": round(th / td - 1.0, 4), "link_gbs_if_serial": round(moved / max(th - td, 1e-9) / 1e9, 1),
                     "filter_gbs_device": round(model.filter_bytes(N, nnz, n_s, n_b, n_p) / td / 1e9, 1),
                     "filter_gbs_host": round(model.filter_bytes(N, nnz, n_s, n_b, n_p) / th / 1e9, 1),
                     "host_equals_device": same})
    torch.cuda.cudart().cudaHostUnregister(Xn.ctypes.data)
    print(json.dumps({"metric": "filter time, search space in host memory vs HBM", "unit": "s", "n_gpus": 1,
                      "steps": a.steps, "warmup": a.warmup, "data": "synthetic", "dtype": "c128",
                      "arith": a.arith,
                      "config": {"workload": "topi-%s" % a.host_lattice, "N": N, "n_s": n_s, "n_b": n_b,
                                 "host_bytes": N * n_s * 16, "storage": "packed", "pinned": True,
                                 "host_layout": a.host_layout},
                      "results": rows}))


def run_sweep(a):
    """Fused-filter throughput (filter with moments, per-step CUDA-event time of
    whole filter applications) on the configurations of the paper's method:
    64x64x32 complex128 with n_b = 8, 16, 32, 64 (n_s = 128); 200x200x100
    complex128 (N = 16e6, n_s = 256 in blocks of 32); 128x128x64 with the
    complex64 filter on a complex128 block (n_s = 256).  Start blocks are
    drawn on the device (seeded torch generator; the largest block is 65 GB).
    GB/s by the minimum-traffic model, Gflop/s by the paper's count and by
    the FP64/FP32 pipe's."""
    import torch
    from paper_1803_02156_gb300 import binding as b
    torch.cuda.set_device(0)
    hbm, hbm_src = measured_hbm_gbs()
    rows = []
    cases = [((64, 64, 32), "c128", "c128", 128, nb, 100) for nb in (8, 16, 32, 64)]
    cases += [((200, 200, 100), "c128", "c128", 256, 32, 40), ((128, 128, 64), "c64", "c128", 256, 32, 50)]
    for lat, ph, px, n_s, n_b, n_p in cases:
        p = b.topi_params(*lat, t=WORKLOAD.t, m=WORKLOAD.m, gamma=WORKLOAD.gamma, seed=WORKLOAD.seed,
                          periodic=WORKLOAD.periodic)
        H = b.cfd_build_matrix(p, 32, 1, ph + "p")
        g = torch.Generator(device="cuda")
        g.manual_seed(WORKLOAD.x_seed)
        dt = torch.complex128 if px == "c128" else torch.complex64
        X = torch.randn(H.N, n_s, dtype=dt, device="cuda", generator=g)
        work = torch.empty(b.cfd_filter_workspace(H.N, n_s, n_b, n_p, ph, px), dtype=torch.uint8, device="cuda")
        mu = torch.empty(n_s, 2 * n_p, dtype=torch.float64, device="cuda")
        blk = b.block_of(X)

        def once():
            b._check(b.lib().cfd_filter(H.ref(), BOUNDS[0], BOUNDS[1], -0.3, 0.3, n_p, blk, n_b, b._ptr(work),
                                        work.numel(), b._ptr(mu), b._stream()))
        ts = []
        for r in range(max(a.warmup, 1) + max(a.steps, 1)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            once()
            e1.record()
            torch.cuda.synchronize()
            if r >= max(a.warmup, 1):
                ts.append(e0.elapsed_time(e1) / 1e3)
        t_step = statistics.median(ts) / (n_p * (n_s // n_b))
        sb = model.step_bytes(H.N, H.nnz, n_b, ph)
        row = {"lattice": "x".join(map(str, lat)), "N": H.N, "nnz": H.nnz, "filter": ph, "block": px, "n_s": n_s,
               "n_b": n_b, "n_p": n_p, "ms_per_step": round(1e3 * t_step, 4), "gbs": round(sb / t_step / 1e9, 1),
               "frac_hbm": round(sb / t_step / 1e9 / hbm, 4),
               "gflops_paper": round(model.step_flops(H.N, H.nnz, n_b) / t_step / 1e9, 1),
               "gflops_pipe": round(model.step_fma_flops(H.N, H.nnz, n_b, packed=True, prepared=True)
                                    / t_step / 1e9, 1)}
        if ph == "c128":
            row["frac_fp64_peak"] = round(row["gflops_pipe"] / FP64_PEAK_GFLOPS, 4)
        rows.append(row)
        del X, work, H
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "fused filter SpMMV GB/s and Gflop/s per configuration", "unit": "GB/s",
                      "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "data": "synthetic",
                      "hbm_peak_gbs": hbm, "hbm_peak_source": hbm_src, "fp64_peak_gflops": round(FP64_PEAK_GFLOPS, 1),
                      "traffic_model": "nnz (s + 4) + 5 N n_b s bytes per step",
                      "flops_paper": "(8 nnz + 42 N) n_b per step", "results": rows}))


def run_tte(a):
    """Time to eigenpairs (residual <= 1e-10, cfd_solve from a device-resident
    random start block, after the untimed matrix build, Lanczos bounds and KPM
    window) for the fp64 policy and the mixed policy (complex64 filter, fp64
    SVQB, Rayleigh-Ritz and residuals, then fp64 filter sweeps) on one
    workload, with the per-eigenvalue difference between the two."""
    import torch
    from paper_1803_02156_gb300 import binding as b
    torch.cuda.set_device(0)
    w = workloads.ALL[a.tte_workload] if a.tte_workload else TTE_WORKLOAD
    p, H, lmin, lmax, lam_l, lam_r, kpm = setup_problem(b, w, w.seed, a.storage, with_kpm=True)
    res = time_to_eigenpairs(b, w, p, H, lmin, lmax, lam_l, lam_r, a.storage, tuple(a.tte_policies.split(",")))
    res["kpm_count_in_window"] = round(kpm, 2)
    print(json.dumps({"metric": "time to eigenpairs, fp64 vs mixed", "unit": "s", "n_gpus": 1, "data": "synthetic",
                      "higher_is_better": False,
                      "config": {"workload": w.name, "lattice": list(w.lattice), "N": H.N, "n_s": w.n_s,
                                 "n_t": w.n_t, "n_p": w.n_p, "n_b": w.n_b, "window": [lam_l, lam_r],
                                 "bounds": [lmin, lmax]},
                      "time_to_eigenpairs": res}))


def run_kernel(a):
    """Small case for profiling one kernel: --steps filter calls of one n_b
    block of the 64x64x32 lattice (N = 524288) with --n-p fused steps and
    moments, after --warmup calls (complex128 with --arith, or complex64)."""
    import torch
    from paper_1803_02156_gb300 import binding as b, inputs
    torch.cuda.set_device(0)
    w = WORKLOAD
    prec = a.prec
    H = b.cfd_build_matrix(b.topi_params(*w.lattice, seed=w.seed), 32, 1, prec + "p")
    dt = torch.complex128 if prec == "c128" else torch.complex64
    X = inputs.gaussian_block_device(H.N, a.n_b, seed=w.x_seed, dtype=dt)
    dw = prec == "c128" and a.arith == "dw"
    ts = []
    for r in range(a.warmup + a.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.cfd_filter_ex(H, *BOUNDS, -0.3, 0.3, a.n_p, X, a.n_b, moments=not a.no_moments, arith=1 if dw else 0,
                        gather=a.gather, vpt=a.vpt, footprint=a.footprint)
        e1.record()
        torch.cuda.synchronize()
        if r >= a.warmup:
            ts.append(e0.elapsed_time(e1) / 1e3)
    t = statistics.median(ts) / a.n_p
    print(json.dumps({"metric": "filter call, ms per step", "unit": "ms", "workload": w.name, "prec": prec,
                      "arith": "dw" if dw else "native", "gather": a.gather, "vpt": a.vpt, "footprint": a.footprint,
                      "moments": not a.no_moments, "n_b": a.n_b, "n_p": a.n_p,
                      "ms_per_step": round(1e3 * t, 4),
                      "model_gbs": round(model.step_bytes(H.N, H.nnz, a.n_b, prec) / t / 1e9, 1)}))


def run_dist(a):
    """The filter distributed over z-slabs of the 200x200x100 lattice, one slab
    per rank and GPU (Sect. 6), halo planes exchanged with NCCL
    (cfd_filter_slab_nccl): --dist-mode 0 vector mode (Algorithm 3), 1
    pipelined mode (Algorithm 4).  One step = one n_b block filtered with n_p
    fused steps; strong scaling (the lattice is fixed).  Under torchrun rank 0
    makes the NCCL id and torch.distributed hands it to the others."""
    import torch
    import torch.distributed as dist
    from paper_1803_02156_gb300 import binding as b, inputs
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("gloo")
    w = LARGE
    n_b, n_p = a.n_b, a.n_p
    uid = b.cfd_nccl_unique_id() if rank == 0 else None
    if world > 1:
        box = [uid]
        dist.broadcast_object_list(box, src=0)
        uid = box[0]
    comm = b.cfd_nccl_comm_init(uid, world, rank)
    p = b.topi_params(*w.lattice, t=w.t, m=w.m, gamma=w.gamma, seed=w.seed, periodic=w.periodic)
    s = b.cfd_slab_plan(p, world, rank)
    H = b.cfd_build_matrix_slab(p, s, w.sell_C, w.sell_sigma, "c128p")
    X = inputs.gaussian_block_device(w.N, n_b, seed=w.x_seed)[s.row0:s.row0 + s.n_local].contiguous()
    arith = 1 if a.arith == "dw" else 0
    mode = a.dist_mode

    def step():
        b.cfd_filter_slab_nccl(s, H, BOUNDS[0], BOUNDS[1], -0.3, 0.3, n_p, X, n_b, comm, mode=mode, moments=True,
                               arith=arith)
    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    t = max_over_ranks(e0.elapsed_time(e1) / 1e3)
    b.cfd_nccl_comm_destroy(comm)
    if rank == 0:
        byts = a.steps * n_p * model.step_bytes(w.N, w.nnz, n_b, "c128")
        print(json.dumps({"metric": METRIC + " (distributed over z-slabs)", "value": round(byts / t / 1e9, 3),
                          "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
                          "ms_per_step": round(1e3 * t / a.steps, 3), "higher_is_better": True, "scaling": "strong",
                          "dtype": "f32x2" if arith else "c128", "data": "synthetic",
                          "config": {"workload": w.name, "N": w.N, "n_b": n_b, "n_p": n_p,
                                     "mode": "pipelined" if mode else "vector", "parallelism": "z-slabs x%d" % world}}))
    if world > 1:
        dist.destroy_process_group()


def run_peaks(a):
    """Measured FMA rates of the fp64 and fp32 pipes (the library's probe)."""
    import torch
    from paper_1803_02156_gb300 import binding as b
    torch.cuda.set_device(0)
    out = {}
    for prec in ("c128", "c64"):
        rates = [b.cfd_probe_fma(prec, 1 << 15) / 1e9 for _ in range(max(a.steps, 1))]
        out[{"c128": "fp64", "c64": "fp32"}[prec]] = {"gflops_median": round(statistics.median(rates), 1),
                                                       "gflops_max": round(max(rates), 1)}
    print(json.dumps({"metric": "FMA pipe peaks", "unit": "GFLOP/s", "n_gpus": 1, "steps": a.steps,
                      "nominal_fp64_gflops": round(FP64_PEAK_GFLOPS, 1), "results": out}))


def run_dense(a):
    """The dense kernels of SVQB and Rayleigh-Ritz on an N x n complex-double
    block (N = --dense-n, n = 256, the 128x128x64 solve's shape by default):
    the Gram X^H Y (cfd_block_gram_ex) and one SVQB orthonormalisation (two
    Hermitian Grams and two in-place projections, cfd_orthogonalize_ex), in
    fp64 on the FP64 tensor cores and in double-word arithmetic on the fp32
    pipe.  GFLOP/s count 8 N n^2 real flops per Gram (the full product) and
    per projection, so SVQB's two passes count 4 x 8 N n^2 (its Hermitian
    Grams compute about half of that); CUDA events, median of --steps after
    --warmup."""
    import torch
    from paper_1803_02156_gb300 import binding as b, inputs
    torch.cuda.set_device(0)
    N, n = a.dense_n, 256
    X = inputs.gaussian_block_device(N, n, seed=5)
    Y = inputs.gaussian_block_device(N, n, seed=6)
    out = {}
    for arith, name in ((0, "fp64_tensor"), (1, "double_word")):
        def timed(fn):
            ts = []
            for r in range(a.warmup + a.steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                torch.cuda.synchronize()
                if r >= a.warmup:
                    ts.append(e0.elapsed_time(e1) / 1e3)
            return statistics.median(ts)
        tg = timed(lambda: b.cfd_block_gram(X, Y, arith=arith))
        Z = X.clone()

        def orth():
            Z.copy_(X)
            b.cfd_orthogonalize(Z, arith=arith)
        t0 = timed(lambda: Z.copy_(X))
        to = timed(orth) - t0
        flops = 8.0 * N * n * n
        out[name] = {"gram_s": round(tg, 5), "gram_gflops": round(flops / tg / 1e9, 1),
                     "svqb_s": round(to, 5),
                     "svqb_gflops": round(4 * flops / to / 1e9, 1)}
    out["speedup_gram"] = round(out["fp64_tensor"]["gram_s"] / out["double_word"]["gram_s"], 3)
    out["speedup_svqb"] = round(out["fp64_tensor"]["svqb_s"] / out["double_word"]["svqb_s"], 3)
    print(json.dumps({"metric": "dense SVQB / Rayleigh-Ritz kernels", "unit": "s", "n_gpus": 1, "steps": a.steps,
                      "warmup": a.warmup, "config": {"N": N, "n": n, "block": "complex double, Gaussian"},
                      "results": out}))


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.mode == "batch":
        run_batch(a)
    elif a.mode == "fusion":
        run_fusion(a)
    elif a.mode == "host":
        run_host(a)
    elif a.mode == "sweep":
        run_sweep(a)
    elif a.mode == "tte":
        run_tte(a)
    elif a.mode == "peaks":
        run_peaks(a)
    elif a.mode == "dense":
        run_dense(a)
    elif a.mode == "kernel":
        run_kernel(a)
    elif a.mode == "dist":
        run_dist(a)
    elif a.mode == "iteration":
        run_iteration(a)
    else:
        run_filter(a)


if __name__ == "__main__":
    main()
