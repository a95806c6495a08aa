"""Autotuner for the fused ChebFD filter: picks the subspace block width n_b,
the SELL chunk height C and sorting window sigma, the threads per row
(vectors per thread), the matrix value storage and the launch style for one
matrix shape and precision on the current GPU.

Search (staged, each stage keeps the best of the previous ones):
  1. n_b in {8, 16, 32, 64} (dividing n_s) x vectors per thread {1, 2}
  2. C in {8, 16, 32, 64, 128}
  3. sigma in {1, C, 8 C}
  4. value storage {packed real/imaginary, complex} and launch {per step, persistent}
Cost of a candidate: device time of `steps` fused steps on one n_b block,
divided by n_b (the whole filter costs n_s / n_b blocks of n_p steps), median
of `repeats` CUDA-event timings.  Results are cached per (lattice, precision,
n_s, device) in a JSON file.

Every candidate computes the same filtered block: the options only change
speed (the kernel tests check this bit for bit).
"""
import json
import os
import statistics

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "cfd_autotune.json")


def candidate_blocks(n_s):
    return [nb for nb in (8, 16, 32, 64) if n_s % nb == 0]


def candidate_vpt(prec, n_b):
    return [v for v in (1, 2) if not (v == 1 and n_b > 32)]


def cache_key(lattice, prec, n_s, device_name):
    return "%s|%s|%d|%s" % ("x".join(str(v) for v in lattice), prec, n_s, device_name)


def load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(path, cache):
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def staged_search(n_s, prec, measure):
    """Run the staged search with `measure(cfg) -> seconds per vector-step`
    (cfg: dict with n_b, vpt, C, sigma, storage, persistent).  Returns
    (best cfg, list of (cfg, cost))."""
    log = []

    def run(cfg):
        c = measure(dict(cfg))
        log.append((dict(cfg), c))
        return c

    best = None
    base = {"C": 32, "sigma": 1, "storage": "packed", "persistent": 0}
    for nb in candidate_blocks(n_s):
        for vpt in candidate_vpt(prec, nb):
            cfg = dict(base, n_b=nb, vpt=vpt)
            c = run(cfg)
            if best is None or c < best[1]:
                best = (cfg, c)
    for C in (8, 16, 64, 128):
        cfg = dict(best[0], C=C)
        c = run(cfg)
        if c < best[1]:
            best = (cfg, c)
    C = best[0]["C"]
    for sigma in (C, 8 * C):
        cfg = dict(best[0], sigma=sigma)
        c = run(cfg)
        if c < best[1]:
            best = (cfg, c)
    for storage, pers in (("complex", 0), ("packed", 1), ("complex", 1)):
        cfg = dict(best[0], storage=storage, persistent=pers)
        if cfg == best[0]:
            continue
        c = run(cfg)
        if c < best[1]:
            best = (cfg, c)
    return best[0], log


def autotune(params, prec="c128", n_s=128, steps=6, repeats=3, cache_path=DEFAULT_CACHE, refresh=False):
    """Tune the filter for the Topi parameters `params` (binding.topi_params)
    on the current CUDA device; returns the best configuration dict with its
    measured cost ("sec_per_vector_step")."""
    import torch
    from . import binding as b

    dev = torch.cuda.get_device_name()
    lattice = (params.Nx, params.Ny, params.Nz)
    key = cache_key(lattice, prec, n_s, dev)
    cache = load_cache(cache_path) if cache_path else {}
    if key in cache and not refresh:
        return cache[key]

    cdt = torch.complex128 if prec == "c128" else torch.complex64
    N = 4 * params.Nx * params.Ny * params.Nz
    mats = {}
    X0 = torch.randn(N, 64, dtype=cdt, device="cuda")

    def matrix(C, sigma, storage):
        k = (C, sigma, storage)
        if k not in mats:
            mats.clear()
            mats[k] = b.cfd_build_matrix(params, C, sigma, prec + ("p" if storage == "packed" else ""))
        return mats[k]

    def measure(cfg):
        H = matrix(cfg["C"], cfg["sigma"], cfg["storage"])
        nb = cfg["n_b"]
        X = X0[:, :nb].clone()
        ws = b.cfd_filter_workspace(N, nb, nb, steps, prec, prec)
        work = torch.empty(ws, dtype=torch.uint8, device="cuda")
        times = []
        for r in range(repeats + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b.cfd_filter_ex(H, -9.0, 9.0, -0.5, 0.5, steps, X, nb, vpt=cfg["vpt"],
                            persistent=cfg["persistent"], work=work)
            e1.record()
            torch.cuda.synchronize()
            if r:
                times.append(e0.elapsed_time(e1) * 1e-3)
        return statistics.median(times) / (steps * nb)

    best, log = staged_search(n_s, prec, measure)
    best = dict(best, sec_per_vector_step=min(c for _, c in log if _ == best),
                log=[dict(cfg, cost=c) for cfg, c in log])
    if cache_path:
        cache[key] = best
        save_cache(cache_path, cache)
    return best
