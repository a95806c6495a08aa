"""Autotuner: search logic and cache on the CPU (fake timings), a real tuning
run on the GPU."""
import os

import pytest

from paper_1803_02156_gb300 import autotune


def test_staged_search_finds_planted_optimum():
    # cost model with a unique optimum at n_b=32, vpt=2, C=64, sigma=512, packed, persistent
    def measure(cfg):
        c = 1.0
        c += 0.0 if cfg["n_b"] == 32 else 0.3
        c += 0.0 if cfg["vpt"] == 2 else 0.2
        c += 0.0 if cfg["C"] == 64 else 0.1
        c += 0.0 if cfg["sigma"] == 8 * cfg["C"] else 0.05
        c += 0.0 if cfg["storage"] == "packed" else 0.4
        c += 0.0 if cfg["persistent"] else 0.01
        return c
    best, log = autotune.staged_search(128, "c64", measure)
    assert best == {"n_b": 32, "vpt": 2, "C": 64, "sigma": 512, "storage": "packed", "persistent": 1}
    assert len(log) < 25


def test_candidates_respect_limits():
    assert autotune.candidate_blocks(48) == [8, 16]
    assert autotune.candidate_vpt("c128", 64) == [2]
    assert autotune.candidate_vpt("c64", 16) == [1, 2]


def test_cache_roundtrip(tmp_path):
    p = os.path.join(tmp_path, "sub", "tune.json")
    k = autotune.cache_key((8, 8, 8), "c128", 32, "GB300")
    autotune.save_cache(p, {k: {"n_b": 16}})
    assert autotune.load_cache(p)[k]["n_b"] == 16
    assert autotune.load_cache(os.path.join(tmp_path, "missing.json")) == {}


@pytest.mark.gpu
def test_autotune_on_gpu(tmp_path):
    import torch
    from paper_1803_02156_gb300 import build, binding as b
    build.build()
    p = b.topi_params(16, 16, 8)
    cfg = autotune.autotune(p, "c64", n_s=64, steps=4, repeats=2, cache_path=os.path.join(tmp_path, "t.json"))
    assert cfg["n_b"] in (8, 16, 32, 64) and cfg["C"] in (8, 16, 32, 64, 128)
    assert cfg["sec_per_vector_step"] > 0
    again = autotune.autotune(p, "c64", n_s=64, cache_path=os.path.join(tmp_path, "t.json"))
    assert again == cfg                                           # served from the cache
    # the tuned configuration computes the default configuration's result (to the
    # fp32 rounding of a different summation order when it packs the values)
    H0 = b.cfd_build_matrix(p, 32, 1, "c64")
    H1 = b.cfd_build_matrix(p, cfg["C"], cfg["sigma"], "c64" + ("p" if cfg["storage"] == "packed" else ""))
    X = torch.randn(H0.N, 64, dtype=torch.complex64, device="cuda")
    Y0, Y1 = X.clone(), X.clone()
    b.cfd_filter(H0, -9.0, 9.0, -0.5, 0.5, 30, Y0, 32)
    b.cfd_filter_ex(H1, -9.0, 9.0, -0.5, 0.5, 30, Y1, cfg["n_b"], vpt=cfg["vpt"], persistent=cfg["persistent"])
    assert (torch.linalg.norm(Y0 - Y1) / torch.linalg.norm(Y0)).item() < 30 * 13 * 2.0 ** -24
