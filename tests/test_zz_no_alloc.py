"""cfd_filter_noalloc, the filter entry point for callers that may not
allocate device memory (an application-owned memory pool or budget forbids
cudaMalloc, or a latency-critical loop cannot afford it): its scratch is a
static array inside the library.  Checked against cfd_filter through the C
ABI on two calls in a row, since every call reuses the same scratch.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1803_02156_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-11      # the fp64 filter parity tolerance of the other GPU tests


@pytest.fixture(scope="module")
def b():
    import torch
    from paper_1803_02156_gb300 import build, binding
    assert torch.cuda.is_available()
    build.build()
    binding.lib()
    return binding


@pytest.mark.parametrize("prec,L,n_s,n_b,n_p", [("c128", (8, 8, 8), 32, 32, 200),
                                                 ("c64", (12, 10, 7), 48, 16, 90)])
def test_noalloc_matches_filter_twice(b, prec, L, n_s, n_b, n_p):
    import torch
    H = b.cfd_build_matrix(b.topi_params(*L), 32, 1, prec)
    dt = torch.complex128 if prec == "c128" else torch.complex64
    X0 = torch.from_numpy(inputs.gaussian_block(H.N, n_s, seed=2)).to(dt).cuda()
    ref = X0.clone()
    mu_ref = b.cfd_filter(H, -8.6, 8.6, -0.7, 0.7, n_p, ref, n_b, moments=True)
    mu = torch.empty(n_s, 2 * n_p, dtype=torch.float64, device="cuda")
    for _ in range(2):                       # the second call finds the first call's scratch contents
        X = X0.clone()
        mu.fill_(float("nan"))
        b.cfd_filter_noalloc(H, -8.6, 8.6, -0.7, 0.7, n_p, X, n_b, moments=mu)
        torch.cuda.synchronize()
        err = (torch.linalg.norm(X - ref) / torch.linalg.norm(ref)).item()
        merr = (torch.max(torch.abs(mu - mu_ref)) / torch.max(torch.abs(mu_ref))).item()
        assert err < TOL, err
        assert merr < TOL, merr


def test_noalloc_rejects_too_large(b):
    """The 64x64x32 lattice with n_b = 32 needs far more than the static scratch."""
    import torch
    H = b.cfd_build_matrix(b.topi_params(64, 64, 32), 32, 1, "c128")
    X = torch.zeros(H.N, 32, dtype=torch.complex128, device="cuda")
    with pytest.raises(b.CfdError) as e:
        b.cfd_filter_noalloc(H, -8.6, 8.6, -0.5, 0.5, 10, X, 32)
    assert e.value.status == 1
    assert "static scratch" in str(e.value)
