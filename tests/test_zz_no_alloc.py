"""cfd_filter_noalloc, the filter entry point for callers that may not
allocate device memory (an application-owned memory pool or budget forbids
cudaMalloc, or a latency-critical loop cannot afford it): its scratch is a
static array inside the library.  Checked against cfd_filter through the C
ABI on two calls in a row of two problems with different scratch layouts,
with the scratch's device status read after every call, since every call
reuses the same scratch.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1803_02156_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-11      # the fp64 filter parity tolerance of the other GPU tests
TOL_C64 = 1e-6   # same fp32 kernels on the same input: only the reduction order of the moments may differ


@pytest.fixture(scope="module")
def b():
    import torch
    from paper_1803_02156_gb300 import build, binding
    assert torch.cuda.is_available()
    build.build()
    binding.lib()
    return binding


# Two problems with different layouts of the shared scratch (precision, N,
# n_b, n_p), called alternately, so each call finds the other's leftovers at
# different offsets: status word, CTA ticket, recurrence blocks, dot partials.
CASES = [("c128", (8, 8, 8), 32, 32, 200, (-0.7, 0.7)),
         ("c64", (12, 10, 7), 48, 16, 90, (-0.6, 0.4))]


def test_noalloc_matches_filter_alternating(b):
    import torch
    refs = []
    for prec, L, n_s, n_b, n_p, win in CASES:
        H = b.cfd_build_matrix(b.topi_params(*L), 32, 1, prec)
        dt = torch.complex128 if prec == "c128" else torch.complex64
        X0 = torch.from_numpy(inputs.gaussian_block(H.N, n_s, seed=2)).to(dt).cuda()
        ref = X0.clone()
        mu_ref = b.cfd_filter(H, -8.6, 8.6, win[0], win[1], n_p, ref, n_b, moments=True)
        tol = TOL if prec == "c128" else TOL_C64
        refs.append((H, X0, ref, mu_ref, n_b, n_p, win, tol))
    for rep in range(2):                     # two calls in a row of each, interleaved
        for H, X0, ref, mu_ref, n_b, n_p, win, tol in refs:
            X = X0.clone()
            mu = torch.full((X0.shape[1], 2 * n_p), float("nan"), dtype=torch.float64, device="cuda")
            b.cfd_filter_noalloc(H, -8.6, 8.6, win[0], win[1], n_p, X, n_b, moments=mu)
            b.cfd_filter_noalloc_status()    # raises on a recorded device-side error
            err = (torch.linalg.norm(X - ref) / torch.linalg.norm(ref)).item()
            merr = (torch.max(torch.abs(mu - mu_ref)) / torch.max(torch.abs(mu_ref))).item()
            assert err < tol, (rep, err)
            assert merr < tol, (rep, merr)


def test_noalloc_status_reports_bad_bounds(b):
    """Bounds that cut the spectrum make the moments grow: the status of the
    static scratch reports CFD_ERR_BOUNDS, and the next good call clears it."""
    import torch
    H = b.cfd_build_matrix(b.topi_params(8, 8, 4), 32, 1, "c128")
    X0 = torch.from_numpy(inputs.gaussian_block(H.N, 16, seed=14)).cuda()
    mu = torch.empty(16, 80, dtype=torch.float64, device="cuda")
    X = X0.clone()
    b.cfd_filter_noalloc(H, -2.0, 2.0, -0.5, 0.5, 40, X, 16, moments=mu)
    with pytest.raises(b.CfdError) as e:
        b.cfd_filter_noalloc_status()
    assert e.value.status == 4               # CFD_ERR_BOUNDS
    X = X0.clone()
    b.cfd_filter_noalloc(H, -8.6, 8.6, -0.5, 0.5, 40, X, 16, moments=mu)
    b.cfd_filter_noalloc_status()


def test_noalloc_reports_argument_errors_first(b):
    """An invalid block width on a problem too large for the scratch is
    reported as the argument error, not as a size error."""
    import torch
    H = b.cfd_build_matrix(b.topi_params(64, 64, 32), 32, 1, "c128")
    X = torch.zeros(H.N, 32, dtype=torch.complex128, device="cuda")
    with pytest.raises(b.CfdError) as e:
        b.cfd_filter_noalloc(H, -8.6, 8.6, -0.5, 0.5, 10, X, 7)
    assert e.value.status == 1
    assert "n_b=7" in str(e.value)


def test_noalloc_rejects_too_large(b):
    """The 64x64x32 lattice with n_b = 32 needs far more than the static scratch."""
    import torch
    H = b.cfd_build_matrix(b.topi_params(64, 64, 32), 32, 1, "c128")
    X = torch.zeros(H.N, 32, dtype=torch.complex128, device="cuda")
    with pytest.raises(b.CfdError) as e:
        b.cfd_filter_noalloc(H, -8.6, 8.6, -0.5, 0.5, 10, X, 32)
    assert e.value.status == 1
    assert "static scratch" in str(e.value)
