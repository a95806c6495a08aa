"""GPU parity of the complex-double filter whose general steps run in
double-word arithmetic on the fp32 pipe (cfd_filter_opts.arith = 1), against
the CPU oracle, through the C ABI.

The double-word steps round each operation at a few units of 2^-48 relative
to the magnitudes of its terms instead of 2^-53, so the filtered block and
the moments carry about 30 times the native step's rounding; the tolerance
is the fp64 filter's bar of 1e-11 relative (Frobenius for the block, of
max |mu| for the moments)."""
import numpy as np
import pytest

import oracle
from paper_1803_02156_gb300 import inputs, workloads

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def b():
    import torch
    from paper_1803_02156_gb300 import build, binding
    assert torch.cuda.is_available()
    build.build()
    binding.lib()
    return binding


def _compare(b, L, n_s, n_b, n_p, win, C=32, sigma=1, seed=1, gather=0, tol=TOL):
    import torch
    H = b.cfd_build_matrix(b.topi_params(*L, seed=seed), C, sigma, "c128p")
    ref = oracle.topi_csr(*L, seed=seed)
    X = inputs.gaussian_block(ref.N, n_s, seed=2)
    Xg = torch.from_numpy(X).cuda()
    mu = b.cfd_filter_ex(H, -8.6, 8.6, win[0], win[1], n_p, Xg, n_b, moments=True, arith=1, gather=gather)
    torch.cuda.synchronize()
    Y, dots = oracle.chebfd_filter(ref, -8.6, 8.6, win[0], win[1], n_p, X, n_b)
    err = np.linalg.norm(Xg.cpu().numpy() - Y) / np.linalg.norm(Y)
    muref = oracle.kpm_moments(dots)
    merr = np.max(np.abs(mu.cpu().numpy() - muref)) / np.max(np.abs(muref))
    assert err < tol, err
    assert merr < tol, merr
    return Xg, mu, err, merr


@pytest.mark.parametrize("n_b", [8, 16, 32, 64])
def test_dw_filter_parity_small_config(b, n_b):
    """8x8x8 (N = 2048), n_s = 64, n_p = 200: block and moments vs oracle."""
    w = workloads.SMALL
    _compare(b, w.lattice, 64, n_b, w.n_p, (-0.7, 0.7))


@pytest.mark.parametrize("L,n_s,n_b,n_p,C,sigma", [((13, 7, 5), 48, 16, 25, 32, 64),
                                                   ((9, 10, 3), 16, 16, 3, 32, 1),
                                                   ((16, 16, 9), 64, 32, 40, 16, 1),
                                                   ((5, 4, 6), 16, 8, 30, 8, 32)])
def test_dw_filter_parity_ragged(b, L, n_s, n_b, n_p, C, sigma):
    """Ragged tails, sigma-sorted rows, a single general step (n_p = 3), and
    chunk heights other than 32 (the kernel with the height at run time)."""
    _compare(b, L, n_s, n_b, n_p, (-1.1, 0.4), C=C, sigma=sigma)


def test_dw_full_size_parity(b):
    """The 64x64x32 lattice (N = 524288), n_b = 32, 12 steps, against the oracle."""
    w = workloads.MEDIUM
    _compare(b, w.lattice, 32, 32, 12, (-0.3, 0.3))


def test_dw_full_degree_against_native(b):
    """64x64x32 at the full degree n_p = 1000: the double-word filter against
    the native fp64 one (itself within the oracle's bar), block and moments."""
    import torch
    w = workloads.MEDIUM
    H = b.cfd_build_matrix(b.topi_params(*w.lattice), 32, 1, "c128p")
    X0 = torch.from_numpy(inputs.gaussian_block(w.N, 32, seed=2)).cuda()
    Xn, Xd = X0.clone(), X0.clone()
    mn = b.cfd_filter(H, -8.6, 8.6, -0.3, 0.3, w.n_p, Xn, 32, moments=True)
    md = b.cfd_filter_ex(H, -8.6, 8.6, -0.3, 0.3, w.n_p, Xd, 32, moments=True, arith=1)
    torch.cuda.synchronize()
    assert (torch.linalg.norm(Xd - Xn) / torch.linalg.norm(Xn)).item() < TOL
    assert (torch.max(torch.abs(md - mn)) / torch.max(torch.abs(mn))).item() < TOL


@pytest.mark.parametrize("n_b", [16, 32])
def test_dw_vectors_per_thread_bitwise_equal(b, n_b):
    """One or two vectors per thread change no element's arithmetic: bitwise
    equal block; moments equal up to the order of their reduction."""
    import torch
    H = b.cfd_build_matrix(b.topi_params(12, 10, 7), 32, 1, "c128p")
    X0 = torch.from_numpy(inputs.gaussian_block(H.N, 64, seed=9)).cuda()
    Xa, Xb = X0.clone(), X0.clone()
    ma = b.cfd_filter_ex(H, -8.6, 8.6, -0.6, 0.4, 50, Xa, n_b, moments=True, arith=1, vpt=1)
    mb = b.cfd_filter_ex(H, -8.6, 8.6, -0.6, 0.4, 50, Xb, n_b, moments=True, arith=1, vpt=2)
    torch.cuda.synchronize()
    assert torch.equal(Xa, Xb)
    assert (torch.max(torch.abs(ma - mb)) / torch.max(torch.abs(ma))).item() < 1e-13


def test_dw_block_width_invariance(b):
    """The double-word filtered block does not depend on n_b (each vector's
    arithmetic is the same whatever block it is filtered in)."""
    import torch
    H = b.cfd_build_matrix(b.topi_params(12, 10, 7), 32, 1, "c128p")
    X = torch.from_numpy(inputs.gaussian_block(H.N, 64, seed=4)).cuda()
    outs = []
    for n_b in (8, 16, 32, 64):
        Xg = X.clone()
        b.cfd_filter_ex(H, -8.6, 8.6, -0.5, 0.5, 60, Xg, n_b, arith=1)
        outs.append(Xg)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])


def test_dw_degree_two_is_native(b):
    """n_p = 2 has no general step: the result equals the native filter's."""
    import torch
    H = b.cfd_build_matrix(b.topi_params(8, 8, 4), 32, 1, "c128p")
    X0 = torch.from_numpy(inputs.gaussian_block(H.N, 16, seed=5)).cuda()
    Xa, Xb = X0.clone(), X0.clone()
    b.cfd_filter(H, -8.6, 8.6, -0.5, 0.5, 2, Xa, 16)
    b.cfd_filter_ex(H, -8.6, 8.6, -0.5, 0.5, 2, Xb, 16, arith=1)
    assert torch.equal(Xa, Xb)


def test_dw_wait_timeout_reported(b):
    """The bounded waits of the double-word step made to expire (staged = 2):
    CFD_ERR_TIMEOUT in the workspace status, the context still usable."""
    import torch
    H = b.cfd_build_matrix(b.topi_params(8, 8, 4), 32, 1, "c128p")
    X = torch.from_numpy(inputs.gaussian_block(H.N, 16, seed=6)).cuda()
    work = torch.empty(b.cfd_filter_workspace(H.N, 16, 16, 10, "c128", "c128"), dtype=torch.uint8, device="cuda")
    b.cfd_filter_ex(H, -8.6, 8.6, -0.5, 0.5, 10, X, 16, arith=1, staged=2, work=work)
    with pytest.raises(b.CfdError) as e:
        b.cfd_workspace_status(work)
    assert e.value.status == 5
    assert "still have been in flight" not in str(e.value)     # the drain completed
    X2 = X.clone()
    b.cfd_filter_ex(H, -8.6, 8.6, -0.5, 0.5, 10, X2, 16, arith=1, work=work)
    b.cfd_workspace_status(work)


@pytest.mark.parametrize("prec", ["c128", "c64p"])
def test_dw_rejects_unsupported(b, prec):
    import torch
    H = b.cfd_build_matrix(b.topi_params(4, 4, 4), 32, 1, prec)
    dt = torch.complex64 if prec.startswith("c64") else torch.complex128
    X = torch.zeros(H.N, 16, dtype=dt, device="cuda")
    with pytest.raises(b.CfdError) as e:
        b.cfd_filter_ex(H, -8.6, 8.6, -0.5, 0.5, 10, X, 16, arith=1)
    assert e.value.status == 1
