"""GPU parity of the unfused filter (separate SpMMV and BLAS-1 kernels, the
fusion baseline of Sect. 4, Fig. 2) against the CPU oracle and against the
fused filter, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1803_02156_gb300 import inputs, workloads

pytestmark = pytest.mark.gpu

TOL_C128 = 1e-11


@pytest.fixture(scope="module")
def b():
    import torch
    from paper_1803_02156_gb300 import build, binding
    assert torch.cuda.is_available()
    build.build()
    binding.lib()
    return binding


def _run(b, L, n_s, n_b, n_p, win, prec, fused, X, bounds=(-8.6, 8.6)):
    import torch
    H = b.cfd_build_matrix(b.topi_params(*L, seed=1), 32, 1, prec)
    cdt = torch.complex64 if prec.startswith("c64") and X.dtype == np.complex64 else torch.complex128
    Xg = torch.from_numpy(np.ascontiguousarray(X)).to(cdt).cuda()
    f = b.cfd_filter if fused else b.cfd_filter_unfused
    mu = f(H, bounds[0], bounds[1], win[0], win[1], n_p, Xg, n_b, moments=True)
    torch.cuda.synchronize()
    return Xg.cpu().numpy().astype(np.complex128), mu.cpu().numpy()


def _oracle(L, n_p, win, X, n_b, bounds=(-8.6, 8.6)):
    ref = oracle.topi_csr(*L, seed=1)
    Y, dots = oracle.chebfd_filter(ref, bounds[0], bounds[1], win[0], win[1], n_p, X, n_b)
    return Y, oracle.kpm_moments(dots)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["c128", "c128p"])
@pytest.mark.parametrize("L,n_s,n_b,n_p", [(workloads.SMALL.lattice, 32, 32, 200), ((13, 7, 5), 48, 16, 25),
                                           ((9, 10, 3), 8, 8, 2), ((16, 16, 9), 64, 64, 40)])
def test_unfused_parity_c128(b, prec, L, n_s, n_b, n_p):
    """Filtered block and moments vs the oracle (1e-11), several chunks and ragged tails."""
    N = 4 * L[0] * L[1] * L[2]
    X = inputs.gaussian_block(N, n_s, seed=2)
    Y, mu = _run(b, L, n_s, n_b, n_p, (-1.1, 0.4), prec, False, X)
    Yr, mur = _oracle(L, n_p, (-1.1, 0.4), X, n_b)
    assert _rel(Y, Yr) < TOL_C128
    assert np.max(np.abs(mu - mur)) / np.max(np.abs(mur)) < TOL_C128


@pytest.mark.parametrize("prec", ["c64", "c64p"])
def test_unfused_parity_c64(b, prec):
    """complex64 chain vs the fp64 oracle within the fp32 bar of the fused path
    (n_p x 13 x 2^-24 relative)."""
    L, n_s, n_b, n_p = (8, 8, 8), 32, 32, 200
    X = inputs.gaussian_block(4 * 512, n_s, seed=2).astype(np.complex64)
    Y, mu = _run(b, L, n_s, n_b, n_p, (-0.7, 0.7), prec, False, X)
    Yr, mur = _oracle(L, n_p, (-0.7, 0.7), X.astype(np.complex128), n_b)
    tol = n_p * 13 * 2.0 ** -24
    assert _rel(Y, Yr) < tol
    assert np.max(np.abs(mu - mur)) / np.max(np.abs(mur)) < tol


def test_unfused_mixed_blocks(b):
    """complex64 matrix with complex128 blocks (narrowed per block, widened back)."""
    L, n_s, n_b, n_p = (8, 8, 8), 32, 16, 100
    X = inputs.gaussian_block(4 * 512, n_s, seed=3)
    Yu, mu_u = _run(b, L, n_s, n_b, n_p, (-0.7, 0.7), "c64p", False, X)
    Yf, mu_f = _run(b, L, n_s, n_b, n_p, (-0.7, 0.7), "c64p", True, X)
    Yr, _ = _oracle(L, n_p, (-0.7, 0.7), X, n_b)
    tol = n_p * 13 * 2.0 ** -24
    assert _rel(Yu, Yr) < tol and _rel(Yf, Yr) < tol


def test_unfused_matches_fused_c128(b):
    """Fused and unfused compute the same recurrence: they agree to rounding."""
    L, n_s, n_b, n_p = (16, 16, 8), 64, 32, 120
    X = inputs.gaussian_block(4 * 16 * 16 * 8, n_s, seed=4)
    Yu, mu_u = _run(b, L, n_s, n_b, n_p, (-0.5, 0.5), "c128p", False, X)
    Yf, mu_f = _run(b, L, n_s, n_b, n_p, (-0.5, 0.5), "c128p", True, X)
    assert _rel(Yu, Yf) < 1e-12
    assert np.max(np.abs(mu_u - mu_f)) / np.max(np.abs(mu_f)) < 1e-12


def test_unfused_deterministic(b):
    L, n_s, n_b, n_p = (12, 10, 7), 32, 16, 30
    X = inputs.gaussian_block(4 * 12 * 10 * 7, n_s, seed=5)
    a = _run(b, L, n_s, n_b, n_p, (-0.5, 0.5), "c128", False, X)
    c = _run(b, L, n_s, n_b, n_p, (-0.5, 0.5), "c128", False, X)
    assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1])


def test_unfused_argument_errors(b):
    import torch
    H = b.cfd_build_matrix(b.topi_params(4, 4, 4), 32, 1, "c128")
    X = torch.zeros(256, 16, dtype=torch.complex128, device="cuda")
    with pytest.raises(b.CfdError):
        b.cfd_filter_unfused(H, -8.6, 8.6, -0.5, 0.5, 1, X, 16)          # n_p < 2
    with pytest.raises(b.CfdError):
        b.cfd_filter_unfused(H, -8.6, 8.6, -0.5, 0.5, 10, X, 12)         # n_b not allowed
    with pytest.raises(b.CfdError):
        b.cfd_filter_unfused(H, -8.6, 8.6, 0.5, -0.5, 10, X, 16)         # empty window
