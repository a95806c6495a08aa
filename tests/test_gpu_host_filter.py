"""GPU tests of the filter over a search space held in host memory: the
blocks go through two device staging buffers, so the filtered block and the
moments must equal the device-resident filter bit for bit."""
import numpy as np
import pytest

from paper_1803_02156_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def b():
    import torch
    from paper_1803_02156_gb300 import build, binding
    assert torch.cuda.is_available()
    build.build()
    binding.lib()
    return binding


@pytest.mark.parametrize("L,n_s,n_b,n_p,prec,pinned", [
    ((16, 16, 8), 128, 32, 40, "c128p", True),     # 4 blocks
    ((13, 7, 5), 48, 16, 25, "c128", True),        # 3 blocks, ragged rows
    ((8, 8, 8), 32, 32, 60, "c128p", False),       # one block, pageable memory
    ((12, 10, 7), 64, 16, 30, "c64p", True),       # mixed: complex64 matrix, complex128 blocks
])
def test_host_filter_equals_device_filter(b, L, n_s, n_b, n_p, prec, pinned):
    import torch
    H = b.cfd_build_matrix(b.topi_params(*L, seed=1), 32, 1, prec)
    X = torch.from_numpy(inputs.gaussian_block(H.N, n_s, seed=2))
    Xd = X.cuda()
    mu_d = b.cfd_filter(H, -8.6, 8.6, -0.6, 0.4, n_p, Xd, n_b, moments=True)
    Xh = X.clone().pin_memory() if pinned else X.clone()
    mu_h = b.cfd_filter_host(H, -8.6, 8.6, -0.6, 0.4, n_p, Xh, n_b, moments=True)
    torch.cuda.synchronize()
    assert np.array_equal(Xh.numpy(), Xd.cpu().numpy())
    assert np.array_equal(mu_h.cpu().numpy(), mu_d.cpu().numpy())
    assert not np.array_equal(Xh.numpy(), X.numpy())


@pytest.mark.parametrize("prec,tol", [("c128p", 1e-11), ("c64p", 60 * 13 * 2.0 ** -24)])
def test_host_filter_vs_oracle(b, prec, tol):
    """The host-memory filter against the oracle directly (block and moments):
    8x8x8, n_s = 64 in two blocks of 32, n_p = 60."""
    import torch
    import oracle
    L, n_s, n_b, n_p, win = (8, 8, 8), 64, 32, 60, (-0.7, 0.7)
    H = b.cfd_build_matrix(b.topi_params(*L, seed=1), 32, 1, prec)
    ref = oracle.topi_csr(*L, seed=1)
    X = inputs.gaussian_block(ref.N, n_s, seed=2)
    Xh = torch.from_numpy(X.copy()).pin_memory()
    mu = b.cfd_filter_host(H, -8.6, 8.6, win[0], win[1], n_p, Xh, n_b, moments=True)
    Y, dots = oracle.chebfd_filter(ref, -8.6, 8.6, win[0], win[1], n_p, X, n_b)
    err = np.linalg.norm(Xh.numpy() - Y) / np.linalg.norm(Y)
    muref = oracle.kpm_moments(dots)
    merr = np.max(np.abs(mu.cpu().numpy() - muref)) / np.max(np.abs(muref))
    assert err < tol, err
    assert merr < tol, merr


@pytest.mark.parametrize("prec,arith,pinned,n_p", [("c128p", 1, True, 30), ("c128p", 0, False, 30), ("c64p", 0, True, 30),
                                                   ("c128p", 1, True, 50), ("c64p", 0, False, 50)])
def test_host_filter_blocked_equals_device_filter(b, prec, arith, pinned, n_p):
    """A search space stored block after block in host memory (one contiguous
    copy per block) gives the device filter's block and moments bit for bit,
    with the overlapped copies of low degrees (n_p = 30) and the serial
    copies of high degrees (n_p = 50)."""
    import torch
    L, n_s, n_b = (12, 10, 7), 64, 16
    H = b.cfd_build_matrix(b.topi_params(*L, seed=1), 32, 1, prec)
    dt = torch.complex64 if prec.startswith("c64") else torch.complex128
    X = torch.from_numpy(inputs.gaussian_block(H.N, n_s, seed=2)).to(dt)
    Xd = X.cuda()
    mu_d = b.cfd_filter_ex(H, -8.6, 8.6, -0.6, 0.4, n_p, Xd, n_b, moments=True, arith=arith)
    Xb = X.reshape(H.N, n_s // n_b, n_b).permute(1, 0, 2).contiguous()
    if pinned:
        Xb = Xb.pin_memory()
    mu_h = b.cfd_filter_host_blocked(H, -8.6, 8.6, -0.6, 0.4, n_p, Xb, n_b, moments=True, arith=arith)
    torch.cuda.synchronize()
    got = Xb.permute(1, 0, 2).reshape(H.N, n_s)
    assert torch.equal(got, Xd.cpu())
    assert torch.equal(mu_h, mu_d)


def test_host_filter_strided_host_block(b):
    """A column window of a wider host array (ld > n_s) is filtered in place;
    the other columns are untouched."""
    import torch
    H = b.cfd_build_matrix(b.topi_params(8, 8, 4, seed=1), 32, 1, "c128p")
    big = torch.from_numpy(inputs.gaussian_block(H.N, 48, seed=3)).pin_memory()
    ref = big.clone()
    win = big[:, 8:40]
    b.cfd_filter_host(H, -8.6, 8.6, -0.5, 0.5, 20, win, 16)
    Xd = ref[:, 8:40].contiguous().cuda()
    b.cfd_filter(H, -8.6, 8.6, -0.5, 0.5, 20, Xd, 16)
    assert np.array_equal(big[:, 8:40].numpy(), Xd.cpu().numpy())
    assert np.array_equal(big[:, :8].numpy(), ref[:, :8].numpy())
    assert np.array_equal(big[:, 40:].numpy(), ref[:, 40:].numpy())


def test_host_filter_rejects_device_block(b):
    import torch
    from paper_1803_02156_gb300.binding import CfdError, block_of, lib, _ptr, _stream
    H = b.cfd_build_matrix(b.topi_params(4, 4, 4), 32, 1, "c128")
    Xd = torch.zeros(H.N, 16, dtype=torch.complex128, device="cuda")
    work = torch.empty(b.cfd_filter_host_workspace(H.N, 16, 16, 10, "c128", "c128"), dtype=torch.uint8,
                       device="cuda")
    st = lib().cfd_filter_host(H.ref(), -8.6, 8.6, -0.5, 0.5, 10, block_of(Xd), 16, _ptr(work), work.numel(),
                               _ptr(None), _stream())
    assert st == 1          # CFD_ERR_ARG
    with pytest.raises(ValueError):
        b.cfd_filter_host(H, -8.6, 8.6, -0.5, 0.5, 10, Xd, 16)
    with pytest.raises(CfdError):
        b.cfd_filter_host(H, -8.6, 8.6, -0.5, 0.5, 10, Xd.cpu(), 12)
