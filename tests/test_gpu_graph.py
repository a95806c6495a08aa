"""The filter captured as a CUDA graph (cfd_filter_opts.graph = 1): the first
call captures and launches, later calls with the same arguments replay the
cached graph; results are bit for bit those of the kernel-by-kernel launch."""
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


@pytest.mark.parametrize("prec,arith", [("c128p", 0), ("c128p", 1), ("c64p", 0)])
def test_graph_filter_equals_launches(b, prec, arith):
    import torch
    dt = torch.complex64 if prec.startswith("c64") else torch.complex128
    H = b.cfd_build_matrix(b.topi_params(12, 10, 7), 32, 1, prec)
    X0 = torch.from_numpy(inputs.gaussian_block(H.N, 64, seed=3)).to(dt).cuda()
    work = torch.empty(b.cfd_filter_workspace(H.N, 64, 32, 40, prec, prec), dtype=torch.uint8, device="cuda")
    for win in ((-0.6, 0.4), (-0.2, 0.9)):            # a second window: a second graph
        ref = X0.clone()
        mref = b.cfd_filter_ex(H, -8.6, 8.6, win[0], win[1], 40, ref, 32, moments=True, arith=arith, work=work)
        X = torch.empty_like(X0)
        mu = torch.empty(64, 80, dtype=torch.float64, device="cuda")
        for rep in range(3):                            # capture, then two replays into the same buffers
            X.copy_(X0)
            n0 = b.cfd_launch_count()
            o = b.cfd_filter_opts(0, 0, 0, 0, 0, 0, arith, 1)
            b._check(b.lib().cfd_filter_ex(H.ref(), -8.6, 8.6, win[0], win[1], 40, b.block_of(X), 32, b._ptr(work),
                                           work.numel(), b._ptr(mu), b.ctypes.byref(o), b._stream()))
            torch.cuda.synchronize()
            assert b.cfd_launch_count() - n0 >= 40      # the graph's kernels are counted when launched
            assert torch.equal(X, ref), rep
            assert torch.equal(mu, mref), rep


def test_graph_batched_filter_equals_launches(b):
    import torch
    lat = inputs.batched_lattices(3)
    params = [b.topi_params(nx // 2, ny // 2, nz // 2, seed=sd) for (nx, ny, nz, sd) in lat]
    B = b.cfd_build_batch(params, 32, 1, "c64p")
    win = torch.tensor([[-8.6, 8.6, -0.5, 0.5]] * B.R, dtype=torch.float64, device="cuda")
    X0 = torch.from_numpy(inputs.gaussian_block(B.N, 32, seed=4)).to(torch.complex64).cuda()
    end = b.batch_row_end(B)
    for r in range(B.R):
        X0[end[r]:B.row_off[r + 1]] = 0
    ref = X0.clone()
    b.cfd_filter_batched(B, win, 60, ref, 32)
    work = torch.empty(b.lib().cfd_filter_batched_workspace(B.N, B.R, 32, 32, 60, B.prec, B.prec),
                       dtype=torch.uint8, device="cuda")
    X = torch.empty_like(X0)
    for rep in range(2):
        X.copy_(X0)
        b.cfd_filter_batched(B, win, 60, X, 32, graph=1, work=work)
        torch.cuda.synchronize()
        assert torch.equal(X, ref), rep


def test_graph_option_rejected(b):
    import torch
    H = b.cfd_build_matrix(b.topi_params(4, 4, 4), 32, 1, "c128p")
    X = torch.zeros(H.N, 16, dtype=torch.complex128, device="cuda")
    with pytest.raises(b.CfdError):
        b.cfd_filter_ex(H, -8.6, 8.6, -0.5, 0.5, 10, X, 16, graph=2)
