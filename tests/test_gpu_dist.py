"""GPU tests of the distributed filter on one device (Sect. 6, Algorithms 3
and 4): the slab matrices against the oracle's rows, and every slab of a
lattice filtered in one process with the halo planes exchanged by device
copies — the filtered rows must equal cfd_filter on the whole matrix bit for
bit (each slab row keeps the canonical row's entries and order), the
moments to the rounding of their summation order."""
import numpy as np
import pytest

import oracle
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


@pytest.mark.parametrize("L,per_z,nranks,prec", [((6, 5, 7), 0, 3, "c128p"), ((4, 6, 5), 1, 2, "c64p"),
                                                  ((4, 4, 6), 1, 3, "c128")])
def test_slab_matrix_rows_match_oracle(b, L, per_z, nranks, prec):
    import torch
    per = (1, 1, per_z)
    p = b.topi_params(*L, periodic=per, seed=5)
    ref = oracle.topi_csr(*L, periodic=per, seed=5)
    for r in range(nranks):
        s = b.cfd_slab_plan(p, nranks, r)
        H = b.cfd_build_matrix_slab(p, s, 32, 1, prec)
        assert H.N == s.n_local
        rowptr, col, val = b.cfd_matrix_export_csr(H)
        torch.cuda.synchronize()
        rowptr, col, val = rowptr.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy()
        want_dt = np.complex64 if prec.startswith("c64") else np.complex128
        for i in range(s.n_local):
            g = s.row0 + i
            gc = ref.col[ref.rowptr[g]:ref.rowptr[g + 1]]
            gv = ref.val[ref.rowptr[g]:ref.rowptr[g + 1]].astype(want_dt)
            lc = np.array([b.cfd_slab_local_col(s, int(c)) for c in gc])
            o = np.argsort(lc)
            ec, ev = col[rowptr[i]:rowptr[i + 1]], val[rowptr[i]:rowptr[i + 1]]
            oe = np.argsort(ec)                 # the export's order within a row is not the point
            assert np.array_equal(ec[oe], lc[o]), (r, i)
            assert np.array_equal(ev[oe], gv[o]), (r, i)


@pytest.mark.parametrize("L,per_z,nranks", [((8, 8, 6), 0, 2), ((8, 4, 7), 1, 3), ((6, 6, 5), 0, 1),
                                            ((8, 8, 4), 1, 2)])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("prec,arith", [("c128p", 0), ("c128p", 1), ("c64p", 0)])
def test_filter_slabs_equals_whole_matrix(b, L, per_z, nranks, mode, prec, arith):
    import torch
    per = (1, 1, per_z)
    n_s, n_b, n_p, win = 32, 16, 40, (-0.6, 0.4)
    dt = torch.complex64 if prec.startswith("c64") else torch.complex128
    p = b.topi_params(*L, periodic=per)
    H = b.cfd_build_matrix(p, 32, 1, prec)
    X0 = torch.from_numpy(inputs.gaussian_block(H.N, n_s, seed=3)).to(dt).cuda()
    ref = X0.clone()
    mu_ref = b.cfd_filter_ex(H, -8.6, 8.6, win[0], win[1], n_p, ref, n_b, moments=True, arith=arith)
    slabs = [b.cfd_slab_plan(p, nranks, r) for r in range(nranks)]
    Hs = [b.cfd_build_matrix_slab(p, s, 32, 1, prec) for s in slabs]
    Xs = [X0[s.row0:s.row0 + s.n_local].clone() for s in slabs]
    mu = b.cfd_filter_slabs(slabs, Hs, -8.6, 8.6, win[0], win[1], n_p, Xs, n_b, mode=mode, moments=True,
                            arith=arith)
    got = torch.cat(Xs, dim=0)
    assert torch.equal(got, ref)
    tol = 1e-13 if prec.startswith("c128") else 1e-5
    assert (torch.max(torch.abs(mu - mu_ref)) / torch.max(torch.abs(mu_ref))).item() < tol


def test_filter_slabs_vs_oracle(b):
    """Three slabs of the 8x8x8 parity case (n_p = 200), pipelined, against the
    oracle's filtered block and moments."""
    import torch
    L, n_s, n_b, n_p, win = (8, 8, 8), 32, 16, 200, (-0.7, 0.7)
    p = b.topi_params(*L)
    ref = oracle.topi_csr(*L)
    X = inputs.gaussian_block(ref.N, n_s, seed=2)
    slabs = [b.cfd_slab_plan(p, 3, r) for r in range(3)]
    Hs = [b.cfd_build_matrix_slab(p, s, 32, 1, "c128p") for s in slabs]
    Xs = [torch.from_numpy(X[s.row0:s.row0 + s.n_local].copy()).cuda() for s in slabs]
    mu = b.cfd_filter_slabs(slabs, Hs, -8.6, 8.6, win[0], win[1], n_p, Xs, n_b, mode=1, moments=True)
    Y, dots = oracle.chebfd_filter(ref, -8.6, 8.6, win[0], win[1], n_p, X, n_b)
    got = torch.cat(Xs).cpu().numpy()
    assert np.linalg.norm(got - Y) / np.linalg.norm(Y) < 1e-11
    muref = oracle.kpm_moments(dots)
    assert np.max(np.abs(mu.cpu().numpy() - muref)) / np.max(np.abs(muref)) < 1e-11


def test_filter_slabs_rejects_bad_plan(b):
    import torch
    p = b.topi_params(4, 4, 4)
    slabs = [b.cfd_slab_plan(p, 2, r) for r in range(2)]
    Hs = [b.cfd_build_matrix_slab(p, s, 32, 1, "c128p") for s in slabs]
    Xs = [torch.zeros(s.n_local, 16, dtype=torch.complex128, device="cuda") for s in slabs]
    with pytest.raises(b.CfdError):
        b.cfd_filter_slabs(slabs[::-1], Hs[::-1], -8.6, 8.6, -0.5, 0.5, 10, Xs[::-1], 16)
    with pytest.raises(b.CfdError):
        b.cfd_filter_slabs(slabs, Hs, -8.6, 8.6, -0.5, 0.5, 10, Xs, 16, mode=2)


@pytest.mark.parametrize("mode,arith", [(0, 1), (1, 0)])
def test_filter_slab_nccl_single_rank(b, mode, arith):
    """The NCCL path with one rank (no halo partner; the moment all-reduce
    still runs through NCCL) equals cfd_filter on the whole matrix bit for
    bit, moments to rounding."""
    import torch
    p = b.topi_params(8, 8, 6)
    H = b.cfd_build_matrix(p, 32, 1, "c128p")
    X0 = torch.from_numpy(inputs.gaussian_block(H.N, 32, seed=4)).cuda()
    ref = X0.clone()
    mu_ref = b.cfd_filter_ex(H, -8.6, 8.6, -0.5, 0.5, 30, ref, 16, moments=True, arith=arith)
    try:
        uid = b.cfd_nccl_unique_id()
    except b.CfdError as e:
        pytest.skip("NCCL not loadable here: %s" % e)
    comm = b.cfd_nccl_comm_init(uid, 1, 0)
    s = b.cfd_slab_plan(p, 1, 0)
    Hs = b.cfd_build_matrix_slab(p, s, 32, 1, "c128p")
    X = X0.clone()
    mu = b.cfd_filter_slab_nccl(s, Hs, -8.6, 8.6, -0.5, 0.5, 30, X, 16, comm, mode=mode, moments=True, arith=arith)
    torch.cuda.synchronize()
    b.cfd_nccl_comm_destroy(comm)
    assert torch.equal(X, ref)
    assert (torch.max(torch.abs(mu - mu_ref)) / torch.max(torch.abs(mu_ref))).item() < 1e-13


@pytest.mark.parametrize("L,per_z,nranks", [((8, 8, 6), 0, 2), ((8, 4, 7), 1, 3)])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("prec,arith", [("c128p", 1), ("c64p", 0)])
def test_filter_slabs_footprint_equals_whole_matrix(b, L, per_z, nranks, mode, prec, arith):
    """The slabs with the footprint-staged general steps (forced at this size;
    the footprints reach into the halo rows) against the whole matrix with
    the gathered steps: bit for bit."""
    import torch
    per = (1, 1, per_z)
    n_s, n_b, n_p, win = 32, 32, 25, (-0.6, 0.4)
    dt = torch.complex64 if prec.startswith("c64") else torch.complex128
    p = b.topi_params(*L, periodic=per)
    H = b.cfd_build_matrix(p, 32, 1, prec)
    X0 = torch.from_numpy(inputs.gaussian_block(H.N, n_s, seed=7)).to(dt).cuda()
    ref = X0.clone()
    mu_ref = b.cfd_filter_ex(H, -8.6, 8.6, win[0], win[1], n_p, ref, n_b, moments=True, arith=arith, footprint=-1)
    slabs = [b.cfd_slab_plan(p, nranks, r) for r in range(nranks)]
    Hs = [b.cfd_build_matrix_slab(p, s, 32, 1, prec) for s in slabs]
    Xs = [X0[s.row0:s.row0 + s.n_local].clone() for s in slabs]
    mu = b.cfd_filter_slabs(slabs, Hs, -8.6, 8.6, win[0], win[1], n_p, Xs, n_b, mode=mode, moments=True,
                            arith=arith, footprint=65535)
    assert torch.equal(torch.cat(Xs, dim=0), ref)
    tol = 1e-13 if prec.startswith("c128") else 1e-5
    assert (torch.max(torch.abs(mu - mu_ref)) / torch.max(torch.abs(mu_ref))).item() < tol
