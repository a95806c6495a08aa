"""The distributed filter's host-side logic on the CPU (Sect. 6, Algorithms 3
and 4): the z-slab plan and the local column numbering of the library
(cfd_slab_plan, cfd_slab_local_col, host only), and the halo-exchange
protocol the NCCL path follows (every rank sends its top plane to hi_rank and
its bottom plane to lo_rank, and receives its lower halo from lo_rank and its
upper halo from hi_rank), run on gloo ranks with the recurrence written out
in numpy on each rank's slab.  The gathered result must equal the oracle's
filter on the whole matrix, for the vector and the pipelined schedules."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1803_02156_gb300 import inputs


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _binding():
    from paper_1803_02156_gb300 import build, binding
    build.build()
    binding.lib()
    return binding


@pytest.mark.parametrize("L,per_z", [((6, 5, 7), 0), ((4, 6, 5), 1), ((3, 4, 3), 1)])
def test_slab_plan_partitions_the_lattice(L, per_z):
    b = _binding()
    per = (1, 1, per_z)
    p = b.topi_params(*L, periodic=per)
    H = oracle.topi_csr(*L, periodic=per)
    plane = 4 * L[0] * L[1]
    for nranks in range(1, L[2] + 1):
        slabs = [b.cfd_slab_plan(p, nranks, r) for r in range(nranks)]
        assert slabs[0].z0 == 0 and slabs[-1].z1 == L[2]
        for r, s in enumerate(slabs):
            assert s.z1 > s.z0 and s.row0 == plane * s.z0 and s.n_local == plane * (s.z1 - s.z0)
            if r + 1 < nranks:
                assert slabs[r + 1].z0 == s.z1
            # neighbours: the owners of the planes next to the slab
            if nranks > 1 and (s.z0 > 0 or per_z):
                lo = slabs[s.lo_rank]
                assert s.lo_base == lo.row0 + lo.n_local - plane
            else:
                assert s.lo_rank == -1 and s.lo_base == -1
            if nranks > 1 and (s.z1 < L[2] or per_z):
                assert s.hi_base == slabs[s.hi_rank].row0
            else:
                assert s.hi_rank == -1 and s.hi_base == -1
            # every column of the slab's rows has a local index; own rows map
            # onto themselves, the others onto the halo planes' rows
            ext = s.n_local + (2 * plane if nranks > 1 else 0)
            for i in range(s.row0, s.row0 + s.n_local):
                for c in H.col[H.rowptr[i]:H.rowptr[i + 1]]:
                    lc = b.cfd_slab_local_col(s, int(c))
                    assert 0 <= lc < max(ext, s.n_local), (nranks, r, i, c, lc)
                    if s.row0 <= c < s.row0 + s.n_local:
                        assert lc == c - s.row0
                    elif lc < s.n_local + plane:
                        assert c == s.lo_base + (lc - s.n_local)
                    else:
                        assert c == s.hi_base + (lc - s.n_local - plane)


# ------------------------------------------------------- gloo ranks --

def _local_csr(b, H, s):
    """Rows [row0, row0 + n_local) of the canonical CSR with columns in the
    slab's numbering (as cfd_build_matrix_slab stores them)."""
    import scipy.sparse as sp
    r0, r1 = s.row0, s.row0 + s.n_local
    rp = H.rowptr[r0:r1 + 1] - H.rowptr[r0]
    cols = np.array([b.cfd_slab_local_col(s, int(c)) for c in H.col[H.rowptr[r0]:H.rowptr[r1]]], dtype=np.int64)
    assert (cols >= 0).all()
    return sp.csr_matrix((H.val[H.rowptr[r0]:H.rowptr[r1]], cols, rp), shape=(s.n_local, s.n_local + 2 * s.plane))


def _exchange(dist, s, V, tag):
    """Halo planes of V (n_local + 2 plane rows) from the neighbours."""
    import torch
    n, pl = s.n_local, s.plane
    reqs = []
    top = torch.from_numpy(np.ascontiguousarray(V[n - pl:n]))
    bot = torch.from_numpy(np.ascontiguousarray(V[:pl]))
    lo = torch.empty_like(top)
    hi = torch.empty_like(top)
    if s.hi_rank >= 0:
        reqs.append(dist.isend(top, s.hi_rank, tag=2 * tag))
    if s.lo_rank >= 0:
        reqs.append(dist.isend(bot, s.lo_rank, tag=2 * tag + 1))
    if s.lo_rank >= 0:
        reqs.append(dist.irecv(lo, s.lo_rank, tag=2 * tag))
    if s.hi_rank >= 0:
        reqs.append(dist.irecv(hi, s.hi_rank, tag=2 * tag + 1))
    for q in reqs:
        q.wait()
    if s.lo_rank >= 0:
        V[n:n + pl] = lo.numpy()
    if s.hi_rank >= 0:
        V[n + pl:] = hi.numpy()


def _worker(rank, world, port, L, per, n_s, n_b, n_p, win, pipelined, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _binding()
    s = b.cfd_slab_plan(b.topi_params(*L, periodic=per), world, rank)
    H = oracle.topi_csr(*L, periodic=per)
    Hl = _local_csr(b, H, s)
    X = inputs.gaussian_block(H.N, n_s, seed=2)[s.row0:s.row0 + s.n_local].copy()
    a, bb = oracle.spectral_map(-8.6, 8.6)
    gc = oracle.filter_coeffs(win[0], win[1], -8.6, 8.6, n_p)
    n, ext = s.n_local, s.n_local + 2 * s.plane
    n_blocks = n_s // n_b

    def apply(V):
        return a * (Hl @ V) + bb * V[:n]

    dots = np.zeros((n_s, n_p, 2))
    # per block: V_cur (U) and V_prev (W), each with the two halo planes
    U = [None] * n_blocks
    W = [None] * n_blocks
    tag = 0

    def xchg(V):
        nonlocal tag
        _exchange(dist, s, V, tag)
        tag += 1

    def seed(k):
        sl = slice(k * n_b, (k + 1) * n_b)
        Xb = X[:, sl].copy()
        A = np.zeros((ext, n_b), complex)
        A[:n] = Xb
        xchg(A)
        V1 = apply(A)
        dots[sl, 0, 0] = np.sum(np.abs(Xb) ** 2, axis=0)
        dots[sl, 0, 1] = np.real(np.sum(np.conj(V1) * Xb, axis=0))
        B = np.zeros((ext, n_b), complex)
        B[:n] = V1
        xchg(B)
        V2 = 2 * apply(B) - Xb
        dots[sl, 1, 0] = np.sum(np.abs(V1) ** 2, axis=0)
        dots[sl, 1, 1] = np.real(np.sum(np.conj(V2) * V1, axis=0))
        X[:, sl] = gc[0] * Xb + gc[1] * V1 + gc[2] * V2
        A[:n] = V2
        U[k], W[k] = A, B                       # cur = V2, prev = V1

    def general(k, p):                          # U[k]'s halo already exchanged
        sl = slice(k * n_b, (k + 1) * n_b)
        cur, prev = U[k], W[k]
        new = 2 * apply(cur) - prev[:n]
        dots[sl, p - 1, 0] = np.sum(np.abs(cur[:n]) ** 2, axis=0)
        dots[sl, p - 1, 1] = np.real(np.sum(np.conj(new) * cur[:n], axis=0))
        X[:, sl] += gc[p] * new
        prev[:n] = new
        U[k], W[k] = prev, cur

    if not pipelined:                           # Algorithm 3: block by block
        for k in range(n_blocks):
            seed(k)
            for p in range(3, n_p + 1):
                xchg(U[k])
                general(k, p)
    else:                                       # Algorithm 4: degree outside, blocks inside
        for k in range(n_blocks):
            seed(k)
        for p in range(3, n_p + 1):
            for k in range(n_blocks):
                xchg(U[k])
                general(k, p)
    t = torch.from_numpy(dots)
    dist.all_reduce(t)
    out[rank] = (s.row0, X, t.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,L,per_z,pipelined", [(2, (4, 4, 6), 0, False), (2, (4, 4, 5), 1, True),
                                                     (3, (3, 4, 7), 0, True), (3, (4, 3, 6), 1, False)])
def test_distributed_filter_gloo(world, L, per_z, pipelined):
    per = (1, 1, per_z)
    n_s, n_b, n_p, win = 16, 8, 30, (-0.6, 0.4)
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), L, per, n_s, n_b, n_p, win, pipelined, out), nprocs=world,
             join=True)
    H = oracle.topi_csr(*L, periodic=per)
    X = inputs.gaussian_block(H.N, n_s, seed=2)
    Y, dots = oracle.chebfd_filter(H, -8.6, 8.6, win[0], win[1], n_p, X, n_b)
    got = np.zeros_like(Y)
    for r in range(world):
        row0, Xr, dr = out[r]
        got[row0:row0 + Xr.shape[0]] = Xr
        assert np.max(np.abs(dr - dots)) <= 1e-12 * np.max(np.abs(dots))
    assert np.linalg.norm(got - Y) / np.linalg.norm(Y) < 1e-13
