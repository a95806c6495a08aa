"""The large single instance, 200x200x100 (N = 16e6): the filter at full size
in both precisions, with 64-bit element offsets (N x 256 block), checked on
sampled rows that the oracle computes one by one from each row's neighbourhood."""
import numpy as np
import pytest

import oracle
from paper_1803_02156_gb300 import inputs, workloads

pytestmark = pytest.mark.gpu

N_P = 3


@pytest.fixture(scope="module")
def b():
    import torch
    from paper_1803_02156_gb300 import build, binding
    assert torch.cuda.is_available()
    build.build()
    binding.lib()
    return binding


@pytest.fixture(scope="module")
def csr():
    w = workloads.LARGE
    return oracle.topi_csr(*w.lattice, seed=w.seed)


def _neighbourhood(H, rows, hops):
    out = set(rows)
    front = set(rows)
    for _ in range(hops):
        nxt = set()
        for i in front:
            nxt.update(H.col[H.rowptr[i]:H.rowptr[i + 1]].tolist())
        front = nxt - out
        out |= nxt
    return sorted(out)


def _apply(H, V, rows, a, b):
    """(a H + b) V restricted to `rows` (V: dict row -> vector)."""
    out = {}
    for i in rows:
        s, e = H.rowptr[i], H.rowptr[i + 1]
        acc = sum(H.val[k] * V[H.col[k]] for k in range(s, e))
        out[i] = a * acc + b * V[i]
    return out


def _sampled_filter(H, X_rows, rows, lmin, lmax, wl, wr):
    """Rows of sum_{k<=3} g_k c_k T_k(aH + b) X from 3-hop neighbourhoods
    (Algorithm 1 with n_p = 3, evaluated row by row)."""
    a, bb = oracle.spectral_map(lmin, lmax)
    gc = oracle.filter_coeffs(wl, wr, lmin, lmax, N_P)
    R2 = _neighbourhood(H, rows, 2)
    R1 = _neighbourhood(H, rows, 1)
    T1 = _apply(H, X_rows, R2, a, bb)
    T2 = {i: 2 * v - X_rows[i] for i, v in _apply(H, T1, R1, a, bb).items()}
    T3 = {i: 2 * v - T1[i] for i, v in _apply(H, T2, rows, a, bb).items()}
    return {i: gc[0] * X_rows[i] + gc[1] * T1[i] + gc[2] * T2[i] + gc[3] * T3[i] for i in rows}


def _sample_rows(N, Nxy4):
    rng = np.random.default_rng(5)
    rows = [0, 1, 2, 3, Nxy4 - 1, Nxy4, N // 2, N // 2 + 7, N - Nxy4 - 1, N - Nxy4, N - 2, N - 1]
    rows += rng.integers(0, N, 40).tolist()
    return sorted(set(int(r) for r in rows))


@pytest.mark.parametrize("prec,n_s,col0,tol", [("c64p", 256, 224, 3e-5), ("c128p", 32, 0, 1e-11)])
def test_large_instance_sampled_rows(b, csr, prec, n_s, col0, tol):
    import torch
    w = workloads.LARGE
    Nx, Ny, Nz = w.lattice
    H = b.cfd_build_matrix(b.topi_params(*w.lattice, seed=w.seed), 32, 1, prec)
    assert H.N == csr.N == 16_000_000
    dt = torch.complex64 if prec.startswith("c64") else torch.complex128
    X = torch.zeros(H.N, n_s, dtype=dt, device="cuda")
    X[:, col0:col0 + 32] = inputs.gaussian_block_device(H.N, 32, seed=77, dtype=dt)
    rows = _sample_rows(H.N, 4 * Nx * Ny)
    need = _neighbourhood(csr, rows, 3)
    idx = torch.tensor(need, device="cuda")
    Xin = X[idx, col0:col0 + 32].cpu().numpy().astype(np.complex128)
    X_rows = {i: Xin[k] for k, i in enumerate(need)}
    n0 = (torch.linalg.norm(X[:, col0:col0 + 32].to(torch.complex128), dim=0) ** 2).cpu().numpy()
    mu = b.cfd_filter(H, -8.6, 8.6, -0.5, 0.5, N_P, X, 32, moments=True)[col0:col0 + 32].cpu().numpy()
    got = X[torch.tensor(rows, device="cuda"), col0:col0 + 32].cpu().numpy().astype(np.complex128)
    ref = _sampled_filter(csr, X_rows, rows, -8.6, 8.6, -0.5, 0.5)
    for k, i in enumerate(rows):
        err = np.linalg.norm(got[k] - ref[i]) / max(np.linalg.norm(ref[i]), 1e-30)
        assert err < tol, (i, err)
    # moments of the filtered block, properties that hold at any size:
    # mu_0 = ||x||^2 and |mu_m| <= mu_0 (|T_m| <= 1 on the scaled spectrum)
    assert np.allclose(mu[:, 0], n0, rtol=tol)
    assert np.all(np.abs(mu) <= mu[:, :1] * (1 + 1e-5))
    if col0:                 # the other column blocks were zero and stay zero
        assert torch.count_nonzero(X[:, :col0]).item() == 0
