"""GPU parity of the fp64 dense path (Gram on the FP64 tensor cores, Jacobi
eigensolver, SVQB, Rayleigh-Ritz), the Lanczos bounds and the ChebFD solve,
through the C ABI, against numpy / the CPU oracle / dense truth."""
import numpy as np
import pytest

import oracle
from paper_1803_02156_gb300 import inputs, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def b():
    import torch
    from paper_1803_02156_gb300 import build, binding
    assert torch.cuda.is_available()
    build.build()
    binding.lib()
    return binding


def _cuda(A):
    import torch
    return torch.from_numpy(np.ascontiguousarray(A)).cuda()


@pytest.mark.parametrize("N,nx,ny", [(2048, 32, 32), (5001, 24, 40), (100003, 128, 128), (77, 8, 16),
                                     (300, 256, 256)])
def test_gram_vs_numpy(b, N, nx, ny):
    X = inputs.gaussian_block(N, nx, seed=1)
    Y = inputs.gaussian_block(N, ny, seed=2)
    S = b.cfd_block_gram(_cuda(X), _cuda(Y)).cpu().numpy()
    ref = X.conj().T @ Y
    assert np.max(np.abs(S - ref)) < 1e-13 * np.sqrt(N) * 4


def test_gram_strided_view(b):
    """Blocks that are column windows of a wider array (ld > n)."""
    X = inputs.gaussian_block(4000, 64, seed=3)
    Xg = _cuda(X)
    S = b.cfd_block_gram(Xg[:, 16:48], Xg[:, 8:24]).cpu().numpy()
    assert np.max(np.abs(S - X[:, 16:48].conj().T @ X[:, 8:24])) < 1e-11


def _random_hermitian(n, seed, spectrum=None):
    rng = np.random.default_rng(seed)
    if spectrum is None:
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        return 0.5 * (A + A.conj().T)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    return (Q * spectrum) @ Q.conj().T


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 17, 32, 40, 64, 100, 128, 256])
def test_eigh_vs_numpy(b, n):
    A = _random_hermitian(n, n)
    ev, Q = b.cfd_eigh(_cuda(A))
    ev, Q = ev.cpu().numpy(), Q.cpu().numpy()
    ref = np.linalg.eigvalsh(A)
    nA = np.linalg.norm(A, 2)
    assert np.max(np.abs(ev - ref)) <= 1e-13 * nA * max(1, n / 32)
    assert np.linalg.norm(A @ Q - Q * ev) <= 1e-12 * nA * np.sqrt(n)
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(n)) <= 1e-12 * np.sqrt(n)
    assert np.all(np.diff(ev) >= 0)


def test_eigh_degenerate_and_tridiagonal(b):
    spec = np.repeat(np.linspace(-3, 3, 16), 2)                 # doubly degenerate levels
    A = _random_hermitian(32, 5, spec)
    ev, Q = b.cfd_eigh(_cuda(A))
    assert np.max(np.abs(ev.cpu().numpy() - np.sort(spec))) < 1e-13 * 3
    T = np.diag(np.linspace(0, 1, 40)) + np.diag(np.full(39, 0.3), 1) + np.diag(np.full(39, 0.3), -1)
    ev, _ = b.cfd_eigh(_cuda(T.astype(np.complex128)))
    assert np.max(np.abs(ev.cpu().numpy() - np.linalg.eigvalsh(T))) < 1e-14 * 10


@pytest.mark.parametrize("N,n", [(4096, 32), (20000, 128), (3001, 256)])
def test_orthogonalize_random(b, N, n):
    X = inputs.gaussian_block(N, n, seed=7)
    Xg = _cuda(X)
    rank = b.cfd_orthogonalize(Xg)
    Q = Xg.cpu().numpy()
    assert rank == n
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(n)) <= 1e-13
    P = Q @ (Q.conj().T @ X)
    assert np.linalg.norm(X - P) <= 1e-12 * np.linalg.norm(X)


def test_orthogonalize_filtered_block(b):
    """The ill-conditioned output of the filter (8x8x8, n_p = 200) is made orthonormal."""
    H = oracle.topi_csr(8, 8, 8)
    X = inputs.gaussian_block(H.N, 32, seed=2)
    Y, _ = oracle.chebfd_filter(H, -8.6, 8.6, -0.7, 0.7, 200, X, 32)
    Yg = _cuda(Y)
    b.cfd_orthogonalize(Yg)
    Q = Yg.cpu().numpy()
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(32)) <= 1e-13
    # the leading directions of the filtered block are kept: the oracle's MGS basis
    # spans the same space up to the numerically-deficient tail
    Qo = oracle.mgs2(Y)
    s = np.linalg.svd(Qo[:, :16].conj().T @ Q, compute_uv=False)
    assert np.min(s) > 1 - 1e-8


def test_rayleigh_ritz_exact_subspace(b):
    """RR on a rotated exact eigenbasis returns its eigenvalues with ~0 residuals."""
    Hc = oracle.topi_csr(8, 8, 8)
    lam, V = np.linalg.eigh(Hc.dense())
    rng = np.random.default_rng(3)
    U, _ = np.linalg.qr(rng.standard_normal((32, 32)) + 1j * rng.standard_normal((32, 32)))
    X = V[:, 1000:1032] @ U
    H = b.cfd_build_matrix(b.topi_params(8, 8, 8), 32, 1, "c128")
    Xg = _cuda(X)
    th, r = b.cfd_rayleigh_ritz(H, Xg)
    assert np.max(np.abs(th.cpu().numpy() - lam[1000:1032])) < 1e-12
    assert np.max(r.cpu().numpy()) < 1e-12


def test_rayleigh_ritz_vs_oracle(b):
    Hc = oracle.topi_csr(6, 7, 5)
    X = oracle.mgs2(inputs.gaussian_block(Hc.N, 24, seed=9))
    th0, X0, r0 = oracle.rayleigh_ritz(Hc, X)
    H = b.cfd_build_matrix(b.topi_params(6, 7, 5), 32, 1, "c128")
    Xg = _cuda(X)
    th, r = b.cfd_rayleigh_ritz(H, Xg)
    assert np.max(np.abs(th.cpu().numpy() - th0)) < 1e-12
    assert np.max(np.abs(r.cpu().numpy() - r0)) < 1e-11
    # Ritz vectors agree up to phase (the Ritz values here are simple)
    G = np.abs(np.sum(X0.conj() * Xg.cpu().numpy(), axis=0))
    assert np.min(G) > 1 - 1e-10


@pytest.mark.parametrize("L", [(8, 8, 8), (6, 6, 6), (16, 16, 8)])
def test_spectral_bounds(b, L):
    H = b.cfd_build_matrix(b.topi_params(*L), 32, 1, "c128")
    lo, hi = b.cfd_spectral_bounds(H, 40, seed=3)
    Hc = oracle.topi_csr(*L)
    glo, ghi = oracle.gershgorin(Hc)
    assert glo - 1e-12 <= lo < hi <= ghi + 1e-12
    if Hc.N <= 2048:
        ev = np.linalg.eigvalsh(Hc.dense())
        assert lo <= ev[0] and ev[-1] <= hi
    v0 = inputs.gaussian_block(Hc.N, 1, seed=3, tag=2)[:, 0]
    olo, ohi = oracle.lanczos_bounds(Hc, 40, v0)
    spread = ohi - olo
    assert abs(lo - olo) < 0.03 * spread and abs(hi - ohi) < 0.03 * spread


def _small_truth():
    Hc = oracle.topi_csr(8, 8, 8)
    ev = np.linalg.eigvalsh(Hc.dense())
    delta, k = oracle.window_from_dense(ev, 16)
    return ev, delta, k


def test_solve_fp64_small_config(b):
    """8x8x8, n_s = 32, n_p = 200: converged in-window eigenvalues equal dense
    eigh's to 1e-10 with residuals <= 1e-10."""
    import torch
    ev, delta, k = _small_truth()
    w = workloads.SMALL
    H = b.cfd_build_matrix(b.topi_params(*w.lattice), 32, 1, "c128")
    X = torch.empty(w.N, w.n_s, dtype=torch.complex128, device="cuda")
    th, rs, res = b.cfd_solve(H, X, -delta, delta, w.n_p, w.n_b, n_t=k, tol=1e-10, seed=2)
    inside = (th >= -delta) & (th <= delta) & (rs <= 1e-10)
    exact = np.sort(ev[np.abs(ev) < delta])
    assert res.n_conv == k == inside.sum()
    assert np.max(np.abs(np.sort(th[inside]) - exact)) < 1e-10
    assert np.max(rs[inside]) <= 1e-10
    assert res.lmin <= ev[0] and ev[-1] <= res.lmax
    # the returned block is orthonormal
    Q = X.cpu().numpy()
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(w.n_s)) < 1e-12


def test_solve_mixed_matches_fp64(b):
    """Mixed policy (fp32 filter, then fp64) on 8x8x8: same eigenvalues to 1e-10."""
    import torch
    ev, delta, k = _small_truth()
    w = workloads.SMALL
    H = b.cfd_build_matrix(b.topi_params(*w.lattice), 32, 1, "c128")
    Hl = b.cfd_build_matrix(b.topi_params(*w.lattice), 32, 1, "c64")
    X = torch.empty(w.N, w.n_s, dtype=torch.complex128, device="cuda")
    th, rs, res = b.cfd_solve(H, X, -delta, delta, w.n_p, w.n_b, H_low=Hl, policy=b.CFD_POLICY_MIXED, n_t=k,
                              tol=1e-10, seed=2)
    inside = (th >= -delta) & (th <= delta) & (rs <= 1e-10)
    exact = np.sort(ev[np.abs(ev) < delta])
    assert res.n_conv == k and res.iters_low >= 1 and res.iters > res.iters_low
    assert np.max(np.abs(np.sort(th[inside]) - exact)) < 1e-10
    assert np.max(rs[inside]) <= 1e-10


def test_solve_stable_count_rule(b):
    """Without a target count the solve stops when the converged count is stable."""
    import torch
    ev, delta, k = _small_truth()
    H = b.cfd_build_matrix(b.topi_params(8, 8, 8), 32, 1, "c128")
    X = torch.empty(2048, 32, dtype=torch.complex128, device="cuda")
    th, rs, res = b.cfd_solve(H, X, -delta, delta, 200, 32, n_t=0, tol=1e-10, seed=2)
    assert res.n_conv == k


def test_solve_argument_errors(b):
    import torch
    H = b.cfd_build_matrix(b.topi_params(8, 8, 8), 32, 1, "c128")
    X = torch.empty(2048, 32, dtype=torch.complex128, device="cuda")
    with pytest.raises(b.CfdError) as e:
        b.cfd_solve(H, X, -20.0, 0.5, 50, 32, lmin=-9, lmax=9)          # window outside bounds
    assert e.value.status == 1
    with pytest.raises(b.CfdError) as e:
        b.cfd_solve(H, X, -0.5, 0.5, 50, 32, policy=b.CFD_POLICY_MIXED)  # no low-precision matrix
    assert e.value.status == 1
    with pytest.raises(b.CfdError) as e:
        b.cfd_solve(H, X, -0.5, 0.5, 20, 32, max_iter=1, lmin=-9, lmax=9, n_t=16)
    assert e.value.status == 6


# ----------------------------------------------- double-word Gram and SVQB --
# Every double split once into hi + lo floats, every multiply-add a
# double-word one: each operation accurate to a few units of 2^-48 of the
# magnitudes of its terms (2^-53 for fp64), a split's sum of K' terms to
# about sqrt(K') of them.  The Gram's bar is therefore elementwise,
# 8 sqrt(K) 2^-48 (|X|^H |Y|).


def _dw_gram_bound(X, Y):
    return 8 * np.sqrt(X.shape[0]) * 2.0 ** -48 * (np.abs(X).T @ np.abs(Y))

@pytest.mark.parametrize("N,nx,ny", [(2048, 32, 32), (5001, 24, 40), (100003, 128, 128), (77, 8, 16),
                                     (300, 256, 256), (20000, 256, 200)])
def test_gram_dw_vs_numpy(b, N, nx, ny):
    X = inputs.gaussian_block(N, nx, seed=1)
    Y = inputs.gaussian_block(N, ny, seed=2)
    S = b.cfd_block_gram(_cuda(X), _cuda(Y), arith=1).cpu().numpy()
    ref = X.conj().T @ Y
    assert np.all(np.abs(S - ref) <= _dw_gram_bound(X, Y))


def test_gram_dw_hermitian_and_strided(b):
    """X^H X of a column window (ld > n): the Hermitian path (tiles below the
    diagonal mirrored by the fold) against numpy, Hermitian to its rounding."""
    X = inputs.gaussian_block(30011, 256, seed=4)
    Xg = _cuda(X)
    S = b.cfd_block_gram(Xg[:, 0:192], Xg[:, 0:192], arith=1).cpu().numpy()
    ref = X[:, :192].conj().T @ X[:, :192]
    assert np.all(np.abs(S - ref) <= _dw_gram_bound(X[:, :192], X[:, :192]))
    assert np.all(np.abs(S - S.conj().T) <= 2 * _dw_gram_bound(X[:, :192], X[:, :192]))
    S2 = b.cfd_block_gram(Xg[:, 16:48], Xg[:, 8:24], arith=1).cpu().numpy()
    assert np.all(np.abs(S2 - X[:, 16:48].conj().T @ X[:, 8:24]) <= _dw_gram_bound(X[:, 16:48], X[:, 8:24]))


@pytest.mark.parametrize("N,n", [(4096, 32), (20000, 128), (3001, 256), (100003, 256)])
def test_orthogonalize_dw_random(b, N, n):
    """SVQB with double-word Grams and projections: orthonormal to the fp64
    bar times 2^5 (the ratio of 2^-48 to 2^-53), times sqrt(N / 4096) past
    4096 rows (a double-word sum of K terms is good to about sqrt(K) 2^-48),
    and the same span as the input."""
    X = inputs.gaussian_block(N, n, seed=7)
    Xg = _cuda(X)
    rank = b.cfd_orthogonalize(Xg, arith=1)
    Q = Xg.cpu().numpy()
    assert rank == n
    grow = max(1.0, np.sqrt(N / 4096))
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(n)) <= 32 * 1e-13 * grow
    P = Q @ (Q.conj().T @ X)
    assert np.linalg.norm(X - P) <= 32 * 1e-12 * grow * np.linalg.norm(X)


def test_orthogonalize_dw_filtered_block(b):
    """The ill-conditioned filter output (8x8x8, n_p = 200) through the
    double-word SVQB: orthonormal, leading directions of the oracle's basis kept."""
    H = oracle.topi_csr(8, 8, 8)
    X = inputs.gaussian_block(H.N, 32, seed=2)
    Y, _ = oracle.chebfd_filter(H, -8.6, 8.6, -0.7, 0.7, 200, X, 32)
    Yg = _cuda(Y)
    b.cfd_orthogonalize(Yg, arith=1)
    Q = Yg.cpu().numpy()
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(32)) <= 32 * 1e-13
    Qo = oracle.mgs2(Y)
    s = np.linalg.svd(Qo[:, :16].conj().T @ Q, compute_uv=False)
    assert np.min(s) > 1 - 1e-8


def test_dense_dw_option_rejected(b):
    X = _cuda(inputs.gaussian_block(100, 8, seed=1))
    with pytest.raises(b.CfdError) as e:
        b.cfd_block_gram(X, X, arith=2)
    assert e.value.status == 1


@pytest.mark.parametrize("policy", ["fp64_dw", "mixed_dw"])
def test_solve_dw_policies(b, policy):
    """The double-word policies (filter, SVQB and Rayleigh-Ritz in double-word
    arithmetic; mixed: complex-float filter first) on 8x8x8: converged
    in-window eigenvalues equal dense eigh's to 1e-10, residuals <= 1e-10,
    the returned block orthonormal."""
    import torch
    ev, delta, k = _small_truth()
    w = workloads.SMALL
    H = b.cfd_build_matrix(b.topi_params(*w.lattice), 32, 1, "c128p")
    Hl = b.cfd_build_matrix(b.topi_params(*w.lattice), 32, 1, "c64p")
    X = torch.empty(w.N, w.n_s, dtype=torch.complex128, device="cuda")
    pol = b.CFD_POLICY_FP64_DW if policy == "fp64_dw" else b.CFD_POLICY_MIXED_DW
    th, rs, res = b.cfd_solve(H, X, -delta, delta, w.n_p, w.n_b, H_low=Hl if policy == "mixed_dw" else None,
                              policy=pol, n_t=k, tol=1e-10, seed=2)
    inside = (th >= -delta) & (th <= delta) & (rs <= 1e-10)
    exact = np.sort(ev[np.abs(ev) < delta])
    assert res.n_conv == k == inside.sum()
    assert np.max(np.abs(np.sort(th[inside]) - exact)) < 1e-10
    assert np.max(rs[inside]) <= 1e-10
    Q = X.cpu().numpy()
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(w.n_s)) < 1e-11
