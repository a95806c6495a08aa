"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(closed forms, invariants, independent quadrature, brute force), never against
itself.  CPU only."""
import json
import math
import os

import numpy as np
import pytest
import scipy.integrate as si
from numpy.polynomial import chebyshev as npcheb

import oracle
from paper_1803_02156_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _clean_spectrum(L, t=1.0, m=2.0):
    """Clean periodic Topi spectrum: H(k) = (m - t sum cos k_j) Gamma_1 -
    t sum sin k_j Gamma_{j+2} with anticommuting Gammas, so
    E(k) = +-sqrt((m - t sum cos k_j)^2 + t^2 sum sin^2 k_j), each twice."""
    E = []
    for nx in range(L[0]):
        for ny in range(L[1]):
            for nz in range(L[2]):
                k = 2 * np.pi * np.array([nx / L[0], ny / L[1], nz / L[2]])
                e = math.sqrt((m - t * np.cos(k).sum()) ** 2 + t * t * (np.sin(k) ** 2).sum())
                E += [e, e, -e, -e]
    return np.sort(E)


# ------------------------------------------------------------ matrix (P1, P3) --

@pytest.mark.parametrize("L,per", [((3, 3, 3), (1, 1, 1)), ((4, 5, 3), (1, 1, 0)),
                                   ((8, 8, 8), (1, 1, 0)), ((4, 3, 1), (1, 1, 0)),
                                   ((5, 4, 6), (0, 1, 0))])
def test_topi_hermitian_nnz_values(L, per):
    H = oracle.topi_csr(*L, periodic=per, seed=7)
    A = H.dense()
    assert np.array_equal(A, A.conj().T)                 # bitwise Hermitian
    Nx, Ny, Nz = L
    exp = 13 * H.N
    for j, n_other in enumerate((Ny * Nz, Nx * Nz, Nx * Ny)):
        if not per[j]:
            exp -= 16 * n_other        # 2 per row on each open side (4 if L_j = 1)
    assert H.nnz == exp
    # every row: 1 on-site entry and 2 per existing neighbour; off-diagonal
    # values are +-1/2 or +-i/2; the diagonal is +-(m + V), |V| <= gamma/2.
    for i in range(H.N):
        s, e = H.rowptr[i], H.rowptr[i + 1]
        assert np.all(np.diff(H.col[s:e]) > 0)
        for c, v in zip(H.col[s:e], H.val[s:e]):
            if c == i:
                assert v.imag == 0.0 and 1.5 <= abs(v.real) <= 2.5
            else:
                assert (abs(v.real), abs(v.imag)) in ((0.5, 0.0), (0.0, 0.5))


def test_topi_blocks_golden():
    g = json.load(open(os.path.join(GOLD, "topi_blocks.json")))
    L = (4, 4, 4)
    H = oracle.topi_csr(*L, periodic=(1, 1, 1), seed=3, m=2.0, gamma=1.0)
    A = H.dense()

    def site(x, y, z):
        return x + L[0] * (y + L[1] * z)

    s0 = site(1, 2, 1)
    for j, name in enumerate(("T_x", "T_y", "T_z")):
        T = np.zeros((4, 4), complex)
        for r, c, re, im in g[name]:
            T[r, c] = re + 1j * im
        e = [0, 0, 0]
        e[j] = 1
        s1 = site(1 + e[0], 2 + e[1], 1 + e[2])
        blk = A[4 * s1:4 * s1 + 4, 4 * s0:4 * s0 + 4]          # (site + e_j, site)
        assert np.array_equal(blk, T)
        assert np.array_equal(A[4 * s0:4 * s0 + 4, 4 * s1:4 * s1 + 4], T.conj().T)
    on = A[4 * s0:4 * s0 + 4, 4 * s0:4 * s0 + 4]
    v = on[0, 0].real
    assert np.array_equal(on, np.diag(np.array(g["Gamma1_diag"]) * v))


@pytest.mark.parametrize("L", [(4, 4, 4), (3, 5, 4), (6, 3, 3)])
def test_clean_periodic_closed_form(L):
    H = oracle.topi_csr(*L, periodic=(1, 1, 1), gamma=0.0)
    ev = np.linalg.eigvalsh(H.dense())
    E = _clean_spectrum(L)
    assert np.max(np.abs(ev - E)) < 1e-12
    # every level at least doubly degenerate
    assert np.max(np.abs(ev[0::2] - ev[1::2])) < 1e-12


def test_disorder_uniform():
    H = oracle.topi_csr(16, 16, 8, seed=11, gamma=1.0, m=2.0)
    d = np.array([H.val[H.rowptr[i]:H.rowptr[i + 1]][H.col[H.rowptr[i]:H.rowptr[i + 1]] == i][0].real
                  for i in range(0, H.N, 4)])              # orbital 0: +(m + V)
    V = d - 2.0
    assert V.min() >= -0.5 and V.max() < 0.5
    assert abs(V.mean()) < 0.02 and abs(V.var() - 1.0 / 12) < 0.005
    # orbital 2 of the same site carries -(m + V)
    d2 = np.array([H.val[H.rowptr[i]:H.rowptr[i + 1]][H.col[H.rowptr[i]:H.rowptr[i + 1]] == i][0].real
                   for i in range(2, H.N, 4)])
    assert np.array_equal(d2, -d)


def test_gershgorin_contains_spectrum():
    H = oracle.topi_csr(5, 5, 4, seed=5)
    lo, hi = oracle.gershgorin(H)
    ev = np.linalg.eigvalsh(H.dense())
    assert lo <= ev[0] and ev[-1] <= hi
    assert hi <= 2.5 + 6.0 + 1e-12


# ------------------------------------------------------------- coefficients (P2) --

@pytest.mark.parametrize("win", [(-0.3, 0.4), (-0.9, -0.2), (0.05, 0.95)])
def test_window_coeffs_quadrature(win):
    lmin, lmax = -3.0, 5.0
    a, b = oracle.spectral_map(lmin, lmax)
    xl, xr = a * win[0] + b, a * win[1] + b
    c = oracle.window_coeffs(*win, lmin, lmax, 60)
    for k in range(61):
        Tk = npcheb.Chebyshev.basis(k)
        val, err = si.quad(lambda x: Tk(x) / math.sqrt(1 - x * x), xl, xr,
                           epsabs=1e-14, epsrel=1e-14, limit=200)
        ref = (1.0 if k == 0 else 2.0) / math.pi * val
        assert abs(c[k] - ref) < 1e-12, (k, c[k], ref)


def test_full_window_is_identity_polynomial():
    c = oracle.window_coeffs(-2.0, 2.0, -2.0, 2.0, 50)
    assert abs(c[0] - 1.0) < 1e-15
    assert np.max(np.abs(c[1:])) < 1e-14


@pytest.mark.parametrize("n_p", [10, 200, 1000])
def test_jackson_kernel(n_p):
    g = oracle.jackson(n_p)
    M = n_p + 1
    assert abs(g[0] - 1.0) < 1e-14
    assert abs(g[1] - math.cos(math.pi / (M + 1))) < 1e-14
    assert np.all(g > 0) and np.all(g <= 1.0 + 1e-15)
    assert np.all(np.diff(g) < 0)
    # positivity of the Jackson-damped delta expansion (the kernel is positive)
    x0 = 0.3137
    xs = np.linspace(-1, 1, 4001)
    k = np.arange(n_p + 1)
    w = np.where(k == 0, 1.0, 2.0) * g * np.cos(k * math.acos(x0))
    vals = np.cos(np.outer(np.arccos(xs), k)) @ w
    assert vals.min() > -1e-10 * vals.max()


@pytest.mark.parametrize("n_p,win", [(60, (-0.5, 0.5)), (300, (-0.1, 0.2)), (1000, (0.0, 0.05))])
def test_filter_polynomial_bounded(n_p, win):
    # Jackson damping keeps the indicator's approximation inside [0, 1]
    gc = oracle.filter_coeffs(*win, -1.0, 1.0, n_p)
    xs = np.linspace(-1, 1, 20001)
    p = oracle.filter_polynomial(xs, gc)
    assert p.min() > -1e-12 and p.max() < 1 + 1e-12
    mid = 0.5 * (win[0] + win[1])
    assert oracle.filter_polynomial(np.array([mid]), gc)[0] > 0.5


# ---------------------------------------------------------------- filter (P4-P6) --

def _diag_csr(lam):
    N = len(lam)
    return oracle.CSR(np.arange(N + 1, dtype=np.int64), np.arange(N, dtype=np.int32),
                      np.asarray(lam, dtype=np.complex128))


def test_filter_diagonal_matrix():
    rng = np.random.default_rng(0)
    lam = rng.uniform(-2.0, 3.0, 97)
    H = _diag_csr(lam)
    X = inputs.gaussian_block(97, 4, seed=9)
    n_p, lmin, lmax, wl, wr = 150, -2.0, 3.0, -0.4, 0.7
    Y, _ = oracle.chebfd_filter(H, lmin, lmax, wl, wr, n_p, X, 2)
    a, b = oracle.spectral_map(lmin, lmax)
    gc = oracle.filter_coeffs(wl, wr, lmin, lmax, n_p)
    k = np.arange(n_p + 1)
    pv = np.cos(np.outer(np.arccos(np.clip(a * lam + b, -1, 1)), k)) @ gc
    assert np.max(np.abs(Y - pv[:, None] * X)) < 1e-13


def test_filter_full_window_returns_input():
    H = oracle.topi_csr(4, 4, 3, seed=2)
    X = inputs.gaussian_block(H.N, 4, seed=1)
    lo, hi = -9.0, 9.0
    Y, _ = oracle.chebfd_filter(H, lo, hi, lo, hi, 80, X, 4)
    assert np.linalg.norm(Y - X) / np.linalg.norm(X) < 1e-13


@pytest.mark.parametrize("L,n_p,n_s,n_b", [((4, 4, 4), 120, 8, 4), ((5, 3, 4), 60, 6, 3)])
def test_filter_brute_force(L, n_p, n_s, n_b):
    H = oracle.topi_csr(*L, seed=4)
    Hd = H.dense()
    X = inputs.gaussian_block(H.N, n_s, seed=5)
    lmin, lmax, wl, wr = -8.6, 8.6, -1.0, 1.2
    Y, dots = oracle.chebfd_filter(H, lmin, lmax, wl, wr, n_p, X, n_b)
    Yref = oracle.dense_filter(Hd, lmin, lmax, wl, wr, n_p, X)
    assert np.linalg.norm(Y - Yref) / np.linalg.norm(Yref) < 1e-11
    mu = oracle.kpm_moments(dots)
    muref = oracle.dense_moments(Hd, lmin, lmax, X, 2 * n_p)
    assert np.max(np.abs(mu - muref)) / np.max(np.abs(muref)) < 1e-11


def test_filter_small_config_brute_force():
    """The 8x8x8 parity configuration end to end against dense eigh."""
    H = oracle.topi_csr(8, 8, 8, seed=1)
    Hd = H.dense()
    X = inputs.gaussian_block(H.N, 32, seed=2)
    Y, dots = oracle.chebfd_filter(H, -8.5, 8.5, -0.7, 0.7, 200, X, 32)
    Yref = oracle.dense_filter(Hd, -8.5, 8.5, -0.7, 0.7, 200, X)
    assert np.linalg.norm(Y - Yref) / np.linalg.norm(Yref) < 1e-11


def test_filter_block_width_invariance():
    H = oracle.topi_csr(4, 4, 4, seed=6)
    X = inputs.gaussian_block(H.N, 8, seed=3)
    ref, dref = oracle.chebfd_filter(H, -8.6, 8.6, -0.5, 0.5, 50, X, 8)
    for n_b in (1, 2, 4):
        Y, d = oracle.chebfd_filter(H, -8.6, 8.6, -0.5, 0.5, 50, X, n_b)
        assert np.array_equal(Y, ref)
        assert np.array_equal(d, dref)


# ------------------------------------------------- orthogonalisation, RR, bounds --

def test_mgs2_orthonormal_and_span():
    X = inputs.gaussian_block(300, 12, seed=8)
    X[:, 5] = X[:, 4] + 1e-6 * X[:, 5]                    # ill-conditioned
    Q = oracle.mgs2(X)
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(12)) < 1e-13
    P = Q @ Q.conj().T
    assert np.linalg.norm(X - P @ X) < 1e-12 * np.linalg.norm(X)


def test_rayleigh_ritz_exact_subspace():
    H = oracle.topi_csr(4, 4, 3, seed=9)
    lam, V = np.linalg.eigh(H.dense())
    rng = np.random.default_rng(1)
    Qm, _ = np.linalg.qr(rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8)))
    X = V[:, 100:108] @ Qm                                 # rotated exact eigenbasis
    th, Xr, r = oracle.rayleigh_ritz(H, X)
    assert np.max(np.abs(th - lam[100:108])) < 1e-12
    assert np.max(r) < 1e-12


def test_lanczos_bounds_contain_spectrum():
    H = oracle.topi_csr(6, 6, 6, seed=1)
    ev = np.linalg.eigvalsh(H.dense())
    v0 = inputs.gaussian_block(H.N, 1, seed=3, tag=2)[:, 0]
    lo, hi = oracle.lanczos_bounds(H, 40, v0)
    glo, ghi = oracle.gershgorin(H)
    assert glo <= lo <= ev[0] and ev[-1] <= hi <= ghi


def test_solve_small_config_matches_dense():
    """The 8x8x8 parity configuration: n_s = 32, n_p = 200, window holding
    about 16 eigenvalues; eigenvalues to 1e-10 of dense eigh, residual <= 1e-10.
    Also without a target count (stable-count rule)."""
    H = oracle.topi_csr(8, 8, 8, seed=1)
    ev = np.linalg.eigvalsh(H.dense())
    delta, k = oracle.window_from_dense(ev, 16)
    v0 = inputs.gaussian_block(H.N, 1, seed=3, tag=2)[:, 0]
    lmin, lmax = oracle.lanczos_bounds(H, 40, v0)
    X0 = inputs.gaussian_block(H.N, 32, seed=2)
    th, r, X, it, ok = oracle.solve(H, lmin, lmax, -delta, delta, 200, X0, 32, n_t=k)
    assert ok, (it, r)
    exact = np.sort(ev[np.abs(ev) < delta])
    assert len(th) == len(exact) == k
    assert np.max(np.abs(np.sort(th) - exact)) < 1e-10
    assert np.max(r) <= 1e-10
    th2, r2, _, it2, ok2 = oracle.solve(H, lmin, lmax, -delta, delta, 200, X0, 32)
    assert ok2 and len(th2) == k and it2 >= it
    assert np.max(np.abs(np.sort(th2) - exact)) < 1e-10


# ------------------------------------------------------- planted mistakes --

def test_pins_catch_planted_mistakes(monkeypatch):
    """A wrong coefficient convention (c_0 halved) fails the quadrature pin,
    a wrong Jackson order (M = n_p) fails g_1 = cos(pi / (M + 1)), and a
    wrong spectral map fails the brute-force pin."""
    lmin, lmax, win = -3.0, 5.0, (-0.3, 0.4)
    a, b = oracle.spectral_map(lmin, lmax)
    c = oracle.window_coeffs(*win, lmin, lmax, 4)
    Tk = npcheb.Chebyshev.basis(0)
    val, _ = si.quad(lambda x: Tk(x) / math.sqrt(1 - x * x), a * win[0] + b, a * win[1] + b)
    assert abs(0.5 * c[0] - val / math.pi) > 1e-3

    g_wrong = oracle.jackson(99)                           # M = 100 instead of 101 for n_p = 100
    assert abs(g_wrong[1] - math.cos(math.pi / (100 + 2))) > 1e-9     # pin tolerance is 1e-14

    H = oracle.topi_csr(3, 3, 3, seed=4)
    X = inputs.gaussian_block(H.N, 2, seed=5)
    ref = oracle.dense_filter(H.dense(), -8.6, 8.6, -1.0, 1.0, 40, X)
    real_map = oracle.spectral_map
    monkeypatch.setattr(oracle, "spectral_map", lambda lo, hi: (real_map(lo, hi)[0], -real_map(lo, hi)[1] + 0.01))
    Y, _ = oracle.chebfd_filter(H, -8.6, 8.6, -1.0, 1.0, 40, X, 2)
    assert np.linalg.norm(Y - ref) / np.linalg.norm(ref) > 1e-6


# ----------------------------------------------------------- traffic model (P12) --

def test_traffic_model_reproduces_table3_and_eq2():
    from paper_1803_02156_gb300 import model
    g = json.load(open(os.path.join(GOLD, "paper_table3_eq2.json")))
    t3 = g["table3_minimum"]
    N = 4 * np.prod(t3["lattice"])
    assert N == t3["n"]
    rd, wr = model.step_read_write_bytes(N, t3["nnzr"] * N, t3["n_b"])
    assert round(rd / 1e9, 2) == t3["read_gb"]
    assert round(wr / 1e9, 2) == t3["write_gb"]
    assert abs(model.intensity(1e12) - g["eq2"]["limit"]) <= 0.0051   # 146 / 80 = 1.825, printed as 1.83
    assert model.step_flops(1, 13, 1) == g["eq2"]["numerator_flops"]
    assert model.step_bytes(1, 13, 1) == g["eq2"]["matrix_bytes_per_row"] + g["eq2"]["vector_bytes_per_row"]
    for r in g["roofline_gflops"]:
        v = model.roofline(r["n_b"], r["bandwidth_gbs"])
        assert abs(v - r["value"]) / r["value"] < 0.01, (r, v)


# ------------------------------------------------------------ KPM counting --

def test_kpm_count_exact_with_full_basis():
    """With the full standard basis as 'random' vectors the trace estimate is
    exact for the damped window: sum_i p(lambda_i) over the dense spectrum."""
    H = oracle.topi_csr(4, 4, 3, seed=8)
    Hd = H.dense()
    lam = np.linalg.eigvalsh(Hd)
    E = np.eye(H.N, dtype=np.complex128)
    n_p = 60
    _, dots = oracle.chebfd_filter(H, -8.6, 8.6, -1.0, 1.0, n_p, E, 16)
    mu = oracle.kpm_moments(dots)
    cnt = oracle.kpm_count(mu, H.N, -8.6, 8.6, -0.8, 0.9)
    a, b = oracle.spectral_map(-8.6, 8.6)
    gc = oracle.jackson(2 * n_p - 1) * oracle.window_coeffs(-0.8, 0.9, -8.6, 8.6, 2 * n_p - 1)
    ref = oracle.filter_polynomial(a * lam + b, gc).sum()
    assert abs(cnt - ref) < 1e-9 * H.N


def test_kpm_count_estimates_dense_count():
    H = oracle.topi_csr(8, 8, 8, seed=1)
    ev = np.linalg.eigvalsh(H.dense())
    X = inputs.gaussian_block(H.N, 64, seed=21)
    _, dots = oracle.chebfd_filter(H, -8.6, 8.6, -0.7, 0.7, 400, X, 32)
    mu = oracle.kpm_moments(dots)
    cnt = oracle.kpm_count(mu, H.N, -8.6, 8.6, -2.0, 2.0)
    true = np.sum(np.abs(ev) <= 2.0)
    assert abs(cnt - true) < 0.1 * true


def test_library_kpm_functions_match_oracle():
    """The library's host KPM count equals the oracle's on the same moments;
    its window bisection hits the target count."""
    from paper_1803_02156_gb300 import build, binding as b
    build.build()
    H = oracle.topi_csr(6, 6, 6, seed=2)
    X = inputs.gaussian_block(H.N, 16, seed=4)
    _, dots = oracle.chebfd_filter(H, -8.6, 8.6, -0.7, 0.7, 150, X, 16)
    mu = oracle.kpm_moments(dots)
    for win in [(-0.5, 0.5), (-3.0, 1.0), (2.0, 8.0)]:
        assert abs(b.cfd_kpm_count(mu, H.N, -8.6, 8.6, *win) - oracle.kpm_count(mu, H.N, -8.6, 8.6, *win)) < 1e-9
    lo, hi = b.cfd_kpm_window(mu, H.N, -8.6, 8.6, 0.0, 40.0)
    assert abs(oracle.kpm_count(mu, H.N, -8.6, 8.6, lo, hi) - 40.0) < 1e-6
    assert abs(lo + hi) < 1e-12


def test_fma_pipe_flop_model_counts_the_step():
    """The ALU roofline's flop count tallies the fused step's fp64 FMAs per row
    and vector at 13 stored entries: packed values 2 per entry (26), shift /
    scale / subtraction 4, X update 2, two dots 4 = 36 FMAs (72 flops); with
    the prepared values of 2 alpha (H - beta) the 4 for the map vanish (32);
    complex values cost 4 FMAs per entry."""
    from paper_1803_02156_gb300 import model
    assert model.step_fma_flops(1, 13, 1, packed=True) == 2 * 36
    assert model.step_fma_flops(1, 13, 1, packed=True, prepared=True) == 2 * 32
    assert model.step_fma_flops(1, 13, 1, packed=False) == 2 * (13 * 4 + 10)
    # scales with the rows and the block width, the matrix term with nnz
    assert model.step_fma_flops(524288, 6750208, 32, packed=True, prepared=True) == (4 * 6750208 + 12 * 524288) * 32
