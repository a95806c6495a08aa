"""ChebFD oracle: a plain, slow, obviously correct CPU implementation.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference arm may import or run anything under oracle/.  The
CUDA library never calls it, and the oracle imports nothing from the library:
the two share no code.  Inputs (start blocks) come from the seeded generator
module paper_1803_02156_gb300.inputs, which holds none of the method's
arithmetic, or are passed in by the caller.

Everything is fp64 (complex128).  Each function cites the part of arxiv
1803.02156 (Kreutzer et al., "Chebyshev Filter Diagonalization on Modern
Manycore Processors and GPGPUs") it follows.  Where the paper leaves a
definition to its references (window coefficients c_k, Jackson kernel g_k,
spectral bounds, the Hamiltonian's conventions), the reading taken is stated
in the docstring.

The matrix build, CSR SpMMV and the filter recurrence (Algorithms 1 and 2) are
plain C in oracle.c; the dense linear algebra is numpy.
"""
import ctypes
import math

import numpy as np

from . import build as _build

_LIB = None


def lib():
    """Load (building first if needed) the oracle's C library."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i64, i32, u64, dbl, ptr = (ctypes.c_int64, ctypes.c_int, ctypes.c_uint64,
                                   ctypes.c_double, ctypes.c_void_p)
        L.orc_splitmix64.restype = u64
        L.orc_splitmix64.argtypes = [u64, u64, u64]
        L.orc_uniform.restype = dbl
        L.orc_uniform.argtypes = [u64, u64, u64]
        L.orc_topi_nnz.restype = i64
        L.orc_topi_nnz.argtypes = [i32, i32, i32, ptr]
        L.orc_topi_csr.restype = i32
        L.orc_topi_csr.argtypes = [i32, i32, i32, ptr, dbl, dbl, dbl, u64, ptr, ptr, ptr]
        L.orc_csr_spmmv.restype = None
        L.orc_csr_spmmv.argtypes = [i64, ptr, ptr, ptr, ptr, i64, ptr, i64, i32]
        L.orc_chebfd_filter.restype = i32
        L.orc_chebfd_filter.argtypes = [i64, ptr, ptr, ptr, dbl, dbl, i32, ptr, ptr, i64,
                                        i32, i32, ptr]
        L.orc_num_threads.restype = i32
        L.orc_num_threads.argtypes = []
        _LIB = L
    return _LIB


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------- matrix --

class CSR:
    """Canonical CSR of a complex Hermitian matrix: rows in lattice order
    (row = 4 site + orbital, site = x + Nx (y + Ny z)), columns ascending."""

    def __init__(self, rowptr, col, val):
        self.rowptr = rowptr          # int64 [N + 1]
        self.col = col                # int32 [nnz]
        self.val = val                # complex128 [nnz]
        self.N = len(rowptr) - 1
        self.nnz = len(col)

    def dense(self):
        A = np.zeros((self.N, self.N), dtype=np.complex128)
        for i in range(self.N):
            s, e = self.rowptr[i], self.rowptr[i + 1]
            A[i, self.col[s:e]] = self.val[s:e]
        return A

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.N, self.N))


def topi_nnz(Nx, Ny, Nz, periodic=(1, 1, 0)):
    per = np.array(periodic, dtype=np.int32)
    return int(lib().orc_topi_nnz(Nx, Ny, Nz, _p(per)))


def topi_csr(Nx, Ny, Nz, t=1.0, m=2.0, gamma=1.0, seed=1, periodic=(1, 1, 0)):
    """Topological-insulator Hamiltonian Topi-Nx-Ny-Nz (Sect. 2.1): a sparse
    complex Hermitian matrix of dimension n = 4 Nx Ny Nz with 13 nonzeros per
    interior row.  The paper defers the model to its references; the reading
    used here: Gamma_1 = s_z (x) 1, Gamma_{2,3,4} = s_x (x) s_{x,y,z} (index of
    s_a (x) s_b entry is 2a + b); on-site block (m + V_s) Gamma_1 with
    V_s = gamma (u_s - 1/2), u_s uniform from counter-based SplitMix64
    (seed, tag 0, s); hop block T_j = -(t/2) Gamma_1 + i (t/2) Gamma_{j+2} at
    block (site + e_j, site), T_j^H at (site, site + e_j); axes with
    periodic[j] wrap, the others are open."""
    per = np.array(periodic, dtype=np.int32)
    N = 4 * Nx * Ny * Nz
    nnz = topi_nnz(Nx, Ny, Nz, periodic)
    rowptr = np.zeros(N + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    val = np.zeros(nnz, dtype=np.complex128)
    rc = lib().orc_topi_csr(Nx, Ny, Nz, _p(per), float(t), float(m), float(gamma),
                            int(seed), _p(rowptr), _p(col), _p(val))
    if rc != 0:
        raise ValueError("invalid lattice %dx%dx%d periodic=%s" % (Nx, Ny, Nz, periodic))
    return CSR(rowptr, col, val)


def splitmix64(seed, tag, i):
    return int(lib().orc_splitmix64(seed, tag, i))


def uniform(seed, tag, i):
    return float(lib().orc_uniform(seed, tag, i))


def spmmv(H, X):
    """Y = H X for a row-major complex block X (N x nb) via the C CSR SpMMV."""
    X = np.ascontiguousarray(X, dtype=np.complex128)
    if X.ndim == 1:
        X = X[:, None]
    nb = X.shape[1]
    Y = np.zeros_like(X)
    lib().orc_csr_spmmv(H.N, _p(H.rowptr), _p(H.col), _p(H.val), _p(X), nb, _p(Y), nb, nb)
    return Y


def gershgorin(H):
    """Interval containing every eigenvalue: [min_i (H_ii - R_i), max_i (H_ii + R_i)]
    with R_i the off-diagonal absolute row sum (Gershgorin circle theorem)."""
    lo, hi = np.inf, -np.inf
    for i in range(H.N):
        s, e = H.rowptr[i], H.rowptr[i + 1]
        c = H.col[s:e]
        v = H.val[s:e]
        d = v[c == i].real.sum()
        r = np.abs(v[c != i]).sum()
        lo = min(lo, d - r)
        hi = max(hi, d + r)
    return lo, hi


# ---------------------------------------------------- filter coefficients --

def spectral_map(lmin, lmax):
    """Algorithm 1's affine map a H + b 1 taking [lmin, lmax] onto [-1, 1]:
    a = 2 / (lmax - lmin), b = -(lmax + lmin) / (lmax - lmin)."""
    a = 2.0 / (lmax - lmin)
    b = -(lmax + lmin) / (lmax - lmin)
    return a, b


def window_coeffs(lam_l, lam_r, lmin, lmax, n_p):
    """Chebyshev coefficients c_0..c_{n_p} of the indicator function of the
    search interval [lam_l, lam_r] (Sect. 2: "window function"; the paper
    defers the definition to its ref. Pieper15).  Reading: on the scaled axis
    x = a lam + b, with theta = arccos(x), the expansion of the indicator of
    [x_l, x_r] in T_k has c_0 = (theta_l - theta_r) / pi and
    c_k = 2 (sin k theta_l - sin k theta_r) / (k pi) for k >= 1."""
    a, b = spectral_map(lmin, lmax)
    xl = min(max(a * lam_l + b, -1.0), 1.0)
    xr = min(max(a * lam_r + b, -1.0), 1.0)
    tl, tr = math.acos(xl), math.acos(xr)
    c = np.zeros(n_p + 1)
    c[0] = (tl - tr) / math.pi
    for k in range(1, n_p + 1):
        c[k] = 2.0 * (math.sin(k * tl) - math.sin(k * tr)) / (k * math.pi)
    return c


def jackson(n_p):
    """Jackson kernel damping factors g_0..g_{n_p} (Sect. 2 and Algorithm 1
    use g_k; definition from the kernel polynomial method literature) for
    M = n_p + 1 moments:
    g_k = [(M - k + 1) cos(pi k / (M + 1)) + sin(pi k / (M + 1)) cot(pi / (M + 1))] / (M + 1)."""
    M = n_p + 1
    q = math.pi / (M + 1)
    g = np.zeros(n_p + 1)
    for k in range(n_p + 1):
        g[k] = ((M - k + 1) * math.cos(q * k) + math.sin(q * k) / math.tan(q)) / (M + 1)
    return g


def filter_coeffs(lam_l, lam_r, lmin, lmax, n_p):
    """gc_k = g_k c_k, the weights of T_k in the filter polynomial (Algorithm 1)."""
    return jackson(n_p) * window_coeffs(lam_l, lam_r, lmin, lmax, n_p)


def filter_polynomial(x, gc):
    """p(x) = sum_k gc_k T_k(x) evaluated via T_k(x) = cos(k arccos x) on [-1, 1]."""
    th = np.arccos(np.clip(x, -1.0, 1.0))
    k = np.arange(len(gc))
    return np.cos(np.outer(th, k)) @ gc


# ---------------------------------------------------------------- filter --

def chebfd_filter(H, lmin, lmax, lam_l, lam_r, n_p, X, n_b):
    """Apply the ChebFD polynomial filter (Algorithm 1) to the columns of X,
    n_b at a time (Algorithm 2), via the plain C recurrence.  Returns the
    filtered block and the per-step dot products dots[j, p-1] =
    (<T_{p-1} x_j, T_{p-1} x_j>, Re <T_p x_j, T_{p-1} x_j>) for p = 1..n_p."""
    X = np.array(X, dtype=np.complex128, order="C", copy=True)
    N, n_s = X.shape
    if N != H.N:
        raise ValueError("X rows do not match H")
    a, b = spectral_map(lmin, lmax)
    gc = np.ascontiguousarray(filter_coeffs(lam_l, lam_r, lmin, lmax, n_p))
    dots = np.zeros((n_s, n_p, 2))
    rc = lib().orc_chebfd_filter(H.N, _p(H.rowptr), _p(H.col), _p(H.val), a, b, n_p, _p(gc),
                                 _p(X), n_s, n_s, n_b, _p(dots))
    if rc != 0:
        raise ValueError("oracle filter rejected its arguments")
    return X, dots


def kpm_moments(dots):
    """Chebyshev (KPM) moments mu_m = <x, T_m x>, m = 0..2 n_p - 1, from the
    per-step dots of Algorithm 1 lines 10-11, using T_k T_l = (T_{k+l} + T_{|k-l|}) / 2:
    mu_{2p-2} = 2 <T_{p-1}x, T_{p-1}x> - mu_0 and mu_{2p-1} = 2 <T_p x, T_{p-1}x> - mu_1."""
    n_s, n_p, _ = dots.shape
    mu = np.zeros((n_s, 2 * n_p))
    mu[:, 0] = dots[:, 0, 0]
    mu[:, 1] = dots[:, 0, 1]
    for p in range(2, n_p + 1):
        mu[:, 2 * p - 2] = 2.0 * dots[:, p - 1, 0] - mu[:, 0]
        mu[:, 2 * p - 1] = 2.0 * dots[:, p - 1, 1] - mu[:, 1]
    return mu


def dense_filter(Hd, lmin, lmax, lam_l, lam_r, n_p, X):
    """Brute-force filter X_ref = V p(a Lambda + b) V^H X from a dense
    Hermitian eigendecomposition H = V Lambda V^H (truth for small lattices)."""
    lam, V = np.linalg.eigh(Hd)
    a, b = spectral_map(lmin, lmax)
    gc = filter_coeffs(lam_l, lam_r, lmin, lmax, n_p)
    pv = filter_polynomial(a * lam + b, gc)
    return V @ (pv[:, None] * (V.conj().T @ X))


def dense_moments(Hd, lmin, lmax, X, n_mom):
    """mu_m[j] = sum_i |v_i^H x_j|^2 T_m(a lambda_i + b) from dense eigh."""
    lam, V = np.linalg.eigh(Hd)
    a, b = spectral_map(lmin, lmax)
    w = np.abs(V.conj().T @ X) ** 2                      # [N, n_s]
    th = np.arccos(np.clip(a * lam + b, -1.0, 1.0))
    T = np.cos(np.outer(np.arange(n_mom), th))           # [n_mom, N]
    return (T @ w).T


# ------------------------------------------------ bounds, orth, Rayleigh-Ritz --

def lanczos_bounds(H, steps, v0):
    """Spectral bounds for the affine map (not specified by the paper; reading:
    `steps` Lanczos steps with full reorthogonalisation from v0; the extreme
    Ritz values theta_1, theta_m are widened by their residual bounds
    |beta_m y_{m,i}| plus 1% of theta_m - theta_1, then clipped to the
    Gershgorin interval)."""
    v = np.asarray(v0, dtype=np.complex128).copy()
    v /= np.linalg.norm(v)
    Vs = [v]
    alpha, beta = [], []
    prev, bprev = np.zeros_like(v), 0.0
    bm = 0.0
    for k in range(steps):
        w = spmmv(H, Vs[-1])[:, 0] - bprev * prev
        ak = float(np.vdot(Vs[-1], w).real)
        w = w - ak * Vs[-1]
        Q = np.array(Vs).T
        w = w - Q @ (Q.conj().T @ w)
        bk = float(np.linalg.norm(w))
        alpha.append(ak)
        if k == steps - 1 or bk == 0.0:
            bm = bk
            break
        beta.append(bk)
        prev, bprev = Vs[-1], bk
        Vs.append(w / bk)
    m = len(alpha)
    T = np.diag(alpha) + np.diag(beta[:m - 1], 1) + np.diag(beta[:m - 1], -1)
    th, Y = np.linalg.eigh(T)
    spread = th[-1] - th[0]
    lo = th[0] - abs(bm * Y[-1, 0]) - 0.01 * spread
    hi = th[-1] + abs(bm * Y[-1, -1]) + 0.01 * spread
    glo, ghi = gershgorin(H)
    return max(lo, glo), min(hi, ghi)


def mgs2(X):
    """Orthonormalise the columns of X by modified Gram-Schmidt, applied twice
    (the oracle's stand-in for the rank-revealing orthogonalisation the paper
    names, SVQB or TSQR, Sect. 2)."""
    Q = np.array(X, dtype=np.complex128, copy=True)
    n = Q.shape[1]
    for _ in range(2):
        for j in range(n):
            for k in range(j):
                Q[:, j] -= np.vdot(Q[:, k], Q[:, j]) * Q[:, k]
            Q[:, j] /= np.linalg.norm(Q[:, j])
    return Q


def rayleigh_ritz(H, X):
    """Rayleigh-Ritz on the orthonormal block X (the restart step implied in
    Sect. 2): G = X^H H X, G = Y diag(theta) Y^H, Ritz vectors X Y and residual
    norms ||H x_i - theta_i x_i||_2.  Returns (theta ascending, X Y, r)."""
    Z = spmmv(H, X)
    G = X.conj().T @ Z
    G = 0.5 * (G + G.conj().T)
    th, Y = np.linalg.eigh(G)
    Xr = X @ Y
    Zr = Z @ Y
    r = np.linalg.norm(Zr - Xr * th[None, :], axis=0)
    return th, Xr, r


def solve(H, lmin, lmax, lam_l, lam_r, n_p, X0, n_b, tol=1e-10, max_iter=50, n_t=0):
    """ChebFD restart loop (Sect. 2): filter, orthogonalise, Rayleigh-Ritz.
    The paper gives no stopping rule; reading: a Ritz pair inside
    [lam_l, lam_r] is converged when its residual is <= tol; the loop stops
    when the number of converged in-window pairs reaches n_t (n_t > 0), or
    when that number is >= 1 and unchanged over three consecutive iterations
    while the smallest residual of the unconverged in-window pairs did not
    halve in either of the last two (no pair is still converging).  In-window
    Ritz values inside a spectral gap (mixtures of states from both sides of
    the window) never converge and are not counted.  Returns (theta, r, X,
    iterations, converged) with theta, r the converged in-window pairs."""
    X = np.array(X0, dtype=np.complex128, copy=True)
    hist, mres = [], []
    th = r = None
    for it in range(1, max_iter + 1):
        X, _ = chebfd_filter(H, lmin, lmax, lam_l, lam_r, n_p, X, n_b)
        X = mgs2(X)
        th, X, r = rayleigh_ritz(H, X)
        inside = (th >= lam_l) & (th <= lam_r)
        conv = inside & (r <= tol)
        hist.append(int(conv.sum()))
        rest = r[inside & ~conv]
        mres.append(float(rest.min()) if rest.size else 1e300)      # none left: nothing improves
        stable = (len(hist) >= 3 and hist[-1] >= 1 and hist[-1] == hist[-2] == hist[-3]
                  and mres[-1] > 0.5 * mres[-2] and mres[-2] > 0.5 * mres[-3])
        if (n_t > 0 and hist[-1] >= n_t) or stable:
            return th[conv], r[conv], X, it, True
    conv = (th >= lam_l) & (th <= lam_r) & (r <= tol)
    return th[conv], r[conv], X, max_iter, False


def window_from_dense(evals, target):
    """Search window [-delta, delta] centred at 0 holding about `target`
    eigenvalues: sort |lambda|, take the count k nearest `target` at which
    |lambda|_(k+1) - |lambda|_(k) > 1e-8 (degenerate levels do not straddle the
    edge) and delta the midpoint of that gap.  Returns (delta, k)."""
    a = np.sort(np.abs(np.asarray(evals)))
    best = None
    for k in range(1, len(a)):
        if a[k] - a[k - 1] > 1e-8:
            if best is None or abs(k - target) < abs(best - target):
                best = k
    return 0.5 * (a[best - 1] + a[best]), best


def kpm_count(mu, N, lmin, lmax, lam_l, lam_r):
    """Kernel-polynomial estimate of the number of eigenvalues in [lam_l, lam_r]
    (Sect. 2: the Chebyshev moments monitor the number of states in the search
    interval): the trace of the Jackson-damped window function, estimated with
    the random vectors whose moments are the rows of mu,
    count = N / R sum_r (sum_m g_m c_m mu_m(r)) / mu_0(r), with g_m the Jackson
    kernel for M = n_mom moments and c_m the window coefficients."""
    mu = np.atleast_2d(np.asarray(mu, dtype=np.float64))
    n_mom = mu.shape[1]
    c = window_coeffs(lam_l, lam_r, lmin, lmax, n_mom - 1)
    g = jackson(n_mom - 1)
    per = (mu @ (g * c)) / mu[:, 0]
    return N * per.mean()

