"""GPU parity of the matrix build and the fused ChebFD filter against the CPU
oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1803_02156_gb300 import inputs, workloads

pytestmark = pytest.mark.gpu

# filtered block vs oracle (relative Frobenius) and moments (relative to max |mu|), fp64 path
TOL_C128 = 1e-11


@pytest.fixture(scope="module")
def b():
    import torch
    from paper_1803_02156_gb300 import build, binding
    assert torch.cuda.is_available()
    build.build()
    binding.lib()
    return binding


def _gpu_block(X, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(X)).to(dtype).cuda()


@pytest.mark.parametrize("L,per,C,sigma", [((8, 8, 8), (1, 1, 0), 32, 1), ((17, 23, 9), (1, 1, 0), 32, 64),
                                           ((4, 4, 4), (1, 1, 1), 8, 1), ((5, 4, 6), (0, 1, 0), 16, 32),
                                           ((3, 3, 1), (1, 1, 0), 4, 1)])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_matrix_build_bitexact(b, L, per, C, sigma, prec):
    import torch
    p = b.topi_params(*L, seed=17, periodic=per)
    H = b.cfd_build_matrix(p, C, sigma, prec)
    rowptr, col, val = b.cfd_matrix_export_csr(H)
    torch.cuda.synchronize()
    ref = oracle.topi_csr(*L, seed=17, periodic=per)
    assert np.array_equal(rowptr.cpu().numpy(), ref.rowptr)
    assert np.array_equal(col.cpu().numpy(), ref.col)
    v = val.cpu().numpy()
    want = ref.val if prec == "c128" else ref.val.astype(np.complex64)
    assert np.array_equal(v.view(np.uint8), want.view(np.uint8))           # bit-exact


def test_filter_coeffs_match_oracle(b):
    for (lmin, lmax, wl, wr, n_p) in [(-8.5, 8.5, -0.7, 0.7, 200), (-3.0, 5.0, 1.0, 1.5, 1000), (-1, 1, -1, 1, 10)]:
        gc = b.cfd_filter_coeffs(lmin, lmax, wl, wr, n_p).cpu().numpy()
        ref = oracle.filter_coeffs(wl, wr, lmin, lmax, n_p)
        assert np.max(np.abs(gc - ref)) < 1e-14


def _compare_filter(b, L, n_s, n_b, n_p, win, prec="c128", seed=1, tol=TOL_C128, bounds=(-8.6, 8.6)):
    import torch
    H = b.cfd_build_matrix(b.topi_params(*L, seed=seed), 32, 1, prec)
    ref = oracle.topi_csr(*L, seed=seed)
    X = inputs.gaussian_block(ref.N, n_s, seed=2)
    Xg = _gpu_block(X, torch.complex128 if prec == "c128" else torch.complex64)
    mu = b.cfd_filter(H, bounds[0], bounds[1], win[0], win[1], n_p, Xg, n_b, moments=True)
    torch.cuda.synchronize()
    Y, dots = oracle.chebfd_filter(ref, bounds[0], bounds[1], win[0], win[1], n_p, X, n_b)
    Yg = Xg.cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(Yg - Y) / np.linalg.norm(Y)
    muref = oracle.kpm_moments(dots)
    merr = np.max(np.abs(mu.cpu().numpy() - muref)) / np.max(np.abs(muref))
    assert err < tol, err
    assert merr < tol, merr
    return Xg, err, merr


@pytest.mark.parametrize("n_b", [8, 16, 32])
def test_filter_parity_small_config(b, n_b):
    """8x8x8 (N = 2048), n_s = 32, n_p = 200: block and moments vs oracle."""
    w = workloads.SMALL
    _compare_filter(b, w.lattice, w.n_s, n_b, w.n_p, (-0.7, 0.7))


@pytest.mark.parametrize("L,n_s,n_b,n_p", [((16, 16, 9), 64, 64, 40), ((13, 7, 5), 48, 16, 25),
                                           ((9, 10, 3), 8, 8, 2)])
def test_filter_parity_ragged(b, L, n_s, n_b, n_p):
    """Several chunks and a ragged tail (N not a multiple of C or of the CTA's rows)."""
    _compare_filter(b, L, n_s, n_b, n_p, (-1.1, 0.4))


def test_filter_block_width_invariance(b):
    """The fp64 filtered block is bitwise identical for every n_b."""
    import torch
    L = (12, 10, 7)
    H = b.cfd_build_matrix(b.topi_params(*L), 32, 1, "c128")
    X = inputs.gaussian_block(4 * 12 * 10 * 7, 64, seed=4)
    outs = []
    for n_b in (8, 16, 32, 64):
        Xg = _gpu_block(X, torch.complex128)
        b.cfd_filter(H, -8.6, 8.6, -0.5, 0.5, 60, Xg, n_b)
        outs.append(Xg.cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_filter_deterministic_moments(b):
    import torch
    L = (16, 16, 8)
    H = b.cfd_build_matrix(b.topi_params(*L), 32, 1, "c128")
    X = inputs.gaussian_block(4 * 16 * 16 * 8, 32, seed=5)
    res = []
    for _ in range(2):
        Xg = _gpu_block(X, torch.complex128)
        mu = b.cfd_filter(H, -8.6, 8.6, -0.5, 0.5, 30, Xg, 32, moments=True)
        res.append((Xg.cpu().numpy(), mu.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_filter_full_window_is_identity(b):
    import torch
    L = (8, 8, 4)
    H = b.cfd_build_matrix(b.topi_params(*L), 32, 1, "c128")
    X = inputs.gaussian_block(4 * 8 * 8 * 4, 16, seed=6)
    Xg = _gpu_block(X, torch.complex128)
    b.cfd_filter(H, -9.0, 9.0, -9.0, 9.0, 100, Xg, 16)
    assert np.linalg.norm(Xg.cpu().numpy() - X) / np.linalg.norm(X) < 1e-13


# fp32 arithmetic: the rounding of each step is about nnzr * u32 relative and
# the three-term recurrence adds it up linearly over the n_p steps, so the
# filtered block of the n_p = 200 configuration is within n_p * 13 * 2^-24
# (1.6e-4) of the fp64 oracle; moments likewise.
TOL_C64_200 = 200 * 13 * 2.0 ** -24


def test_filter_c64_small_config(b):
    w = workloads.SMALL
    _compare_filter(b, w.lattice, w.n_s, 32, w.n_p, (-0.7, 0.7), prec="c64", tol=TOL_C64_200)


def test_filter_mixed_precision_block(b):
    """c64 matrix with a c128 block: narrowed, filtered in fp32, widened."""
    import torch
    w = workloads.SMALL
    H = b.cfd_build_matrix(b.topi_params(*w.lattice), 32, 1, "c64")
    ref = oracle.topi_csr(*w.lattice)
    X = inputs.gaussian_block(ref.N, 32, seed=2)
    Xg = _gpu_block(X, torch.complex128)
    b.cfd_filter(H, -8.6, 8.6, -0.7, 0.7, 200, Xg, 16)
    Y, _ = oracle.chebfd_filter(ref, -8.6, 8.6, -0.7, 0.7, 200, X, 16)
    err = np.linalg.norm(Xg.cpu().numpy() - Y) / np.linalg.norm(Y)
    assert err < TOL_C64_200, err


def test_filter_parity_full_size_few_steps(b):
    """The 64x64x32 lattice (N = 524288) in the bench's launch configuration
    (n_b = 32, SELL C = 32, sigma = 1) for a few steps, against the oracle."""
    w = workloads.MEDIUM
    _compare_filter(b, w.lattice, 32, 32, 6, (-0.3, 0.3))


# fp32 bound for the 12-step full-size run below (same derivation as TOL_C64_200)
TOL_C64_12 = 12 * 13 * 2.0 ** -24


@pytest.mark.parametrize("prec,tol", [("c128p", TOL_C128), ("c64p", TOL_C64_12)])
def test_bench_kernel_full_size_parity(b, prec, tol):
    """The benchmark's kernel variant at full size: the 64x64x32 lattice
    (N = 524288), packed real-or-imaginary values prepared as 2 alpha (H - beta),
    TMA-staged general steps with moments, SELL C = 32, n_b = 32, for 12 steps
    (10 general steps), against the oracle's filtered block and moments.
    complex64: the fp32 filter on a complex128 block, as the mixed policy runs it."""
    import torch
    w = workloads.MEDIUM
    n_s, n_b, n_p, win = 32, 32, 12, (-0.3, 0.3)
    H = b.cfd_build_matrix(b.topi_params(*w.lattice, seed=w.seed), 32, 1, prec)
    assert H.packed
    ref = oracle.topi_csr(*w.lattice, seed=w.seed)
    X = inputs.gaussian_block(ref.N, n_s, seed=2)
    Xg = _gpu_block(X, torch.complex128)
    mu = b.cfd_filter(H, -8.6, 8.6, win[0], win[1], n_p, Xg, n_b, moments=True)
    torch.cuda.synchronize()
    Y, dots = oracle.chebfd_filter(ref, -8.6, 8.6, win[0], win[1], n_p, X, n_b)
    err = np.linalg.norm(Xg.cpu().numpy() - Y) / np.linalg.norm(Y)
    muref = oracle.kpm_moments(dots)
    merr = np.max(np.abs(mu.cpu().numpy() - muref)) / np.max(np.abs(muref))
    assert err < tol, err
    assert merr < tol, merr


def test_filter_full_size_properties(b):
    """Full degree n_p = 1000 on 64x64x32: properties that hold at any size.
    mu_0 = ||x||^2 and |mu_m| <= mu_0 (|T_m| <= 1 on the scaled spectrum);
    the Jackson-damped filter has 0 <= p <= 1 on the spectrum, so no column
    grows; the result is bitwise independent of n_b."""
    import torch
    w = workloads.MEDIUM
    H = b.cfd_build_matrix(b.topi_params(*w.lattice), 32, 1, "c128")
    X = inputs.gaussian_block(w.N, 64, seed=2)
    outs = []
    for n_b in (32, 64):
        Xg = _gpu_block(X, torch.complex128)
        mu = b.cfd_filter(H, -8.6, 8.6, -0.3, 0.3, w.n_p, Xg, n_b, moments=True)
        outs.append(Xg.cpu().numpy())
    mu = mu.cpu().numpy()
    n0 = np.linalg.norm(X, axis=0) ** 2
    assert np.allclose(mu[:, 0], n0, rtol=1e-12)
    assert np.all(np.abs(mu) <= mu[:, :1] * (1 + 1e-9))
    assert np.all(np.linalg.norm(outs[0], axis=0) ** 2 <= n0 * (1 + 1e-9))
    assert np.array_equal(outs[0], outs[1])


# --------------------------------------------------- packed real/imaginary values --

@pytest.mark.parametrize("L,per,C,sigma", [((8, 8, 8), (1, 1, 0), 32, 1), ((17, 23, 9), (1, 1, 0), 32, 64),
                                           ((5, 4, 6), (0, 1, 0), 16, 32)])
@pytest.mark.parametrize("prec", ["c128p", "c64p"])
def test_packed_matrix_exports_oracle_csr(b, L, per, C, sigma, prec):
    import torch
    H = b.cfd_build_matrix(b.topi_params(*L, seed=17, periodic=per), C, sigma, prec)
    assert H.packed
    rowptr, col, val = b.cfd_matrix_export_csr(H)
    torch.cuda.synchronize()
    ref = oracle.topi_csr(*L, seed=17, periodic=per)
    assert np.array_equal(rowptr.cpu().numpy(), ref.rowptr)
    assert np.array_equal(col.cpu().numpy(), ref.col)
    want = ref.val if prec == "c128p" else ref.val.astype(np.complex64)
    assert np.array_equal(val.cpu().numpy(), want)


@pytest.mark.parametrize("prec,n_b", [("c128", 32), ("c128", 64), ("c64", 32), ("c64", 16)])
def test_packed_filter_equals_complex_storage(b, prec, n_b):
    """Skipping the multiplications by exact zeros changes only the order of
    the row sums (real group, then imaginary group): the filtered block and
    the moments agree with the complex storage's to rounding."""
    import torch
    dt = torch.complex128 if prec == "c128" else torch.complex64
    L = (12, 10, 7)
    Hc = b.cfd_build_matrix(b.topi_params(*L), 32, 1, prec)
    Hp = b.cfd_build_matrix(b.topi_params(*L), 32, 1, prec + "p")
    X0 = torch.from_numpy(inputs.gaussian_block(Hc.N, 64, seed=8)).to(dt).cuda()
    Xc, Xp = X0.clone(), X0.clone()
    mc = b.cfd_filter(Hc, -8.6, 8.6, -0.6, 0.4, 70, Xc, n_b, moments=True)
    mp = b.cfd_filter(Hp, -8.6, 8.6, -0.6, 0.4, 70, Xp, n_b, moments=True)
    tol = 1e-12 if prec == "c128" else 70 * 13 * 2.0 ** -24
    assert (torch.linalg.norm(Xc - Xp) / torch.linalg.norm(Xc)).item() < tol
    assert (torch.max(torch.abs(mc - mp)) / torch.max(torch.abs(mc))).item() < tol


def test_packed_filter_parity_small_config(b):
    w = workloads.SMALL
    import torch
    H = b.cfd_build_matrix(b.topi_params(*w.lattice), 32, 1, "c128p")
    ref = oracle.topi_csr(*w.lattice)
    X = inputs.gaussian_block(ref.N, w.n_s, seed=2)
    Xg = torch.from_numpy(X).cuda()
    b.cfd_filter(H, -8.6, 8.6, -0.7, 0.7, w.n_p, Xg, 32)
    Y, _ = oracle.chebfd_filter(ref, -8.6, 8.6, -0.7, 0.7, w.n_p, X, 32)
    assert np.linalg.norm(Xg.cpu().numpy() - Y) / np.linalg.norm(Y) < TOL_C128


def test_packed_solve_and_bounds(b):
    """Lanczos bounds and the solve accept the packed matrix."""
    import torch
    Hc = oracle.topi_csr(8, 8, 8)
    ev = np.linalg.eigvalsh(Hc.dense())
    delta, k = oracle.window_from_dense(ev, 16)
    H = b.cfd_build_matrix(b.topi_params(8, 8, 8), 32, 1, "c128p")
    lo, hi = b.cfd_spectral_bounds(H, 40)
    assert lo <= ev[0] and ev[-1] <= hi
    X = torch.empty(2048, 32, dtype=torch.complex128, device="cuda")
    th, rs, res = b.cfd_solve(H, X, -delta, delta, 200, 32, n_t=k)
    inside = (th >= -delta) & (th <= delta) & (rs <= 1e-10)
    assert np.max(np.abs(np.sort(th[inside]) - np.sort(ev[np.abs(ev) < delta]))) < 1e-10


def test_kpm_moments_only(b):
    """Moments without the accumulation (Algorithm 1 without line 12) equal the
    filter's moments and the oracle's; the vectors are left unchanged."""
    import torch
    L = (9, 8, 6)
    H = b.cfd_build_matrix(b.topi_params(*L), 32, 1, "c128p")
    ref = oracle.topi_csr(*L)
    R = inputs.gaussian_block(ref.N, 16, seed=31)
    Rg = torch.from_numpy(R).cuda()
    mu = b.cfd_kpm_moments(H, -8.6, 8.6, 120, Rg, 16).cpu().numpy()
    assert np.array_equal(Rg.cpu().numpy(), R)
    _, dots = oracle.chebfd_filter(ref, -8.6, 8.6, -0.5, 0.5, 120, R, 16)
    muref = oracle.kpm_moments(dots)
    assert np.max(np.abs(mu - muref)) / np.max(np.abs(muref)) < 1e-11
    Hc = b.cfd_build_matrix(b.topi_params(*L), 32, 1, "c64p")
    mu32 = b.cfd_kpm_moments(Hc, -8.6, 8.6, 120, Rg.to(torch.complex64), 16).cpu().numpy()
    assert np.max(np.abs(mu32 - muref)) / np.max(np.abs(muref)) < 120 * 13 * 2.0 ** -24


# ------------------------------------------ gathers in flight (staged steps) --

@pytest.mark.parametrize("prec,n_b", [("c64", 32), ("c64", 16), ("c64", 64), ("c128", 32)])
@pytest.mark.parametrize("gather", [8, 16])
def test_gather_all_equals_grouped(b, prec, n_b, gather):
    """Staged general steps that issue all of a row's gathers at once (the
    first 8 or 16 slots, the rest in groups of four) add the same products in
    the same order as groups of four: the filtered block is bitwise equal.
    The open-z lattice has interior chunks of 9 real + 4 imaginary slots and
    boundary chunks of 8 + 3, so gather=8 runs both remainder branches.
    Moments differ only in the order of the cross-CTA reduction."""
    import torch
    dt = torch.complex128 if prec == "c128" else torch.complex64
    L = (8, 6, 5)
    H = b.cfd_build_matrix(b.topi_params(*L), 32, 1, prec + "p")
    X0 = torch.from_numpy(inputs.gaussian_block(H.N, 64, seed=9)).to(dt).cuda()
    Xa, Xb = X0.clone(), X0.clone()
    ma = b.cfd_filter_ex(H, -8.6, 8.6, -0.6, 0.4, 40, Xa, n_b, staged=1, gather=4, moments=True)
    mb = b.cfd_filter_ex(H, -8.6, 8.6, -0.6, 0.4, 40, Xb, n_b, staged=1, gather=gather, moments=True)
    torch.cuda.synchronize()
    assert torch.equal(Xa, Xb)
    tol = 1e-13 if prec == "c128" else 1e-5
    assert (torch.max(torch.abs(ma - mb)) / torch.max(torch.abs(ma))).item() < tol


def test_gather_all_c64_parity_small_config(b):
    """The complex64 filter with all gathers in flight against the fp64 oracle
    on the 8x8x8 configuration (n_p = 200), at the fp32 bound."""
    import torch
    w = workloads.SMALL
    H = b.cfd_build_matrix(b.topi_params(*w.lattice), 32, 1, "c64p")
    ref = oracle.topi_csr(*w.lattice)
    X = inputs.gaussian_block(ref.N, w.n_s, seed=2)
    Xg = torch.from_numpy(X).to(torch.complex64).cuda()
    mu = b.cfd_filter_ex(H, -8.6, 8.6, -0.7, 0.7, w.n_p, Xg, 32, staged=1, gather=16, moments=True)
    torch.cuda.synchronize()
    Y, dots = oracle.chebfd_filter(ref, -8.6, 8.6, -0.7, 0.7, w.n_p, X, 32)
    err = np.linalg.norm(Xg.cpu().numpy().astype(np.complex128) - Y) / np.linalg.norm(Y)
    muref = oracle.kpm_moments(dots)
    merr = np.max(np.abs(mu.cpu().numpy() - muref)) / np.max(np.abs(muref))
    assert err < TOL_C64_200 and merr < TOL_C64_200, (err, merr)


def test_gather_option_rejected(b):
    import torch
    H = b.cfd_build_matrix(b.topi_params(4, 4, 4), 32, 1, "c64p")
    X = torch.zeros(H.N, 16, dtype=torch.complex64, device="cuda")
    with pytest.raises(RuntimeError, match="gather"):
        b.cfd_filter_ex(H, -8.6, 8.6, -0.6, 0.4, 10, X, 16, gather=5)


@pytest.mark.parametrize("prec,n_b,gather", [("c64", 32, 4), ("c64", 16, 16), ("c64", 64, 4), ("c128", 32, 4),
                                             ("c128", 16, 4)])
def test_fixed_chunk_kernel_equals_generic(b, prec, n_b, gather):
    """The staged step compiled for chunk height 32 (immediate shared-memory
    offsets, 32-bit gather offsets) adds the same products in the same order
    as the generic staged step: bitwise equal filtered block, moments equal up
    to the order of the cross-CTA reduction."""
    import torch
    dt = torch.complex128 if prec == "c128" else torch.complex64
    L = (8, 6, 5)
    H = b.cfd_build_matrix(b.topi_params(*L), 32, 1, prec + "p")
    X0 = torch.from_numpy(inputs.gaussian_block(H.N, 64, seed=10)).to(dt).cuda()
    Xa, Xb = X0.clone(), X0.clone()
    ma = b.cfd_filter_ex(H, -8.6, 8.6, -0.6, 0.4, 40, Xa, n_b, staged=1, gather=gather, fixed_chunk=-1,
                         moments=True)
    mb = b.cfd_filter_ex(H, -8.6, 8.6, -0.6, 0.4, 40, Xb, n_b, staged=1, gather=gather, fixed_chunk=1,
                         moments=True)
    torch.cuda.synchronize()
    assert torch.equal(Xa, Xb)
    tol = 1e-13 if prec == "c128" else 1e-5
    assert (torch.max(torch.abs(ma - mb)) / torch.max(torch.abs(ma))).item() < tol


def test_fixed_chunk_kernel_parity_ragged(b):
    """Chunk height 32 with a ragged last chunk (N = 4 * 13 * 7 * 5 = 1820
    rows, not a multiple of 32) and sigma-sorted rows, complex128 staged,
    against the oracle."""
    import torch
    L, n_s, n_b, n_p = (13, 7, 5), 32, 16, 30
    H = b.cfd_build_matrix(b.topi_params(*L), 32, 64, "c128p")
    ref = oracle.topi_csr(*L)
    X = inputs.gaussian_block(ref.N, n_s, seed=2)
    Xg = torch.from_numpy(X).cuda()
    mu = b.cfd_filter_ex(H, -8.6, 8.6, -1.1, 0.4, n_p, Xg, n_b, staged=1, moments=True)
    torch.cuda.synchronize()
    Y, dots = oracle.chebfd_filter(ref, -8.6, 8.6, -1.1, 0.4, n_p, X, n_b)
    assert np.linalg.norm(Xg.cpu().numpy() - Y) / np.linalg.norm(Y) < TOL_C128
    muref = oracle.kpm_moments(dots)
    assert np.max(np.abs(mu.cpu().numpy() - muref)) / np.max(np.abs(muref)) < TOL_C128


@pytest.mark.parametrize("prec", ["c128p", "c64p"])
def test_bounds_guard_reports_bad_bounds(b, prec):
    """Spectral bounds that cut the spectrum (here [-2, 2] against |lambda| up
    to about 8.5) make the Chebyshev moments grow; the filter records
    CFD_ERR_BOUNDS in its workspace status.  Correct bounds leave it clear."""
    import torch
    dt = torch.complex128 if prec.startswith("c128") else torch.complex64
    H = b.cfd_build_matrix(b.topi_params(8, 8, 4), 32, 1, prec)
    ws = b.cfd_filter_workspace(H.N, 16, 16, 40, prec, prec)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    X0 = torch.from_numpy(inputs.gaussian_block(H.N, 16, seed=14)).to(dt).cuda()
    X = X0.clone()
    b.cfd_filter(H, -8.6, 8.6, -0.5, 0.5, 40, X, 16, moments=True, work=work)
    b.cfd_workspace_status(work)                       # clear with bounds that contain the spectrum
    X = X0.clone()
    b.cfd_filter(H, -2.0, 2.0, -0.5, 0.5, 40, X, 16, moments=True, work=work)
    with pytest.raises(b.CfdError) as e:
        b.cfd_workspace_status(work)
    assert e.value.status == 4                         # CFD_ERR_BOUNDS
