"""GPU checks of the batched (block-diagonal, per-realisation map) filter, the
persistent single-launch filter and the kernel options, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1803_02156_gb300 import inputs

pytestmark = pytest.mark.gpu

LATTICES = [(5, 6, 3, 11), (7, 3, 4, 12), (4, 4, 5, 13), (3, 5, 2, 14), (6, 6, 6, 15)]


@pytest.fixture(scope="module")
def b():
    import torch
    from paper_1803_02156_gb300 import build, binding
    assert torch.cuda.is_available()
    build.build()
    binding.lib()
    return binding


def _params(b):
    return [b.topi_params(nx, ny, nz, seed=s) for (nx, ny, nz, s) in LATTICES]


@pytest.mark.parametrize("C,sigma,prec", [(32, 1, "c128"), (8, 64, "c128"), (32, 1, "c64")])
def test_batch_matrix_is_block_diagonal_oracle(b, C, sigma, prec):
    import torch
    B = b.cfd_build_batch(_params(b), C, sigma, prec)
    rowptr, col, val = b.cfd_matrix_export_csr(B)
    torch.cuda.synchronize()
    rowptr, col, val = rowptr.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy()
    for r, (nx, ny, nz, s) in enumerate(LATTICES):
        ref = oracle.topi_csr(nx, ny, nz, seed=s)
        o = B.row_off[r]
        rp = rowptr[o:o + ref.N + 1] - rowptr[o]
        assert np.array_equal(rp, ref.rowptr)
        seg = slice(rowptr[o], rowptr[o + ref.N])
        assert np.array_equal(col[seg], ref.col + o)
        want = ref.val if prec == "c128" else ref.val.astype(np.complex64)
        assert np.array_equal(val[seg].view(np.uint8), want.view(np.uint8))
        assert rowptr[B.row_off[r + 1]] == rowptr[o + ref.N]          # padding rows are empty


def _windows(b):
    import torch
    w = []
    for r in range(len(LATTICES)):
        w.append([-8.6 - 0.1 * r, 8.6 + 0.05 * r, -0.9 + 0.1 * r, 0.4 + 0.2 * r])
    return torch.tensor(w, dtype=torch.float64, device="cuda"), w


@pytest.mark.parametrize("persistent", [1, 0])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_batched_filter_equals_looped(b, persistent, prec):
    """Per realisation the batched filter equals cfd_filter on that realisation
    alone, bit for bit (same kernel arithmetic, same weights, same prepared
    matrix values).  The persistent launch runs the unstaged general step, so
    its reference is the unstaged per-realisation filter (the staged step's
    prepared values round differently)."""
    import torch
    dt = torch.complex128 if prec == "c128" else torch.complex64
    B = b.cfd_build_batch(_params(b), 32, 1, prec)
    wt, w = _windows(b)
    n_s, n_b, n_p = 16, 16, 60
    X = torch.zeros(B.N, n_s, dtype=dt, device="cuda")
    blocks = []
    for r, (nx, ny, nz, s) in enumerate(LATTICES):
        N = 4 * nx * ny * nz
        Xr = torch.from_numpy(inputs.gaussian_block(N, n_s, seed=100 + r)).to(dt).cuda()
        X[B.row_off[r]:B.row_off[r] + N] = Xr
        blocks.append(Xr)
    b.cfd_filter_batched(B, wt, n_p, X, n_b, persistent=persistent)
    for r, (nx, ny, nz, s) in enumerate(LATTICES):
        N = 4 * nx * ny * nz
        H = b.cfd_build_matrix(b.topi_params(nx, ny, nz, seed=s), 32, 1, prec)
        Y = blocks[r].clone()
        b.cfd_filter_ex(H, w[r][0], w[r][1], w[r][2], w[r][3], n_p, Y, n_b, staged=-1 if persistent else 0)
        got = X[B.row_off[r]:B.row_off[r] + N]
        assert torch.equal(got, Y), r
        pad = X[B.row_off[r] + N:B.row_off[r + 1]]
        assert torch.count_nonzero(pad).item() == 0


def test_batched_filter_vs_oracle(b):
    import torch
    B = b.cfd_build_batch(_params(b), 32, 64, "c128")
    wt, w = _windows(b)
    n_s, n_b, n_p = 8, 8, 45
    X = torch.zeros(B.N, n_s, dtype=torch.complex128, device="cuda")
    refs = []
    for r, (nx, ny, nz, s) in enumerate(LATTICES):
        H = oracle.topi_csr(nx, ny, nz, seed=s)
        Xr = inputs.gaussian_block(H.N, n_s, seed=200 + r)
        X[B.row_off[r]:B.row_off[r] + H.N] = torch.from_numpy(Xr).cuda()
        refs.append(oracle.chebfd_filter(H, w[r][0], w[r][1], w[r][2], w[r][3], n_p, Xr, n_b)[0])
    b.cfd_filter_batched(B, wt, n_p, X, n_b)
    for r, Y in enumerate(refs):
        got = X[B.row_off[r]:B.row_off[r] + Y.shape[0]].cpu().numpy()
        assert np.linalg.norm(got - Y) / np.linalg.norm(Y) < 1e-11


@pytest.mark.parametrize("prec,n_b,vpt", [("c128", 32, 1), ("c128", 32, 2), ("c64", 16, 1), ("c64", 64, 2)])
def test_persistent_and_options_bitwise(b, prec, n_b, vpt):
    """Every vectors-per-thread choice gives the per-step result bit for bit;
    the single-launch persistent filter (unstaged general steps) gives the
    unstaged per-step result bit for bit, and the staged one to rounding."""
    import torch
    dt = torch.complex128 if prec == "c128" else torch.complex64
    L = (10, 9, 6)
    H = b.cfd_build_matrix(b.topi_params(*L), 32, 1, prec)
    X0 = torch.from_numpy(inputs.gaussian_block(H.N, 64, seed=3)).to(dt).cuda()
    ref = X0.clone()
    b.cfd_filter(H, -8.6, 8.6, -0.5, 0.5, 80, ref, n_b)
    ref_unstaged = X0.clone()
    b.cfd_filter_ex(H, -8.6, 8.6, -0.5, 0.5, 80, ref_unstaged, n_b, staged=-1)
    Y = X0.clone()
    b.cfd_filter_ex(H, -8.6, 8.6, -0.5, 0.5, 80, Y, n_b, vpt=vpt)
    assert torch.equal(Y, ref)
    Y = X0.clone()
    b.cfd_filter_ex(H, -8.6, 8.6, -0.5, 0.5, 80, Y, n_b, vpt=vpt, persistent=1, grid_cap=200)
    assert torch.equal(Y, ref_unstaged)
    tol = 1e-12 if prec == "c128" else 80 * 13 * 2.0 ** -24
    assert (torch.linalg.norm(Y - ref) / torch.linalg.norm(ref)).item() < tol


@pytest.mark.parametrize("prec,n_b", [("c64p", 32), ("c64p", 16), ("c128p", 32), ("c128p", 64)])
def test_persistent_staged_equals_per_step(b, prec, n_b):
    """With packed values the persistent filter runs steps 1 and 2 as single
    launches and steps 3..n_p in one cooperative launch of the staged step:
    bit for bit the per-step staged filter (same row arithmetic), also with
    fewer CTAs than chunks and a ragged last chunk."""
    import torch
    dt = torch.complex128 if prec.startswith("c128") else torch.complex64
    L = (10, 9, 7)
    H = b.cfd_build_matrix(b.topi_params(*L), 32, 1, prec)
    X0 = torch.from_numpy(inputs.gaussian_block(H.N, 64, seed=3)).to(dt).cuda()
    ref = X0.clone()
    b.cfd_filter(H, -8.6, 8.6, -0.5, 0.5, 80, ref, n_b)
    for cap in (0, 7):
        Y = X0.clone()
        b.cfd_filter_ex(H, -8.6, 8.6, -0.5, 0.5, 80, Y, n_b, persistent=1, grid_cap=cap)
        torch.cuda.synchronize()
        assert torch.equal(Y, ref), cap


def test_persistent_staged_batched_equals_looped(b):
    """The batched filter with the staged persistent launch (packed complex64
    batch) equals the per-realisation filter bit for bit."""
    import torch
    B = b.cfd_build_batch(_params(b), 32, 1, "c64p")
    wt, w = _windows(b)
    n_s, n_b, n_p = 16, 16, 60
    X = torch.zeros(B.N, n_s, dtype=torch.complex64, device="cuda")
    blocks = []
    for r, (nx, ny, nz, s) in enumerate(LATTICES):
        N = 4 * nx * ny * nz
        Xr = torch.from_numpy(inputs.gaussian_block(N, n_s, seed=100 + r)).to(torch.complex64).cuda()
        X[B.row_off[r]:B.row_off[r] + N] = Xr
        blocks.append(Xr)
    b.cfd_filter_batched(B, wt, n_p, X, n_b, persistent=1)
    for r, (nx, ny, nz, s) in enumerate(LATTICES):
        N = 4 * nx * ny * nz
        H = b.cfd_build_matrix(b.topi_params(nx, ny, nz, seed=s), 32, 1, "c64p")
        Y = blocks[r].clone()
        b.cfd_filter(H, w[r][0], w[r][1], w[r][2], w[r][3], n_p, Y, n_b)
        assert torch.equal(X[B.row_off[r]:B.row_off[r] + N], Y), r


def test_persistent_staged_wait_timeout(b):
    """The staged persistent launch with its bounded waits made to expire
    (staged = 2): CFD_ERR_TIMEOUT in the status, every CTA leaves at the same
    grid barrier, and the context stays usable."""
    import torch
    H = b.cfd_build_matrix(b.topi_params(8, 8, 4), 32, 1, "c64p")
    X = torch.from_numpy(inputs.gaussian_block(H.N, 16, seed=6)).to(torch.complex64).cuda()
    work = torch.empty(b.cfd_filter_workspace(H.N, 16, 16, 10, "c64", "c64"), dtype=torch.uint8, device="cuda")
    b.cfd_filter_ex(H, -8.6, 8.6, -0.5, 0.5, 10, X, 16, persistent=1, staged=2, work=work)
    with pytest.raises(b.CfdError) as e:
        b.cfd_workspace_status(work)
    assert e.value.status == 5
    assert "still have been in flight" not in str(e.value)
    Y = X.clone()
    b.cfd_filter_ex(H, -8.6, 8.6, -0.5, 0.5, 10, Y, 16, persistent=1, work=work)
    b.cfd_workspace_status(work)


def test_graph_capture_replays_filter(b):
    """The n_p-step recurrence captured as a CUDA graph (torch capture of the
    C-ABI call on a side stream) replays to the same result."""
    import torch
    L = (8, 8, 4)
    H = b.cfd_build_matrix(b.topi_params(*L), 32, 1, "c128")
    X0 = torch.from_numpy(inputs.gaussian_block(H.N, 32, seed=7)).cuda()
    ref = X0.clone()
    b.cfd_filter(H, -8.6, 8.6, -0.5, 0.5, 50, ref, 32)
    X = X0.clone()
    ws = b.cfd_filter_workspace(H.N, 32, 32, 50, "c128", "c128")
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.cfd_filter(H, -8.6, 8.6, -0.5, 0.5, 50, X, 32, work=work)     # warm-up outside capture
        X.copy_(X0)
    torch.cuda.current_stream().wait_stream(s)
    with torch.cuda.graph(g):
        b.cfd_filter(H, -8.6, 8.6, -0.5, 0.5, 50, X, 32, work=work)
    X.copy_(X0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(X, ref)


# ------------------------------------------------------------ batched solve --

SOLVE_LATTICES = [(6, 6, 4, 21), (5, 7, 4, 22), (8, 4, 3, 23), (6, 5, 6, 24)]


def _batch_truth(target=8):
    wins, nts, exact = [], [], []
    for (nx, ny, nz, s) in SOLVE_LATTICES:
        H = oracle.topi_csr(nx, ny, nz, seed=s)
        ev = np.linalg.eigvalsh(H.dense())
        delta, k = oracle.window_from_dense(ev, target)
        lo, hi = oracle.gershgorin(H)
        wins.append([lo - 0.05, hi + 0.05, -delta, delta])
        nts.append(k)
        exact.append(np.sort(ev[np.abs(ev) < delta]))
    return np.array(wins), np.array(nts, dtype=np.int32), exact


@pytest.mark.parametrize("policy", ["fp64", "mixed"])
def test_batched_solve_matches_dense(b, policy):
    """Four uneven realisations solved together: each realisation's converged
    in-window eigenvalues equal its dense eigh to 1e-10, residuals <= 1e-10."""
    import torch
    params = [b.topi_params(nx, ny, nz, seed=s) for (nx, ny, nz, s) in SOLVE_LATTICES]
    B = b.cfd_build_batch(params, 32, 1, "c128p")
    Bl = b.cfd_build_batch(params, 32, 1, "c64p") if policy == "mixed" else None
    wins, nts, exact = _batch_truth()
    X = torch.empty(B.N, 32, dtype=torch.complex128, device="cuda")
    ev, rs, res = b.cfd_solve_batched(B, X, wins, nts, 150, 32, B_low=Bl,
                                      policy=b.CFD_POLICY_MIXED if policy == "mixed" else b.CFD_POLICY_FP64)
    for r in range(len(SOLVE_LATTICES)):
        d = wins[r][3]
        conv = (ev[r] >= -d) & (ev[r] <= d) & (rs[r] <= 1e-10)
        assert res[r].n_conv == nts[r] == conv.sum(), (r, res[r].n_conv, nts[r])
        assert np.max(np.abs(np.sort(ev[r][conv]) - exact[r])) < 1e-10
    if policy == "mixed":
        assert max(x.iters_low for x in res) >= 1
    # padding rows stay zero
    for r in range(len(SOLVE_LATTICES)):
        end = B.row_off[r] + 4 * np.prod(SOLVE_LATTICES[r][:3])
        assert torch.count_nonzero(X[end:B.row_off[r + 1]]).item() == 0


def test_batched_solve_equals_single(b):
    """Realisation by realisation, the batched solve returns the eigenvalues the
    single-matrix solve finds."""
    import torch
    params = [b.topi_params(nx, ny, nz, seed=s) for (nx, ny, nz, s) in SOLVE_LATTICES[:2]]
    B = b.cfd_build_batch(params, 32, 1, "c128")
    wins, nts, exact = _batch_truth()
    X = torch.empty(B.N, 16, dtype=torch.complex128, device="cuda")
    ev, rs, res = b.cfd_solve_batched(B, X, wins[:2], nts[:2], 150, 16)
    for r, p in enumerate(params):
        H = b.cfd_build_matrix(p, 32, 1, "c128")
        Y = torch.empty(H.N, 16, dtype=torch.complex128, device="cuda")
        th, rr, _ = b.cfd_solve(H, Y, wins[r][2], wins[r][3], 150, 16, lmin=wins[r][0], lmax=wins[r][1],
                                n_t=int(nts[r]))
        c1 = np.sort(ev[r][(ev[r] >= wins[r][2]) & (ev[r] <= wins[r][3]) & (rs[r] <= 1e-10)])
        c2 = np.sort(th[(th >= wins[r][2]) & (th <= wins[r][3]) & (rr <= 1e-10)])
        assert len(c1) == len(c2) and np.max(np.abs(c1 - c2)) < 1e-10


# ------------------------------------------------------- TMA-staged kernel --

@pytest.mark.parametrize("prec,n_b,C", [("c64p", 32, 32), ("c64", 16, 8), ("c128p", 32, 16), ("c128", 64, 32),
                                        ("c64p", 64, 128)])
def test_staged_kernel_matches_unstaged(b, prec, n_b, C):
    """The staged general step reads matrix values prepared as
    2 alpha (H - beta) from shared memory and starts each row sum at -V_prev;
    the unstaged step sums H V_cur, then shifts, scales and subtracts.  Both
    compute the same recurrence, rounded differently: the filtered blocks
    agree to rounding (fp64: 1e-12 relative; fp32: the n_p * 13 * 2^-24
    bound of the complex64 filter)."""
    import torch
    dt = torch.complex128 if prec.startswith("c128") else torch.complex64
    L = (13, 11, 7)
    H = b.cfd_build_matrix(b.topi_params(*L), C, 1, prec)
    X0 = torch.from_numpy(inputs.gaussian_block(H.N, 64, seed=12)).to(dt).cuda()
    outs = []
    for staged in (-1, 1):
        Y = X0.clone()
        b.cfd_filter_ex(H, -8.6, 8.6, -0.4, 0.6, 45, Y, n_b, staged=staged)
        outs.append(Y)
    tol = 1e-12 if dt == torch.complex128 else 45 * 13 * 2.0 ** -24
    assert (torch.linalg.norm(outs[0] - outs[1]) / torch.linalg.norm(outs[0])).item() < tol


def test_staged_timeout_is_reported(b):
    """A wait that cannot succeed (test hook: barriers expect 16 bytes more than
    are copied) ends with CFD_ERR_TIMEOUT in the workspace status, no fault,
    and the context keeps working."""
    import torch
    H = b.cfd_build_matrix(b.topi_params(8, 8, 4), 32, 1, "c64p")
    X = torch.from_numpy(inputs.gaussian_block(H.N, 32, seed=3)).to(torch.complex64).cuda()
    ws = b.cfd_filter_workspace(H.N, 32, 32, 4, "c64", "c64")
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    b.cfd_filter_ex(H, -8.6, 8.6, -0.4, 0.6, 4, X, 32, staged=2, work=work)
    with pytest.raises(b.CfdError) as e:
        b.cfd_workspace_status(work)
    assert e.value.status == 5
    # the next call clears the status and works normally
    Y = torch.from_numpy(inputs.gaussian_block(H.N, 32, seed=3)).to(torch.complex64).cuda()
    b.cfd_filter_ex(H, -8.6, 8.6, -0.4, 0.6, 4, Y, 32, staged=1, work=work)
    b.cfd_workspace_status(work)
    assert torch.isfinite(torch.view_as_real(Y)).all()
