"""GPU tests of the footprint-staged general steps (cfd_filter_opts.footprint):
each SELL chunk's V_cur rows copied into shared memory by TMA before the
chunk is computed.  Every row's arithmetic is that of the gathered steps, so
the filtered block must equal the gathered steps' (footprint = -1) bit for
bit, for staged chunks, for chunks whose footprint exceeds the row cap (then
gathered from global memory inside the same launch) and for a mix of both;
the moments agree to the rounding of their cross-row sums.  Parity against
the oracle at the ragged and the full-size cases, the bounded waits' timeout
path, and graph replay."""
import numpy as np
import pytest

import oracle
from paper_1803_02156_gb300 import inputs, workloads

pytestmark = pytest.mark.gpu

MOM_TOL = {"c64p": 1e-5, "c128p": 1e-13}
FORCE = 65535      # footprint steps at any matrix size, no row cap below the stage's own


@pytest.fixture(scope="module")
def b():
    import torch
    from paper_1803_02156_gb300 import build, binding
    assert torch.cuda.is_available()
    build.build()
    binding.lib()
    return binding


def _pair(b, L, prec, n_s, n_p, win, footprint, per=(1, 1, 1), mixed=False, seed=3, graph=0):
    """The filter with the footprint steps (option `footprint`) and with the
    gathered steps, on the same seeded block."""
    import torch
    H = b.cfd_build_matrix(b.topi_params(*L, periodic=per), 32, 1, prec)
    dt = torch.complex128 if (prec == "c128p" or mixed) else torch.complex64
    arith = 1 if prec == "c128p" else 0
    X0 = torch.from_numpy(inputs.gaussian_block(H.N, n_s, seed=seed)).to(dt).cuda()
    Xf, Xg = X0.clone(), X0.clone()
    muf = b.cfd_filter_ex(H, -8.6, 8.6, win[0], win[1], n_p, Xf, 32, moments=True, arith=arith,
                          footprint=footprint, graph=graph)
    mug = b.cfd_filter_ex(H, -8.6, 8.6, win[0], win[1], n_p, Xg, 32, moments=True, arith=arith, footprint=-1)
    torch.cuda.synchronize()
    return Xf, Xg, muf, mug


def _mom_close(muf, mug, prec):
    import torch
    rel = (torch.max(torch.abs(muf - mug)) / torch.max(torch.abs(mug))).item()
    assert rel < MOM_TOL[prec], rel


@pytest.mark.parametrize("prec", ["c64p", "c128p"])
@pytest.mark.parametrize("L,per", [((8, 8, 8), (1, 1, 1)), ((3, 3, 3), (1, 1, 1)), ((13, 7, 5), (0, 1, 1)),
                                   ((16, 16, 9), (1, 0, 0)), ((5, 4, 6), (1, 1, 0))])
def test_footprint_equals_gathered(b, prec, L, per):
    """Staged footprints on lattices with ragged last chunks (3x3x3: N = 108),
    chunks spanning several x-lines and open boundaries: bit for bit."""
    import torch
    Xf, Xg, muf, mug = _pair(b, L, prec, 64, 30, (-0.6, 0.4), FORCE, per=per)
    assert torch.equal(Xf, Xg)
    _mom_close(muf, mug, prec)


@pytest.mark.parametrize("prec", ["c64p", "c128p"])
@pytest.mark.parametrize("cap", [1, 120, 150])
def test_footprint_row_cap_falls_back(b, prec, cap):
    """A row cap below every chunk's footprint (1: all chunks gathered from
    global memory inside the footprint launch), and caps that stage some
    chunks and not others (the chunks of the 16x16x9 lattice, periodic in x
    only, need 104, 136 or 168 rows): still bit for bit."""
    import torch
    Xf, Xg, muf, mug = _pair(b, (16, 16, 9), prec, 32, 20, (-0.5, 0.5), cap, per=(1, 0, 0))
    assert torch.equal(Xf, Xg)
    _mom_close(muf, mug, prec)


def test_footprint_mixed_precision_block(b):
    """The complex-float matrix on a complex-double block (narrowed per block,
    the mixed policy's filter): bit for bit."""
    import torch
    Xf, Xg, muf, mug = _pair(b, (8, 8, 8), "c64p", 64, 25, (-0.7, 0.7), FORCE, mixed=True)
    assert Xf.dtype == torch.complex128
    assert torch.equal(Xf, Xg)
    _mom_close(muf, mug, "c64p")


@pytest.mark.parametrize("prec,tol", [("c64p", 200 * 13 * 2.0 ** -24), ("c128p", 1e-11)])
def test_footprint_parity_small_config(b, prec, tol):
    """8x8x8, n_s = 64, n_b = 32, n_p = 200 (the small configuration) against
    the oracle: block and moments."""
    import torch
    w = workloads.SMALL
    H = b.cfd_build_matrix(b.topi_params(*w.lattice, seed=w.seed), 32, 1, prec)
    ref = oracle.topi_csr(*w.lattice, seed=w.seed)
    X = inputs.gaussian_block(ref.N, 64, seed=2)
    Xg = torch.from_numpy(X).cuda()
    mu = b.cfd_filter_ex(H, -8.6, 8.6, -0.7, 0.7, w.n_p, Xg, 32, moments=True,
                         arith=1 if prec == "c128p" else 0, footprint=FORCE)
    torch.cuda.synchronize()
    Y, dots = oracle.chebfd_filter(ref, -8.6, 8.6, -0.7, 0.7, w.n_p, X, 32)
    err = np.linalg.norm(Xg.cpu().numpy() - Y) / np.linalg.norm(Y)
    muref = oracle.kpm_moments(dots)
    merr = np.max(np.abs(mu.cpu().numpy() - muref)) / np.max(np.abs(muref))
    assert err < tol, err
    assert merr < tol, merr


@pytest.mark.parametrize("prec", ["c64p", "c128p"])
def test_footprint_full_size_equals_gathered(b, prec):
    """The benchmark's kernel workload, 64x64x32 (N = 524288), n_b = 32,
    12 steps: bit for bit against the gathered steps."""
    import torch
    Xf, Xg, muf, mug = _pair(b, workloads.MEDIUM.lattice, prec, 32, 12, (-0.3, 0.3), 0,
                             mixed=(prec == "c64p"))
    assert torch.equal(Xf, Xg)
    _mom_close(muf, mug, prec)


@pytest.mark.parametrize("prec", ["c64p", "c128p"])
def test_footprint_graph_replay(b, prec):
    """Captured as a CUDA graph (footprint build included) and replayed."""
    import torch
    for _ in range(2):
        Xf, Xg, muf, mug = _pair(b, (8, 8, 6), prec, 32, 15, (-0.5, 0.5), FORCE, graph=1)
        assert torch.equal(Xf, Xg)
        _mom_close(muf, mug, prec)


@pytest.mark.parametrize("prec", ["c64p", "c128p"])
def test_footprint_wait_timeout_reported(b, prec):
    """The footprint step's bounded waits made to expire (staged = 2): every
    stage expects 16 bytes more than are copied; CFD_ERR_TIMEOUT in the
    workspace status, all copies drained, the context still usable."""
    import torch
    H = b.cfd_build_matrix(b.topi_params(8, 8, 4), 32, 1, prec)
    dt = torch.complex128 if prec == "c128p" else torch.complex64
    arith = 1 if prec == "c128p" else 0
    X = torch.from_numpy(inputs.gaussian_block(H.N, 32, seed=6)).to(dt).cuda()
    pw = "c128" if prec == "c128p" else "c64"
    work = torch.empty(b.cfd_filter_workspace(H.N, 32, 32, 10, pw, pw), dtype=torch.uint8, device="cuda")
    b.cfd_filter_ex(H, -8.6, 8.6, -0.5, 0.5, 10, X, 32, arith=arith, staged=2, footprint=FORCE, work=work)
    with pytest.raises(b.CfdError) as e:
        b.cfd_workspace_status(work)
    assert e.value.status == 5
    assert "still have been in flight" not in str(e.value)
    X2 = X.clone()
    b.cfd_filter_ex(H, -8.6, 8.6, -0.5, 0.5, 10, X2, 32, arith=arith, work=work)
    b.cfd_workspace_status(work)


def test_footprint_option_rejected(b):
    import torch
    H = b.cfd_build_matrix(b.topi_params(4, 4, 4), 32, 1, "c64p")
    X = torch.zeros(H.N, 32, dtype=torch.complex64, device="cuda")
    with pytest.raises(b.CfdError) as e:
        b.cfd_filter_ex(H, -8.6, 8.6, -0.5, 0.5, 10, X, 32, footprint=-2)
    assert e.value.status == 1


@pytest.mark.parametrize("prec", ["c64p", "c128p"])
def test_footprint_batched_equals_per_realisation(b, prec):
    """The batched filter (block-diagonal matrix of five uneven lattices,
    about 3100 chunks, enough for the default to take the footprint steps;
    each chunk's weight taken from its realisation): per realisation bit for
    bit cfd_filter on that lattice alone with the gathered steps."""
    import torch
    lattices = [(24, 20, 12, 11), (20, 22, 10, 12), (18, 16, 14, 13), (26, 18, 11, 14), (22, 22, 12, 15)]
    arith = 1 if prec == "c128p" else 0
    dt = torch.complex128 if prec == "c128p" else torch.complex64
    B = b.cfd_build_batch([b.topi_params(nx, ny, nz, seed=s) for (nx, ny, nz, s) in lattices], 32, 1, prec)
    w = [[-8.6 - 0.1 * r, 8.6 + 0.05 * r, -0.9 + 0.1 * r, 0.4 + 0.2 * r] for r in range(len(lattices))]
    wt = torch.tensor(w, dtype=torch.float64, device="cuda")
    n_s, n_p = 32, 40
    X = torch.zeros(B.N, n_s, dtype=dt, device="cuda")
    blocks = []
    for r, (nx, ny, nz, s) in enumerate(lattices):
        N = 4 * nx * ny * nz
        Xr = torch.from_numpy(inputs.gaussian_block(N, n_s, seed=300 + r)).to(dt).cuda()
        X[B.row_off[r]:B.row_off[r] + N] = Xr
        blocks.append(Xr)
    b.cfd_filter_batched(B, wt, n_p, X, 32, arith=arith)
    for r, (nx, ny, nz, s) in enumerate(lattices):
        N = 4 * nx * ny * nz
        H = b.cfd_build_matrix(b.topi_params(nx, ny, nz, seed=s), 32, 1, prec)
        Y = blocks[r].clone()
        b.cfd_filter_ex(H, w[r][0], w[r][1], w[r][2], w[r][3], n_p, Y, 32, arith=arith, footprint=-1)
        assert torch.equal(X[B.row_off[r]:B.row_off[r] + N], Y), r
