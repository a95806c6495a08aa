"""CPU checks of the C ABI: the library loads, exports every function the
header declares, and rejects bad arguments before touching the GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    txt = open(os.path.join(ROOT, "include", "cfd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cfd_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def L():
    from paper_1803_02156_gb300 import build, binding
    build.build()
    return binding.lib()


def test_library_exports_every_declared_symbol(L):
    from paper_1803_02156_gb300 import binding
    declared = _header_functions()
    assert len(declared) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (cfd_\w+)", out))
    missing = [f for f in declared if f not in exported]
    assert not missing, missing
    # the binding covers the whole header
    assert set(binding.declared_symbols()) == set(declared)


def test_status_strings(L):
    assert L.cfd_status_string(0) == b"CFD_OK"
    assert L.cfd_status_string(3) == b"CFD_ERR_OOM"


def test_query_size_matches_formula(L):
    from paper_1803_02156_gb300 import binding as b, workloads
    for w in (workloads.SMALL, workloads.MEDIUM, workloads.LARGE):
        s = b.cfd_matrix_query_size(b.topi_params(*w.lattice), 32, 1, "c128")
        assert s.n_rows == w.N and s.nnz == w.nnz and s.n_slots >= s.nnz
    with pytest.raises(b.CfdError) as e:
        b.cfd_matrix_query_size(b.topi_params(2, 8, 8), 32, 1, "c128")     # periodic axis of 2
    assert e.value.status == 1
    with pytest.raises(b.CfdError):
        b.cfd_matrix_query_size(b.topi_params(8, 8, 8), 24, 1, "c128")     # C not a power of 2


def test_filter_argument_validation_on_host(L):
    """Validation happens before any GPU work, so fake (aligned) pointers suffice."""
    from paper_1803_02156_gb300 import binding as b
    m = b.cfd_matrix(n_rows=2048, nnz=25600, n_chunks=64, n_slots=25600, C=32, sigma=1, prec=0,
                     val=4096, col=4096, chunk_ptr=4096, chunk_len=4096, perm=None)
    X = b.cfd_block(ptr=1 << 20, n_rows=2048, ld=32, n_cols=32, prec=0)

    def call(**kw):
        args = dict(lmin=-9.0, lmax=9.0, ll=-0.5, lr=0.5, n_p=20, X=X, n_b=32, work=1 << 24, wb=1 << 40)
        args.update(kw)
        return L.cfd_filter(ctypes.byref(m), args["lmin"], args["lmax"], args["ll"], args["lr"], args["n_p"],
                            args["X"], args["n_b"], ctypes.c_void_p(args["work"]), args["wb"], None, None)

    assert call(n_b=24) == 1
    assert call(n_b=64) == 1                                    # does not divide n_s = 32
    assert call(ll=-10.0) == 1                                  # window outside bounds
    assert call(ll=0.6) == 1                                    # empty window
    assert call(n_p=1) == 1
    assert call(wb=1000) == 3                                   # workspace too small
    Xbad = b.cfd_block(ptr=(1 << 20) + 8, n_rows=2048, ld=32, n_cols=32, prec=0)
    assert call(X=Xbad) == 1                                    # misaligned
    Xrows = b.cfd_block(ptr=1 << 20, n_rows=2000, ld=32, n_cols=32, prec=0)
    assert call(X=Xrows) == 1
    X64 = b.cfd_block(ptr=1 << 20, n_rows=2048, ld=32, n_cols=32, prec=1)
    assert call(X=X64) == 1                                     # c128 matrix with c64 block
    assert b"n_b" in L.cfd_last_error() or len(L.cfd_last_error()) > 0


def _fake_matrix(b, n_rows=2048, nnz=25600, C=32):
    return b.cfd_matrix(n_rows=n_rows, nnz=nnz, n_chunks=(n_rows + C - 1) // C, n_slots=nnz, C=C, sigma=1, prec=0,
                        val=4096, col=4096, chunk_ptr=4096, chunk_len=4096, perm=None)


def test_filter_options_validated_on_host(L):
    """Kernel options out of range are rejected before any GPU work."""
    from paper_1803_02156_gb300 import binding as b
    m = _fake_matrix(b)
    X = b.cfd_block(ptr=1 << 20, n_rows=2048, ld=32, n_cols=32, prec=0)

    def call(**kw):
        o = b.cfd_filter_opts(**kw)
        return L.cfd_filter_ex(ctypes.byref(m), -9.0, 9.0, -0.5, 0.5, 20, X, 32, ctypes.c_void_p(1 << 24), 1 << 40,
                               None, ctypes.byref(o), None)

    assert call(gather=5) == 1
    assert call(gather=12) == 1
    assert call(staged=3) == 1
    assert call(grid_cap=-1) == 1


def test_filter_workspace_holds_prepared_values(L):
    """The filter workspace holds the two N x n_b recurrence blocks and the
    matrix values prepared as 2 alpha (H - beta), 13 per row (the matrices
    this library builds), and grows with N, n_b and n_p."""
    from paper_1803_02156_gb300 import binding as b
    for prec, s in ((0, 16), (1, 8)):
        for N, n_b in ((2048, 32), (524288, 32), (16000000, 64)):
            ws = L.cfd_filter_workspace(N, 4 * n_b, n_b, 100, prec, prec)
            assert ws >= 2 * N * n_b * s + 13 * N * s
            assert L.cfd_filter_workspace(N + 4096, 4 * n_b, n_b, 100, prec, prec) > ws
            assert L.cfd_filter_workspace(N, 4 * n_b, n_b, 1000, prec, prec) > ws
    # mixed precision (complex-float matrix, complex-double block) also holds the narrowed block
    assert L.cfd_filter_workspace(2048, 64, 32, 100, 1, 0) > L.cfd_filter_workspace(2048, 64, 32, 100, 1, 1)


def test_noalloc_rejects_oversize_on_host(L):
    """A problem whose workspace exceeds the static scratch is rejected with
    CFD_ERR_ARG before the library touches a GPU."""
    from paper_1803_02156_gb300 import binding as b
    N = 4 * 64 * 64 * 32
    m = _fake_matrix(b, n_rows=N, nnz=13 * N)
    X = b.cfd_block(ptr=1 << 20, n_rows=N, ld=32, n_cols=32, prec=0)
    st = L.cfd_filter_noalloc(ctypes.byref(m), -9.0, 9.0, -0.5, 0.5, 20, X, 32, None, None)
    assert st == 1
    assert b"static scratch" in L.cfd_last_error()


def test_sell_layout_has_no_padding_on_the_benchmark_lattices(L):
    """SELL-C-sigma with C = 32: chunks of 8 sites never straddle a z-plane
    when Nx Ny is a multiple of 8, so every slot holds a nonzero (packed or
    complex values); uneven lattices pad only the chunks that straddle."""
    from paper_1803_02156_gb300 import binding as b, workloads
    for w in (workloads.SMALL, workloads.MEDIUM, workloads.LARGE, workloads.MIXED):
        for prec in ("c128", "c128p", "c64p"):
            s = b.cfd_matrix_query_size(b.topi_params(*w.lattice), 32, 1, prec)
            assert s.n_slots == s.nnz == w.nnz
    s = b.cfd_matrix_query_size(b.topi_params(37, 26, 17), 32, 1, "c64p")
    assert s.nnz < s.n_slots < 1.001 * s.nnz
