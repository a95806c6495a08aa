"""Thin ctypes binding of libcfd.so (include/cfd.h).

Argument marshalling only: torch supplies device memory and the current CUDA
stream, every computation runs in the library's kernels.  Function names
match the C ABI.  There is no fallback: if the library is missing or no GPU
is present the calls raise.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcfd.so")

CFD_C128, CFD_C64 = 0, 1
CFD_PACK_RI = 0x100
# "p": values packed as real-or-imaginary scalars (CFD_PACK_RI)
PREC = {"c128": CFD_C128, "c64": CFD_C64, "c128p": CFD_C128 | CFD_PACK_RI, "c64p": CFD_C64 | CFD_PACK_RI}
TORCH_DTYPE = {CFD_C128: torch.complex128, CFD_C64: torch.complex64}
SCALAR_BYTES = {CFD_C128: 16, CFD_C64: 8}

STATUS = {0: "CFD_OK", 1: "CFD_ERR_ARG", 2: "CFD_ERR_CUDA", 3: "CFD_ERR_OOM", 4: "CFD_ERR_BOUNDS",
          5: "CFD_ERR_TIMEOUT", 6: "CFD_ERR_NOCONV", 7: "CFD_ERR_INTERNAL"}


class CfdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


# ------------------------------------------------------------ structs --

class cfd_topi_params(ctypes.Structure):
    _fields_ = [("Nx", ctypes.c_int32), ("Ny", ctypes.c_int32), ("Nz", ctypes.c_int32),
                ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
                ("periodic_z", ctypes.c_int32), ("t", ctypes.c_double), ("m", ctypes.c_double),
                ("gamma", ctypes.c_double), ("seed", ctypes.c_uint64)]


class cfd_matrix_sizes(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "n_rows", "nnz", "n_chunks", "n_slots", "bytes_val", "bytes_col", "bytes_chunk_ptr",
        "bytes_chunk_len", "bytes_perm", "bytes_work")]


class cfd_matrix_buffers(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("val", "col", "chunk_ptr", "chunk_len", "perm", "work")]


class cfd_matrix(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("nnz", ctypes.c_int64), ("n_chunks", ctypes.c_int64),
                ("n_slots", ctypes.c_int64), ("C", ctypes.c_int32), ("sigma", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("flags", ctypes.c_int32), ("val", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("chunk_ptr", ctypes.c_void_p),
                ("chunk_len", ctypes.c_void_p), ("perm", ctypes.c_void_p)]


class cfd_block(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p), ("n_rows", ctypes.c_int64), ("ld", ctypes.c_int64),
                ("n_cols", ctypes.c_int32), ("prec", ctypes.c_int32)]


class cfd_filter_opts(ctypes.Structure):
    _fields_ = [("vpt", ctypes.c_int32), ("grid_cap", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("staged", ctypes.c_int32), ("gather", ctypes.c_int32),
                ("fixed_chunk", ctypes.c_int32), ("arith", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("footprint", ctypes.c_int32)]


class cfd_solve_params(ctypes.Structure):
    _fields_ = [("lam_l", ctypes.c_double), ("lam_r", ctypes.c_double), ("lmin", ctypes.c_double),
                ("lmax", ctypes.c_double), ("tol", ctypes.c_double), ("switch_tol", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("n_s", ctypes.c_int32), ("n_p", ctypes.c_int32),
                ("n_b", ctypes.c_int32), ("n_t", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("policy", ctypes.c_int32), ("bounds_steps", ctypes.c_int32), ("start", ctypes.c_int32)]


class cfd_solve_result(ctypes.Structure):
    _fields_ = [("n_conv", ctypes.c_int32), ("iters", ctypes.c_int32), ("iters_low", ctypes.c_int32),
                ("rank_min", ctypes.c_int32), ("lmin", ctypes.c_double), ("lmax", ctypes.c_double),
                ("t_filter", ctypes.c_double), ("t_orth", ctypes.c_double), ("t_rr", ctypes.c_double),
                ("t_total", ctypes.c_double)]


class cfd_slab(ctypes.Structure):
    _fields_ = [("nranks", ctypes.c_int32), ("rank", ctypes.c_int32), ("z0", ctypes.c_int32), ("z1", ctypes.c_int32),
                ("row0", ctypes.c_int64), ("n_local", ctypes.c_int64), ("plane", ctypes.c_int64),
                ("lo_rank", ctypes.c_int32), ("hi_rank", ctypes.c_int32), ("lo_base", ctypes.c_int64),
                ("hi_base", ctypes.c_int64)]


CFD_POLICY_FP64, CFD_POLICY_MIXED, CFD_POLICY_FP64_DW, CFD_POLICY_MIXED_DW = 0, 1, 2, 3
CFD_DIST_VECTOR, CFD_DIST_PIPELINED = 0, 1

# ---------------------------------------------------------------- load --

_LIB = None

_PROTOS = {
    "cfd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "cfd_last_error": (ctypes.c_char_p, []),
    "cfd_version": (ctypes.c_char_p, []),
    "cfd_launch_count": (ctypes.c_ulonglong, []),
    "cfd_matrix_query_size": (ctypes.c_int, [ctypes.POINTER(cfd_topi_params), ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.POINTER(cfd_matrix_sizes)]),
    "cfd_build_matrix": (ctypes.c_int, [ctypes.POINTER(cfd_topi_params), ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.POINTER(cfd_matrix_buffers),
                                        ctypes.POINTER(cfd_matrix), ctypes.c_void_p]),
    "cfd_export_csr_workspace": (ctypes.c_size_t, [ctypes.POINTER(cfd_matrix)]),
    "cfd_matrix_export_csr": (ctypes.c_int, [ctypes.POINTER(cfd_matrix), ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                             ctypes.c_void_p]),
    "cfd_filter_coeffs": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "cfd_filter_workspace": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_int]),
    "cfd_filter": (ctypes.c_int, [ctypes.POINTER(cfd_matrix), ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_int, cfd_block, ctypes.c_int,
                                  ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p]),
    "cfd_filter_ex": (ctypes.c_int, [ctypes.POINTER(cfd_matrix), ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int, cfd_block, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                     ctypes.POINTER(cfd_filter_opts), ctypes.c_void_p]),
    "cfd_filter_unfused_workspace": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                       ctypes.c_int, ctypes.c_int]),
    "cfd_filter_unfused": (ctypes.c_int, [ctypes.POINTER(cfd_matrix), ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int, cfd_block, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p]),
    "cfd_filter_host_workspace": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                    ctypes.c_int, ctypes.c_int]),
    "cfd_filter_host": (ctypes.c_int, [ctypes.POINTER(cfd_matrix), ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int, cfd_block, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p]),
    "cfd_filter_host_ex": (ctypes.c_int, [ctypes.POINTER(cfd_matrix), ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int, cfd_block, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                          ctypes.POINTER(cfd_filter_opts), ctypes.c_void_p]),
    "cfd_filter_host_blocked": (ctypes.c_int, [ctypes.POINTER(cfd_matrix), ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_int, cfd_block,
                                               ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                               ctypes.POINTER(cfd_filter_opts), ctypes.c_void_p]),
    "cfd_workspace_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "cfd_kpm_moments": (ctypes.c_int, [ctypes.POINTER(cfd_matrix), ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       cfd_block, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "cfd_kpm_count": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_double)]),
    "cfd_kpm_window": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "cfd_batch_query_size": (ctypes.c_int, [ctypes.POINTER(cfd_topi_params), ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, ctypes.POINTER(cfd_matrix_sizes),
                                            ctypes.c_void_p]),
    "cfd_build_batch": (ctypes.c_int, [ctypes.POINTER(cfd_topi_params), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.POINTER(cfd_matrix_buffers), ctypes.c_void_p,
                                       ctypes.POINTER(cfd_matrix), ctypes.c_void_p]),
    "cfd_filter_batched_workspace": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                       ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "cfd_filter_batched": (ctypes.c_int, [ctypes.POINTER(cfd_matrix), ctypes.c_void_p, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_int, cfd_block, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_size_t, ctypes.POINTER(cfd_filter_opts), ctypes.c_void_p]),
    "cfd_spectral_bounds_workspace": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int]),
    "cfd_spectral_bounds": (ctypes.c_int, [ctypes.POINTER(cfd_matrix), ctypes.c_int, ctypes.c_uint64,
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                           ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "cfd_gram_workspace": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int, ctypes.c_int]),
    "cfd_block_gram": (ctypes.c_int, [cfd_block, cfd_block, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_size_t, ctypes.c_void_p]),
    "cfd_block_gram_ex": (ctypes.c_int, [cfd_block, cfd_block, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p]),
    "cfd_eigh_workspace": (ctypes.c_size_t, [ctypes.c_int]),
    "cfd_eigh": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "cfd_orthogonalize_workspace": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int]),
    "cfd_orthogonalize": (ctypes.c_int, [cfd_block, ctypes.c_double, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p,
                                         ctypes.c_size_t, ctypes.c_void_p]),
    "cfd_orthogonalize_ex": (ctypes.c_int, [cfd_block, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                            ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p]),
    "cfd_rayleigh_ritz_workspace": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int]),
    "cfd_rayleigh_ritz": (ctypes.c_int, [ctypes.POINTER(cfd_matrix), cfd_block, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "cfd_solve_workspace": (ctypes.c_size_t, [ctypes.POINTER(cfd_matrix), ctypes.POINTER(cfd_matrix),
                                              ctypes.POINTER(cfd_solve_params)]),
    "cfd_solve": (ctypes.c_int, [ctypes.POINTER(cfd_matrix), ctypes.POINTER(cfd_matrix),
                                 ctypes.POINTER(cfd_solve_params), cfd_block, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(cfd_solve_result),
                                 ctypes.c_void_p]),
    "cfd_solve_batched_workspace": (ctypes.c_size_t, [ctypes.POINTER(cfd_matrix), ctypes.c_int,
                                                      ctypes.POINTER(cfd_solve_params)]),
    "cfd_solve_batched": (ctypes.c_int, [ctypes.POINTER(cfd_matrix), ctypes.POINTER(cfd_matrix), ctypes.c_void_p,
                                         ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.POINTER(cfd_solve_params), cfd_block,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(cfd_solve_result),
                                         ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "cfd_filter_noalloc": (ctypes.c_int, [ctypes.POINTER(cfd_matrix), ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int, cfd_block,
                                          ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "cfd_filter_noalloc_status": (ctypes.c_int, [ctypes.c_void_p]),
    "cfd_slab_plan": (ctypes.c_int, [ctypes.POINTER(cfd_topi_params), ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(cfd_slab)]),
    "cfd_slab_local_col": (ctypes.c_int64, [ctypes.POINTER(cfd_slab), ctypes.c_int64]),
    "cfd_slab_query_size": (ctypes.c_int, [ctypes.POINTER(cfd_topi_params), ctypes.POINTER(cfd_slab), ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, ctypes.POINTER(cfd_matrix_sizes)]),
    "cfd_build_matrix_slab": (ctypes.c_int, [ctypes.POINTER(cfd_topi_params), ctypes.POINTER(cfd_slab), ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, ctypes.POINTER(cfd_matrix_buffers),
                                             ctypes.POINTER(cfd_matrix), ctypes.c_void_p]),
    "cfd_filter_slab_workspace": (ctypes.c_size_t, [ctypes.POINTER(cfd_slab), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                    ctypes.c_int, ctypes.c_int]),
    "cfd_filter_slabs": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(cfd_slab), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, ctypes.POINTER(cfd_block), ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t, ctypes.c_void_p,
                                        ctypes.POINTER(cfd_filter_opts), ctypes.c_void_p]),
    "cfd_nccl_unique_id": (ctypes.c_int, [ctypes.c_void_p]),
    "cfd_nccl_comm_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "cfd_nccl_comm_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "cfd_filter_slab_nccl": (ctypes.c_int, [ctypes.POINTER(cfd_slab), ctypes.POINTER(cfd_matrix), ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                            cfd_block, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_size_t, ctypes.c_void_p, ctypes.POINTER(cfd_filter_opts),
                                            ctypes.c_void_p, ctypes.c_void_p]),
    "cfd_probe_fma_workspace": (ctypes.c_size_t, []),
    "cfd_probe_fma": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p,
                                     ctypes.c_size_t, ctypes.c_void_p]),
}


def lib():
    """Load libcfd.so (built in-tree by __graft_entry__.build())."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libcfd.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def declared_symbols():
    """Names of the entry points this binding expects the library to export."""
    return sorted(_PROTOS)


def _check(st):
    if st != 0:
        raise CfdError(st, lib().cfd_last_error().decode())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _workspace(nbytes, device):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _prec(p):
    return PREC[p] if isinstance(p, str) else int(p)


def cfd_version():
    return lib().cfd_version().decode()


def cfd_launch_count():
    """Kernels launched by the library so far in this process."""
    return int(lib().cfd_launch_count())


# -------------------------------------------------------------- matrix --

def topi_params(Nx, Ny, Nz, t=1.0, m=2.0, gamma=1.0, seed=1, periodic=(1, 1, 0)):
    return cfd_topi_params(Nx, Ny, Nz, int(periodic[0]), int(periodic[1]), int(periodic[2]),
                           float(t), float(m), float(gamma), int(seed))


def cfd_matrix_query_size(params, C=32, sigma=1, prec="c128"):
    sz = cfd_matrix_sizes()
    _check(lib().cfd_matrix_query_size(ctypes.byref(params), C, sigma, _prec(prec), ctypes.byref(sz)))
    return sz


class Matrix:
    """A built SELL-C-sigma matrix: the C struct plus the torch buffers it points into."""

    def __init__(self, cmat, buffers, params):
        self.c = cmat
        self.buffers = buffers
        self.params = params

    @property
    def N(self):
        return self.c.n_rows

    @property
    def nnz(self):
        return self.c.nnz

    @property
    def prec(self):
        return self.c.prec

    @property
    def packed(self):
        return bool(self.c.flags & 1)

    def ref(self):
        return ctypes.byref(self.c)


def cfd_build_matrix(params, C=32, sigma=1, prec="c128", device="cuda", stream=None):
    """Allocate the SELL-C-sigma buffers with torch and build Topi into them."""
    prec = _prec(prec)
    sz = cfd_matrix_query_size(params, C, sigma, prec)
    dev = torch.device(device)
    bufs = {
        "val": _workspace(sz.bytes_val, dev), "col": _workspace(sz.bytes_col, dev),
        "chunk_ptr": _workspace(sz.bytes_chunk_ptr, dev), "chunk_len": _workspace(sz.bytes_chunk_len, dev),
        "perm": _workspace(sz.bytes_perm, dev) if sz.bytes_perm else None,
        "work": _workspace(sz.bytes_work, dev),
    }
    b = cfd_matrix_buffers(*[(bufs[k].data_ptr() if bufs[k] is not None else None)
                             for k in ("val", "col", "chunk_ptr", "chunk_len", "perm", "work")])
    out = cfd_matrix()
    _check(lib().cfd_build_matrix(ctypes.byref(params), C, sigma, prec, ctypes.byref(b), ctypes.byref(out),
                                  _stream(stream)))
    return Matrix(out, bufs, params)


def cfd_matrix_export_csr(H, stream=None):
    """Canonical CSR of H as torch device tensors (rowptr int64, col int32, val complex)."""
    dev = H.buffers["val"].device
    rowptr = torch.empty(H.N + 1, dtype=torch.int64, device=dev)
    col = torch.empty(H.nnz, dtype=torch.int32, device=dev)
    val = torch.empty(H.nnz, dtype=TORCH_DTYPE[H.prec], device=dev)
    ws = lib().cfd_export_csr_workspace(H.ref())
    work = _workspace(ws, dev)
    _check(lib().cfd_matrix_export_csr(H.ref(), _ptr(rowptr), _ptr(col), _ptr(val), _ptr(work), ws,
                                       _stream(stream)))
    return rowptr, col, val


# -------------------------------------------------------------- filter --

def cfd_filter_coeffs(lmin, lmax, lam_l, lam_r, n_p, device="cuda", stream=None):
    gc = torch.empty(n_p + 1, dtype=torch.float64, device=device)
    _check(lib().cfd_filter_coeffs(lmin, lmax, lam_l, lam_r, n_p, _ptr(gc), _stream(stream)))
    return gc


def block_of(X):
    """cfd_block describing a 2-D torch complex tensor with unit column stride."""
    if X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("block must be a 2-D tensor with unit column stride")
    prec = {torch.complex128: CFD_C128, torch.complex64: CFD_C64}[X.dtype]
    return cfd_block(X.data_ptr(), X.shape[0], X.stride(0), X.shape[1], prec)


def cfd_filter_workspace(N, n_s, n_b, n_p, prec_H, prec_X):
    return lib().cfd_filter_workspace(N, n_s, n_b, n_p, _prec(prec_H), _prec(prec_X))


def cfd_filter(H, lmin, lmax, lam_l, lam_r, n_p, X, n_b, moments=False, work=None, stream=None):
    """Filter the columns of X (N x n_s complex, row-major) in place.  Returns the
    [n_s, 2 n_p] Chebyshev moments (float64 device tensor) when moments=True."""
    blk = block_of(X)
    ws = cfd_filter_workspace(H.N, blk.n_cols, n_b, n_p, H.prec, blk.prec)
    if work is None or work.numel() < ws:
        work = _workspace(ws, X.device)
    mu = torch.empty(blk.n_cols, 2 * n_p, dtype=torch.float64, device=X.device) if moments else None
    _check(lib().cfd_filter(H.ref(), lmin, lmax, lam_l, lam_r, n_p, blk, n_b, _ptr(work), work.numel(),
                            _ptr(mu), _stream(stream)))
    return mu


def cfd_filter_ex(H, lmin, lmax, lam_l, lam_r, n_p, X, n_b, vpt=0, grid_cap=0, moments=False, work=None,
                  stream=None, persistent=0, staged=0, gather=0, fixed_chunk=0, arith=0, graph=0, footprint=0):
    """cfd_filter with the kernel options (vectors per thread, CTA cap, persistent
    launch, TMA staging: 1 on, -1 off, 0 default; gathers in flight per row in
    staged steps: 16 all at once, 4 groups of four, 0 default; fixed_chunk -1:
    generic staged kernel instead of the one compiled for C = 32; arith 1:
    complex-double general steps in double-word arithmetic on the fp32 pipe;
    graph 1: the call captured once as a CUDA graph and replayed; footprint
    0: general steps stage each chunk's V_cur rows by TMA where they apply,
    -1 never, n > 0 at most n rows per chunk)."""
    blk = block_of(X)
    ws = cfd_filter_workspace(H.N, blk.n_cols, n_b, n_p, H.prec, blk.prec)
    if work is None or work.numel() < ws:
        work = _workspace(ws, X.device)
    mu = torch.empty(blk.n_cols, 2 * n_p, dtype=torch.float64, device=X.device) if moments else None
    o = cfd_filter_opts(vpt, grid_cap, persistent, staged, gather, fixed_chunk, arith, graph, footprint)
    _check(lib().cfd_filter_ex(H.ref(), lmin, lmax, lam_l, lam_r, n_p, blk, n_b, _ptr(work), work.numel(),
                               _ptr(mu), ctypes.byref(o), _stream(stream)))
    return mu


def cfd_filter_unfused_workspace(N, n_s, n_b, n_p, prec_H, prec_X):
    return lib().cfd_filter_unfused_workspace(N, n_s, n_b, n_p, _prec(prec_H), _prec(prec_X))


def cfd_filter_unfused(H, lmin, lmax, lam_l, lam_r, n_p, X, n_b, moments=False, work=None, stream=None):
    """The filter as a chain of separate SpMMV and BLAS-1 kernels (fusion
    baseline); same arguments and result as cfd_filter."""
    blk = block_of(X)
    ws = cfd_filter_unfused_workspace(H.N, blk.n_cols, n_b, n_p, H.prec, blk.prec)
    if work is None or work.numel() < ws:
        work = _workspace(ws, X.device)
    mu = torch.empty(blk.n_cols, 2 * n_p, dtype=torch.float64, device=X.device) if moments else None
    _check(lib().cfd_filter_unfused(H.ref(), lmin, lmax, lam_l, lam_r, n_p, blk, n_b, _ptr(work), work.numel(),
                                    _ptr(mu), _stream(stream)))
    return mu


def cfd_filter_host_workspace(N, n_s, n_b, n_p, prec_H, prec_X):
    return lib().cfd_filter_host_workspace(N, n_s, n_b, n_p, _prec(prec_H), _prec(prec_X))


def cfd_filter_host(H, lmin, lmax, lam_l, lam_r, n_p, X, n_b, moments=False, work=None, stream=None,
                    device="cuda", arith=0):
    """cfd_filter for X in host memory (a CPU tensor, pinned for overlap); X is
    filtered in place once the stream is synchronised (this call synchronises
    it).  Returns the device moments when moments=True.  arith 1: double-word
    complex-double steps (cfd_filter_host_ex)."""
    if X.is_cuda:
        raise ValueError("cfd_filter_host takes a host (CPU) tensor")
    blk = block_of(X)
    ws = cfd_filter_host_workspace(H.N, blk.n_cols, n_b, n_p, H.prec, blk.prec)
    if work is None or work.numel() < ws:
        work = _workspace(ws, device)
    mu = torch.empty(blk.n_cols, 2 * n_p, dtype=torch.float64, device=device) if moments else None
    o = cfd_filter_opts(0, 0, 0, 0, 0, 0, arith, 0)
    _check(lib().cfd_filter_host_ex(H.ref(), lmin, lmax, lam_l, lam_r, n_p, blk, n_b, _ptr(work), work.numel(),
                                    _ptr(mu), ctypes.byref(o), _stream(stream)))
    (stream or torch.cuda.current_stream()).synchronize()
    return mu


def cfd_filter_host_blocked(H, lmin, lmax, lam_l, lam_r, n_p, Xb, n_b, moments=False, work=None, stream=None,
                            device="cuda", arith=0):
    """The host-memory filter for a search space stored block after block: Xb
    is a CPU tensor [n_s / n_b, N, n_b] (block b of n_b columns contiguous,
    pinned for overlap), filtered in place (this call synchronises the
    stream).  Returns the device moments when moments=True."""
    if Xb.is_cuda or Xb.dim() != 3 or Xb.shape[2] != n_b or not Xb.is_contiguous():
        raise ValueError("Xb must be a contiguous CPU tensor [n_s / n_b, N, n_b]")
    prec = {torch.complex128: CFD_C128, torch.complex64: CFD_C64}[Xb.dtype]
    nblk, N = Xb.shape[0], Xb.shape[1]
    blk = cfd_block(Xb.data_ptr(), N, n_b, nblk * n_b, prec)
    ws = cfd_filter_host_workspace(H.N, blk.n_cols, n_b, n_p, H.prec, blk.prec)
    if work is None or work.numel() < ws:
        work = _workspace(ws, device)
    mu = torch.empty(blk.n_cols, 2 * n_p, dtype=torch.float64, device=device) if moments else None
    o = cfd_filter_opts(0, 0, 0, 0, 0, 0, arith, 0)
    _check(lib().cfd_filter_host_blocked(H.ref(), lmin, lmax, lam_l, lam_r, n_p, blk, n_b, _ptr(work), work.numel(),
                                         _ptr(mu), ctypes.byref(o), _stream(stream)))
    (stream or torch.cuda.current_stream()).synchronize()
    return mu


def cfd_workspace_status(work, stream=None):
    """Device status of a filter workspace: raises CfdError on a recorded timeout
    (CFD_ERR_TIMEOUT) or a moment that exceeded mu_0 (CFD_ERR_BOUNDS)."""
    _check(lib().cfd_workspace_status(_ptr(work), _stream(stream)))


def cfd_kpm_moments(H, lmin, lmax, n_p, R, n_b, work=None, stream=None):
    """[n_s, 2 n_p] Chebyshev moments of the columns of R (not modified)."""
    blk = block_of(R)
    ws = cfd_filter_workspace(H.N, blk.n_cols, n_b, n_p, H.prec, blk.prec)
    if work is None or work.numel() < ws:
        work = _workspace(ws, R.device)
    mu = torch.empty(blk.n_cols, 2 * n_p, dtype=torch.float64, device=R.device)
    _check(lib().cfd_kpm_moments(H.ref(), lmin, lmax, n_p, blk, n_b, _ptr(work), work.numel(), _ptr(mu),
                                 _stream(stream)))
    return mu


def cfd_kpm_count(mu, N, lmin, lmax, lam_l, lam_r):
    """Estimated eigenvalue count in [lam_l, lam_r] from host moments mu [n_vec, n_mom]."""
    import numpy as np
    m = np.ascontiguousarray(mu, dtype=np.float64)
    out = ctypes.c_double()
    _check(lib().cfd_kpm_count(m.ctypes.data_as(ctypes.c_void_p), m.shape[0], m.shape[1], N, lmin, lmax, lam_l,
                               lam_r, ctypes.byref(out)))
    return out.value


def cfd_kpm_window(mu, N, lmin, lmax, center, target):
    """(lam_l, lam_r) centred at `center` whose KPM count is `target`."""
    import numpy as np
    m = np.ascontiguousarray(mu, dtype=np.float64)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(lib().cfd_kpm_window(m.ctypes.data_as(ctypes.c_void_p), m.shape[0], m.shape[1], N, lmin, lmax, center,
                                target, ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


class Batch(Matrix):
    """A built batch: the block-diagonal matrix, its chunk -> realisation map and row offsets."""

    def __init__(self, cmat, buffers, params, chunk_rid, row_off):
        super().__init__(cmat, buffers, params)
        self.chunk_rid = chunk_rid
        self.row_off = row_off
        self.R = len(row_off) - 1


def cfd_build_batch(params_list, C=32, sigma=1, prec="c128", device="cuda", stream=None):
    """Build R realisations (list of cfd_topi_params) as one block-diagonal matrix."""
    import numpy as np
    prec = _prec(prec)
    R = len(params_list)
    P = (cfd_topi_params * R)(*params_list)
    sz = cfd_matrix_sizes()
    off = np.zeros(R + 1, dtype=np.int64)
    _check(lib().cfd_batch_query_size(P, R, C, sigma, prec, ctypes.byref(sz), off.ctypes.data_as(ctypes.c_void_p)))
    dev = torch.device(device)
    bufs = {
        "val": _workspace(sz.bytes_val, dev), "col": _workspace(sz.bytes_col, dev),
        "chunk_ptr": _workspace(sz.bytes_chunk_ptr, dev), "chunk_len": _workspace(sz.bytes_chunk_len, dev),
        "perm": _workspace(sz.bytes_perm, dev) if sz.bytes_perm else None,
        "work": _workspace(sz.bytes_work, dev),
    }
    rid = torch.empty(sz.n_chunks, dtype=torch.int32, device=dev)
    b = cfd_matrix_buffers(*[(bufs[k].data_ptr() if bufs[k] is not None else None)
                             for k in ("val", "col", "chunk_ptr", "chunk_len", "perm", "work")])
    out = cfd_matrix()
    _check(lib().cfd_build_batch(P, R, C, sigma, prec, ctypes.byref(b), _ptr(rid), ctypes.byref(out),
                                 _stream(stream)))
    return Batch(out, bufs, list(params_list), rid, off)


def cfd_filter_batched(B, windows, n_p, X, n_b, persistent=0, vpt=0, work=None, stream=None, graph=0, arith=0):
    """Filter every realisation of batch B at once; windows: float64 device tensor [R, 4]
    (lmin, lmax, lam_l, lam_r per realisation); graph 1: captured once as a CUDA
    graph and replayed; arith 1: double-word general steps (complex double)."""
    blk = block_of(X)
    ws = lib().cfd_filter_batched_workspace(B.N, B.R, blk.n_cols, n_b, n_p, B.prec, blk.prec)
    if work is None or work.numel() < ws:
        work = _workspace(ws, X.device)
    o = cfd_filter_opts(vpt, 0, persistent, 0, 0, 0, arith, graph)
    _check(lib().cfd_filter_batched(B.ref(), _ptr(B.chunk_rid), B.R, _ptr(windows), n_p, blk, n_b, _ptr(work),
                                    work.numel(), ctypes.byref(o), _stream(stream)))


# ------------------------------------------------------- bounds, dense --

def cfd_spectral_bounds(H, steps=40, seed=3, stream=None):
    """(lmin, lmax) enclosing the spectrum of the complex-double matrix H."""
    ws = lib().cfd_spectral_bounds_workspace(H.N, steps)
    work = _workspace(ws, H.buffers["val"].device)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(lib().cfd_spectral_bounds(H.ref(), steps, seed, ctypes.byref(lo), ctypes.byref(hi), _ptr(work), ws,
                                     _stream(stream)))
    return lo.value, hi.value


def cfd_block_gram(X, Y, stream=None, arith=0):
    """S = X^H Y (complex double device tensor); arith 1: double-word
    arithmetic on the fp32 pipe (cfd_block_gram_ex)."""
    bx, by = block_of(X), block_of(Y)
    S = torch.empty(bx.n_cols, by.n_cols, dtype=torch.complex128, device=X.device)
    ws = lib().cfd_gram_workspace(bx.n_rows, bx.n_cols, by.n_cols)
    work = _workspace(ws, X.device)
    if arith:
        _check(lib().cfd_block_gram_ex(bx, by, _ptr(S), S.stride(0), _ptr(work), ws, arith, _stream(stream)))
    else:
        _check(lib().cfd_block_gram(bx, by, _ptr(S), S.stride(0), _ptr(work), ws, _stream(stream)))
    return S


def cfd_eigh(A, stream=None):
    """(evals ascending, Q) of the Hermitian part of a complex double device matrix."""
    n = A.shape[0]
    ev = torch.empty(n, dtype=torch.float64, device=A.device)
    Q = torch.empty(n, n, dtype=torch.complex128, device=A.device)
    ws = lib().cfd_eigh_workspace(n)
    work = _workspace(ws, A.device)
    _check(lib().cfd_eigh(_ptr(A), A.stride(0), n, _ptr(ev), _ptr(Q), Q.stride(0), _ptr(work), ws,
                          _stream(stream)))
    return ev, Q


def cfd_orthogonalize(X, tol=0.0, stream=None, arith=0):
    """SVQB-orthonormalise the columns of X in place; returns the rank of the
    first pass.  arith 1: Grams and projections in double-word arithmetic."""
    blk = block_of(X)
    ws = lib().cfd_orthogonalize_workspace(blk.n_rows, blk.n_cols)
    work = _workspace(ws, X.device)
    rank = ctypes.c_int()
    if arith:
        _check(lib().cfd_orthogonalize_ex(blk, tol, ctypes.byref(rank), _ptr(work), ws, arith, _stream(stream)))
    else:
        _check(lib().cfd_orthogonalize(blk, tol, ctypes.byref(rank), _ptr(work), ws, _stream(stream)))
    return rank.value


def cfd_rayleigh_ritz(H, X, stream=None):
    """Rayleigh-Ritz in place on X; returns (theta, residual norms) as device tensors."""
    blk = block_of(X)
    ev = torch.empty(blk.n_cols, dtype=torch.float64, device=X.device)
    rs = torch.empty(blk.n_cols, dtype=torch.float64, device=X.device)
    ws = lib().cfd_rayleigh_ritz_workspace(blk.n_rows, blk.n_cols)
    work = _workspace(ws, X.device)
    _check(lib().cfd_rayleigh_ritz(H.ref(), blk, _ptr(ev), _ptr(rs), _ptr(work), ws, _stream(stream)))
    return ev, rs


def cfd_solve(H, X, lam_l, lam_r, n_p, n_b, H_low=None, policy=CFD_POLICY_FP64, lmin=0.0, lmax=0.0,
              tol=1e-10, n_t=0, max_iter=50, seed=2, start=0, switch_tol=0.0, bounds_steps=40, work=None,
              stream=None, raise_noconv=True):
    """Run the ChebFD solve on the N x n_s complex double tensor X (in: start block
    when start=1; out: Ritz vectors).  Returns (evals, resid, cfd_solve_result)
    with host numpy arrays of all n_s Ritz values and residuals."""
    import numpy as np
    blk = block_of(X)
    p = cfd_solve_params(lam_l=lam_l, lam_r=lam_r, lmin=lmin, lmax=lmax, tol=tol, switch_tol=switch_tol,
                         seed=seed, n_s=blk.n_cols, n_p=n_p, n_b=n_b, n_t=n_t, max_iter=max_iter, policy=policy,
                         bounds_steps=bounds_steps, start=start)
    hl = H_low.ref() if H_low is not None else None
    ws = lib().cfd_solve_workspace(H.ref(), hl, ctypes.byref(p))
    if work is None or work.numel() < ws:
        work = _workspace(ws, X.device)
    ev = np.zeros(blk.n_cols)
    rs = np.zeros(blk.n_cols)
    res = cfd_solve_result()
    st = lib().cfd_solve(H.ref(), hl, ctypes.byref(p), blk, ev.ctypes.data_as(ctypes.c_void_p),
                         rs.ctypes.data_as(ctypes.c_void_p), _ptr(work), work.numel(), ctypes.byref(res),
                         _stream(stream))
    if st != 0 and (raise_noconv or st != 6):
        _check(st)
    return ev, rs, res


def batch_row_end(B):
    """End of each realisation's real rows in a batch."""
    import numpy as np
    return np.array([B.row_off[r] + 4 * p.Nx * p.Ny * p.Nz for r, p in enumerate(B.params)], dtype=np.int64)


def cfd_solve_batched(B, X, windows, n_t, n_p, n_b, B_low=None, policy=CFD_POLICY_FP64, tol=1e-10, max_iter=50,
                      seed=2, start=0, switch_tol=0.0, work=None, stream=None, raise_noconv=True):
    """Batched ChebFD solve.  windows: host array [R, 4]; n_t: host ints [R].
    Returns (evals [R, n_s], resid [R, n_s], list of cfd_solve_result)."""
    import numpy as np
    blk = block_of(X)
    R = B.R
    win = np.ascontiguousarray(windows, dtype=np.float64).reshape(R, 4)
    nt = np.ascontiguousarray(n_t, dtype=np.int32).reshape(R)
    off = np.ascontiguousarray(B.row_off, dtype=np.int64)
    end = batch_row_end(B)
    p = cfd_solve_params(lam_l=0, lam_r=0, lmin=0, lmax=0, tol=tol, switch_tol=switch_tol, seed=seed,
                         n_s=blk.n_cols, n_p=n_p, n_b=n_b, n_t=0, max_iter=max_iter, policy=policy,
                         bounds_steps=0, start=start)
    ws = lib().cfd_solve_batched_workspace(B.ref(), R, ctypes.byref(p))
    if work is None or work.numel() < ws:
        work = _workspace(ws, X.device)
    ev = np.zeros((R, blk.n_cols))
    rs = np.zeros((R, blk.n_cols))
    res = (cfd_solve_result * R)()

    def vp(a):
        return a.ctypes.data_as(ctypes.c_void_p)

    st = lib().cfd_solve_batched(B.ref(), B_low.ref() if B_low is not None else None, _ptr(B.chunk_rid), R,
                                 vp(off), vp(end), vp(win), vp(nt), ctypes.byref(p), blk, vp(ev), vp(rs), res,
                                 _ptr(work), work.numel(), _stream(stream))
    if st != 0 and (raise_noconv or st != 6):
        _check(st)
    return ev, rs, list(res)


NOALLOC_SCRATCH_BYTES = 64 * 1024 * 1024


def cfd_filter_noalloc(H, lmin, lmax, lam_l, lam_r, n_p, X, n_b, moments=None, stream=None):
    """cfd_filter for callers that may not allocate device memory: the library's
    static 64 MiB device scratch replaces the workspace.  `moments`, if given,
    is a caller-owned float64 device tensor [n_s, 2 n_p]; nothing is allocated
    here.  Calls must not overlap on the GPU (they share the scratch)."""
    blk = block_of(X)
    _check(lib().cfd_filter_noalloc(H.ref(), lmin, lmax, lam_l, lam_r, n_p, blk, n_b, _ptr(moments),
                                    _stream(stream)))


def cfd_filter_noalloc_status(stream=None):
    """Device status of the last cfd_filter_noalloc call on this device: raises
    CfdError on a recorded timeout or moment growth (as cfd_workspace_status)."""
    _check(lib().cfd_filter_noalloc_status(_stream(stream)))


def cfd_probe_fma(prec="c128", iters=1 << 16, device="cuda", stream=None):
    """Measured FMA rate of the current GPU in flop/s: "c128" the fp64 pipe, "c64" the fp32 pipe."""
    work = _workspace(lib().cfd_probe_fma_workspace(), device)
    out = ctypes.c_double()
    _check(lib().cfd_probe_fma(_prec(prec), int(iters), ctypes.byref(out), _ptr(work), work.numel(),
                               _stream(stream)))
    return out.value


# ------------------------------------------------- distributed (z-slabs) --

def cfd_slab_plan(params, nranks, rank):
    """The z-slab of `rank` among nranks (host only)."""
    out = cfd_slab()
    _check(lib().cfd_slab_plan(ctypes.byref(params), nranks, rank, ctypes.byref(out)))
    return out


def cfd_slab_local_col(slab, col):
    return int(lib().cfd_slab_local_col(ctypes.byref(slab), int(col)))


def cfd_build_matrix_slab(params, slab, C=32, sigma=1, prec="c128", device="cuda", stream=None):
    """Allocate and build one slab's rows of Topi (columns in the slab's numbering)."""
    prec = _prec(prec)
    sz = cfd_matrix_sizes()
    _check(lib().cfd_slab_query_size(ctypes.byref(params), ctypes.byref(slab), C, sigma, prec, ctypes.byref(sz)))
    dev = torch.device(device)
    bufs = {
        "val": _workspace(sz.bytes_val, dev), "col": _workspace(sz.bytes_col, dev),
        "chunk_ptr": _workspace(sz.bytes_chunk_ptr, dev), "chunk_len": _workspace(sz.bytes_chunk_len, dev),
        "perm": _workspace(sz.bytes_perm, dev) if sz.bytes_perm else None,
        "work": _workspace(sz.bytes_work, dev),
    }
    b = cfd_matrix_buffers(*[(bufs[k].data_ptr() if bufs[k] is not None else None)
                             for k in ("val", "col", "chunk_ptr", "chunk_len", "perm", "work")])
    out = cfd_matrix()
    _check(lib().cfd_build_matrix_slab(ctypes.byref(params), ctypes.byref(slab), C, sigma, prec, ctypes.byref(b),
                                       ctypes.byref(out), _stream(stream)))
    return Matrix(out, bufs, params)


def cfd_filter_slabs(slabs, Hs, lmin, lmax, lam_l, lam_r, n_p, Xs, n_b, mode=CFD_DIST_VECTOR, moments=False,
                     arith=0, stream=None, footprint=0):
    """The distributed filter with every slab in this process (halo exchange by
    device copies).  Xs: the slabs' local blocks (filtered in place).  Returns
    the moments of the whole vectors when moments=True.  footprint: as in
    cfd_filter_ex."""
    n = len(slabs)
    S = (cfd_slab * n)(*slabs)
    blks = [block_of(X) for X in Xs]
    B = (cfd_block * n)(*blks)
    Hp = (ctypes.c_void_p * n)(*[ctypes.addressof(H.c) for H in Hs])
    ws = max(lib().cfd_filter_slab_workspace(ctypes.byref(slabs[r]), blks[r].n_cols, n_b, n_p, Hs[r].prec, mode)
             for r in range(n))
    works = [_workspace(ws, Xs[0].device) for _ in range(n)]
    W = (ctypes.c_void_p * n)(*[w.data_ptr() for w in works])
    mu = torch.empty(blks[0].n_cols, 2 * n_p, dtype=torch.float64, device=Xs[0].device) if moments else None
    o = cfd_filter_opts(0, 0, 0, 0, 0, 0, arith, 0, footprint)
    _check(lib().cfd_filter_slabs(n, S, Hp, lmin, lmax, lam_l, lam_r, n_p, B, n_b, mode, W, ws, _ptr(mu),
                                  ctypes.byref(o), _stream(stream)))
    (stream or torch.cuda.current_stream()).synchronize()      # the workspaces are freed on return
    del works
    return mu


def cfd_nccl_unique_id():
    """128-byte NCCL unique id (bytes), to be shared with every rank."""
    buf = ctypes.create_string_buffer(128)
    _check(lib().cfd_nccl_unique_id(buf))
    return buf.raw


def cfd_nccl_comm_init(uid, nranks, rank):
    comm = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(bytes(uid), 128)
    _check(lib().cfd_nccl_comm_init(buf, nranks, rank, ctypes.byref(comm)))
    return comm


def cfd_nccl_comm_destroy(comm):
    _check(lib().cfd_nccl_comm_destroy(comm))


def cfd_filter_slab_nccl(slab, H, lmin, lmax, lam_l, lam_r, n_p, X, n_b, comm, mode=CFD_DIST_VECTOR,
                         moments=False, arith=0, work=None, stream=None, footprint=0):
    """One rank's part of the distributed filter (one slab per process and GPU,
    halo exchange over NCCL).  Every rank receives the global moments.
    footprint: as in cfd_filter_ex."""
    blk = block_of(X)
    ws = lib().cfd_filter_slab_workspace(ctypes.byref(slab), blk.n_cols, n_b, n_p, H.prec, mode)
    if work is None or work.numel() < ws:
        work = _workspace(ws, X.device)
    mu = torch.empty(blk.n_cols, 2 * n_p, dtype=torch.float64, device=X.device) if moments else None
    o = cfd_filter_opts(0, 0, 0, 0, 0, 0, arith, 0, footprint)
    _check(lib().cfd_filter_slab_nccl(ctypes.byref(slab), H.ref(), lmin, lmax, lam_l, lam_r, n_p, blk, n_b, mode,
                                      _ptr(work), work.numel(), _ptr(mu), ctypes.byref(o), comm, _stream(stream)))
    return mu
