"""Minimum-traffic and flop model of one ChebFD filter step (Sect. 3.4, Eq. 2).

Per matrix row and block step: the row's nonzeros are read once per block of
n_b vectors (value + 4-byte index each), and each of the n_b vectors moves
five complex words: U read once, W read and written, X read and written
(Algorithm 1, lines 9-12).  With 13 nonzeros per row and 16-byte complex
values this gives the paper's 260 / n_b + 80 bytes per row per vector.

Flops per row per vector: 8 per complex multiply-add of the SpMMV and 42 for
the shift, scaling, subtraction, two dot products and the update, the split
that reproduces the paper's 146 at 13 nonzeros per row.  The FP64/FP32 pipe
executes 4 fused multiply-adds per complex multiply-add and 10 per row for
the rest (8 nnz + 20 flops per row per vector), the count the ALU roofline
uses.
"""

IDX_BYTES = 4


def scalar_bytes(prec):
    return {"c128": 16, "c64": 8}[prec]


def step_bytes(N, nnz, n_b, prec="c128"):
    """Minimum DRAM bytes of one fused step over an N x n_b block:
    nnz (s + 4) + 5 N n_b s."""
    s = scalar_bytes(prec)
    return nnz * (s + IDX_BYTES) + 5 * N * n_b * s


def step_read_write_bytes(N, nnz, n_b, prec="c128"):
    """(read, write) split of step_bytes: matrix + U + W + X read; W + X written."""
    s = scalar_bytes(prec)
    return nnz * (s + IDX_BYTES) + 3 * N * n_b * s, 2 * N * n_b * s


def unfused_step_bytes(N, nnz, n_b, prec="c128", moments=True):
    """Minimum DRAM bytes of one step computed by separate calls (SpMMV into a
    third block Y, then W = 2 alpha Y - W, W -= 2 alpha beta U, X += g W, and
    the dots <U, U>, <W, U>): the matrix plus 2 + 3 + 3 + 3 (+ 1 + 2) block
    vectors, 14 with the moments against the fused step's 5."""
    s = scalar_bytes(prec)
    return nnz * (s + IDX_BYTES) + (14 if moments else 11) * N * n_b * s


def step_flops(N, nnz, n_b):
    """Paper-convention flops of one fused step: (8 nnz + 42 N) n_b."""
    return (8 * nnz + 42 * N) * n_b


def step_fma_flops(N, nnz, n_b, packed=False, prepared=False):
    """Flops the multiply-add pipe must execute for one fused step with
    moments: (8 nnz + 20 N) n_b with complex matrix values; (4 nnz + 20 N) n_b
    when every value is stored as one real-or-imaginary scalar (two fused
    multiply-adds per nonzero).  prepared: the step reads the values of
    2 alpha (H - beta), prepared once per filter application, and starts each
    row sum at -V_prev, so the shift, scale and subtraction (8 flops per row
    and vector) vanish: (4 or 8) nnz n_b + 12 N n_b (X update, two dots)."""
    return ((4 if packed else 8) * nnz + (12 if prepared else 20) * N) * n_b


def intensity(n_b, nnzr=13, prec="c128"):
    """Eq. 2: flops per byte for one row, 146 / (nnzr (s + 4) / n_b + 5 s)."""
    s = scalar_bytes(prec)
    return (8 * nnzr + 42) / (nnzr * (s + IDX_BYTES) / n_b + 5 * s)


def roofline(n_b, bandwidth_gbs, nnzr=13, prec="c128"):
    """Eq. 1 memory bound P* = I(n_b) b in Gflop/s."""
    return intensity(n_b, nnzr, prec) * bandwidth_gbs


def filter_bytes(N, nnz, n_s, n_b, n_p, prec="c128"):
    """Minimum bytes of a whole filter application: n_s / n_b blocks of n_p steps."""
    return (n_s // n_b) * n_p * step_bytes(N, nnz, n_b, prec)


def filter_flops(N, nnz, n_s, n_b, n_p):
    return (n_s // n_b) * n_p * step_flops(N, nnz, n_b)
