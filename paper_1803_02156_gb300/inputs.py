"""Seeded synthetic inputs shared by the oracle-side and the GPU-side tests.

This module holds none of the method's arithmetic: it only turns a seed into
numbers.  It implements counter-based SplitMix64 (Steele, Lea, Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014) in numpy:
draw i of stream (seed, tag) is mix(key + (i + 1) GAMMA), with
key = mix(seed + GAMMA (2 tag + 1)), mix the SplitMix64 output function.

Tags: 0 on-site disorder, 1 start block, 2 Lanczos start vector,
3 orthogonalisation refill, 4 lattice-size draws of the batched workload.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed, tag, idx):
    """uint64 draws idx (array) of stream (seed, tag)."""
    with np.errstate(over="ignore"):
        key = _mix(np.uint64(seed) + GAMMA * np.uint64(2 * tag + 1))
        i = np.asarray(idx, dtype=np.uint64)
        return _mix(key + (i + np.uint64(1)) * GAMMA)


def uniform(seed, tag, idx):
    """Doubles in [0, 1) from the top 53 bits of each draw."""
    return (splitmix64(seed, tag, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def gaussian_block(N, n_s, seed, tag=1):
    """Complex Gaussian N x n_s block (row-major), unit variance per entry:
    entry k = i n_s + j uses draws 2k, 2k + 1 with Box-Muller,
    r = sqrt(-2 ln(1 - u1)), value = r exp(2 pi i u2) / sqrt(2)."""
    k = np.arange(N * n_s, dtype=np.uint64)
    u1 = uniform(seed, tag, 2 * k)
    u2 = uniform(seed, tag, 2 * k + np.uint64(1))
    r = np.sqrt(-2.0 * np.log1p(-u1))
    z = r * np.exp(2j * np.pi * u2) / np.sqrt(2.0)
    return z.reshape(N, n_s).astype(np.complex128)


def batched_lattices(count, base_seed=1000):
    """Uneven lattice sizes of the batched workload: realisation r draws
    Nx, Ny uniformly from 16..48 and Nz from 8..24 out of stream
    (base_seed + r, tag 4); its disorder seed is base_seed + r."""
    out = []
    for r in range(count):
        d = splitmix64(base_seed + r, 4, np.arange(3, dtype=np.uint64))
        nx = 16 + int(d[0] % np.uint64(33))
        ny = 16 + int(d[1] % np.uint64(33))
        nz = 8 + int(d[2] % np.uint64(17))
        out.append((nx, ny, nz, base_seed + r))
    return out


def gaussian_block_device(N, n_s, seed, dtype=None, device="cuda"):
    """Complex Gaussian N x n_s block generated on the device with a seeded
    torch generator (for blocks too large to build on the host); any row can
    be read back as an input for the oracle."""
    import torch
    dtype = dtype or torch.complex128
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    real = torch.float64 if dtype == torch.complex128 else torch.float32
    z = torch.randn(N, n_s, 2, generator=g, device=device, dtype=real) * (0.5 ** 0.5)
    return torch.view_as_complex(z).contiguous()


def fill_gaussian_device(X, seed):
    """Overwrite the complex device tensor X (contiguous) in place with the
    values gaussian_block_device(X.shape[0], X.shape[1], seed, X.dtype) draws,
    without allocating a second block."""
    import torch
    g = torch.Generator(device=X.device)
    g.manual_seed(int(seed))
    r = torch.view_as_real(X)
    torch.randn(r.shape, generator=g, device=X.device, dtype=r.dtype, out=r)
    r.mul_(0.5 ** 0.5)
    return X
