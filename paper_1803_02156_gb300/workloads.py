"""Named synthetic workloads: topological-insulator lattices and ChebFD
search parameters (sizes only, no arithmetic).

Topi-Nx-Ny-Nz: n = 4 Nx Ny Nz rows, t = 1, m = 2, disorder gamma = 1 (V uniform
in [-1/2, 1/2]), periodic in x and y, open in z.
"""
from dataclasses import dataclass, field


@dataclass(frozen=True)
class Workload:
    name: str
    lattice: tuple          # (Nx, Ny, Nz)
    n_s: int                # search vectors
    n_p: int                # filter degree
    n_b: int                # subspace block width
    prec: str = "c128"      # filter arithmetic
    n_t: int = 0            # target eigenpair count (window holds about n_t states)
    periodic: tuple = (1, 1, 0)
    t: float = 1.0
    m: float = 2.0
    gamma: float = 1.0
    seed: int = 1           # disorder seed
    x_seed: int = 2         # start block seed
    lanczos_seed: int = 3
    sell_C: int = 32
    sell_sigma: int = 1

    @property
    def N(self):
        Nx, Ny, Nz = self.lattice
        return 4 * Nx * Ny * Nz

    @property
    def nnz(self):
        """13 per row, less one hop pair per open boundary side (2 nonzeros)."""
        Nx, Ny, Nz = self.lattice
        n = 13 * self.N
        if not self.periodic[2]:
            n -= 16 * Nx * Ny
        if not self.periodic[1]:
            n -= 16 * Nx * Nz
        if not self.periodic[0]:
            n -= 16 * Ny * Nz
        return n


# Parity case: 8x8x8 (N = 2048), window holding about 16 eigenvalues.
SMALL = Workload("topi-8x8x8-c128", (8, 8, 8), n_s=32, n_p=200, n_b=32, n_t=16)
# Headline filter workload: 64x64x32 (N = 524288), n_s = 128, n_p ~ 1000.
MEDIUM = Workload("topi-64x64x32-c128", (64, 64, 32), n_s=128, n_p=1000, n_b=32, n_t=64)
# Large single instance: 200x200x100 (N = 16e6), n_s = 256 in blocks of 32.
LARGE = Workload("topi-200x200x100-c128", (200, 200, 100), n_s=256, n_p=100, n_b=32)
# Mixed precision: 128x128x64 (N = 4.2e6), n_s = 256, complex64 filter.
MIXED = Workload("topi-128x128x64-c64", (128, 128, 64), n_s=256, n_p=500, n_b=32,
                 prec="c64", n_t=128)
# Batched: 64 realisations, n_s = 64, n_p = 500, complex64 filter.
BATCH_COUNT = 64
BATCH = Workload("topi-batch64-c64", (32, 32, 16), n_s=64, n_p=500, n_b=32, prec="c64", n_t=32)

ALL = {w.name: w for w in (SMALL, MEDIUM, LARGE, MIXED, BATCH)}
