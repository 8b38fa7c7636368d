"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the spectral-element method: it only names
the workloads (box sizes, polynomial order, deformation switch) and draws
seeded random arrays with numpy's PCG64 generator.  Both the CPU oracle and
the CUDA library receive what it produces; neither imports the other.

Random right-hand sides that are defined per *global* node are not drawn
here: both sides implement the SplitMix64 counter-based generator from its
published definition (Steele, Lea & Flood, OOPSLA 2014) and draw them
themselves, keyed by (seed, global node id).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class BoxCase:
    """A box mesh of kx*ky*kz hexahedra on [lo, hi]^3 at polynomial order N."""

    kx: int
    ky: int
    kz: int
    N: int
    deform: bool = False
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)

    @property
    def n(self) -> int:
        return self.N + 1

    @property
    def E(self) -> int:
        return self.kx * self.ky * self.kz

    @property
    def L(self) -> int:
        """Local (unassembled) degrees of freedom E*(N+1)^3."""
        return self.E * self.n ** 3

    @property
    def U(self) -> int:
        """Unique global nodes of the box numbering."""
        return (self.kx * self.N + 1) * (self.ky * self.N + 1) * (self.kz * self.N + 1)


# The workloads, named by what they are.
SINE_4x4x4_N7 = BoxCase(4, 4, 4, 7, deform=False)             # 32,768 local DOFs
DEFORMED_32x32x32_N7 = BoxCase(32, 32, 32, 7, deform=True)    # 16.8 M local DOFs


def order_sweep_case(N: int) -> BoxCase:
    """Deformed cube with about 2^24 local DOFs at order N (k = round((2^24/n^3)^(1/3)))."""
    n = N + 1
    k = int(round((2 ** 24 / n ** 3) ** (1.0 / 3.0)))
    return BoxCase(k, k, k, N, deform=True)


def uniform_local(L: int, seed: int, dtype=np.float64) -> np.ndarray:
    """L values uniform in [-1, 1) from PCG64(seed); an unassembled local vector."""
    g = np.random.Generator(np.random.PCG64(seed))
    return (2.0 * g.random(L) - 1.0).astype(dtype)


def uniform_matrix(rows: int, cols: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """rows x cols values uniform in [-scale, scale) from PCG64(seed)."""
    g = np.random.Generator(np.random.PCG64(seed))
    return scale * (2.0 * g.random((rows, cols)) - 1.0)


def batched_cases(count: int = 64, seed: int = 1, kmin: int = 8, kmax: int = 24,
                  orders=(5, 7, 9)):
    """Box sizes k (E = k^3) and orders N of a batch of independent problems,
    drawn from PCG64(seed); problem i's right-hand side uses seed 1000 + i."""
    g = np.random.Generator(np.random.PCG64(seed))
    ks = g.integers(kmin, kmax + 1, size=count)
    Ns = g.choice(np.asarray(orders), size=count)
    return [(int(k), int(N)) for k, N in zip(ks, Ns)]
