"""Seeded synthetic inputs for the triangle-lattice truss solves.

This module is shared by the CPU oracle, the tests and the benchmark.  It holds
random number generation and the recipes of the workloads only -- none of the
solver's arithmetic (no geometry, no stiffness, no residual).

The paper loads every node of its lattice with "a force which is random both
in magnitude and direction" (Sec. 3.1).  The readings used here:

* loads: iid Uniform(-1, 1) per degree of freedom (x and y of every node);
* bar stiffness EA: 1, or lognormal(0, 0.3) per bar, EA = exp(0.3 z),
  z ~ N(0, 1) by the Box-Muller transform;
* supports: the bottom row of nodes (j = 0) clamped in x and y.

All draws come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11), a counter-based generator, keyed
by the seed and indexed by node, so an entry never depends on the lattice
size or on how the array is produced.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "philox4x32_10", "uniform01", "loads", "loads_torch", "ea_lognormal", "clamp_bottom",
    "LatticeCase", "CASES",
]

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)

# stream tags (the fourth counter word), one per kind of draw
TAG_LOAD = 0x4C4F4144  # "LOAD"
TAG_EA = 0x45414541    # "EAEA"
TAG_BATCH = 0x42415443  # "BATC"
TAG_SERVE = 0x53525645  # "SRVE"


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds (SC'11, Sec. 3.3 / Random123 reference).

    Each round multiplies counter words 0 and 2 by the constants M0, M1 into
    64-bit products (hi, lo), permutes and xors them with the other two words
    and the round key; the key is bumped by the Weyl constants W0, W1 between
    rounds.  All arguments broadcast; returns four uint32 arrays.
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint32) for c in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    c0, c1, c2, c3 = (c.astype(np.uint32, copy=True) for c in (c0, c1, c2, c3))
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    for rnd in range(10):
        if rnd:
            k0 = np.uint32((int(k0) + int(_W0)) & 0xFFFFFFFF)
            k1 = np.uint32((int(k1) + int(_W1)) & 0xFFFFFFFF)
        p0 = c0.astype(np.uint64) * _M0
        p1 = c2.astype(np.uint64) * _M1
        hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
        lo0 = (p0 & _MASK32).astype(np.uint32)
        hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
        lo1 = (p1 & _MASK32).astype(np.uint32)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def uniform01(w):
    """Map uint32 words to doubles strictly inside (0, 1): (w + 1/2) / 2^32."""
    return (np.asarray(w, dtype=np.float64) + 0.5) * (1.0 / 4294967296.0)


def _node_counters(nx, ny):
    idx = np.arange(nx * ny, dtype=np.uint64)
    lo = (idx & _MASK32).astype(np.uint32)
    hi = (idx >> np.uint64(32)).astype(np.uint32)
    return lo, hi


def loads(nx: int, ny: int, seed: int, rhs: int = 0) -> np.ndarray:
    """Nodal loads, iid Uniform(-1, 1) per DOF; float64 array [ny, nx, 2].

    Node n = j*nx + i draws counter (n_lo, n_hi, rhs, TAG_LOAD) under key
    (seed, 0); its x load uses word 0 and its y load word 1.  Loads on
    constrained DOFs are generated like all others; the solver ignores them.
    """
    lo, hi = _node_counters(nx, ny)
    w0, w1, _, _ = philox4x32_10(lo, hi, np.uint32(rhs), np.uint32(TAG_LOAD),
                                 seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    out = np.empty((ny, nx, 2), dtype=np.float64)
    out[..., 0] = (2.0 * uniform01(w0) - 1.0).reshape(ny, nx)
    out[..., 1] = (2.0 * uniform01(w1) - 1.0).reshape(ny, nx)
    return out


def _mulhilo_t(a, m: int):
    """High and low 32-bit words of a * m (a: int64 tensor of uint32 values,
    m < 2^32), by 16-bit halves so that no int64 product overflows."""
    m1, m0 = m >> 16, m & 0xFFFF
    a1, a0 = a >> 16, a & 0xFFFF
    mid = a1 * m0 + a0 * m1
    t = a0 * m0 + ((mid & 0xFFFF) << 16)
    return a1 * m1 + (mid >> 16) + (t >> 32), t & 0xFFFFFFFF


def loads_torch(nx: int, ny: int, seed: int, rhs: int = 0, device="cpu", chunk: int = 1 << 25):
    """The loads of `loads` (the same Philox4x32-10 draws, bit for bit) as a
    torch float64 tensor [ny, nx, 2] made on `device`, chunk nodes at a time:
    for lattices whose loads are too large to draw on the host (10^9 DOFs)."""
    import torch

    out = torch.empty((ny * nx, 2), dtype=torch.float64, device=device)
    k0, k1 = seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF
    inv = 1.0 / 4294967296.0
    for n0 in range(0, nx * ny, chunk):
        n = torch.arange(n0, min(n0 + chunk, nx * ny), dtype=torch.int64, device=device)
        c0, c1 = n & 0xFFFFFFFF, n >> 32
        c2 = torch.full_like(n, rhs & 0xFFFFFFFF)
        c3 = torch.full_like(n, TAG_LOAD)
        a0, a1 = k0, k1
        for rnd in range(10):
            if rnd:
                a0 = (a0 + int(_W0)) & 0xFFFFFFFF
                a1 = (a1 + int(_W1)) & 0xFFFFFFFF
            hi0, lo0 = _mulhilo_t(c0, int(_M0))
            hi1, lo1 = _mulhilo_t(c2, int(_M1))
            c0, c1, c2, c3 = hi1 ^ c1 ^ a0, lo1, hi0 ^ c3 ^ a1, lo0
        out[n0:n0 + n.numel(), 0] = 2.0 * ((c0.double() + 0.5) * inv) - 1.0
        out[n0:n0 + n.numel(), 1] = 2.0 * ((c1.double() + 0.5) * inv) - 1.0
    return out.view(ny, nx, 2)


def ea_lognormal(nx: int, ny: int, seed: int, sigma: float = 0.3) -> np.ndarray:
    """Per-bar EA = exp(sigma z), z ~ N(0,1); float64 array [3, ny, nx].

    Plane d = 0, 1, 2 holds the bar of direction E, NE, NW owned by node
    (i, j).  Node n draws counter (n_lo, n_hi, 0, TAG_EA) under key
    (seed, 1); Box-Muller on (w0, w1) gives z_E = rho cos(theta),
    z_NE = rho sin(theta), and on (w2, w3) gives z_NW = rho' cos(theta').
    Entries of bars that do not exist (lattice edges) are generated and
    ignored.
    """
    lo, hi = _node_counters(nx, ny)
    w0, w1, w2, w3 = philox4x32_10(lo, hi, np.uint32(0), np.uint32(TAG_EA),
                                   seed & 0xFFFFFFFF, ((seed >> 32) + 1) & 0xFFFFFFFF)
    r0 = np.sqrt(-2.0 * np.log(uniform01(w0)))
    t0 = 2.0 * math.pi * uniform01(w1)
    r1 = np.sqrt(-2.0 * np.log(uniform01(w2)))
    t1 = 2.0 * math.pi * uniform01(w3)
    z = np.stack([r0 * np.cos(t0), r0 * np.sin(t0), r1 * np.cos(t1)])
    return np.exp(sigma * z).reshape(3, ny, nx)


def clamp_bottom(nx: int, ny: int) -> np.ndarray:
    """Constrained-DOF mask [ny, nx, 2] (uint8, 1 = fixed): row j = 0 clamped."""
    fixed = np.zeros((ny, nx, 2), dtype=np.uint8)
    fixed[0] = 1
    return fixed


@dataclasses.dataclass(frozen=True)
class LatticeCase:
    """One named workload: lattice size, set tile, stiffness and stop rule."""
    name: str
    nx: int
    ny: int
    sx: int
    sy: int
    ea: str            # "uniform" or "lognormal"
    tol: float         # 1-norm relative residual of Eq. 19
    precision: str     # "fp64" or "mixed"
    nrhs: int = 1
    seed: int = 0

    def ea_array(self):
        if self.ea == "uniform":
            return None
        return ea_lognormal(self.nx, self.ny, self.seed + 1000)

    def load_array(self, rhs: int = 0):
        return loads(self.nx, self.ny, self.seed, rhs)

    @property
    def dofs(self) -> int:
        return 2 * self.nx * self.ny


# The paper's test problems are square triangle-lattice trusses under random
# loads (Sec. 3.1); these are the sizes this project measures and tests.
CASES = {
    "lattice64_fp64": LatticeCase("lattice64_fp64", 64, 64, 16, 16, "uniform", 1e-8, "fp64"),
    "lattice1024_lognormal_fp64": LatticeCase(
        "lattice1024_lognormal_fp64", 1024, 1024, 64, 64, "lognormal", 1e-10, "fp64"),
    "lattice1024_lognormal_mixed": LatticeCase(
        "lattice1024_lognormal_mixed", 1024, 1024, 64, 64, "lognormal", 1e-10, "mixed"),
    "lattice22361_mixed": LatticeCase(
        "lattice22361_mixed", 22361, 22361, 64, 64, "uniform", 1e-10, "mixed"),
}


@dataclasses.dataclass(frozen=True)
class BatchLattice:
    """One lattice of a batch: size, load-vector count and its load seed."""
    nx: int
    ny: int
    nrhs: int
    seed: int

    def load_array(self):
        """[nrhs, 2*nx*ny] loads, load vector r from counter rhs = r."""
        return np.stack([loads(self.nx, self.ny, self.seed, r).reshape(-1) for r in range(self.nrhs)])


def batched_lattices(count: int = 256, seed: int = 7, side_min: int = 32, side_max: int = 512,
                     aspect_max: float = 4.0, nrhs_max: int = 8):
    """Independent lattices of uneven shape: lattice k draws counter
    (k, 0, 0, TAG_BATCH) under key (seed, 2); the long side is log-uniform in
    [side_min, side_max] (word 0), the aspect ratio Uniform[1, aspect_max]
    (word 1), the short side max(2, round(long / aspect)), the orientation a
    coin flip (word 2) and the load-vector count 1 + floor(nrhs_max u)
    (word 3).  Lattice k's loads use seed 1000 + k."""
    k = np.arange(count, dtype=np.uint64)
    w0, w1, w2, w3 = philox4x32_10(k.astype(np.uint32), np.zeros(count, np.uint32), np.uint32(0),
                                   np.uint32(TAG_BATCH), seed & 0xFFFFFFFF, ((seed >> 32) + 2) & 0xFFFFFFFF)
    lo, hi = math.log(side_min), math.log(side_max)
    longs = np.rint(np.exp(lo + (hi - lo) * uniform01(w0))).astype(int)
    aspect = 1.0 + (aspect_max - 1.0) * uniform01(w1)
    shorts = np.maximum(2, np.rint(longs / aspect).astype(int))
    flip = uniform01(w2) < 0.5
    nrhs = 1 + np.minimum(nrhs_max - 1, np.floor(nrhs_max * uniform01(w3)).astype(int))
    out = []
    for i in range(count):
        nx, ny = (int(longs[i]), int(shorts[i])) if flip[i] else (int(shorts[i]), int(longs[i]))
        out.append(BatchLattice(nx, ny, int(nrhs[i]), 1000 + i))
    return out


@dataclasses.dataclass(frozen=True)
class ServeRequest:
    """One request of the serving workload: arrival time (s), lattice, loads."""
    arrival: float
    nx: int
    ny: int
    nrhs: int
    seed: int

    def ea_array(self):
        return ea_lognormal(self.nx, self.ny, self.seed + 1)

    def load_array(self):
        return np.stack([loads(self.nx, self.ny, self.seed, r).reshape(-1) for r in range(self.nrhs)])


def serving_requests(count: int = 64, seed: int = 5, rate: float = 200.0, side_min: int = 64,
                     side_max: int = 2048, width_max: int | None = None, nrhs_max: int = 16):
    """Poisson arrivals (mean rate per second) of lattice solves: request k
    draws counter (k, 0, 0, TAG_SERVE) under key (seed, 3): the gap to the
    previous arrival is exponential (word 0), the width nx and the height ny
    are log-uniform in [side_min, side_max] (words 1, 2), the load-vector
    count is 1 + floor(nrhs_max u) (word 3).  width_max (None: no cap) caps
    nx; request k's loads use seed 2000 + k."""
    k = np.arange(count, dtype=np.uint64)
    w0, w1, w2, w3 = philox4x32_10(k.astype(np.uint32), np.zeros(count, np.uint32), np.uint32(0),
                                   np.uint32(TAG_SERVE), seed & 0xFFFFFFFF, ((seed >> 32) + 3) & 0xFFFFFFFF)
    gaps = -np.log(uniform01(w0)) / rate
    t = np.cumsum(gaps) - gaps[0]
    lo, hi = math.log(side_min), math.log(side_max)
    a = np.rint(np.exp(lo + (hi - lo) * uniform01(w1))).astype(int)
    b = np.rint(np.exp(lo + (hi - lo) * uniform01(w2))).astype(int)
    nrhs = 1 + np.minimum(nrhs_max - 1, np.floor(nrhs_max * uniform01(w3)).astype(int))
    out = []
    for i in range(count):
        nx, ny = int(a[i]), int(b[i])
        if width_max is not None:
            nx = min(nx, width_max)
        out.append(ServeRequest(float(t[i]), int(nx), int(ny), int(nrhs[i]), 2000 + i))
    return out
