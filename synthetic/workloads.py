"""Seeded workload generators for the 2D type-II inverse NUDFT (points, coefficients, noise).

Point sets follow the jittered-grid recipe: an m_x-by-m_y lattice whose nodes are shifted
independently per coordinate by theta ~ U[lo, hi] lattice cells and wrapped into [0, 1)
(paper Sec. 1: sample points lie anywhere in [0, 1)^2; M >= N = n_x n_y).  Coefficients are
complex with independent N(0, 1) real and imaginary parts.  Nothing here evaluates the
NUDFT; right-hand sides f = A c are formed by whichever side (oracle or device) the caller
is testing.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def jittered_grid(mx: int, my: int, lo: float, hi: float, seed: int):
    """Points x=((i+theta)/mx) mod 1, y=((j+theta')/my) mod 1, i-major order, theta iid U[lo,hi]."""
    rng = _rng(seed)
    i, j = np.meshgrid(np.arange(mx, dtype=np.float64), np.arange(my, dtype=np.float64), indexing="ij")
    tx = rng.uniform(lo, hi, size=i.size)
    ty = rng.uniform(lo, hi, size=j.size)
    x = np.mod((i.ravel() + tx) / mx, 1.0)
    y = np.mod((j.ravel() + ty) / my, 1.0)
    # a value that rounds to exactly 1.0 after the wrap belongs to 0 (half-open [0, 1))
    x[x >= 1.0] = 0.0
    y[y >= 1.0] = 0.0
    return x, y


def uniform_grid(mx: int, my: int):
    """Unperturbed lattice x=i/mx, y=j/my (i-major), the closed-form special case."""
    i, j = np.meshgrid(np.arange(mx, dtype=np.float64), np.arange(my, dtype=np.float64), indexing="ij")
    return (i.ravel() / mx), (j.ravel() / my)


def complex_normal(shape, seed: int) -> np.ndarray:
    """complex128 with iid N(0,1) real and imaginary parts."""
    rng = _rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def noise_like(f0: np.ndarray, rel: float, seed: int) -> np.ndarray:
    """Noise e = rel * ||f0|| * w / ||w|| per column, w iid complex normal."""
    w = complex_normal(f0.shape, seed)
    if f0.ndim == 1:
        return rel * np.linalg.norm(f0) * w / np.linalg.norm(w)
    return rel * np.linalg.norm(f0, axis=0) * w / np.linalg.norm(w, axis=0)


@dataclass(frozen=True)
class Workload:
    """One synthetic problem: sizes, grid recipe, solver options."""
    name: str
    nx: int
    ny: int
    mx: int
    my: int
    theta: tuple
    nrhs: int
    levels: int          # equal depth of both 1D trees; product leaf = (nx>>L) x (ny>>L)
    eps: float
    noise: float = 0.0
    mixed: bool = False
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.nx * self.ny

    @property
    def M(self) -> int:
        return self.mx * self.my


WORKLOADS = {
    # plain FP64 solve, N=256, M=512 on a 32x16 jittered grid, product leaf 4x4
    "fp64_n16": Workload("fp64_n16", 16, 16, 32, 16, (-0.25, 0.25), 1, 2, 1e-10, seed=1),
    # plain FP64 solve at scale, N=16384, M=32768, leaf 8x8, 1e-12 relative noise, 4 RHS
    "fp64_n128": Workload("fp64_n128", 128, 128, 256, 128, (-0.3, 0.3), 4, 4, 1e-10, noise=1e-12, seed=2),
    # mixed precision, N=65536, M=131072, leaf 8x8, 16 RHS, FP64 refinement
    "mixed_n256": Workload("mixed_n256", 256, 256, 512, 256, (-0.3, 0.3), 16, 5, 1e-10, mixed=True, seed=3),
    # differentiation workload, N=16384, M=32768, 16 RHS
    "grad_n128": Workload("grad_n128", 128, 128, 256, 128, (-0.3, 0.3), 16, 4, 1e-10, seed=5),
    # mid-size case the dense oracle finishes in seconds: several tiles, ragged leaves
    "fp64_n32": Workload("fp64_n32", 32, 32, 64, 32, (-0.3, 0.3), 3, 3, 1e-10, seed=11),
    # intermediate sizes of the same recipe (scaling and profiling cases)
    "fp64_n64": Workload("fp64_n64", 64, 64, 128, 64, (-0.3, 0.3), 4, 3, 1e-10, seed=12),
    "mixed_n64": Workload("mixed_n64", 64, 64, 128, 64, (-0.3, 0.3), 16, 3, 1e-10, mixed=True, seed=13),
    "mixed_n128": Workload("mixed_n128", 128, 128, 256, 128, (-0.3, 0.3), 16, 4, 1e-10, mixed=True, seed=14),
}


def make_workload(w: Workload):
    """Return (x, y, c_true) for a workload; c_true is (N, nrhs) in lexicographic ky + kx*ny order."""
    x, y = jittered_grid(w.mx, w.my, w.theta[0], w.theta[1], w.seed)
    c = complex_normal((w.N, w.nrhs), w.seed + 1000)
    return x, y, c


BATCH_SIZES = (32, 48, 64, 96, 128, 192, 256)


def batched_uneven(count: int = 64, seed: int = 100, sizes=BATCH_SIZES, nrhs: int = 8,
                   ratio=(1.5, 4.0), theta=(-0.25, 0.35)):
    """Independent problems of uneven size (the batched workload): problem p draws n_x, n_y
    uniformly from `sizes` and an oversampling rho ~ U[ratio] from seed + p, then takes a
    jittered m_x x m_y grid with m_x = round(n_x sqrt(rho)), m_y = round(n_y sqrt(rho)) (so
    M ~ rho N, and M > N since rho >= 1.5) and theta ~ U[theta], plus nrhs iid complex normal
    coefficient columns.
    Returns a list of dicts with nx, ny, x, y, c_true (N x nrhs, lexicographic ky + kx*ny)."""
    out = []
    for p in range(count):
        rng = _rng(seed + p)
        nx = int(rng.choice(sizes))
        ny = int(rng.choice(sizes))
        rho = float(rng.uniform(*ratio))
        mx = int(np.round(nx * np.sqrt(rho)))
        my = int(np.round(ny * np.sqrt(rho)))
        x, y = jittered_grid(mx, my, theta[0], theta[1], seed + p + 10_000)
        c = complex_normal((nx * ny, nrhs), seed + p + 20_000)
        out.append({"nx": nx, "ny": ny, "x": x, "y": y, "c_true": c, "rho": rho})
    return out


def polar_grid(n: int, beta: float = 0.6):
    """The modified polar grid of the paper's experiments: the centre (1/2, 1/2) and the points
    x = 1/2 + r_p cos(2 pi t_q), y = 1/2 + r_p sin(2 pi t_q), r_p = (sqrt(2)/2) p / n_r,
    t_q = q / n_t, p = 1..n_r-1, q = 0..n_t-1, with n_r = n and n_t = ceil(beta n log2 n);
    points outside [0, 1)^2 are dropped.  Deterministic (no seed)."""
    nr = n
    nt = int(np.ceil(beta * n * np.log2(n)))
    r = (np.sqrt(2.0) / 2.0) * np.arange(1, nr, dtype=np.float64) / nr
    t = np.arange(nt, dtype=np.float64) / nt
    R, T = np.meshgrid(r, t, indexing="ij")
    x = np.concatenate([[0.5], (0.5 + R * np.cos(2 * np.pi * T)).ravel()])
    y = np.concatenate([[0.5], (0.5 + R * np.sin(2 * np.pi * T)).ravel()])
    keep = (x >= 0) & (x < 1) & (y >= 0) & (y < 1)
    return x[keep], y[keep]


def random_grid(M: int, seed: int):
    """M points drawn independently and uniformly from [0, 1)^2 (the paper's random grid)."""
    rng = _rng(seed)
    return rng.random(M), rng.random(M)
