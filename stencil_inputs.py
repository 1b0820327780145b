"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no stencil arithmetic: it only draws grids, coefficient
tensors and workload lists from a counter-based generator, so that the oracle
and the GPU library see exactly the same problem.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  Element i of the stream for a seed is the
SplitMix64 finaliser applied to ``seed + (i + 1) * 0x9E3779B97F4A7C15``
(mod 2^64); uniform[0,1) is ``(x >> 11) * 2^-53`` and uniform[lo,hi) is
``lo + (hi - lo) * u``.  Grids are filled in C order over the interior points.

Problem conventions (the paper's statement of the problem, Sec. 2.2 and the
footnote of Sec. 4.1): arrays are C-ordered with the last index contiguous;
``shape`` lists the interior (updated) points; the coefficient tensor is the
gather-mode matrix C^g of Eq. (stencil-2d9p-cm), side 2r+1 per dimension,
where r is the stencil order (radius).  A star stencil is a box whose
off-axis entries are zero (Sec. 3.3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STAR = "star"
BOX = "box"
DIRICHLET = "dirichlet"
PERIODIC = "periodic"


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Elements offset..offset+n-1 of the SplitMix64 stream for ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0, offset: int = 0) -> np.ndarray:
    """n doubles uniform in [lo, hi) from the SplitMix64 stream."""
    u = (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    if lo == 0.0 and hi == 1.0:
        return u
    return lo + (hi - lo) * u


def field_uniform(shape: Sequence[int], seed: int, lo: float = 0.0, hi: float = 1.0,
                  chunk: int = 1 << 24) -> np.ndarray:
    """A float64 grid of the given shape, uniform[lo,hi), C order."""
    n = int(np.prod(shape))
    out = np.empty(n, dtype=np.float64)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        out[s:s + m] = uniform(seed, m, lo, hi, offset=s)
    return out.reshape(tuple(shape))


def round_to(x: np.ndarray, dtype: str) -> np.ndarray:
    """Round a float64 array to the storage dtype ('f32'|'f64') and back to float64.

    The oracle is given exactly the values the GPU stores, so a comparison
    measures the GPU arithmetic only, not input quantisation.
    """
    if dtype == "f32":
        return x.astype(np.float32).astype(np.float64)
    if dtype == "f64":
        return np.asarray(x, dtype=np.float64)
    raise ValueError(dtype)


def star_mask(ndim: int, r: int) -> np.ndarray:
    """Boolean (2r+1)^ndim mask of the on-axis (star) positions."""
    w = 2 * r + 1
    m = np.zeros((w,) * ndim, dtype=bool)
    for ax in range(ndim):
        idx = [r] * ndim
        for t in range(w):
            idx[ax] = t
            m[tuple(idx)] = True
    return m


def coeffs_random(ndim: int, r: int, kind: str, seed: int, normalise: bool = True,
                  dtype: str = "f64") -> np.ndarray:
    """C^g with entries uniform[0,1) (zero off-axis for a star), optionally
    normalised to sum 1 in float64, then rounded to the storage dtype."""
    w = 2 * r + 1
    c = uniform(seed, w ** ndim).reshape((w,) * ndim)
    if kind == STAR:
        c = np.where(star_mask(ndim, r), c, 0.0)
    elif kind != BOX:
        raise ValueError(kind)
    if normalise:
        c = c / c.sum()
    return round_to(c, dtype)


def coeffs_jacobi_2d5p() -> np.ndarray:
    """2D 5-point star Jacobi weights: centre 0.5, four axis neighbours 0.125."""
    c = np.zeros((3, 3))
    c[1, 1] = 0.5
    c[0, 1] = c[2, 1] = c[1, 0] = c[1, 2] = 0.125
    return c


def coeffs_symmetric_3d7p() -> np.ndarray:
    """3D 7-point star: centre 0.4, six axis neighbours 0.1."""
    c = np.zeros((3, 3, 3))
    c[1, 1, 1] = 0.4
    for ax in range(3):
        for t in (0, 2):
            idx = [1, 1, 1]
            idx[ax] = t
            c[tuple(idx)] = 0.1
    return c


def coeffs_separable_3d27p() -> np.ndarray:
    """3D 27-point box: outer product (1/4, 1/2, 1/4)^(x3)."""
    v = np.array([0.25, 0.5, 0.25])
    return np.einsum("i,j,k->ijk", v, v, v)


# ---------------------------------------------------------------------------
# Workloads.  Each is a seeded recipe; sizes follow the paper's synthetic grid
# experiments scaled to GB300 memory (box/star, r = 1..3, 2D and 3D).
# ---------------------------------------------------------------------------

@dataclass
class Problem:
    ndim: int
    shape: tuple
    r: int
    kind: str
    coeffs: np.ndarray          # dense C^g, float64 (already rounded to dtype)
    dtype: str                  # 'f32' | 'f64'
    bc: str                     # 'dirichlet' | 'periodic'
    steps: int
    field_seed: int
    field_lo: float = 0.0
    field_hi: float = 1.0
    name: str = ""
    field_kind: str = "uniform"   # 'uniform' (seeded) | 'sine' (lowest Dirichlet mode)

    def field(self) -> np.ndarray:
        if self.field_kind == "sine":
            return round_to(sine_mode(self.shape), self.dtype)
        return round_to(field_uniform(self.shape, self.field_seed, self.field_lo, self.field_hi),
                        self.dtype)

    @property
    def points(self) -> int:
        return int(np.prod(self.shape))

    @property
    def updates(self) -> int:
        return self.points * self.steps


def sine_mode(shape: Sequence[int]) -> np.ndarray:
    """prod_k sin(pi (x_k + 1) / (n_k + 1)): the lowest mode of the zero-Dirichlet
    grid of the given interior shape."""
    f = np.ones(tuple(shape))
    for k, n in enumerate(shape):
        s = np.sin(np.pi * (np.arange(n, dtype=np.float64) + 1) / (n + 1))
        f = f * s.reshape([n if j == k else 1 for j in range(len(shape))])
    return f


def sine_cube_512(kind: str, steps: int = 1000, side: int = 512) -> Problem:
    """Long FP64 run: 512^3, 7-point star (centre 0.4, neighbours 0.1) or
    27-point separable box ((1/4, 1/2, 1/4)^3), zero Dirichlet, started from
    the lowest sine mode, so the exact result is a known multiple of it."""
    cg = coeffs_symmetric_3d7p() if kind == STAR else coeffs_separable_3d27p()
    return Problem(3, (side,) * 3, 1, kind, cg, "f64", DIRICHLET, steps, 0, field_kind="sine",
                   name=f"3d{'7p' if kind == STAR else '27p'}-sine-{side}-f64")


def jacobi_256(steps: int = 10) -> Problem:
    """2D 5-point star Jacobi, 256x256 FP64, zero Dirichlet halo, 10 steps."""
    return Problem(2, (256, 256), 1, STAR, coeffs_jacobi_2d5p(), "f64", DIRICHLET, steps, 1,
                   name="2d5p-jacobi-256-f64")


def box25_8192(dtype: str = "f32", steps: int = 100, side: int = 8192) -> Problem:
    """2D radius-2 box (25 point), side^2, uniform[0,1) coefficients normalised
    to sum 1, periodic, 100 steps."""
    return Problem(2, (side, side), 2, BOX, coeffs_random(2, 2, BOX, 102, dtype=dtype), dtype,
                   PERIODIC, steps, 2, name=f"2d25p-box-{side}-{dtype}")


def cube_512(kind: str, dtype: str = "f32", steps: int = 50, side: int = 512, r: int = 1) -> Problem:
    """3D star or box of order r (7-point star and 27-point box at r = 1),
    side^3, interior uniform[-1,1), zero Dirichlet halo, random normalised
    coefficients (seed 103)."""
    points = 6 * r + 1 if kind == STAR else (2 * r + 1) ** 3
    return Problem(3, (side,) * 3, r, kind, coeffs_random(3, r, kind, 103, dtype=dtype), dtype,
                   DIRICHLET, steps, 3, -1.0, 1.0, name=f"3d{points}p-{side}-{dtype}")


def batch_1024(n: int = 1024, seed: int = 4, lo: int = 64, hi: int = 2048,
               steps_lo: int = 20, steps_hi: int = 200) -> List[Problem]:
    """Independent 2D 9-point box problems: Ny, Nx log-uniform in [lo, hi]
    (rounded to int), steps uniform in {steps_lo..steps_hi}, random normalised
    3x3 coefficients, uniform[0,1) fields, FP32, zero Dirichlet."""
    u = uniform(seed, 4 * n).reshape(n, 4)
    out = []
    for i in range(n):
        ny = int(round(math.exp(math.log(lo) + u[i, 0] * (math.log(hi) - math.log(lo)))))
        nx = int(round(math.exp(math.log(lo) + u[i, 1] * (math.log(hi) - math.log(lo)))))
        st = steps_lo + int(u[i, 2] * (steps_hi - steps_lo + 1))
        cseed = seed * 1_000_003 + 2 * i + 1
        fseed = seed * 1_000_003 + 2 * i + 2
        out.append(Problem(2, (ny, nx), 1, BOX, coeffs_random(2, 1, BOX, cseed, dtype="f32"),
                           "f32", DIRICHLET, st, fseed, name=f"batch{i}"))
    return out


@dataclass
class Request:
    arrival_s: float
    problem: Problem


def serving_stream(n: int = 2000, rate_per_s: float = 10.0, seed: int = 5,
                   scale: float = 1.0) -> List[Request]:
    """Poisson arrivals of mixed stencil solves: 70% 2D (side log-uniform in
    [128, 4096], r uniform in {1,2,3}, star|box 50/50), 30% 3D (side
    log-uniform in [64, 384], 7- or 27-point), FP32 with 10% FP64, steps
    uniform in {10..500}, random normalised coefficients, zero Dirichlet.
    ``scale`` shrinks every side (for tests)."""
    u = uniform(seed, 8 * n).reshape(n, 8)
    t = 0.0
    out = []
    for i in range(n):
        t += -math.log(1.0 - u[i, 0]) / rate_per_s
        dtype = "f64" if u[i, 1] < 0.1 else "f32"
        steps = 10 + int(u[i, 2] * 491)
        cseed = seed * 7_000_001 + 2 * i + 1
        fseed = seed * 7_000_001 + 2 * i + 2
        if u[i, 3] < 0.7:
            side = int(round(math.exp(math.log(128) + u[i, 4] * (math.log(4096) - math.log(128)))))
            side = max(16, int(side * scale))
            r = 1 + int(u[i, 5] * 3)
            kind = STAR if u[i, 6] < 0.5 else BOX
            p = Problem(2, (side, side), r, kind, coeffs_random(2, r, kind, cseed, dtype=dtype),
                        dtype, DIRICHLET, steps, fseed, name=f"req{i}")
        else:
            side = int(round(math.exp(math.log(64) + u[i, 4] * (math.log(384) - math.log(64)))))
            side = max(8, int(side * scale))
            kind = STAR if u[i, 6] < 0.5 else BOX
            p = Problem(3, (side,) * 3, 1, kind, coeffs_random(3, 1, kind, cseed, dtype=dtype),
                        dtype, DIRICHLET, steps, fseed, name=f"req{i}")
        out.append(Request(t, p))
    return out
