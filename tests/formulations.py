"""Independent restatements of the paper's other formulations, for pinning the
oracle on tiny integer grids (exact in FP64).

Each function is written from the paper's equations, not from the oracle, and
works on a field padded by the boundary rule (``pad``) so the formulation
itself only ever sees interior arithmetic:

* ``scatter``     -- Eq. (stencil-2d9p-scatter) with C^s = J C^g J,
                     Eq. (stencil-2d9p-gm2sm): every input point scatters
                     C^s * A[x] into its (2r+1)^d output neighbourhood.
* ``final_2d``    -- Eq. (final): per n x n output tile, the sum over the 2r+1
                     columns of C^o (Eq. (co)) and the n+2r input rows of
                     coefficient-window (outer) input-row products.  The
                     printed column pairing is only right for left-right
                     symmetric C^g; ``corrected=True`` pairs C^o column j with
                     input columns starting at 2r-j (see the readings of the
                     paper in the design notes).
* ``algorithm1``  -- the blocked 3D update of Sec. 3.4 / Algorithm 1 (box):
                     groups of ui x uk n x n subblocks, each the sum over the
                     (z, x) offsets of a banded coefficient matrix times the
                     shifted input rows (a sum of outer products), written as
                     matrix algebra rather than in the listing's loop order.
"""
from __future__ import annotations

import numpy as np


def pad(a: np.ndarray, r: int, bc: str) -> np.ndarray:
    """Field with a halo of width r filled by the boundary rule."""
    if bc == "dirichlet":
        return np.pad(a, r, mode="constant", constant_values=0.0)
    if bc == "periodic":
        return np.pad(a, r, mode="wrap")
    raise ValueError(bc)


def reversal(n: int) -> np.ndarray:
    """J_n, Eq. (stencil-2d9p-jmatrix): ones on the anti-diagonal."""
    return np.fliplr(np.eye(n))


def scatter_matrix(cg: np.ndarray) -> np.ndarray:
    """C^s = J C^g J for d = 2 (Eq. (stencil-2d9p-gm2sm)); for d = 3 the same
    reversal applied along every axis."""
    if cg.ndim == 2:
        J = reversal(cg.shape[0])
        return J @ cg @ J
    return cg[::-1, ::-1, ::-1].copy()


def scatter(a: np.ndarray, r: int, cg: np.ndarray, bc: str, steps: int) -> np.ndarray:
    cs = scatter_matrix(cg)
    for _ in range(steps):
        p = pad(a, r, bc)
        # Output is accumulated on the interior; contributions landing in the
        # halo are dropped (the halo is not updated).
        b = np.zeros_like(a)
        bp = np.zeros(tuple(s + 2 * r for s in a.shape))
        for x in np.ndindex(*p.shape):
            v = p[x]
            if v == 0.0:
                continue
            # A[x] is scattered to B[x + (o - r)] with weight C^s[o]
            lo = [max(0, xi - r) for xi in x]
            hi = [min(bs, xi + r + 1) for xi, bs in zip(x, bp.shape)]
            cs_sl = tuple(slice(l - (xi - r), h - (xi - r)) for l, h, xi in zip(lo, hi, x))
            bp[tuple(slice(l, h) for l, h in zip(lo, hi))] += cs[cs_sl] * v
        b[...] = bp[tuple(slice(r, r + s) for s in a.shape)]
        a = b
    return a


def coefficient_outer_matrix(cs: np.ndarray, n: int) -> np.ndarray:
    """C^o of Eq. (co): C^s with (n-1) zero rows above and below."""
    w = cs.shape[1]
    z = np.zeros((n - 1, w))
    return np.vstack([z, cs, z])


def final_2d(a: np.ndarray, r: int, cg: np.ndarray, bc: str, steps: int, n: int,
             corrected: bool = True) -> np.ndarray:
    """Eq. (final) applied to every n x n output tile (the grid sides must be
    multiples of n)."""
    ny, nx = a.shape
    assert ny % n == 0 and nx % n == 0
    co = coefficient_outer_matrix(scatter_matrix(cg), n)
    for _ in range(steps):
        p = pad(a, r, bc)
        b = np.empty_like(a)
        for ty in range(0, ny, n):
            for tx in range(0, nx, n):
                # Local input tile A_{0:n+2r, 0:n+2r}; output B_{r:r+n, r:r+n}.
                t = p[ty:ty + n + 2 * r, tx:tx + n + 2 * r]
                acc = np.zeros((n, n))
                for j in range(2 * r + 1):
                    c0 = (2 * r - j) if corrected else j
                    for i in range(n + 2 * r):
                        cvec = co[n + 2 * r - i - 1: 2 * n + 2 * r - i - 1, j]
                        acc += np.outer(cvec, t[i, c0:c0 + n])
                b[ty:ty + n, tx:tx + n] = acc
        a = b
    return a


def banded_coefficients(cg: np.ndarray, a: int, c: int, n: int) -> np.ndarray:
    """The n x (n + 2r) coefficient matrix of one (z offset a, x offset c)
    pair: column j' holds the coefficient vector that input row j' of a
    subblock's slab scatters to the n output rows (output row jj receives
    input row jj + b with weight C^g[a, b, c], b = 0..2r)."""
    w = cg.shape[0]
    v = np.zeros((n, n + w - 1))
    for b in range(w):
        v[np.arange(n), np.arange(n) + b] = cg[a, b, c]
    return v


def algorithm1(a: np.ndarray, r: int, cg: np.ndarray, bc: str, steps: int, n: int,
               ui: int, uk: int) -> np.ndarray:
    """The blocked 3D update of Sec. 3.4 and Algorithm 1, restated as matrix
    algebra: the output is cut into groups of ui planes x n rows x uk n-wide
    column subblocks; each n x n subblock of output plane i is the sum, over
    the z offsets a and x offsets c, of the banded coefficient matrix of (a, c)
    times the n + 2r input rows of plane i + a - r shifted by c - r columns,
    i.e. a sum of (coefficient vector) x (input row vector) outer products.
    The grid sides must be multiples of (ui, n, uk n)."""
    nz, ny, nx = a.shape
    assert nz % ui == 0 and ny % n == 0 and nx % (uk * n) == 0
    w = 2 * r + 1
    vs = {(za, xc): banded_coefficients(cg, za, xc, n) for za in range(w) for xc in range(w)}
    for _ in range(steps):
        p = pad(a, r, bc)
        b = np.empty_like(a)
        for i0 in range(0, nz, ui):
            for j0 in range(0, ny, n):
                for k0 in range(0, nx, uk * n):
                    # padded input slab of the group: planes i0-r .., rows j0-r .., columns k0-r ..
                    slab = p[i0:i0 + ui + 2 * r, j0:j0 + n + 2 * r, k0:k0 + uk * n + 2 * r]
                    for i in range(ui):
                        for k in range(uk):
                            bm = np.zeros((n, n))
                            for za in range(w):
                                for xc in range(w):
                                    rows = slab[i + za, :, k * n + xc: k * n + xc + n]
                                    bm += vs[za, xc] @ rows
                            b[i0 + i, j0:j0 + n, k0 + k * n: k0 + (k + 1) * n] = bm
        a = b
    return a
