"""CPU checks of the boundary decomposition the tensor-core path relies on
(no GPU): a periodic sweep equals the sweep that sees zeros outside the grid
in x and y (and, in 3D, wraps whole planes in z), plus the wrapped terms of
the points within r of an x or y face.

The tensor-core kernels compute the first part (TMA's zero fill; the 3D
producer wraps the plane index) and the boundary-strip kernel adds the
second, enumerating its points as rows within r of a y face in full and the
2r edge columns of every other row.  These tests restate that enumeration
and term rule in numpy and hold their sum to the oracle's periodic sweep, on
grids down to the smallest extent a plan takes (2r + 1), where a point's
halo reaches across both faces.  A plausible mistake in the rule (a missed
corner term, a term counted in both the y and the x pass, a strip one row
too narrow) fails them."""
import numpy as np
import pytest

import oracle
import stencil_inputs as si


def strip_points(ny, nx, r):
    """(y, x) of the boundary strips, each once."""
    pts = []
    for y in range(ny):
        if y < r or y >= ny - r:
            pts.extend((y, x) for x in range(nx))
        else:
            xs = sorted({x for x in list(range(min(r, nx))) + list(range(max(nx - r, 0), nx))})
            pts.extend((y, x) for x in xs)
    return pts


def wrapped_terms(a, r, cg):
    """The boundary-strip kernel's sum: for every strip point, the terms whose
    neighbour leaves the grid in y or x, read at wrapped indices."""
    a3 = a if a.ndim == 3 else a[None]
    c3 = cg if cg.ndim == 3 else cg[None]
    nz, ny, nx = a3.shape
    rz = r if a.ndim == 3 else 0
    out = np.zeros_like(a3)
    for z in range(nz):
        for (y, x) in strip_points(ny, nx, r):
            s = 0.0
            for dz in range(-rz, rz + 1):
                for dy in range(-r, r + 1):
                    for dx in range(-r, r + 1):
                        w = c3[dz + rz, dy + r, dx + r]
                        yy, xx = y + dy, x + dx
                        if w == 0.0 or (0 <= yy < ny and 0 <= xx < nx):
                            continue
                        s += w * a3[(z + dz) % nz, yy % ny, xx % nx]
            out[z, y, x] = s
    return out if a.ndim == 3 else out[0]


def zero_xy_sweep(a, r, cg):
    """One sweep that reads zeros outside the grid in x and y and wraps z
    (the plane index) when 3D: the part the tensor-core kernels compute."""
    a3 = a if a.ndim == 3 else a[None]
    c3 = cg if cg.ndim == 3 else cg[None]
    rz = r if a.ndim == 3 else 0
    nz, ny, nx = a3.shape
    pad = np.zeros((nz, ny + 2 * r, nx + 2 * r))
    pad[:, r:r + ny, r:r + nx] = a3
    out = np.zeros_like(a3)
    for dz in range(-rz, rz + 1):
        plane = np.roll(pad, -dz, axis=0)   # plane z + dz, wrapped
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                w = c3[dz + rz, dy + r, dx + r]
                if w != 0.0:
                    out += w * plane[:, r + dy:r + dy + ny, r + dx:r + dx + nx]
    return out if a.ndim == 3 else out[0]


@pytest.mark.parametrize("r", [1, 2, 3, 4])
@pytest.mark.parametrize("kind", ["star", "box"])
@pytest.mark.parametrize("shape", [(23, 17), "min-y", "min-x", "min-both"])
def test_2d_periodic_is_zero_fill_plus_strip_terms(r, kind, shape):
    m = 2 * r + 1
    shape = {"min-y": (m, 13), "min-x": (11, m), "min-both": (m, m)}.get(shape, shape)
    cg = si.coeffs_random(2, r, kind, 300 + r)
    a = si.field_uniform(shape, 301 + r, -1.0, 1.0)
    # the zero-fill part is the oracle's Dirichlet sweep in 2D
    zero = oracle.gather(a, r, cg, "dirichlet", 1)
    assert np.allclose(zero, zero_xy_sweep(a, r, cg), rtol=0, atol=1e-13)
    got = zero + wrapped_terms(a, r, cg)
    want = oracle.gather(a, r, cg, "periodic", 1)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("r,kind", [(1, "star"), (1, "box"), (2, "box"), (3, "star")])
@pytest.mark.parametrize("shape", [(6, 9, 11), "min"])
def test_3d_periodic_is_zwrapped_zero_fill_plus_strip_terms(r, kind, shape):
    m = 2 * r + 1
    shape = (m, m, m) if shape == "min" else shape
    if min(shape) < m:
        pytest.skip("below the minimum extent")
    cg = si.coeffs_random(3, r, kind, 310 + r)
    a = si.field_uniform(shape, 311 + r, -1.0, 1.0)
    got = zero_xy_sweep(a, r, cg) + wrapped_terms(a, r, cg)
    want = oracle.gather(a, r, cg, "periodic", 1)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


def test_points_off_the_strips_need_no_wrapped_term():
    """Every point whose periodic and zero-fill values differ lies in a strip."""
    r = 2
    cg = si.coeffs_random(2, r, "box", 320)
    a = si.field_uniform((30, 26), 321, -1.0, 1.0)
    diff = np.abs(oracle.gather(a, r, cg, "periodic", 1) - oracle.gather(a, r, cg, "dirichlet", 1)) > 0
    strips = np.zeros_like(diff)
    for (y, x) in strip_points(*a.shape, r):
        strips[y, x] = True
    assert not np.any(diff & ~strips)
    assert np.all(diff[strips])   # random weights: every strip point has a wrapped term
