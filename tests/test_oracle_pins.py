"""Pins for the CPU oracle: results the paper and the mathematics fix, checked
without any GPU.  Each test would fail on a plausible oracle mistake (a dropped
term, a reflected or transposed coefficient tensor, a wrong boundary rule, an
off-by-one in the time loop)."""
import ctypes
import itertools
import math
import os
import shutil
import subprocess
import zlib

import numpy as np
import pytest

import oracle
import stencil_inputs as si
import formulations as fm

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def int_problem(ndim, shape, r, kind, seed):
    """Integer field in [-8, 8] and integer C^g in [-3, 3] (star: zero off-axis);
    every sum the stencil forms stays exact in FP64 for a few steps."""
    rng = np.random.default_rng(seed)
    a = rng.integers(-8, 9, size=shape).astype(np.float64)
    c = rng.integers(-3, 4, size=(2 * r + 1,) * ndim).astype(np.float64)
    if kind == "star":
        c = np.where(si.star_mask(ndim, r), c, 0.0)
    # make sure the tensor is not symmetric in any axis so reflections show
    c.flat[0] = 3.0
    c.flat[-1] = -2.0
    return a, c


# ---------------------------------------------------------------- scatter == gather
@pytest.mark.parametrize("ndim,shape", [(2, (7, 9)), (2, (12, 11)), (3, (5, 6, 7))])
@pytest.mark.parametrize("r", [1, 2, 3])
@pytest.mark.parametrize("kind", ["star", "box"])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_gather_equals_scatter(ndim, shape, r, kind, bc):
    if ndim == 3 and r == 3 and bc == "periodic":
        pytest.skip("covered by the smaller radii; keeps the CPU suite short")
    a, c = int_problem(ndim, shape, r, kind, seed=zlib.crc32(repr((ndim, shape, r, kind, bc)).encode()))
    steps = 2
    got = oracle.gather(a, r, c, bc, steps)
    ref = fm.scatter(a, r, c, bc, steps)
    assert np.array_equal(got, ref)


# ---------------------------------------------------------------- Eq. (final)
@pytest.mark.parametrize("r", [1, 2, 3])
@pytest.mark.parametrize("n", [4, 8])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_gather_equals_final_formula_corrected(r, n, bc):
    a, c = int_problem(2, (2 * n, 3 * n), r, "box", seed=17 * r + n)
    got = oracle.gather(a, r, c, bc, 2)
    ref = fm.final_2d(a, r, c, bc, 2, n, corrected=True)
    assert np.array_equal(got, ref)


def test_final_formula_as_printed_needs_symmetric_columns():
    """The printed column pairing of Eq. (final) matches the gather definition
    only when C^g is left-right symmetric; with an asymmetric C^g it does not.
    This pins the reading recorded for the garbled pairing."""
    r, n = 1, 4
    a, c = int_problem(2, (8, 8), r, "box", seed=5)
    ref = oracle.gather(a, r, c, "periodic", 1)
    assert not np.array_equal(fm.final_2d(a, r, c, "periodic", 1, n, corrected=False), ref)
    cs = 0.5 * (c + c[:, ::-1])
    assert np.array_equal(fm.final_2d(a, r, cs, "periodic", 1, n, corrected=False),
                          oracle.gather(a, r, cs, "periodic", 1))


def test_worked_example_cls_r1():
    """The coefficient vectors of CLS(*,1) for r = 1 (Eq. (stencil-2d9p-scatter-
    extend-2)) are windows of column 1 of C^o, Eq. (co)/(final)."""
    rows = []
    with open(os.path.join(GOLDEN, "eq_scatter_extend2_r1.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    # symbolic C^g: entry (a, b) holds the code 10*a + b + 100 so 0 is free
    cg = np.array([[100 + 10 * a + b for b in range(3)] for a in range(3)], dtype=float)
    n = 3
    co = fm.coefficient_outer_matrix(fm.scatter_matrix(cg), n)
    for off_s, *vec in rows:
        off = int(off_s)
        # output rows i-1..i+1 form the output vector; the input row i+off is
        # row index (off + 2) of the local tile A_{0:n+2r}
        i = off + 2
        window = co[n + 2 - i - 1: 2 * n + 2 - i - 1, 1]
        want = [0.0 if v == "0" else 100 + 10 * int(v[0]) + int(v[1]) for v in vec]
        assert list(window) == want, (off, list(window), want)


# ---------------------------------------------------------------- Algorithm 1
@pytest.mark.parametrize("r,n,ui,uk,shape", [(1, 4, 2, 2, (4, 8, 8)), (2, 4, 2, 1, (4, 4, 8)),
                                              (1, 2, 4, 2, (4, 4, 8))])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_gather_equals_algorithm1(r, n, ui, uk, shape, bc):
    a, c = int_problem(3, shape, r, "box", seed=31 * r + n + ui)
    got = oracle.gather(a, r, c, bc, 2)
    ref = fm.algorithm1(a, r, c, bc, 2, n, ui, uk)
    assert np.array_equal(got, ref)


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("ndim,shape,r,kind", [(2, (9, 13), 2, "box"), (3, (6, 7, 5), 1, "box"),
                                               (2, (10, 10), 3, "star"), (3, (7, 7, 7), 2, "star")])
def test_constant_field_periodic(ndim, shape, r, kind):
    """Periodic A == c gives B == c * (sum C^g)^steps exactly (dyadic weights)."""
    rng = np.random.default_rng(ndim * 10 + r)
    cg = rng.integers(-8, 9, size=(2 * r + 1,) * ndim) / 16.0
    if kind == "star":
        cg = np.where(si.star_mask(ndim, r), cg, 0.0)
    s = cg.sum()
    a = np.full(shape, 3.0)
    for steps in (1, 3):
        got = oracle.gather(a, r, cg, "periodic", steps)
        assert np.all(got == 3.0 * s ** steps)


def test_constant_field_dirichlet_interior():
    """Dirichlet: the constant result holds exactly at points at least
    r*steps away from the boundary, and not next to it."""
    r, steps = 2, 3
    cg = np.full((5, 5), 1.0 / 32.0)
    a = np.full((20, 22), 2.0)
    got = oracle.gather(a, r, cg, "dirichlet", steps)
    inner = got[r * steps: -r * steps, r * steps: -r * steps]
    assert np.all(inner == 2.0 * (25 / 32.0) ** steps)
    assert got[0, 0] != 2.0 * (25 / 32.0) ** steps


@pytest.mark.parametrize("ndim,shape,r", [(2, (11, 9), 2), (3, (6, 5, 7), 1)])
def test_linearity(ndim, shape, r):
    a, c = int_problem(ndim, shape, r, "box", seed=1)
    b, _ = int_problem(ndim, shape, r, "box", seed=2)
    for bc in ("dirichlet", "periodic"):
        lhs = oracle.gather(0.5 * a - 3.0 * b, r, c, bc, 3)
        rhs = 0.5 * oracle.gather(a, r, c, bc, 3) - 3.0 * oracle.gather(b, r, c, bc, 3)
        assert np.array_equal(lhs, rhs)


def test_steps_compose_and_zero_steps():
    a, c = int_problem(2, (9, 8), 1, "box", seed=3)
    for bc in ("dirichlet", "periodic"):
        assert np.array_equal(oracle.gather(a, 1, c, bc, 0), a)
        two = oracle.gather(oracle.gather(a, 1, c, bc, 1), 1, c, bc, 1)
        assert np.array_equal(two, oracle.gather(a, 1, c, bc, 2))


# ---------------------------------------------------------------- polynomial fields
def _grid(shape):
    return np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")


def test_laplacian_quadratic_and_cubic_2d():
    lap = np.zeros((3, 3))
    lap[1, 1] = -4.0
    lap[0, 1] = lap[2, 1] = lap[1, 0] = lap[1, 2] = 1.0
    x, y = _grid((16, 18))
    got = oracle.gather(x ** 2 + y ** 2, 1, lap, "dirichlet", 1)
    assert np.all(got[1:-1, 1:-1] == 4.0)
    f = x ** 3 + 2 * y ** 3 + x * y ** 2
    got = oracle.gather(f, 1, lap, "dirichlet", 1)
    assert np.array_equal(got[1:-1, 1:-1], (6 * x + 12 * y + 2 * x)[1:-1, 1:-1])


def test_laplacian_quadratic_3d():
    lap = np.zeros((3, 3, 3))
    lap[1, 1, 1] = -6.0
    for ax in range(3):
        for t in (0, 2):
            idx = [1, 1, 1]
            idx[ax] = t
            lap[tuple(idx)] = 1.0
    x, y, z = _grid((8, 9, 10))
    got = oracle.gather(x ** 2 + y ** 2 + z ** 2, 1, lap, "dirichlet", 1)
    assert np.all(got[1:-1, 1:-1, 1:-1] == 6.0)


def test_jacobi_linear_and_quadratic():
    """The 2D 5-point Jacobi weights keep linear fields and map x^2 to x^2 + 1/4
    per step (exact away from the boundary)."""
    cg = si.coeffs_jacobi_2d5p()
    x, y = _grid((24, 24))
    steps = 3
    lin = 2.0 + 3.0 * x - 5.0 * y
    got = oracle.gather(lin, 1, cg, "dirichlet", steps)
    s = slice(steps, -steps)
    assert np.array_equal(got[s, s], lin[s, s])
    got = oracle.gather(x ** 2, 1, cg, "dirichlet", steps)
    assert np.array_equal(got[s, s], (x ** 2 + steps / 4.0)[s, s])


# ---------------------------------------------------------------- eigenmodes
@pytest.mark.parametrize("ndim,shape,r,m", [(2, (16, 20), 2, (1, 3)), (3, (8, 10, 12), 1, (1, 2, 1)),
                                            (2, (12, 12), 3, (2, 1))])
def test_periodic_fourier_mode(ndim, shape, r, m):
    """Periodic, any C^g: cos(theta.x) -> |lam|^T cos(theta.x + T arg lam) with
    lam = sum_o C^g[o] exp(i theta.(o - r))."""
    cg = si.coeffs_random(ndim, r, "box", seed=7 + ndim)
    theta = [2 * math.pi * mk / nk for mk, nk in zip(m, shape)]
    lam = 0j
    for o in itertools.product(range(2 * r + 1), repeat=ndim):
        lam += cg[o] * np.exp(1j * sum(t * (oi - r) for t, oi in zip(theta, o)))
    xs = _grid(shape)
    phase = sum(t * x for t, x in zip(theta, xs))
    T = 6
    got = oracle.gather(np.cos(phase), r, cg, "periodic", T)
    want = abs(lam) ** T * np.cos(phase + T * np.angle(lam))
    assert np.max(np.abs(got - want)) <= 1e-13 * max(1.0, abs(lam) ** T) * 10


@pytest.mark.parametrize("cg,shape,m", [(si.coeffs_jacobi_2d5p(), (20, 24), (1, 2)),
                                        (si.coeffs_symmetric_3d7p(), (10, 12, 9), (1, 1, 2)),
                                        (si.coeffs_separable_3d27p(), (9, 8, 11), (2, 1, 1))])
def test_dirichlet_sine_mode(cg, shape, m):
    """Dirichlet, r = 1, C^g symmetric in each axis: prod sin(pi m (x+1)/(N+1)) is
    an eigenvector with lam = sum_o C^g[o] prod cos(pi m (o-1)/(N+1))."""
    ndim = len(shape)
    phi = [math.pi * mk / (nk + 1) for mk, nk in zip(m, shape)]
    lam = 0.0
    for o in itertools.product(range(3), repeat=ndim):
        lam += cg[o] * np.prod([math.cos(p * (oi - 1)) for p, oi in zip(phi, o)])
    xs = _grid(shape)
    f = np.ones(shape)
    for p, x in zip(phi, xs):
        f = f * np.sin(p * (x + 1))
    T = 12
    got = oracle.gather(f, 1, cg, "dirichlet", T)
    assert np.max(np.abs(got - lam ** T * f)) <= 1e-13


# ---------------------------------------------------------------- sampling
@pytest.mark.parametrize("ndim,shape,r,bc,steps", [(2, (40, 37), 2, "periodic", 6),
                                                   (2, (33, 30), 1, "dirichlet", 9),
                                                   (3, (12, 11, 13), 1, "dirichlet", 4),
                                                   (3, (9, 10, 8), 1, "periodic", 7)])
def test_sample_matches_full_sweep_bitwise(ndim, shape, r, bc, steps):
    a = si.field_uniform(shape, 9)
    cg = si.coeffs_random(ndim, r, "box", 11)
    full = oracle.gather(a, r, cg, bc, steps)
    rng = np.random.default_rng(0)
    pts = np.stack([rng.integers(0, s, size=12) for s in shape], axis=1)
    pts[0] = 0
    pts[1] = np.array(shape) - 1
    vals = oracle.sample(a, r, cg, bc, steps, pts)
    assert np.array_equal(vals, full[tuple(pts.T)])


def test_rejects_bad_arguments():
    a = np.zeros((4, 4))
    with pytest.raises(ValueError):
        oracle.gather(a, 1, np.zeros((5, 5)), "dirichlet", 1)
    with pytest.raises(RuntimeError):
        oracle.gather(a, 1, np.zeros((3, 3)), "dirichlet", -1)


# ---------------------------------------------------------------- planted mistakes
_MUTATIONS = {
    "reflected offsets": ("y[d] = x[d] + o - r;", "y[d] = x[d] - o + r;"),
    "dropped last term": ("for (int64_t t = 0; t < nterm; ++t) {\n                /* o =",
                          "for (int64_t t = 0; t + 1 < nterm; ++t) {\n                /* o ="),
    "one step short": ("for (int64_t s = 0; s < steps; ++s) {", "for (int64_t s = 1; s < steps; ++s) {"),
    "periodic read as zero": ("            xi = wrap_index(xi, n[d]);\n        }\n        lin",
                              "            return 0.0;\n        }\n        lin"),
}


@pytest.mark.parametrize("name", sorted(_MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    """A copy of the oracle with one plausible mistake planted in it (on the
    CPU) fails the scatter-form pin."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = open(os.path.join(os.path.dirname(oracle.__file__), "stencil_oracle.c")).read()
    old, new = _MUTATIONS[name]
    assert old in src, name
    mutated = tmp_path / "mut.c"
    mutated.write_text(src.replace(old, new, 1))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so), str(mutated)],
                   check=True)
    lib = ctypes.CDLL(str(so))
    a, c = int_problem(2, (9, 10), 2, "box", seed=99)
    shape = np.array(a.shape, dtype=np.int64)
    out = np.empty_like(a)
    dp = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    lib.oracle_gather(2, shape.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 2, dp(c), 1,
                      ctypes.c_int64(2), dp(a), dp(out))
    assert not np.array_equal(out, fm.scatter(a, 2, c, "periodic", 2))


# ---------------------------------------------------------------- minimal line cover (Sec. 3.5)
def _covers(mask, rows, cols):
    m = np.asarray(mask) != 0
    return all(rows[i] or cols[j] for i, j in zip(*np.nonzero(m)))


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_min_line_cover_box_and_star(r):
    """Table cls-2d: a box needs all 2r+1 lines; a star two (its row and column)."""
    n = 2 * r + 1
    count, rows, cols = oracle.min_line_cover(np.ones((n, n)))
    assert count == n and _covers(np.ones((n, n)), rows, cols)
    star = np.zeros((n, n))
    star[r, :] = 1
    star[:, r] = 1
    count, rows, cols = oracle.min_line_cover(star)
    assert count == 2 and rows[r] and cols[r] and rows.sum() == 1 and cols.sum() == 1


def test_min_line_cover_special_cases():
    assert oracle.min_line_cover(np.zeros((5, 5)))[0] == 0
    one = np.zeros((5, 5))
    one[3, 1] = 1
    assert oracle.min_line_cover(one)[0] == 1
    # no two weights share a line: one line per weight
    perm = np.eye(7)[[3, 0, 6, 2, 5, 1, 4]]
    assert oracle.min_line_cover(perm)[0] == 7
    # a full row plus one weight elsewhere: the row and one more line
    m = np.zeros((5, 5))
    m[2, :] = 1
    m[4, 0] = 1
    assert oracle.min_line_cover(m)[0] == 2


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("density", [0.2, 0.5, 0.8])
def test_min_line_cover_konig(n, density):
    """Konig's theorem: the minimum line cover has as many lines as the largest
    set of weights with no two in one row or column (brute force over
    permutations), and the returned lines cover every weight."""
    for seed in range(6):
        mask = si.uniform(1000 * n + seed + int(100 * density), n * n).reshape(n, n) < density
        count, rows, cols = oracle.min_line_cover(mask)
        assert _covers(mask, rows, cols) and count == rows.sum() + cols.sum()
        matching = max(sum(bool(mask[i, p[i]]) for i in range(n)) for p in itertools.permutations(range(n)))
        assert count == matching
