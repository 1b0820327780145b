"""GPU parity of the CUDA-core gather kernel against the FP64 oracle (through
the C ABI).  Small odd shapes span several tiles plus ragged tails."""
import numpy as np
import pytest

import oracle
import paper_2310_16298_gb300 as sx
import stencil_inputs as si
from gpuutil import TOL, check, run

pytestmark = pytest.mark.gpu


def problem(ndim, shape, r, kind, dtype, seed):
    cg = si.coeffs_random(ndim, r, kind, 100 + seed, dtype=dtype)
    a = si.round_to(si.field_uniform(shape, seed, -1.0, 1.0), dtype)
    return a, cg


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("kind", ["star", "box"])
@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_gather_2d(dtype, bc, kind, r):
    shape = (37 + r, 53 + 2 * r) if r != 2 else (70, 300)
    a, cg = problem(2, shape, r, kind, dtype, seed=r)
    steps = 5
    got, info = run(a, r, kind, cg, dtype, bc, steps, impl="gather")
    assert info["impl"] == 1
    check(got, oracle.gather(a, r, cg, bc, steps), TOL[dtype], f"2d r={r} {kind} {bc} {dtype}")


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("kind", ["star", "box"])
@pytest.mark.parametrize("r", [1, 2, 3])
def test_gather_3d(dtype, bc, kind, r):
    shape = (19, 23, 29 + r) if r < 3 else (13, 40, 35)
    a, cg = problem(3, shape, r, kind, dtype, seed=10 + r)
    steps = 3
    got, _ = run(a, r, kind, cg, dtype, bc, steps, impl="gather")
    check(got, oracle.gather(a, r, cg, bc, steps), TOL[dtype], f"3d r={r} {kind} {bc} {dtype}")


@pytest.mark.parametrize("ndim,shape,r,dtype", [(2, (67, 141), 2, "f64"), (2, (40, 33), 1, "f64"),
                                                (3, (21, 18, 37), 1, "f64"), (3, (12, 12, 40), 2, "f32")])
@pytest.mark.parametrize("tb", [2, 3, 4])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_gather_temporal_blocking(ndim, shape, r, dtype, tb, bc):
    a, cg = problem(ndim, shape, r, "box", dtype, seed=tb)
    steps = 7  # not a multiple of tb: exercises the shorter last sweep
    try:
        got, info = run(a, r, "box", cg, dtype, bc, steps, impl="gather", tb=tb)
    except sx.StencilError as e:
        # a halo of r*tb that does not fit shared memory is refused at plan time
        assert e.status == sx.EUNSUPPORTED and ndim == 3, str(e)
        pytest.skip(str(e))
    assert info["tb"] == tb
    check(got, oracle.gather(a, r, cg, bc, steps), TOL[dtype], f"tb={tb}")


def test_gather_split_runs_bitwise():
    """apply(k) then apply(T-k) equals apply(T) bit for bit (checkpoint/resume)."""
    a, cg = problem(2, (90, 130), 2, "box", "f32", seed=3)
    full, _ = run(a, 2, "box", cg, "f32", "periodic", 9, tb=2)
    part, _ = run(a, 2, "box", cg, "f32", "periodic", 4, tb=2)
    rest, _ = run(part, 2, "box", cg, "f32", "periodic", 5, tb=2)
    assert np.array_equal(full, rest)


@pytest.mark.parametrize("steps", [1, 2, 3])
def test_gather_in_place(steps):
    a, cg = problem(2, (50, 70), 1, "box", "f64", seed=4)
    got, _ = run(a, 1, "box", cg, "f64", "dirichlet", steps, alias=True, check_guard=False)
    check(got, oracle.gather(a, 1, cg, "dirichlet", steps), 1e-12)


def test_gather_zero_steps_copies():
    a, cg = problem(2, (20, 24), 1, "star", "f32", seed=5)
    got, _ = run(a, 1, "star", cg, "f32", "dirichlet", 0)
    assert np.array_equal(got, a)


def test_gather_minimum_extent():
    """Every extent exactly 2r+1 (the smallest valid problem)."""
    for ndim, r in ((2, 3), (3, 1), (3, 2)):
        shape = (2 * r + 1,) * ndim
        a, cg = problem(ndim, shape, r, "box", "f64", seed=6)
        for bc in ("dirichlet", "periodic"):
            got, _ = run(a, r, "box", cg, "f64", bc, 4)
            check(got, oracle.gather(a, r, cg, bc, 4), 1e-12, f"min extent {ndim}d r={r} {bc}")


def test_jacobi_256_f64_10_steps():
    """2D 5-point Jacobi, 256^2 FP64, zero Dirichlet halo, 10 steps: <= 1e-12."""
    p = si.jacobi_256()
    a = p.field()
    got, _ = run(a, 1, "star", p.coeffs, "f64", "dirichlet", 10)
    check(got, oracle.gather(a, 1, p.coeffs, "dirichlet", 10), 1e-12, "jacobi 256")


def test_dirichlet_sine_mode_long_run_f64():
    """FP64, 1000 steps of a symmetric 3D 7-point stencil on a sine eigenmode:
    the result is lam^T times the mode (closed form)."""
    shape = (48, 40, 56)
    m = (1, 1, 1)
    cg = si.coeffs_symmetric_3d7p()
    phi = [np.pi * mk / (nk + 1) for mk, nk in zip(m, shape)]
    lam = sum(cg[o] * np.prod([np.cos(p * (oi - 1)) for p, oi in zip(phi, o)])
              for o in np.ndindex(3, 3, 3))
    xs = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
    f = np.ones(shape)
    for p, x in zip(phi, xs):
        f = f * np.sin(p * (x + 1))
    T = 1000
    got, _ = run(f, 1, "star", cg, "f64", "dirichlet", T, tb=2)
    check(got, lam ** T * f, 1e-12, "sine mode 1000 steps")
