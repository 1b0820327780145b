"""GPU parity of the matrixized (tcgen05 outer-product) kernel against the
FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
import stencil_inputs as si
from gpuutil import TOL, check, run

pytestmark = pytest.mark.gpu


def problem(ndim, shape, r, kind, seed, lo=-1.0, hi=1.0):
    cg = si.coeffs_random(ndim, r, kind, 200 + seed, dtype="f32")
    a = si.round_to(si.field_uniform(shape, seed, lo, hi), "f32")
    return a, cg


@pytest.mark.parametrize("prec", ["tf32x3", "tf32", "bf16x3", "bf16x2", "bf16", "bf16w2"])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("kind", ["box", "star"])
@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_mx_2d(prec, bc, kind, r):
    shape = (300 + r, 196 + 4 * r)  # several tiles in both axes plus ragged tails
    a, cg = problem(2, shape, r, kind, seed=r)
    steps = 3
    got, info = run(a, r, kind, cg, "f32", bc, steps, impl="matrixized", prec=prec)
    assert info["impl"] == 2 and info["device_error"] == 0
    check(got, oracle.gather(a, r, cg, bc, steps), TOL[prec], f"mx 2d r={r} {kind} {bc} {prec}")


@pytest.mark.parametrize("shape", [(5, 8), (37, 20), (129, 68), (128, 64), (256, 128), (130, 4 * 33)])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_mx_2d_shapes(shape, bc):
    r = 2
    if min(shape) < 2 * r + 1:
        pytest.skip("below the minimum extent")
    a, cg = problem(2, shape, r, "box", seed=sum(shape))
    got, info = run(a, r, "box", cg, "f32", bc, 4, impl="matrixized", prec="tf32x3")
    assert info["device_error"] == 0
    check(got, oracle.gather(a, r, cg, bc, 4), 1e-5, f"mx shape {shape} {bc}")


@pytest.mark.parametrize("shape,r,kind", [((3, 64), 1, "box"), ((5, 40), 2, "box"), ((9, 300), 4, "star"),
                                          ((130, 5), 2, "box"), ((7, 7), 3, "box"), ((300, 9), 4, "box")])
def test_mx_2d_periodic_at_the_minimum_extent(shape, r, kind):
    """Extents of 2r + 1 (the smallest a plan takes): the periodic halo of
    every point wraps across both faces, which the boundary-term kernel adds
    (the tensor-core kernel reads zeros outside the grid)."""
    a, cg = problem(2, shape, r, kind, seed=sum(shape) + r)
    got, info = run(a, r, kind, cg, "f32", "periodic", 3, impl="matrixized", prec="tf32x3")
    assert info["impl"] == 2 and info["kernels_per_sweep"] == 2 and info["device_error"] == 0
    check(got, oracle.gather(a, r, cg, "periodic", 3), 1e-5, f"mx small periodic {shape} r={r}")


@pytest.mark.parametrize("shape,r,kind,cover", [((3, 3, 64), 1, "box", "auto"), ((3, 40, 3), 1, "star", "hybrid"),
                                                ((7, 7, 70), 3, "star", "parallel")])
def test_mx_3d_periodic_at_the_minimum_extent(shape, r, kind, cover):
    a, cg = problem(3, shape, r, kind, seed=sum(shape) + 7 * r)
    got, info = run(a, r, kind, cg, "f32", "periodic", 3, impl="matrixized", prec="tf32x3", cover=cover)
    assert info["impl"] == 2 and info["kernels_per_sweep"] == 2 and info["device_error"] == 0
    check(got, oracle.gather(a, r, cg, "periodic", 3), 1e-5, f"mx 3d small periodic {shape} r={r}")


@pytest.mark.parametrize("ndim,kind", [(2, "box"), (3, "star")])
def test_kernels_per_sweep(ndim, kind):
    """One kernel per sweep, plus the boundary-term kernel for periodic
    matrixized plans; a stencil with no off-centre weight in x or y (pure z
    line, 3D) needs no boundary terms."""
    import paper_2310_16298_gb300 as sx
    shape = (64, 64) if ndim == 2 else (16, 32, 64)
    cg = si.coeffs_random(ndim, 1, kind, 5, dtype="f32")
    for impl, bc, want in [("matrixized", "periodic", 2), ("matrixized", "dirichlet", 1), ("gather", "periodic", 1)]:
        plan = sx.Plan(shape, 1, kind, cg, "f32", bc=bc, impl=impl)
        try:
            assert plan.info["kernels_per_sweep"] == want, (impl, bc)
        finally:
            plan.close()
    if ndim == 3:
        zline = np.zeros((3, 3, 3))
        zline[:, 1, 1] = [0.25, 0.5, 0.25]
        plan = sx.Plan(shape, 1, "star", zline, "f32", bc="periodic", impl="matrixized")
        try:
            assert plan.info["kernels_per_sweep"] == 1
        finally:
            plan.close()
        a = si.round_to(si.field_uniform(shape, 9), "f32")
        got, _ = run(a, 1, "star", zline, "f32", "periodic", 2, impl="matrixized", prec="tf32x3")
        check(got, oracle.gather(a, 1, zline, "periodic", 2), 1e-5, "z line")


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_mx_3d_125_point_box_runs_on_the_tensor_cores(prec):
    """The 3D box of order 2: 25 lines of 8 columns plus one all-zero line
    (N = 208, a multiple of 16), five running plane sums."""
    shape = (37, 61, 52)
    a, cg = problem(3, shape, 2, "box", seed=125)
    got, info = run(a, 2, "box", cg, "f32", "dirichlet", 2, impl="matrixized", prec=prec)
    assert info["impl"] == 2 and info["n_lines"] == 25 and info["tile_n"] == 8
    check(got, oracle.gather(a, 2, cg, "dirichlet", 2), TOL[prec], f"125-point box {prec}")


def test_mx_exact_when_operands_are_tf32():
    """Inputs and weights exactly representable in TF32 (small dyadic values):
    the lo parts vanish and TF32x3 matches the FP32 CUDA-core result to 1e-6."""
    rng = np.random.default_rng(1)
    shape = (160, 96)
    a = rng.integers(-64, 65, size=shape) / 64.0
    cg = rng.integers(-8, 9, size=(5, 5)) / 64.0
    mx, _ = run(a, 2, "box", cg, "f32", "periodic", 2, impl="matrixized", prec="tf32x3")
    ga, _ = run(a, 2, "box", cg, "f32", "periodic", 2, impl="gather")
    want = oracle.gather(a, 2, cg, "periodic", 2)
    check(mx, want, 1e-6, "mx exact operands")
    check(ga, want, 1e-6, "gather exact operands")


def test_mx_auto_picks_matrixized_for_f32_box():
    a, cg = problem(2, (64, 64), 1, "box", seed=9)
    _, info = run(a, 1, "box", cg, "f32", "dirichlet", 1, impl="auto")
    assert info["impl"] == 2 and info["prec"] == 2


def test_mx_split_runs_bitwise():
    a, cg = problem(2, (200, 136), 2, "box", seed=11)
    full, _ = run(a, 2, "box", cg, "f32", "periodic", 6, impl="matrixized")
    part, _ = run(a, 2, "box", cg, "f32", "periodic", 2, impl="matrixized")
    rest, _ = run(part, 2, "box", cg, "f32", "periodic", 4, impl="matrixized")
    assert np.array_equal(full, rest)


def test_mx_in_place_and_zero_steps():
    a, cg = problem(2, (140, 72), 1, "box", seed=12)
    got, _ = run(a, 1, "box", cg, "f32", "dirichlet", 3, impl="matrixized", alias=True, check_guard=False)
    check(got, oracle.gather(a, 1, cg, "dirichlet", 3), 1e-5)
    got, _ = run(a, 1, "box", cg, "f32", "dirichlet", 0, impl="matrixized")
    assert np.array_equal(got, a)


def test_mx_takes_unaligned_rows_through_padded_grids():
    """Rows that are not 16-byte multiples run on the tensor-core kernel
    through the plan's padded grids (two of them, reported as scratch)."""
    import paper_2310_16298_gb300 as sx
    plan = sx.stencil_plan_create((64, 66), 1, "box", np.ones((3, 3)) / 9, "f32", sx.make_options(impl="matrixized"))
    try:
        info = sx.stencil_plan_info(plan)
        assert info["impl"] == 2 and info["scratch_bytes"] >= 2 * 64 * 68 * 4
    finally:
        sx.stencil_plan_destroy(plan)


@pytest.mark.parametrize("prec", ["tf32x3", "tf32", "bf16x3", "bf16", "bf16w2"])
@pytest.mark.parametrize("kind,r", [("star", 1), ("box", 1), ("star", 2), ("star", 3), ("box", 2)])
@pytest.mark.parametrize("shape", [(40, 150, 44), (70, 29, 68)])
def test_mx_3d(prec, kind, r, shape):
    """3D matrixized sweep (plane streaming, lines along N) vs the oracle:
    several y tiles, x tiles and z chunks plus ragged tails."""
    if min(shape) < 2 * r + 1:
        pytest.skip("below the minimum extent")
    a, cg = problem(3, shape, r, kind, seed=40 + r)
    steps = 3
    got, info = run(a, r, kind, cg, "f32", "dirichlet", steps, impl="matrixized", prec=prec)
    assert info["impl"] == 2 and info["device_error"] == 0
    check(got, oracle.gather(a, r, cg, "dirichlet", steps), TOL[prec], f"mx 3d {kind} r={r} {shape} {prec}")


@pytest.mark.parametrize("prec", ["tf32x3", "tf32", "bf16x3", "bf16"])
@pytest.mark.parametrize("r", [1, 2, 3])
@pytest.mark.parametrize("cover", ["parallel", "hybrid"])
def test_mx_3d_star_covers(prec, r, cover):
    """Both line covers of a 3D star (Tables cls-3d): the parallel cover puts
    every line on the tensor cores, the hybrid cover only the contiguous-axis
    line (plus an identity band) and applies the 4r off-axis weights on the
    CUDA cores; both match the oracle."""
    shape = (38, 70, 52)
    a, cg = problem(3, shape, r, "star", seed=60 + r)
    steps = 3
    got, info = run(a, r, "star", cg, "f32", "dirichlet", steps, impl="matrixized", prec=prec, cover=cover)
    assert info["impl"] == 2 and info["device_error"] == 0
    assert info["n_scalar"] == (4 * r if cover == "hybrid" else 0)
    check(got, oracle.gather(a, r, cg, "dirichlet", steps), TOL[prec], f"mx 3d star r={r} {cover} {prec}")


def test_mx_hybrid_cover_only_for_3d_stars():
    import paper_2310_16298_gb300 as sx
    cg3 = np.ones((3, 3, 3)) / 27
    with pytest.raises(sx.StencilError) as ei:
        sx.stencil_plan_create((16, 16, 16), 1, "box", cg3, "f32", sx.make_options(impl="matrixized", cover="hybrid"))
    assert ei.value.status == sx.EUNSUPPORTED
    cg2 = np.zeros((3, 3))
    cg2[1, :] = cg2[:, 1] = 0.2
    with pytest.raises(sx.StencilError) as ei:
        sx.stencil_plan_create((64, 64), 1, "star", cg2, "f32", sx.make_options(impl="matrixized", cover="hybrid"))
    assert ei.value.status == sx.EUNSUPPORTED


def test_mx_3d_symmetric_closed_form():
    """Symmetric 7-point star on a Dirichlet sine mode: lam^T times the mode."""
    shape = (36, 40, 48)
    cg = si.coeffs_symmetric_3d7p()
    m = (1, 2, 1)
    phi = [np.pi * mk / (nk + 1) for mk, nk in zip(m, shape)]
    lam = sum(cg[o] * np.prod([np.cos(p * (oi - 1)) for p, oi in zip(phi, o)]) for o in np.ndindex(3, 3, 3))
    xs = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
    f = np.ones(shape)
    for p, x in zip(phi, xs):
        f = f * np.sin(p * (x + 1))
    f = si.round_to(f, "f32")
    T = 20
    got, _ = run(f, 1, "star", cg, "f32", "dirichlet", T, impl="matrixized", prec="tf32x3")
    check(got, oracle.gather(f, 1, cg, "dirichlet", T), 1e-5, "3d sine mode")
    l2, _ = oracle.error_norms(got, lam ** T * f)
    assert l2 < 1e-5


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x2"])
def test_mx_bf16_exact_operands(prec):
    """Inputs and weights exactly representable in BF16: the lower parts vanish
    and the split products reproduce the FP32 result to 1e-6."""
    rng = np.random.default_rng(2)
    shape = (140, 64)
    a = rng.integers(-16, 17, size=shape) / 16.0
    cg = rng.integers(-8, 9, size=(5, 5)) / 64.0
    got, _ = run(a, 2, "box", cg, "f32", "periodic", 2, impl="matrixized", prec=prec)
    check(got, oracle.gather(a, 2, cg, "periodic", 2), 1e-6, f"{prec} exact operands")


def test_mx_cover_auto_picks_a_built_cover_and_matches_it():
    """COVER_AUTO on a 3D star times both covers and keeps one; the plan
    reports it, and its result is bit-identical to the explicit plan's."""
    shape = (40, 120, 64)
    a, cg = problem(3, shape, 2, "star", seed=71)
    got, info = run(a, 2, "star", cg, "f32", "dirichlet", 3, impl="matrixized", prec="tf32x3", cover="auto")
    assert info["cover"] in (1, 2)
    want, info2 = run(a, 2, "star", cg, "f32", "dirichlet", 3, impl="matrixized", prec="tf32x3",
                      cover={1: "parallel", 2: "hybrid"}[info["cover"]])
    assert info2["cover"] == info["cover"]
    assert np.array_equal(got, want)
    # 2D plans run the parallel cover; gather plans report none
    _, i2 = run(a[0], 2, "star", cg[2], "f32", "dirichlet", 1, impl="matrixized")
    assert i2["cover"] == 1
    _, ig = run(a[0], 2, "star", cg[2], "f32", "dirichlet", 1, impl="gather")
    assert ig["cover"] == 0


@pytest.mark.parametrize("pattern", ["diagonal", "anti-diagonal", "random", "ring"])
@pytest.mark.parametrize("impl", ["matrixized", "gather"])
def test_arbitrary_weight_patterns(pattern, impl):
    """Weight patterns that are neither star nor box (Sec. 3.3 diagonal lines,
    Sec. 3.5 arbitrary patterns) run as a box plan whose absent weights are
    zero: every line of the pattern is a (possibly sparse) banded operand."""
    r = 2
    rng = np.random.default_rng(5)
    w = rng.uniform(0.1, 1.0, size=(5, 5))
    a_, b_ = np.meshgrid(np.arange(5), np.arange(5), indexing="ij")
    mask = {"diagonal": a_ == b_, "anti-diagonal": a_ + b_ == 4,
            "random": rng.uniform(size=(5, 5)) < 0.4,
            "ring": np.maximum(abs(a_ - 2), abs(b_ - 2)) == 2}[pattern]
    cg = si.round_to(np.where(mask, w, 0.0) / np.where(mask, w, 0.0).sum(), "f32")
    a = si.round_to(si.field_uniform((300, 196), 77, -1.0, 1.0), "f32")
    got, info = run(a, r, "box", cg, "f32", "periodic", 4, impl=impl, prec="tf32x3" if impl == "matrixized" else "native")
    check(got, oracle.gather(a, r, cg, "periodic", 4), 1e-5, f"{pattern} {impl}")


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "tf32"])
@pytest.mark.parametrize("kind,r,cover", [("star", 1, "hybrid"), ("star", 1, "parallel"), ("box", 1, "auto"),
                                          ("star", 2, "hybrid"), ("star", 3, "parallel"), ("box", 2, "auto")])
@pytest.mark.parametrize("shape", [(40, 150, 44), (70, 29, 68)])
def test_mx_3d_periodic(prec, kind, r, cover, shape):
    """Periodic 3D sweeps: wrapped plane indices and wrapped halo rows and
    columns of the edge tiles (several y and x tiles, ragged tails)."""
    a, cg = problem(3, shape, r, kind, seed=80 + r)
    got, info = run(a, r, kind, cg, "f32", "periodic", 3, impl="matrixized", prec=prec, cover=cover)
    assert info["impl"] == 2
    check(got, oracle.gather(a, r, cg, "periodic", 3), TOL[prec], f"mx 3d periodic {kind} r={r} {cover} {prec}")


@pytest.mark.parametrize("kind,r", [("star", 1), ("box", 1), ("star", 2), ("box", 2)])
def test_mx_3d_unit_depth_does_not_change_the_result(kind, r):
    """The work-unit depth (planes per unit) changes how often halo planes
    are re-read, not the arithmetic: every output plane sums the same input
    planes in the same order, so results are bit-identical."""
    import paper_2310_16298_gb300 as sx
    import torch
    shape = (70, 29, 68)
    a, cg = problem(3, shape, r, kind, seed=90 + r)
    x = torch.tensor(a, dtype=torch.float32, device="cuda")
    outs = []
    for up in (0, 1, 7, 100):
        plan = sx.Plan(shape, r, kind, cg, "f32", bc="dirichlet", impl="matrixized", prec="tf32x3",
                       cover="hybrid" if kind == "star" else "auto", unit_planes=up)
        y = plan.apply(x, steps=3)
        torch.cuda.synchronize()
        assert sx.stencil_plan_info(plan.handle)["device_error"] == 0
        outs.append(y.cpu().numpy())
        plan.close()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    check(outs[0], oracle.gather(a, r, cg, "dirichlet", 3), 1e-5, "unit depth")
