"""GPU parity of the TMA-staged gather kernels against the FP64 oracle.

Rows that are a multiple of 16 bytes take the persistent TMA kernels: 2D
tiles through a ring of shared-memory stages (FP32: 32 x 128 tiles, four
stages; FP64: 64 x 32, two), 3D columns of planes through a ring of 2r + 2
plane buffers.  The shapes span several tiles (units) with ragged tails in
every axis; with a periodic boundary the tiles at the edges are staged by
TMA and then get their cells outside the grid wrapped.  Full-size grids
(many tiles or units per CTA) are checked at sampled points, computed by the
oracle on their dependency cones."""
import numpy as np
import pytest

import oracle
import stencil_inputs as si
from gpuutil import TOL, check, run

pytestmark = pytest.mark.gpu


def problem(shape, r, kind, dtype, seed):
    cg = si.coeffs_random(len(shape), r, kind, 900 + seed, dtype=dtype)
    a = si.round_to(si.field_uniform(shape, 900 + seed, -1.0, 1.0), dtype)
    return a, cg


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("kind", ["star", "box"])
@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_gather_tma_2d(dtype, bc, kind, r):
    shape = (300, 516)   # 128- and 32-column tiles, 32- and 64-row tiles, ragged edges
    a, cg = problem(shape, r, kind, dtype, r)
    got, info = run(a, r, kind, cg, dtype, bc, 3, impl="gather")
    assert info["impl"] == 1
    check(got, oracle.gather(a, r, cg, bc, 3), TOL[dtype], f"tma 2d r={r} {kind} {bc} {dtype}")


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("r,tb", [(1, 2), (1, 4), (2, 2), (2, 3)])
def test_gather_tma_2d_temporal_blocking(dtype, bc, r, tb):
    shape = (300, 516)
    a, cg = problem(shape, r, "box", dtype, 10 + tb)
    steps = 7   # not a multiple of tb
    got, info = run(a, r, "box", cg, dtype, bc, steps, impl="gather", tb=tb)
    assert info["tb"] == tb
    check(got, oracle.gather(a, r, cg, bc, steps), TOL[dtype], f"tma 2d tb={tb}")


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("kind", ["star", "box"])
@pytest.mark.parametrize("r", [1, 2, 3])
def test_gather_tma_3d(dtype, bc, kind, r):
    """150 x 70 x 132: three 64-plane chunks (the last 22 planes), three
    32-row and three 64-column tiles, each with a ragged last one."""
    shape = (150, 70, 132)
    a, cg = problem(shape, r, kind, dtype, 20 + r)
    got, info = run(a, r, kind, cg, dtype, bc, 2, impl="gather")
    assert info["impl"] == 1
    check(got, oracle.gather(a, r, cg, bc, 2), TOL[dtype], f"tma 3d r={r} {kind} {bc} {dtype}")


def seam_points(shape, periods, n, seed):
    """Corners, points on both sides of tile seams, and random points."""
    rng = np.random.default_rng(seed)
    cands = []
    for s, ps in zip(shape, periods):
        c = {0, 1, s // 2, s - 2, s - 1}
        for p in ps:
            for k in (1, s // p // 2, s // p):
                c.update((k * p - 1, k * p))
        cands.append(sorted(v for v in c if 0 <= v < s))
    pts = {tuple(0 if b == 0 else s - 1 for b, s in zip(bits, shape)) for bits in np.ndindex(*([2] * len(shape)))}
    total = int(np.prod([len(c) for c in cands]))
    for _ in range(20 * n):   # bounded: the candidate grid may hold fewer than n points
        if len(pts) >= min(n, total):
            break
        pts.add(tuple(int(rng.choice(c)) for c in cands))
    pts = list(pts) + [tuple(int(rng.integers(0, s)) for s in shape) for _ in range(16)]
    return np.array(pts, dtype=np.int64)


@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_gather_tma_2d_many_tiles_per_cta(bc):
    """4096 x 4096 FP32 (2048 tiles, several per CTA), 4 steps, sampled."""
    import torch
    import paper_2310_16298_gb300 as sx
    shape, r, steps = (4096, 4096), 2, 4
    a, cg = problem(shape, r, "box", "f32", 40)
    plan = sx.Plan(shape, r, "box", cg, "f32", bc=bc, impl="gather")
    try:
        x = torch.tensor(a, dtype=torch.float32, device="cuda")
        y = plan.apply(x, steps=steps)
        torch.cuda.synchronize()
        assert sx.stencil_plan_info(plan.handle)["device_error"] == 0
        pts = seam_points(shape, [(32, 64), (128,)], 96, 1)
        got = y[tuple(torch.as_tensor(c, device="cuda") for c in pts.T)].double().cpu().numpy()
    finally:
        plan.close()
    check(got, oracle.sample(a, r, cg, bc, steps, pts), 1e-5, f"4096^2 gather {bc}")


@pytest.mark.parametrize("kind,dtype", [("box", "f32"), ("star", "f64")])
def test_gather_tma_3d_many_units_per_cta(kind, dtype):
    """512^3 (1024 units of 64 planes x 32 rows x 64 columns), 2 steps, sampled."""
    import torch
    import paper_2310_16298_gb300 as sx
    shape, r, steps = (512, 512, 512), 1, 2
    cg = si.coeffs_random(3, r, kind, 941, dtype=dtype)
    a = si.round_to(si.field_uniform(shape, 941, -1.0, 1.0), dtype)
    td = torch.float32 if dtype == "f32" else torch.float64
    plan = sx.Plan(shape, r, kind, cg, dtype, bc="dirichlet", impl="gather")
    try:
        x = torch.tensor(a, dtype=td, device="cuda")
        y = plan.apply(x, steps=steps)
        torch.cuda.synchronize()
        assert sx.stencil_plan_info(plan.handle)["device_error"] == 0
        pts = seam_points(shape, [(64,), (32,), (64,)], 96, 2)
        got = y[tuple(torch.as_tensor(c, device="cuda") for c in pts.T)].double().cpu().numpy()
        del x, y
    finally:
        plan.close()
    check(got, oracle.sample(a, r, cg, "dirichlet", steps, pts), TOL[dtype], f"512^3 gather {kind} {dtype}")
