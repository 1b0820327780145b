"""GPU checks of batched runs: every problem's result in the batch equals the
same problem run alone (bit for bit: temporal blocking and packing do not
change the arithmetic of any point) and the oracle."""
import math

import numpy as np
import pytest

import oracle
import paper_2310_16298_gb300 as sx
import stencil_inputs as si

pytestmark = pytest.mark.gpu


def make_batch(n, seed, rmix=False):
    u = si.uniform(seed, 4 * n).reshape(n, 4)
    probs = []
    for i in range(n):
        ny = int(round(math.exp(math.log(12) + u[i, 0] * (math.log(180) - math.log(12)))))
        nx = int(round(math.exp(math.log(12) + u[i, 1] * (math.log(180) - math.log(12)))))
        steps = int(u[i, 2] * 13)  # 0..12
        r = 1 + (i % 2) if rmix else 1
        ny, nx = max(ny, 2 * r + 1), max(nx, 2 * r + 1)
        cg = si.coeffs_random(2, r, "box", seed * 1000 + i, dtype="f32")
        a = si.round_to(si.field_uniform((ny, nx), seed * 1000 + 500 + i), "f32")
        probs.append((a, cg, steps, r))
    return probs


def run_batch(probs, tb=0, alias_every=5, launches=1, tile_shape=-1):
    import torch
    plans, ins, outs, keep = [], [], [], []
    for i, (a, cg, steps, r) in enumerate(probs):
        plans.append(sx.stencil_plan_create(a.shape, r, "box", cg, "f32", sx.make_options(impl="gather")))
        x = torch.tensor(a, dtype=torch.float32, device="cuda")
        y = x if (alias_every and i % alias_every == 0) else torch.full_like(x, float("nan"))
        keep += [x, y]
        ins.append(x.data_ptr())
        outs.append(y.data_ptr())
    torch.cuda.synchronize()
    steps = [p[2] for p in probs]
    if tile_shape < 0:
        b = sx.stencil_batch_create(plans, ins, outs, steps, tb)
    else:
        b = sx.stencil_batch_create_ex(plans, ins, outs, steps, tb, tile_shape)
    info = sx.stencil_batch_info(b)
    s = torch.cuda.current_stream().cuda_stream
    sx.stencil_batch_launch(b, s)
    torch.cuda.synchronize()
    results = [keep[2 * i + 1].double().cpu().numpy() for i in range(len(probs))]
    for _ in range(launches - 1):  # replay the graph on the results (more steps)
        sx.stencil_batch_launch(b, s)
    torch.cuda.synchronize()
    sx.stencil_batch_destroy(b)
    for p in plans:
        sx.stencil_plan_destroy(p)
    return results, info


def run_alone(a, cg, steps, r):
    import torch
    plan = sx.stencil_plan_create(a.shape, r, "box", cg, "f32", sx.make_options(impl="gather"))
    x = torch.tensor(a, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    sx.stencil_apply(plan, x.data_ptr(), y.data_ptr(), steps, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    sx.stencil_plan_destroy(plan)
    return y.double().cpu().numpy()


@pytest.mark.parametrize("tb", [0, 1, 3])
def test_batch_equals_alone_and_oracle(tb):
    probs = make_batch(40, seed=7)
    got, info = run_batch(probs, tb=tb)
    assert info["packed"] == 1 and info["tb"] >= 1
    if tb:
        assert info["tb"] == tb
    for (a, cg, steps, r), g in zip(probs, got):
        alone = run_alone(a, cg, steps, r)
        assert np.array_equal(g, alone)
        if steps:
            l2, mx = oracle.error_norms(g, oracle.gather(a, r, cg, "dirichlet", steps))
            assert l2 <= 1e-5 and mx <= 1e-5
        else:
            assert np.array_equal(g, a)


@pytest.mark.parametrize("tile_shape,tb", [(0, 2), (1, 0), (1, 1), (1, 3)])
def test_batch_tile_shapes_equal_alone_and_oracle(tile_shape, tb):
    """Each batch tile shape (64 x 128 and 32 x 64 outputs) gives every problem
    the same result as running it alone, with its ragged edge tiles."""
    probs = make_batch(30, seed=11)
    got, info = run_batch(probs, tb=tb, tile_shape=tile_shape)
    assert info["packed"] == 1 and info["tile_shape"] == tile_shape
    if tb:
        assert info["tb"] == tb
    for (a, cg, steps, r), g in zip(probs, got):
        assert np.array_equal(g, run_alone(a, cg, steps, r))
        if steps:
            l2, mx = oracle.error_norms(g, oracle.gather(a, r, cg, "dirichlet", steps))
            assert l2 <= 1e-5 and mx <= 1e-5


def test_batch_autotune_reports_a_valid_shape():
    probs = make_batch(8, seed=12)
    _, info = run_batch(probs, tb=0)
    assert info["packed"] == 1 and info["tile_shape"] in (0, 1) and 1 <= info["tb"] <= 4


def test_batch_mixed_orders_not_packed():
    probs = make_batch(12, seed=8, rmix=True)
    got, info = run_batch(probs, tb=0)
    assert info["packed"] == 0 and info["tile_shape"] == -1
    for (a, cg, steps, r), g in zip(probs, got):
        assert np.array_equal(g, run_alone(a, cg, steps, r))


def test_batch_rejects_bad_entries():
    with pytest.raises(sx.StencilError):
        sx.stencil_batch_create([0], [0], [0], [1], 0)
