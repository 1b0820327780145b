"""stencil_apply_noalloc: the apply variant for callers that cannot allocate
device memory while they step a field (it keeps its second grid copy in a
static device array).  Its results must equal stencil_apply's, call after
call, whether this file runs alone or after the rest of the suite."""
import numpy as np
import pytest

import paper_2310_16298_gb300 as sx
import stencil_inputs as si

pytestmark = pytest.mark.gpu


def _run_both(shape, r, kind, dtype, bc, impl, steps, in_place=False):
    import torch
    td = torch.float32 if dtype == "f32" else torch.float64
    cg = si.coeffs_random(len(shape), r, kind, 300 + r, dtype=dtype)
    a = si.round_to(si.field_uniform(shape, 31 + r), dtype)
    plan = sx.stencil_plan_create(shape, r, kind, cg, dtype, sx.make_options("native", bc, impl, 0))
    try:
        assert sx.stencil_plan_info(plan)["impl"] == sx.IMPLS[impl]
        x = torch.tensor(a, dtype=td, device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        ref = torch.empty_like(x)
        sx.stencil_apply(plan, x.data_ptr(), ref.data_ptr(), steps, s)
        outs = []
        for _ in range(2):  # two calls in a row share (and reuse) the static array
            if in_place:
                y = x.clone()
                sx.stencil_apply_noalloc(plan, y.data_ptr(), y.data_ptr(), steps, s)
            else:
                y = torch.full_like(x, float("nan"))
                sx.stencil_apply_noalloc(plan, x.data_ptr(), y.data_ptr(), steps, s)
            outs.append(y)
        torch.cuda.synchronize()
        assert sx.stencil_plan_info(plan)["device_error"] == 0
        return ref.cpu().numpy(), [o.cpu().numpy() for o in outs]
    finally:
        sx.stencil_plan_destroy(plan)


@pytest.mark.parametrize("impl,shape,r,kind,dtype,bc", [
    ("matrixized", (300, 196), 2, "box", "f32", "periodic"),
    ("matrixized", (40, 150, 44), 1, "star", "f32", "dirichlet"),
    ("gather", (130, 90), 1, "star", "f64", "dirichlet"),
    ("gather", (21, 18, 33), 1, "box", "f32", "dirichlet"),
])
@pytest.mark.parametrize("steps", [1, 4, 5])
def test_noalloc_matches_apply(impl, shape, r, kind, dtype, bc, steps):
    """Same kernels in the same order as stencil_apply, only another buffer for
    the second grid copy: the results must be identical bit for bit."""
    ref, outs = _run_both(shape, r, kind, dtype, bc, impl, steps)
    for got in outs:
        assert np.all(np.isfinite(got))
        assert np.array_equal(got, ref)


def test_noalloc_in_place():
    ref, outs = _run_both((140, 72), 1, "box", "f32", "dirichlet", "matrixized", 3, in_place=True)
    for got in outs:
        assert np.array_equal(got, ref)


def test_noalloc_rejects_grids_beyond_the_static_scratch():
    import torch
    shape = (2048, 2056)  # 16.06 MiB in FP32: one row more than fits
    plan = sx.stencil_plan_create(shape, 1, "box", np.full((3, 3), 1 / 9), "f32",
                                  sx.make_options("native", "dirichlet", "gather", 0))
    try:
        x = torch.zeros(shape, dtype=torch.float32, device="cuda")
        with pytest.raises(sx.StencilError) as ei:
            sx.stencil_apply_noalloc(plan, x.data_ptr(), x.data_ptr(), 1)
        assert ei.value.status == sx.EINVAL and "16 MiB" in str(ei.value)
    finally:
        sx.stencil_plan_destroy(plan)
