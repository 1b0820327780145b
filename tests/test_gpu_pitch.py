"""Row pitch: grids whose rows are padded (stencil_options.pitch), and packed
grids whose rows are not 16-byte multiples, which the tensor-core kernels run
through padded grids the plan owns.  Results must equal the packed run bit
for bit (same kernels, same arithmetic), the padding must stay untouched, and
the odd extents must match the FP64 oracle."""
import numpy as np
import pytest

import oracle
import paper_2310_16298_gb300 as sx
import stencil_inputs as si
from gpuutil import TOL, check, run

pytestmark = pytest.mark.gpu

CANARY = -777.25


def run_pitched(a, r, kind, cg, dtype, bc, steps, impl, prec, pitch):
    """Run with grids of row stride `pitch` (padding filled with a canary)."""
    import torch
    td = torch.float32 if dtype == "f32" else torch.float64
    rows = int(np.prod(a.shape[:-1]))
    nx = a.shape[-1]
    xin = torch.full((rows, pitch), CANARY, dtype=td, device="cuda")
    xin[:, :nx] = torch.from_numpy(np.ascontiguousarray(a).reshape(rows, nx)).to(td)
    xout = torch.full_like(xin, CANARY)
    plan = sx.stencil_plan_create(a.shape, r, kind, cg, dtype, sx.make_options(prec, bc, impl, 0, "auto", pitch))
    try:
        sx.stencil_apply(plan, xin.data_ptr(), xout.data_ptr(), steps, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        info = sx.stencil_plan_info(plan)
        assert info["device_error"] == 0
    finally:
        sx.stencil_plan_destroy(plan)
    out = xout.double().cpu().numpy()
    assert np.all(out[:, nx:] == CANARY), "padding written"
    assert np.all(xin[:, nx:].double().cpu().numpy() == CANARY), "input padding modified"
    return out[:, :nx].reshape(a.shape), info


@pytest.mark.parametrize("case", [
    ("matrixized", (300, 196), 2, "box", "f32", "periodic", 200),
    ("matrixized", (300, 196), 2, "box", "f32", "dirichlet", 256),
    ("matrixized", (40, 150, 44), 1, "star", "f32", "dirichlet", 48),
    ("matrixized", (40, 150, 44), 1, "box", "f32", "periodic", 52),
    ("gather", (300, 516), 2, "box", "f32", "periodic", 520),
    ("gather", (300, 516), 1, "star", "f64", "dirichlet", 522),
    ("gather", (150, 70, 132), 1, "box", "f32", "periodic", 136),
    ("gather", (19, 23, 30), 2, "star", "f64", "dirichlet", 34),
])
def test_pitched_grids_match_packed(case):
    impl, shape, r, kind, dtype, bc, pitch = case
    cg = si.coeffs_random(len(shape), r, kind, 600 + r, dtype=dtype)
    a = si.round_to(si.field_uniform(shape, 601, -1.0, 1.0), dtype)
    prec = "tf32x3" if impl == "matrixized" else "native"
    got, info = run_pitched(a, r, kind, cg, dtype, bc, 3, impl, prec, pitch)
    want, info0 = run(a, r, kind, cg, dtype, bc, 3, impl=impl, prec=prec)
    assert info["impl"] == info0["impl"]
    assert np.array_equal(got, want)


@pytest.mark.parametrize("shape,r,kind,bc", [
    ((301, 203), 2, "box", "periodic"),
    ((301, 203), 2, "box", "dirichlet"),
    ((257, 130), 1, "star", "periodic"),
    ((2050, 2047), 2, "box", "periodic"),   # many tiles per CTA
    ((40, 150, 43), 1, "star", "dirichlet"),
    ((41, 97, 66), 1, "box", "periodic"),
])
@pytest.mark.parametrize("steps", [3, 4])
def test_unaligned_rows_run_on_the_tensor_cores(shape, r, kind, bc, steps):
    """Packed rows that are not 16-byte multiples (odd contiguous extents)."""
    cg = si.coeffs_random(len(shape), r, kind, 610 + r, dtype="f32")
    a = si.round_to(si.field_uniform(shape, 611, -1.0, 1.0), "f32")
    got, info = run(a, r, kind, cg, "f32", bc, steps, impl="matrixized", prec="tf32x3")
    assert info["impl"] == 2
    check(got, oracle.gather(a, r, cg, bc, steps), 1e-5, f"unaligned {shape} {kind} {bc}")


def test_unaligned_rows_in_place_host_and_noalloc():
    import torch
    shape, r = (131, 97), 1
    cg = si.coeffs_random(2, r, "box", 620, dtype="f32")
    a = si.round_to(si.field_uniform(shape, 621), "f32")
    want = oracle.gather(a, r, cg, "dirichlet", 5)
    got, _ = run(a, r, "box", cg, "f32", "dirichlet", 5, impl="matrixized", alias=True, check_guard=False)
    check(got, want, 1e-5, "in place")
    got0, _ = run(a, r, "box", cg, "f32", "dirichlet", 0, impl="matrixized")
    assert np.array_equal(got0, a)
    plan = sx.stencil_plan_create(shape, r, "box", cg, "f32", sx.make_options("native", "dirichlet", "matrixized"))
    try:
        h_out = np.empty_like(a, dtype=np.float32)
        sx.stencil_apply_host(plan, a.astype(np.float32), h_out, 5)
        check(h_out, want, 1e-5, "apply_host")
        x = torch.tensor(a, dtype=torch.float32, device="cuda")
        with pytest.raises(sx.StencilError) as ei:
            sx.stencil_apply_noalloc(plan, x.data_ptr(), x.data_ptr(), 1)
        assert ei.value.status == sx.EINVAL
    finally:
        sx.stencil_plan_destroy(plan)


@pytest.mark.parametrize("pitch", [-1, 150, 201])
def test_invalid_pitch_is_rejected(pitch):
    """A pitch below the extent, or one that does not give 16-byte rows."""
    with pytest.raises(sx.StencilError) as ei:
        sx.stencil_plan_create((64, 199), 1, "box", np.full((3, 3), 1 / 9), "f32",
                               sx.make_options("native", "dirichlet", "auto", 0, "auto", pitch))
    assert ei.value.status == sx.EINVAL
