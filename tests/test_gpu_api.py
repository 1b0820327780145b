"""GPU tests of the C ABI's asynchronous, host-buffer and batch entry points
(results against the oracle and against stencil_apply), and of the error
bits path: a plan whose kernel gave up a bounded wait must make every call
that runs or completes its work return ECUDA.  The error is raised on the
host (stencil_plan_raise_error), never by making a GPU fault."""
import time

import numpy as np
import pytest

import oracle
import paper_2310_16298_gb300 as sx
import stencil_inputs as si

pytestmark = pytest.mark.gpu


def setup(shape=(300, 196), r=2, kind="box", bc="periodic", impl="matrixized", seed=7):
    import torch
    cg = si.coeffs_random(len(shape), r, kind, 700 + seed, dtype="f32")
    a = si.round_to(si.field_uniform(shape, 700 + seed), "f32")
    plan = sx.stencil_plan_create(shape, r, kind, cg, "f32", sx.make_options("native", bc, impl, 0))
    x = torch.tensor(a, dtype=torch.float32, device="cuda")
    return plan, a, cg, x


@pytest.mark.parametrize("impl", ["matrixized", "gather"])
def test_submit_poll_result_matches_oracle(impl):
    import torch
    plan, a, cg, x = setup(impl=impl)
    try:
        y = torch.full_like(x, float("nan"))
        torch.cuda.synchronize()
        t = sx.stencil_submit(plan, x.data_ptr(), y.data_ptr(), 5)
        deadline = time.time() + 30
        st = sx.stencil_poll(t)
        while st == sx.ENOTREADY and time.time() < deadline:
            time.sleep(0.001)
            st = sx.stencil_poll(t)
        assert st == sx.OK, sx.stencil_last_error()
        # the ticket is released by the poll that returned OK
        assert sx.stencil_poll(t) == sx.EINVAL
        got = y.double().cpu().numpy()
        l2, mx = oracle.error_norms(got, oracle.gather(a, 2, cg, "periodic", 5))
        assert l2 <= 1e-5 and mx <= 1e-5
    finally:
        sx.stencil_plan_destroy(plan)


def test_submit_wait_ok_and_matches_apply():
    import torch
    plan, a, cg, x = setup()
    try:
        y = torch.empty_like(x)
        ref = torch.empty_like(x)
        sx.stencil_apply(plan, x.data_ptr(), ref.data_ptr(), 4, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        t = sx.stencil_submit(plan, x.data_ptr(), y.data_ptr(), 4)
        assert sx.stencil_wait(t, 30000) == sx.OK, sx.stencil_last_error()
        assert torch.equal(y, ref)
        assert sx.stencil_wait(t, 0) == sx.EINVAL
    finally:
        sx.stencil_plan_destroy(plan)


@pytest.mark.parametrize("impl,steps", [("matrixized", 6), ("matrixized", 3), ("gather", 5)])
def test_apply_host_matches_oracle(impl, steps):
    plan, a, cg, _ = setup(impl=impl)
    try:
        h_in = np.ascontiguousarray(a, dtype=np.float32)
        keep = h_in.copy()
        for _ in range(2):   # the second call reuses the plan's staging grid
            h_out = np.full_like(h_in, np.nan)
            sx.stencil_apply_host(plan, h_in, h_out, steps)
            l2, mx = oracle.error_norms(h_out, oracle.gather(a, 2, cg, "periodic", steps))
            assert l2 <= 1e-5 and mx <= 1e-5
        assert np.array_equal(h_in, keep), "input modified"
    finally:
        sx.stencil_plan_destroy(plan)


def test_batch_run_equals_solo_runs():
    import torch
    shapes = [(96, 130), (200, 64), (129, 257)]
    steps = [7, 3, 12]
    plans, xs, ys, want = [], [], [], []
    try:
        for i, sh in enumerate(shapes):
            cg = si.coeffs_random(2, 1, "box", 800 + i, dtype="f32")
            a = si.round_to(si.field_uniform(sh, 800 + i), "f32")
            p = sx.stencil_plan_create(sh, 1, "box", cg, "f32", sx.make_options("native", "dirichlet", "gather", 0))
            plans.append(p)
            x = torch.tensor(a, dtype=torch.float32, device="cuda")
            xs.append(x)
            ys.append(torch.full_like(x, float("nan")))
            want.append(oracle.gather(a, 1, cg, "dirichlet", steps[i]))
        s = torch.cuda.current_stream().cuda_stream
        sx.stencil_batch_run(plans, [x.data_ptr() for x in xs], [y.data_ptr() for y in ys], steps, s)
        for i, p in enumerate(plans):
            solo = torch.empty_like(xs[i])
            sx.stencil_apply(p, xs[i].data_ptr(), solo.data_ptr(), steps[i], s)
            torch.cuda.synchronize()
            l2, mx = oracle.error_norms(ys[i].double().cpu().numpy(), want[i])
            assert l2 <= 1e-5 and mx <= 1e-5
            # the batch's tile shape and depth may differ from the solo plan's:
            # same arithmetic per point, so equal to FP32 rounding
            assert torch.allclose(ys[i], solo, rtol=1e-6, atol=1e-6)
    finally:
        for p in plans:
            sx.stencil_plan_destroy(p)


@pytest.mark.parametrize("impl", ["matrixized", "gather"])
def test_error_bits_turn_into_statuses(impl):
    """Bits raised on the host are reported by every call that runs or
    completes the plan's work, and by plan_info; other plans are unaffected."""
    import torch
    plan, a, cg, x = setup(impl=impl)
    other, _, _, _ = setup(impl=impl, seed=8)
    try:
        y = torch.empty_like(x)
        s = torch.cuda.current_stream().cuda_stream
        t = sx.stencil_submit(plan, x.data_ptr(), y.data_ptr(), 2)
        sx.stencil_plan_raise_error(plan, 4)
        # work submitted before the error completes with the error
        assert sx.stencil_wait(t, 30000) == sx.ECUDA
        assert "bounded wait" in sx.stencil_last_error()
        assert sx.stencil_plan_info(plan)["device_error"] == 4
        for call in (lambda: sx.stencil_apply(plan, x.data_ptr(), y.data_ptr(), 1, s),
                     lambda: sx.stencil_apply_noalloc(plan, x.data_ptr(), y.data_ptr(), 1, s),
                     lambda: sx.stencil_apply_host(plan, a.astype(np.float32), np.empty_like(a, np.float32), 1),
                     lambda: sx.stencil_submit(plan, x.data_ptr(), y.data_ptr(), 1),
                     lambda: sx.stencil_batch_run([plan], [x.data_ptr()], [y.data_ptr()], [1], s)):
            with pytest.raises(sx.StencilError) as ei:
                call()
            assert ei.value.status == sx.ECUDA and "bounded wait" in str(ei.value)
        # a plan without error bits still runs
        sx.stencil_apply(other, x.data_ptr(), y.data_ptr(), 1, s)
        torch.cuda.synchronize()
        assert sx.stencil_plan_info(other)["device_error"] == 0
        with pytest.raises(sx.StencilError) as ei:
            sx.stencil_plan_raise_error(plan, 0)
        assert ei.value.status == sx.EINVAL
    finally:
        sx.stencil_plan_destroy(plan)
        sx.stencil_plan_destroy(other)


def test_batch_launch_reports_error_bits():
    import torch
    plan, a, cg, x = setup(shape=(128, 128), r=1, impl="gather", bc="dirichlet")
    try:
        y = torch.empty_like(x)
        b = sx.stencil_batch_create_ex([plan], [x.data_ptr()], [y.data_ptr()], [3], 1, 0)
        try:
            s = torch.cuda.current_stream().cuda_stream
            sx.stencil_batch_launch(b, s)
            torch.cuda.synchronize()
            sx.stencil_plan_raise_error(plan, 1)
            with pytest.raises(sx.StencilError) as ei:
                sx.stencil_batch_launch(b, s)
            assert ei.value.status == sx.ECUDA
        finally:
            sx.stencil_batch_destroy(b)
    finally:
        sx.stencil_plan_destroy(plan)
