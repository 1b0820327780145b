"""GPU checks of the serving loop: every request's result is the same alone
and in a mix of concurrently served requests, the device-memory budget limits
admission, and errors and timeouts come back as statuses."""
import time

import numpy as np
import pytest

import oracle
import paper_2310_16298_gb300 as sx
import stencil_inputs as si

pytestmark = pytest.mark.gpu


def test_fill_uniform_matches_host_generator():
    import torch
    for dtype, td in (("f32", torch.float32), ("f64", torch.float64)):
        for lo, hi, off in ((0.0, 1.0, 0), (-1.0, 1.0, 12345)):
            n = 100_003
            x = torch.empty(n, dtype=td, device="cuda")
            sx.stencil_fill_uniform(x.data_ptr(), dtype, n, 77, off, lo, hi)
            torch.cuda.synchronize()
            want = si.round_to(si.uniform(77, n, lo, hi, offset=off), dtype)
            assert np.array_equal(x.double().cpu().numpy(), want)


def mixed_requests(n, seed):
    u = si.uniform(seed, 6 * n).reshape(n, 6)
    out = []
    for i in range(n):
        dtype = "f64" if u[i, 0] < 0.25 else "f32"
        steps = 1 + int(u[i, 1] * 40)
        if u[i, 2] < 0.6:
            r = 1 + int(u[i, 3] * 3)
            kind = "star" if u[i, 4] < 0.5 else "box"
            side = 16 + 4 * int(u[i, 5] * 30)
            shape = (side + 3, side)
        else:
            r = 1
            kind = "star" if u[i, 4] < 0.5 else "box"
            side = 12 + 4 * int(u[i, 5] * 8)
            shape = (side, side + 5, side)
        cg = si.coeffs_random(len(shape), r, kind, seed * 100 + i, dtype=dtype)
        out.append(dict(shape=shape, r=r, kind=kind, cg=cg, dtype=dtype, steps=steps, seed=seed * 100 + 50 + i))
    return out


def alone(q):
    import torch
    td = torch.float32 if q["dtype"] == "f32" else torch.float64
    plan = sx.stencil_plan_create(q["shape"], q["r"], q["kind"], q["cg"], q["dtype"])
    a = si.round_to(si.field_uniform(q["shape"], q["seed"]), q["dtype"])
    x = torch.tensor(a, dtype=td, device="cuda")
    y = torch.empty_like(x)
    sx.stencil_apply(plan, x.data_ptr(), y.data_ptr(), q["steps"], torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    sx.stencil_plan_destroy(plan)
    return a, y.double().cpu().numpy()


@pytest.mark.parametrize("budget_mb,max_resident", [(4096, 16), (3, 4)])
def test_server_results_same_alone_and_in_the_mix(budget_mb, max_resident):
    reqs = mixed_requests(24, seed=11)
    srv = sx.stencil_server_create(budget_mb << 20, max_resident, 7, 4)
    try:
        ids, keep = [], []
        host_inputs = {}
        for k, q in enumerate(reqs):
            # every third request sends its input from host memory, the rest name a seeded field
            h_in = None
            if k % 3 == 0:
                h_in = si.round_to(si.field_uniform(q["shape"], q["seed"]), q["dtype"])
                h_in = h_in.astype(np.float32 if q["dtype"] == "f32" else np.float64)
                host_inputs[k] = h_in
            rq, ref = sx.make_request(q["shape"], q["r"], q["kind"], q["cg"], q["dtype"], q["steps"],
                                      h_in=h_in, seed=q["seed"])
            keep.append((rq, ref))
            ids.append(sx.stencil_server_submit(srv, rq))
            if k % 5 == 0:
                time.sleep(0.002)  # arrivals while others run
        for k, (q, rid) in enumerate(zip(reqs, ids)):
            assert sx.stencil_server_wait(srv, rid, 60_000) == sx.OK, sx.stencil_last_error()
            out = np.empty(q["shape"], dtype=np.float32 if q["dtype"] == "f32" else np.float64)
            st = sx.stencil_server_result(srv, rid, out)
            a, want = alone(q)
            assert np.array_equal(out.astype(np.float64), want), (k, q["shape"], q["dtype"])
            assert st["done_s"] >= st["admit_s"] >= st["submit_s"] >= 0
            if k < 4:
                tol = 1e-12 if q["dtype"] == "f64" else 1e-5
                l2, mx = oracle.error_norms(out, oracle.gather(a, q["r"], q["cg"], "dirichlet", q["steps"]))
                assert l2 <= tol and mx <= tol
        stats = sx.stencil_server_stats(srv)
        assert stats["completed"] == len(reqs)
        assert stats["peak_resident"] <= max_resident
        assert stats["peak_bytes"] <= budget_mb << 20  # admission kept the device memory within the budget
        if budget_mb == 3:
            assert stats["peak_resident"] < max_resident
    finally:
        sx.stencil_server_destroy(srv)


def test_server_errors_and_timeouts():
    srv = sx.stencil_server_create(8 << 20, 4, 8, 2)
    try:
        cg = np.full((3, 3), 1 / 9)
        rq, keep = sx.make_request((64, 64), 1, "star", cg, "f32", 5)  # star with off-axis weights
        rid = sx.stencil_server_submit(srv, rq)
        assert sx.stencil_server_wait(srv, rid, 10_000) == sx.EINVAL
        with pytest.raises(sx.StencilError):
            sx.stencil_server_result(srv, rid)
        big, keep2 = sx.make_request((4096, 4096), 1, "box", cg, "f32", 5)
        with pytest.raises(sx.StencilError) as ei:
            sx.stencil_server_submit(srv, big)
        assert ei.value.status == sx.ENOMEM
        slow, keep3 = sx.make_request((512, 512), 1, "box", cg, "f32", 2000)
        rid = sx.stencil_server_submit(srv, slow)
        assert sx.stencil_server_wait(srv, rid, 0) == sx.ETIMEDOUT
        assert sx.stencil_server_wait(srv, rid, 60_000) == sx.OK
        sx.stencil_server_result(srv, rid, None)
        assert sx.stencil_server_poll(srv, 999_999) == sx.EINVAL
    finally:
        sx.stencil_server_destroy(srv)
