"""Helpers for the GPU tests: run a problem through the C ABI on torch device
memory with guard bands around the output, and compare with the oracle."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2310_16298_gb300 as sx

GUARD = 4096  # elements of canary before and after each output grid
CANARY = 1234.5

# Tolerances on rel-L2 and rel-max against the FP64 oracle.  Plain TF32 and
# the BF16 family are set from their operand mantissas (TF32 11 bits, BF16 8,
# BF16x2 16, BF16x3 24); BF16_W2 rounds the field to 8 bits like plain BF16.
TOL = {"f64": 1e-12, "f32": 1e-5, "tf32x3": 1e-5, "bf16x3": 1e-5, "bf16x2": 1e-4, "tf32": 1e-3,
       "bf16": 1e-2, "bf16w2": 1e-2}


def torch_dtype(dtype):
    import torch
    return torch.float32 if dtype == "f32" else torch.float64


def run(field: np.ndarray, r: int, kind: str, cg: np.ndarray, dtype: str, bc: str, steps: int,
        impl: str = "gather", prec: str = "native", tb: int = 0, check_guard: bool = True,
        alias: bool = False, cover: str = "auto"):
    """Returns (result as float64 ndarray, plan info)."""
    import torch
    td = torch_dtype(dtype)
    n = field.size
    buf_in = torch.full((n + 2 * GUARD,), CANARY, dtype=td, device="cuda")
    buf_out = torch.full((n + 2 * GUARD,), CANARY, dtype=td, device="cuda")
    x = buf_in[GUARD:GUARD + n]
    x.copy_(torch.from_numpy(np.ascontiguousarray(field).ravel()).to(td))
    y = x if alias else buf_out[GUARD:GUARD + n]
    plan = sx.stencil_plan_create(field.shape, r, kind, cg, dtype, sx.make_options(prec, bc, impl, tb, cover))
    try:
        stream = torch.cuda.current_stream()
        sx.stencil_apply(plan, x.data_ptr(), y.data_ptr(), steps, stream.cuda_stream)
        torch.cuda.synchronize()
        info = sx.stencil_plan_info(plan)
        assert info["device_error"] == 0, "a kernel gave up a bounded wait"
    finally:
        sx.stencil_plan_destroy(plan)
    if check_guard:
        for buf in (buf_in, buf_out):
            head = buf[:GUARD].double().cpu().numpy()
            tail = buf[GUARD + n:].double().cpu().numpy()
            assert np.all(head == CANARY) and np.all(tail == CANARY), "guard band overwritten"
        if not alias:
            assert np.array_equal(buf_in[GUARD:GUARD + n].cpu().numpy().reshape(field.shape),
                                  np.ascontiguousarray(field).astype(np.float32 if dtype == "f32" else np.float64)), \
                "input grid modified"
    return y.double().cpu().numpy().reshape(field.shape), info


def check(got: np.ndarray, want: np.ndarray, tol: float, what: str = ""):
    l2, mx = oracle.error_norms(got, want)
    assert l2 <= tol and mx <= tol, f"{what}: rel_l2={l2:.3e} rel_max={mx:.3e} tol={tol:.1e}"
    return l2, mx
