"""GPU check of the FP64 error-norm reduction (the accuracy report attached to
every result) against the same four sums formed on the host in FP64."""
import numpy as np
import pytest

import paper_2310_16298_gb300 as sx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("count", [1, 255, 256 * 608 + 17, 3_000_001])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_error_norms_match_host(count, dtype):
    import torch
    rng = np.random.default_rng(count)
    ref = rng.uniform(-2.0, 2.0, size=count)
    got = ref + rng.normal(0.0, 1e-3, size=count)
    got = got.astype(np.float32) if dtype == "f32" else got
    g = torch.from_numpy(got).cuda()
    o = torch.from_numpy(ref).cuda()
    out = sx.stencil_error_norms(g.data_ptr(), dtype, o.data_ptr(), count)
    d = got.astype(np.float64) - ref
    want = np.array([np.dot(d, d), np.dot(ref, ref), np.abs(d).max(), np.abs(ref).max()])
    assert out[2] == want[2] and out[3] == want[3]
    assert np.allclose(out[:2], want[:2], rtol=1e-12, atol=0)


def test_error_norms_empty_and_errors():
    import torch
    g = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = sx.stencil_error_norms(g.data_ptr(), "f64", g.data_ptr(), 0)
    assert np.array_equal(out, np.zeros(4))
    with pytest.raises(sx.StencilError):
        sx.stencil_error_norms(g.data_ptr(), "f64", g.data_ptr(), -1)
