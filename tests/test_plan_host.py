"""Host-side checks of the C library: it loads, exports every symbol the header
declares, and its plan algebra matches what the paper fixes (no GPU needed)."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_2310_16298_gb300 as sx
import stencil_inputs as si

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def header_functions():
    src = open(os.path.join(ROOT, "include", "stencil.h")).read()
    return sorted(set(re.findall(r"STENCIL_API\s+[\w\s\*]+?\b(stencil_\w+)\s*\(", src)))


def test_library_exports_every_header_symbol():
    lib = sx.lib()
    names = header_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(sx.exported_symbols())
    assert "sm_103a" in sx.stencil_version()


def test_band_operand_matches_worked_example():
    """The banded operand of one coefficient line, pad = r, n = 3, reproduces
    the coefficient vectors of Eq. (stencil-2d9p-scatter-extend-2): output q of
    the block (B[i-1], B[i], B[i+1]) receives input row k (A[i-2..i+2])."""
    codes = {(a, b): 100 + 10 * a + b for a in range(3) for b in range(3)}
    line = np.array([codes[(0, 1)], codes[(1, 1)], codes[(2, 1)]], dtype=float)  # C^g column 1
    band = sx.stencil_band_operand(1, line, 3, 1)
    rows = [l.split() for l in open(os.path.join(GOLDEN, "eq_scatter_extend2_r1.txt"))
            if l.strip() and not l.startswith("#")]
    assert band.shape == (5, 3)
    for off_s, *vec in rows:
        k = int(off_s) + 2
        want = [0.0 if v == "0" else codes[(int(v[0]), int(v[1]))] for v in vec]
        assert list(band[k]) == want


def test_band_operand_padding_shifts_window():
    w = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    b2 = sx.stencil_band_operand(2, w, 4, 2)
    b4 = sx.stencil_band_operand(2, w, 4, 4)
    assert b4.shape == (12, 4)
    assert np.array_equal(b4[2:10], b2)
    assert not b4[:2].any() and not b4[10:].any()
    # Toeplitz: constant along diagonals
    for k in range(1, 8):
        for q in range(1, 4):
            assert b2[k, q] == b2[k - 1, q - 1]


def test_band_operand_rejects_bad_pad():
    with pytest.raises(sx.StencilError):
        sx.stencil_band_operand(2, np.ones(5), 4, 1)


@pytest.mark.parametrize("r", [1, 2, 3])
@pytest.mark.parametrize("n", [4, 8, 16])
def test_line_cover_counts_match_tables(r, n):
    # box: (2r+1) lines of 2r+n outer products (Sec. 3.4); 3D box (2r+1)^2 lines
    assert sx.stencil_line_cover(2, r, "box", 0, n) == (2 * r + 1, (2 * r + 1) * (2 * r + n))
    assert sx.stencil_line_cover(3, r, "box", 0, n) == ((2 * r + 1) ** 2, (2 * r + 1) ** 2 * (2 * r + n))
    # Table cls-2d
    assert sx.stencil_line_cover(2, r, "star", 0, n) == (2 * r + 1, (2 * r + n) + 2 * r * n)
    assert sx.stencil_line_cover(2, r, "star", 1, n) == (2, 2 * (2 * r + n))
    # Table cls-3d
    assert sx.stencil_line_cover(3, r, "star", 0, n) == (4 * r + 1, (2 * r + n) + 4 * r * n)
    assert sx.stencil_line_cover(3, r, "star", 1, n) == (3, 3 * (2 * r + n))
    assert sx.stencil_line_cover(3, r, "star", 2, n) == (2 * r + 2, 2 * (2 * r + n) + 2 * r * n)


def test_line_cover_invalid_options():
    with pytest.raises(sx.StencilError):
        sx.stencil_line_cover(2, 1, "box", 1, 8)
    with pytest.raises(sx.StencilError):
        sx.stencil_line_cover(2, 1, "star", 2, 8)


@pytest.mark.parametrize("args,msg", [
    (dict(shape=(16, 16), radius=0, kind="box", coeffs=np.ones((1, 1))), "radius"),
    (dict(shape=(16, 16), radius=5, kind="box", coeffs=np.ones((11, 11))), "radius"),
    (dict(shape=(4, 16), radius=2, kind="box", coeffs=np.ones((5, 5))), "extent"),
    (dict(shape=(16,), radius=1, kind="box", coeffs=np.ones(3)), "ndim"),
    (dict(shape=(16, 16), radius=1, kind="star", coeffs=np.ones((3, 3))), "off-axis"),
    (dict(shape=(16, 16), radius=1, kind="box", coeffs=np.full((3, 3), np.nan)), "finite"),
])
def test_plan_create_rejects_invalid_problems(args, msg):
    with pytest.raises(sx.StencilError) as ei:
        sx.stencil_plan_create(args["shape"], args["radius"], args["kind"], args["coeffs"], "f32")
    assert ei.value.status == sx.EINVAL
    assert msg in str(ei.value)


def test_plan_create_rejects_unknown_cover():
    with pytest.raises(sx.StencilError) as ei:
        sx.stencil_plan_create((16, 16), 1, "box", np.ones((3, 3)), "f32", sx.make_options(cover=7))
    assert ei.value.status == sx.EINVAL
    assert "cover" in str(ei.value)


def test_plan_create_rejects_tensor_precision_for_f64():
    with pytest.raises(sx.StencilError) as ei:
        sx.stencil_plan_create((16, 16), 1, "box", np.ones((3, 3)), "f64", sx.make_options(prec="tf32"))
    assert ei.value.status == sx.EINVAL


@pytest.mark.parametrize("tb,tile_shape", [(9, -1), (-1, 0), (0, 2), (1, -2)])
def test_batch_create_rejects_out_of_range_depth_and_shape(tb, tile_shape):
    # argument checks come before any plan is dereferenced or any device call
    with pytest.raises(sx.StencilError):
        sx.stencil_batch_create_ex([1], [1], [1], [1], tb, tile_shape)


def test_unknown_ticket_is_rejected():
    assert sx.stencil_poll(123456789) == sx.EINVAL
    assert sx.stencil_wait(123456789, 0) == sx.EINVAL


# ---------------------------------------------------------------- minimal line cover (Sec. 3.5)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 9])
@pytest.mark.parametrize("density", [0.15, 0.4, 0.7, 1.0])
def test_min_line_cover_matches_oracle(n, density):
    for seed in range(8):
        mask = si.uniform(7919 * n + seed + int(1000 * density), n * n).reshape(n, n) < density
        count, rows, cols = sx.stencil_min_line_cover(mask)
        want = oracle.min_line_cover(mask)[0]
        assert count == want == rows.sum() + cols.sum()
        assert all(rows[i] or cols[j] for i, j in zip(*np.nonzero(mask)))


def test_min_line_cover_star_and_box_agree_with_line_cover_counts():
    for r in (1, 2, 3, 4):
        n = 2 * r + 1
        star = np.zeros((n, n), dtype=bool)
        star[r, :] = star[:, r] = True
        assert sx.stencil_min_line_cover(star)[0] == sx.stencil_line_cover(2, r, "star", 1, 8)[0] == 2
        assert sx.stencil_min_line_cover(np.ones((n, n)))[0] == sx.stencil_line_cover(2, r, "box", 0, 8)[0] == n


@pytest.mark.parametrize("n", [16, 33, 64])
def test_min_line_cover_large_konig(n):
    """Large patterns: a valid cover whose size equals a maximum matching
    (Konig's theorem), the matching taken from SciPy."""
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    import scipy.sparse as sp
    for seed in range(4):
        mask = si.uniform(31 * n + seed, n * n).reshape(n, n) < 0.08
        count, rows, cols = sx.stencil_min_line_cover(mask)
        assert all(rows[i] or cols[j] for i, j in zip(*np.nonzero(mask)))
        match = csgraph.maximum_bipartite_matching(sp.csr_matrix(mask.astype(np.int8)), perm_type="column")
        assert count == int((match >= 0).sum())


def test_min_line_cover_rejects_bad_sizes():
    with pytest.raises(sx.StencilError):
        sx.stencil_min_line_cover(np.zeros((0, 0)))
    with pytest.raises(sx.StencilError):
        sx.stencil_min_line_cover(np.ones((65, 65)))
