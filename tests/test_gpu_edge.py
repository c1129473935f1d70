"""Edge cases and error behaviour of the C ABI on the GPU.

Malformed problems are rejected by asyrk_create (Section 1: no zero rows; the
CSR rules of asyrk.h); degenerate systems (one row, one column, rows of one
entry, x0 already at x*, max_sweeps = 0) and an inconsistent system (which
never reaches the tolerance) give the documented statuses.
"""
import numpy as np
import pytest

import oracle
from paper_1401_4780_gb300 import asyrk, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    asyrk.load()


def _base():
    row_ptr = np.array([0, 2, 4, 6, 8], dtype=np.int64)
    col = np.array([0, 3, 1, 2, 4, 5, 0, 5], dtype=np.int32)
    val = np.arange(1.0, 9.0)
    b = np.ones(4)
    return row_ptr, col, val, b


@pytest.mark.parametrize("defect", ["zero_row", "unsorted", "duplicate", "out_of_range",
                                    "negative", "nan", "zero_values", "row_ptr0", "b_inf",
                                    "decreasing"])
def test_malformed_problem_is_rejected(defect):
    row_ptr, col, val, b = _base()
    if defect == "zero_row":
        row_ptr = np.array([0, 2, 2, 4, 6], dtype=np.int64)
        col, val = col[:6].copy(), val[:6].copy()
    elif defect == "unsorted":
        col[0], col[1] = 3, 0
    elif defect == "duplicate":
        col[1] = 0
    elif defect == "out_of_range":
        col[7] = 6
    elif defect == "negative":
        col[2] = -1
    elif defect == "nan":
        val[3] = np.nan
    elif defect == "zero_values":
        val[2:4] = 0.0
    elif defect == "row_ptr0":
        row_ptr = row_ptr + 1
    elif defect == "b_inf":
        b[2] = np.inf
    elif defect == "decreasing":
        row_ptr = np.array([0, 4, 2, 6, 8], dtype=np.int64)
    st, h = asyrk.asyrk_create(4, 6, row_ptr, col, val, asyrk.F64, b)
    assert st == asyrk.EINVAL and not h.value, (st, asyrk.asyrk_last_error())
    # the oracle's own checks agree
    if defect != "decreasing":
        assert oracle.validate(4, 6, row_ptr, col, val, b) == oracle.EINVAL


@pytest.mark.parametrize("which", ["frobenius", "b"])
def test_totals_beyond_the_fp64_range_are_rejected(which):
    # every value and every row weight is finite, but ||A||_F^2 (four rows of
    # weight 1e308) or ||b||^2 (b_i = 1e200) is not: the exact sums carry into
    # their top digits and round to infinity, and create refuses the problem
    row_ptr = np.arange(5, dtype=np.int64)
    col = np.arange(4, dtype=np.int32)
    val = np.full(4, 1e154) if which == "frobenius" else np.ones(4)
    b = np.ones(4) if which == "frobenius" else np.full(4, 1e200)
    st, h = asyrk.asyrk_create(4, 4, row_ptr, col, val, asyrk.F64, b)
    assert st == asyrk.EINVAL and not h.value
    assert "not finite" in asyrk.asyrk_last_error()
    if which == "frobenius":  # the oracle's F overflows the same way
        assert oracle.validate(4, 4, row_ptr, col, val, b) == oracle.OK
        assert oracle.row_weights(4, row_ptr, val)[1] == np.inf


def test_well_formed_base_is_accepted():
    row_ptr, col, val, b = _base()
    with asyrk.Problem(4, 6, row_ptr, col, val, asyrk.F64, b) as p:
        assert p.stats()["nnz"] == 8


@pytest.mark.parametrize("bad", [{"gamma": 0.0}, {"gamma": 2.0}, {"max_sweeps": -1},
                                 {"check_every": -1}, {"subwarp": 3}, {"workers": -2},
                                 {"mode": 9}])
def test_solve_argument_errors(bad):
    s = synth.make_system(64, 16, 4, 1)
    with asyrk.Problem.from_system(s) as p:
        kw = dict(gamma=1.0, tol=1e-6, max_sweeps=10)
        opt = {}
        for k, v in bad.items():
            (kw if k in kw else opt).__setitem__(k, v)
        st, info = p.solve(np.zeros(s.n), raise_on_error=False, **kw, **opt)
        assert st == asyrk.EINVAL


def test_one_row_system_solved_in_one_projection():
    n = 37
    rng = np.random.default_rng(0)
    val = rng.standard_normal(n)
    with asyrk.Problem(1, n, np.array([0, n], dtype=np.int64), np.arange(n, dtype=np.int32), val,
                       asyrk.F64, np.array([1.5])) as p:
        x = rng.standard_normal(n)
        st, info = p.solve(x, tol=0.0, max_sweeps=1, mode=asyrk.MODE_SEQUENTIAL)
        assert st == asyrk.OK
        assert abs(val @ x - 1.5) <= 1e-13
        assert info.rel_res <= 1e-13


def test_one_column_system():
    m = 50
    rng = np.random.default_rng(1)
    val = rng.standard_normal(m) + 3.0
    xs = np.array([2.0])
    with asyrk.Problem(m, 1, np.arange(m + 1, dtype=np.int64), np.zeros(m, dtype=np.int32), val,
                       asyrk.F64, val * 2.0) as p:
        x = np.zeros(1)
        st, info = p.solve(x, tol=1e-12, max_sweeps=10, x_true=xs)
        assert st == asyrk.OK and abs(x[0] - 2.0) <= 1e-12 * 2


def test_start_at_solution_does_no_work():
    s = synth.make_system(256, 64, 8, 2)
    with asyrk.Problem.from_system(s) as p:
        x = s.x_true.copy()
        st, info = p.solve(x, tol=1e-10, max_sweeps=10, x_true=s.x_true)
        assert st == asyrk.OK and info.sweeps == 0 and info.projections == 0
        np.testing.assert_array_equal(x, s.x_true)


def test_zero_sweeps_returns_x0():
    s = synth.make_system(256, 64, 8, 2)
    with asyrk.Problem.from_system(s) as p:
        x0 = np.random.default_rng(5).standard_normal(s.n)
        x = x0.copy()
        st, info = p.solve(x, tol=1e-10, max_sweeps=0)
        assert st == asyrk.NOT_CONVERGED and info.projections == 0
        np.testing.assert_array_equal(x, x0)


@pytest.mark.parametrize("mode", [asyrk.MODE_ASYNC, asyrk.MODE_REFINE])
def test_inconsistent_system_reports_not_converged(mode):
    s = synth.make_system(512, 128, 8, 3, value_dtype="f32")
    b = s.b + np.random.default_rng(2).standard_normal(s.m)  # not in the range of A
    with asyrk.Problem(s.m, s.n, s.row_ptr, s.col, s.val_store, asyrk.F32, b) as p:
        x = np.zeros(s.n)
        st, info = p.solve(x, tol=1e-8, max_sweeps=30, mode=mode)
        assert st == asyrk.NOT_CONVERGED
        assert 0.05 < info.rel_res < 1.0 and info.sweeps == 30


def test_single_entry_rows_and_many_workers():
    # diagonal-like system: each row has one entry; RK solves it exactly
    m = n = 1000
    rng = np.random.default_rng(7)
    # |a_i| in [1, 2]: every row is drawn often enough (sampling is ~ a_i^2)
    val = (1.0 + rng.random(m)) * np.sign(rng.standard_normal(m))
    xs = rng.standard_normal(n)
    with asyrk.Problem(m, n, np.arange(m + 1, dtype=np.int64), np.arange(n, dtype=np.int32), val,
                       asyrk.F64, val * xs) as p:
        x = np.zeros(n)
        st, info = p.solve(x, tol=1e-12, max_sweeps=200, x_true=xs, workers=512)
        assert st == asyrk.OK and info.workers == 512
        assert np.max(np.abs(x - xs)) <= 1e-12 * np.max(np.abs(xs))


def test_half_a_billion_rows_64bit_offsets():
    """m = 2^29 + 7 rows of one entry each (padded to 4: 2^31 + 28 stored
    entries, so row starts pass 2^31): the alias table built on the GPU over the
    whole m draws the three weight classes in proportion (chi-square), and one
    sweep solves the diagonal-block system (each column's rows agree)."""
    import torch
    from scipy import stats
    m, n = (1 << 29) + 7, 1 << 20
    dev = "cuda"
    i = torch.arange(m, dtype=torch.int64, device=dev)
    row_ptr = torch.arange(m + 1, dtype=torch.int64, device=dev)
    col = (i % n).to(torch.int32)
    val = (1 + (i % 3)).to(torch.float32)
    x_true = torch.linspace(-1.0, 1.0, n, dtype=torch.float64, device=dev)
    b = val.double() * x_true[col.long()]
    del i
    torch.cuda.synchronize()
    with asyrk.Problem(m, n, row_ptr, col, val, asyrk.F32, b, seed=5, device_ptrs=True) as p:
        del row_ptr, col, b
        st_ = p.stats()
        assert st_["m"] == m and st_["nnz_padded"] == 4 * m and st_["uniform"] == 0
        rows = p.draw_rows(2**33 + 11, 1 << 20)
        assert rows.min() >= 0 and rows.max() < m
        counts = np.bincount(rows % 3, minlength=3)
        sizes = np.array([(m + 2) // 3, (m + 1) // 3, m // 3], dtype=np.float64)
        expected = sizes * np.array([1.0, 4.0, 9.0])
        expected = expected / expected.sum() * rows.size
        assert stats.chisquare(counts, expected).pvalue > 1e-4
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        st, info = p.solve(x, tol=1e-6, max_sweeps=3, device_ptrs=True, x_true=x_true)
        assert st == asyrk.OK, info.as_dict()
    del val
    torch.cuda.empty_cache()


def test_reused_pool_memory_gives_the_same_solve_and_trim():
    # a problem created in memory that another problem used and freed (the
    # pool keeps it) solves bit for bit like the first problem did; trimming
    # the pool between problems changes nothing either
    s = synth.make_system(4096, 1024, 16, 31, row_norms="lognormal", value_dtype="f32")
    other = synth.make_system(8192, 2048, 24, 32, row_norms="lognormal", value_dtype="f32")
    xs = []
    for k in range(3):
        with asyrk.Problem.from_system(s) as p:
            x = np.zeros(s.n)
            st, info = p.solve(x, tol=1e-5, max_sweeps=400, x_true=s.x_true,
                               mode=asyrk.MODE_SEQUENTIAL)
            assert st == asyrk.OK, (st, info.as_dict())
            xs.append(x)
        with asyrk.Problem.from_system(other) as q:
            y = np.full(other.n, 7.0)
            st, _ = q.solve(y, tol=1e-3, max_sweeps=50, x_true=other.x_true)
            assert st == asyrk.OK
        if k == 1:
            assert asyrk.asyrk_trim_memory() == asyrk.OK
    np.testing.assert_array_equal(xs[0], xs[1])
    np.testing.assert_array_equal(xs[0], xs[2])


@pytest.mark.parametrize("lengths", [(30, 42), 36])
def test_host_entries_in_chunks_match_a_device_created_problem(lengths):
    # 151 MB of entries reach the device in three chunks, each chunk's rows set
    # up as it arrives (rows of 30..42 entries: 4-misaligned starts, the padding
    # copy; 36 per row: the staged entries kept as they are).  The same system
    # created from device arrays (one pass) gives the same records, sums, alias
    # table and sequential iterate, and F is the oracle's
    import torch
    m, n = 1 << 19, 1 << 17
    s = synth.make_system(m, n, lengths, 77, row_norms="lognormal", value_dtype="f32")
    assert s.row_ptr[-1] * 8 > 2 * (64 << 20)
    seed = synth.solver_seed(s.seed)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda()
           for a in (s.row_ptr, s.col, s.val_store, s.b)]
    with asyrk.Problem.from_system(s) as ph, \
            asyrk.Problem(m, n, *dev[:3], asyrk.F32, dev[3], seed=seed, device_ptrs=True) as pd:
        sh, sd = ph.stats(), pd.stats()
        for k in ("nnz", "nnz_padded", "max_row_len", "frob2", "uniform"):
            assert sh[k] == sd[k], k
        assert (sh["nnz_padded"] == sh["nnz"]) == (lengths == 36)
        assert sh["frob2"] == oracle.Sampler(m, s.row_ptr, s.val64).F
        np.testing.assert_array_equal(ph.draw_rows(12345, 200000), pd.draw_rows(12345, 200000))
        xs = []
        for p in (ph, pd):
            x = np.zeros(n)
            st, info = p.solve(x, tol=0.0, max_sweeps=1, mode=asyrk.MODE_SEQUENTIAL)
            assert st == asyrk.OK
            xs.append(x)
        np.testing.assert_array_equal(xs[0], xs[1])
        assert np.isfinite(xs[0]).all() and np.linalg.norm(xs[0]) > 0
