"""asyrk_residual_noalloc: the residual entry point that allocates nothing.

Callers that cannot call cudaMalloc (their device memory is all in their own
pool, or cudaMalloc/cudaFree would stall a latency-critical path) use it on a
CSR system they already hold on the device.  Its result must equal the result of
asyrk_residual, the handle-based entry point, on the same system -- on two calls
in a row, since every call reuses the same static scratch array -- and the FP64
oracle's ||b - A x|| and ||b||, for every stored value type.  This file is
collected last, and passes alone in a fresh process as well as after the others.
"""
import numpy as np
import pytest

import oracle
from paper_1401_4780_gb300 import asyrk, synth

pytestmark = pytest.mark.gpu

_DTYPES = {"f64": asyrk.F64, "f32": asyrk.F32, "bf16": asyrk.BF16}


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    asyrk.load()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_noalloc_residual_matches_handle_residual_and_oracle_on_consecutive_calls(dtype):
    import torch
    s = synth.make_system(50_000, 12_000, (3, 40), 77, row_norms="lognormal", value_dtype=dtype)
    rng = np.random.default_rng(9)
    xs = [rng.standard_normal(s.n), s.x_true + 1e-3 * rng.standard_normal(s.n)]
    with asyrk.Problem.from_system(s) as p:
        want = [p.residual(x) for x in xs]  # ||b - Ax|| / ||b|| from the existing entry point
    bnorm = np.linalg.norm(s.b)

    rp, col, val, b = _dev(s.row_ptr), _dev(s.col), _dev(s.val_store), _dev(s.b)
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for x, w in zip(xs, want):  # two calls in a row on the shared scratch
        xd = _dev(x)
        st = asyrk.asyrk_residual_noalloc(s.m, s.n, s.nnz, rp, col, val, _DTYPES[dtype], b, xd,
                                          out, stream=stream)
        assert st == asyrk.OK, asyrk.asyrk_last_error()
        torch.cuda.synchronize()
        r, bn = out.cpu().numpy()
        # the oracle's FP64 residual of the same stored values (widened exactly)
        r_or, _ = oracle.residual(s.m, s.row_ptr, s.col, s.val64, s.b, x)
        assert abs(bn - bnorm) <= 1e-12 * bnorm
        assert abs(r - r_or) <= 1e-12 * r_or, (r, r_or)
        assert abs(r / bn - w) <= 1e-12 * w, (r / bn, w)


@pytest.mark.parametrize("defect", ["column_equal_to_n", "row_ptr_beyond_nnz"])
def test_noalloc_out_of_range_entries_give_nan_without_reading_them(defect):
    # the kernel checks each column against [0, n) and each row's range against
    # [0, nnz) before it reads col, values or x, so these inputs are safe; the
    # documented result is out[0] = NaN, out[1] = ||b||
    import torch
    s = synth.make_system(3000, 700, (2, 20), 5, row_norms="unit", value_dtype="f64")
    col = s.col.copy()
    row_ptr = s.row_ptr.copy()
    if defect == "column_equal_to_n":
        col[int(s.row_ptr[1234]) + 1] = s.n
    else:
        row_ptr[-1] = s.nnz + 3  # the last row would run past the stored entries
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    st = asyrk.asyrk_residual_noalloc(s.m, s.n, s.nnz, _dev(row_ptr), _dev(col), _dev(s.val64),
                                      asyrk.F64, _dev(s.b), _dev(np.zeros(s.n)), out,
                                      stream=torch.cuda.current_stream())
    assert st == asyrk.OK, asyrk.asyrk_last_error()
    torch.cuda.synchronize()
    r, bn = out.cpu().numpy()
    assert np.isnan(r)
    assert abs(bn - np.linalg.norm(s.b)) <= 1e-12 * bn


def test_noalloc_rejects_more_rows_than_its_scratch_holds():
    import torch
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = asyrk.asyrk_residual_noalloc(asyrk.NOALLOC_MAX_ROWS + 1, 4, 4, dummy, dummy, dummy,
                                      asyrk.F64, dummy, dummy, dummy)
    assert st == asyrk.EINVAL
    assert "exceeds" in asyrk.asyrk_last_error()
