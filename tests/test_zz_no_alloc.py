"""asyrk_residual_noalloc: the residual entry point that allocates nothing.

Callers that cannot call cudaMalloc (their device memory is all in their own
pool, or cudaMalloc/cudaFree would stall a latency-critical path) use it on a
CSR system they already hold on the device.  Its result must equal the result of
asyrk_residual, the handle-based entry point, on the same system -- on two calls
in a row, since every call reuses the same static scratch array.  This file is
collected last, and passes alone in a fresh process as well as after the others.
"""
import numpy as np
import pytest

from paper_1401_4780_gb300 import asyrk, synth

pytestmark = pytest.mark.gpu


def test_noalloc_residual_matches_handle_residual_on_consecutive_calls():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    asyrk.load()
    s = synth.make_system(50_000, 12_000, (3, 40), 77, row_norms="lognormal", value_dtype="f32")
    rng = np.random.default_rng(9)
    xs = [rng.standard_normal(s.n), s.x_true + 1e-3 * rng.standard_normal(s.n)]
    with asyrk.Problem.from_system(s) as p:
        want = [p.residual(x) for x in xs]  # ||b - Ax|| / ||b|| from the existing entry point

    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rp, col, val, b = d(s.row_ptr), d(s.col), d(s.val_store), d(s.b)
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for x, w in zip(xs, want):  # two calls in a row on the shared scratch
        xd = d(x)
        st = asyrk.asyrk_residual_noalloc(s.m, s.n, s.nnz, rp, col, val, asyrk.F32, b, xd, out,
                                          stream=stream)
        assert st == asyrk.OK, asyrk.asyrk_last_error()
        torch.cuda.synchronize()
        r, bn = out.cpu().numpy()
        assert abs(bn - np.linalg.norm(s.b)) <= 1e-12 * bn
        assert abs(r / bn - w) <= 1e-12 * w, (r / bn, w)


def test_noalloc_rejects_more_rows_than_its_scratch_holds():
    import torch
    asyrk.load()
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = asyrk.asyrk_residual_noalloc(asyrk.NOALLOC_MAX_ROWS + 1, 4, 4, dummy, dummy, dummy,
                                      asyrk.F64, dummy, dummy, dummy)
    assert st == asyrk.EINVAL
    assert "exceeds" in asyrk.asyrk_last_error()
