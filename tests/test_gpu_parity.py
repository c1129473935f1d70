"""GPU parity of libasyrk.so against the FP64 oracle, through the C ABI.

  * sampler: the GPU's row sequence equals the oracle's bit for bit;
  * single worker (SEQUENTIAL mode): the FP64 iterate matches the oracle's
    sequential RK iterate (Eq. (2)) to 1e-12 relative, on the plain FP64
    workload (m=4096, n=1024, 16 nnz/row) and on ragged rows with every
    sub-warp width, including rows longer than a worker keeps in registers;
  * residual ||b - A x||/||b|| in FP64 matches the oracle's to 1e-12;
  * resuming from a saved position reproduces the uninterrupted run exactly.
"""
import math

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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _oracle_steps(s, seed, nsteps, gamma=1.0, j0=0, x0=None):
    x = np.zeros(s.n) if x0 is None else x0.copy()
    oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x, gamma, seed, 0, j0, nsteps)
    return x


# ---------------------------------------------------------------------------
# sampler
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["unit_f64", "lognormal_f32", "uniform"])
def test_row_sequence_is_bit_exact(kind):
    if kind == "unit_f64":
        s = synth.plain_f64_system()
    elif kind == "lognormal_f32":
        s = synth.make_system(1 << 16, 1 << 14, 32, 99, row_norms="lognormal", value_dtype="f32")
    else:  # every row has the same bit-identical weight: the table is skipped
        m, n = 3000, 500
        s = synth.make_system(m, n, 4, 5, value_dtype="f64")
        s.val_store[:] = 0.5
        s.b = synth.spmv_f64(m, s.row_ptr, s.col, s.val64, s.x_true)
    seed = synth.solver_seed(s.seed)
    samp = oracle.Sampler(s.m, s.row_ptr, s.val64)
    with asyrk.Problem.from_system(s) as p:
        assert p.stats()["uniform"] == samp.uniform
        assert p.stats()["frob2"] == samp.F == math.fsum(samp.w)
        for j0, count, stream in [(0, 1_000_000, 0), (2**32 - 500, 1000, 0), (12345, 5000, 7)]:
            got = p.draw_rows(j0, count, stream)
            want = oracle.draw_rows(seed, stream, j0, count, samp.thr, samp.alias, samp.uniform)
            np.testing.assert_array_equal(got, want)


# ---------------------------------------------------------------------------
# single-worker FP64 iterate
# ---------------------------------------------------------------------------
def test_sequential_iterate_matches_oracle_plain_f64_workload():
    s = synth.plain_f64_system()
    seed = synth.solver_seed(s.seed)
    with asyrk.Problem.from_system(s) as p:
        x = np.zeros(s.n)
        st, info = p.solve(x, tol=0.0, max_sweeps=5, mode=asyrk.MODE_SEQUENTIAL)
        assert st == asyrk.OK and info.projections == 5 * s.m and info.workers == 1
        assert info.skipped == 0
        xo = _oracle_steps(s, seed, 5 * s.m)
        assert _rel(x, xo) <= 1e-12
        # continue to the oracle's converged sweep count: still the same iterate
        xo2 = np.zeros(s.n)
        res = oracle.rk_solve(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, xo2, 1.0, seed, 1e-8, 200,
                              x_true=s.x_true)
        assert res.status == oracle.OK
        p.position = 0
        x2 = np.zeros(s.n)
        st, info = p.solve(x2, tol=1e-8, max_sweeps=200, x_true=s.x_true,
                           mode=asyrk.MODE_SEQUENTIAL)
        assert st == asyrk.OK
        assert info.sweeps == res.sweeps
        assert _rel(x2, xo2) <= 1e-12
        assert info.rel_err <= 1e-8
        assert abs(info.rel_err - res.rel_err) <= 1e-3 * res.rel_err


@pytest.mark.parametrize("subwarp", [1, 2, 4, 8, 16, 32])
def test_sequential_iterate_ragged_rows_every_subwarp(subwarp):
    # row lengths 1..70: unaligned starts (padding path), chunk tails, rows
    # longer than 4*subwarp*2 entries (re-load path); subwarp 1 = one lane per row
    s = synth.make_system(700, 400, (1, 70), 4242, row_norms="lognormal", value_dtype="f64")
    seed = synth.solver_seed(s.seed)
    with asyrk.Problem.from_system(s) as p:
        st_ = p.stats()
        assert st_["nnz"] == s.nnz and st_["nnz_padded"] >= s.nnz and st_["max_row_len"] <= 70
        x0 = np.random.default_rng(1).standard_normal(s.n)
        x = x0.copy()
        st, info = p.solve(x, gamma=0.8, tol=0.0, max_sweeps=3, subwarp=subwarp,
                           mode=asyrk.MODE_SEQUENTIAL)
        assert st == asyrk.OK and info.subwarp == subwarp
        xo = _oracle_steps(s, seed, 3 * s.m, gamma=0.8, x0=x0)
        assert _rel(x, xo) <= 1e-12


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_sequential_iterate_on_narrow_stored_values(dtype):
    # values stored in FP32 / BF16, widened exactly to FP64 on both sides
    s = synth.make_system(2048, 512, 16, 77, row_norms="unit", value_dtype=dtype)
    seed = synth.solver_seed(s.seed)
    with asyrk.Problem.from_system(s) as p:
        x = np.zeros(s.n)
        st, _ = p.solve(x, tol=0.0, max_sweeps=4, mode=asyrk.MODE_SEQUENTIAL)
        assert st == asyrk.OK
        assert _rel(x, _oracle_steps(s, seed, 4 * s.m)) <= 1e-12


def test_resume_from_saved_position_is_exact():
    s = synth.make_system(1024, 256, 12, 3, row_norms="lognormal", value_dtype="f64")
    with asyrk.Problem.from_system(s) as p:
        x_full = np.zeros(s.n)
        p.solve(x_full, tol=0.0, max_sweeps=5, mode=asyrk.MODE_SEQUENTIAL)
        p.position = 0
        x = np.zeros(s.n)
        p.solve(x, tol=0.0, max_sweeps=2, mode=asyrk.MODE_SEQUENTIAL)
        saved_x, saved_j = x.copy(), p.position
        assert saved_j == 2 * s.m
        p.position = 999  # disturb, then restore
        p.position = saved_j
        p.solve(saved_x, tol=0.0, max_sweeps=3, mode=asyrk.MODE_SEQUENTIAL)
        np.testing.assert_array_equal(saved_x, x_full)


def test_residual_matches_oracle():
    s = synth.make_system(3000, 800, (5, 40), 8, row_norms="lognormal", value_dtype="f32")
    x = np.random.default_rng(3).standard_normal(s.n)
    with asyrk.Problem.from_system(s) as p:
        got = p.residual(x)
    nrm, _ = oracle.residual(s.m, s.row_ptr, s.col, s.val64, s.b, x)
    want = nrm / np.linalg.norm(s.b)
    assert abs(got - want) <= 1e-12 * want


def test_device_pointer_create_and_solve():
    import torch
    s = synth.plain_f64_system(m=2048, n=512, L=16)
    seed = synth.solver_seed(s.seed)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rp, col, val, b = d(s.row_ptr), d(s.col), d(s.val_store), d(s.b)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()  # inputs were written on the default stream
    with asyrk.Problem(s.m, s.n, rp, col, val, asyrk.F64, b, seed=seed, device_ptrs=True,
                       stream=stream) as p:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        st, info = p.solve(x, tol=0.0, max_sweeps=2, mode=asyrk.MODE_SEQUENTIAL,
                           device_ptrs=True, stream=stream)
        assert st == asyrk.OK
        stream.synchronize()
        assert _rel(x.cpu().numpy(), _oracle_steps(s, seed, 2 * s.m)) <= 1e-12


@pytest.mark.parametrize("kind", ["spiky", "one_heavy", "near_unit", "tiny_m1", "tiny_m2",
                                  "tiny_m3", "two_levels"])
def test_alias_table_built_on_the_gpu_matches_the_oracle(kind):
    rng = np.random.default_rng(11)
    if kind == "spiky":
        w = np.array([1e-12, 1.0, 1e6, 3.0, 1e-3, 7.0, 2.0] * 300)
    elif kind == "one_heavy":
        w = np.ones(5000)
        w[1234] = 1e7
    elif kind == "near_unit":
        w = 1.0 + rng.integers(-3, 4, size=4096) * np.finfo(np.float64).eps
    elif kind.startswith("tiny_m"):
        w = np.exp(rng.standard_normal(int(kind[-1])))
    else:
        w = np.where(rng.random(70000) < 0.5, 1.0, 2.0)
    m = w.size
    val = np.sqrt(w)
    row_ptr = np.arange(m + 1, dtype=np.int64)
    col = np.arange(m, dtype=np.int32)
    b = val * rng.standard_normal(m)
    samp = oracle.Sampler(m, row_ptr, val)
    with asyrk.Problem(m, m, row_ptr, col, val, asyrk.F64, b, seed=77) as p:
        assert p.stats()["uniform"] == samp.uniform
        # F is the w_i's exact sum rounded once, on both sides
        assert p.stats()["frob2"] == samp.F == math.fsum(samp.w)
        for j0, count in [(0, 300_000), (2**33 + 5, 10_000)]:
            np.testing.assert_array_equal(
                p.draw_rows(j0, count, 3),
                oracle.draw_rows(77, 3, j0, count, samp.thr, samp.alias, samp.uniform))


@pytest.mark.parametrize("kind", ["tiny_rows_beside_unit_rows", "wide_dynamic_range",
                                  "subnormal_weights"])
def test_frobenius_norm_is_the_correctly_rounded_sum(kind):
    # Section 1's probabilities divide by F = ||A||_F^2; both sides take it as
    # the exact sum of the w_i rounded once, so it matches Python's correctly
    # rounded math.fsum bit for bit, where any running or blocked FP64 sum
    # (the GPU's reduction order included) would round away the small rows
    rng = np.random.default_rng(21)
    m = 300_000
    if kind == "tiny_rows_beside_unit_rows":
        val = np.full(m, 2.0**-27)            # w_i = 2^-54, half an ulp of 1 / 2
        val[rng.choice(m, 40, replace=False)] = 1.0
    elif kind == "wide_dynamic_range":
        val = np.exp(60.0 * rng.standard_normal(m))  # weights from ~1e-200 to ~1e200
    else:
        val = np.full(m, 2.0**-530)           # w_i = 2^-1060: subnormal
        val[::7] = 2.0**-520
    row_ptr = np.arange(m + 1, dtype=np.int64)
    col = (np.arange(m) % 1000).astype(np.int32)
    b = val.copy()
    samp = oracle.Sampler(m, row_ptr, val)
    assert samp.F == math.fsum(samp.w)
    with asyrk.Problem(m, 1000, row_ptr, col, val, asyrk.F64, b, seed=5) as p:
        assert p.stats()["frob2"] == samp.F
        assert p.stats()["uniform"] == samp.uniform
        np.testing.assert_array_equal(
            p.draw_rows(0, 200_000, 1),
            oracle.draw_rows(5, 1, 0, 200_000, samp.thr, samp.alias, samp.uniform))


@pytest.mark.parametrize("form", [asyrk.FORM_THROUGHPUT, asyrk.FORM_LATENCY])
@pytest.mark.parametrize("subwarp", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_async_fp32_kernel_with_one_worker_matches_the_oracle(dtype, subwarp, form):
    # the kernels the asynchronous workloads run -- FP32 iterate, FP32 b and
    # 1/||a_i||^2 from the row record, row exclusion on; the throughput form
    # (the large workload's) and the latency form (small systems': records and
    # rows loaded ahead) -- with a single worker apply the projections in
    # order: after two sweeps the iterate is the oracle's sequential RK iterate
    # (Eq. (2)) on the same row sequence, to FP32 accuracy; ragged rows of
    # 1..70 entries exercise the chunk tails and the rows longer than a worker
    # keeps in registers
    s = synth.make_system(3000, 800, (1, 70), 515, row_norms="lognormal", value_dtype=dtype)
    seed = synth.solver_seed(s.seed)
    with asyrk.Problem.from_system(s) as p:
        x = np.zeros(s.n)
        st, info = p.solve(x, tol=0.0, max_sweeps=2, mode=asyrk.MODE_ASYNC, workers=1,
                           subwarp=subwarp, kernel_form=form)
        assert st == asyrk.OK  # tol = 0: the sweep budget ends the solve
        assert info.workers == 1 and info.subwarp == subwarp and info.skipped == 0
        assert info.projections == 2 * s.m
    xo = _oracle_steps(s, seed, 2 * s.m)
    assert _rel(x, xo) <= 2e-5


@pytest.mark.parametrize("form", [asyrk.FORM_THROUGHPUT, asyrk.FORM_LATENCY])
@pytest.mark.parametrize("subwarp", [1, 4, 32])
def test_async_fp64_kernel_with_one_worker_matches_the_oracle(subwarp, form):
    # the ASYNC FP64 kernels of both forms (FP64 iterate, b_i and ||a_i||^2 in
    # FP64, the oracle's division) with one worker: the oracle's iterate to 1e-12
    # after two sweeps of ragged, lognormal rows
    s = synth.make_system(3000, 800, (1, 70), 516, row_norms="lognormal")
    seed = synth.solver_seed(s.seed)
    with asyrk.Problem.from_system(s) as p:
        x = np.zeros(s.n)
        st, info = p.solve(x, tol=0.0, max_sweeps=2, mode=asyrk.MODE_ASYNC, workers=1,
                           subwarp=subwarp, kernel_form=form)
        assert st == asyrk.OK and info.workers == 1 and info.projections == 2 * s.m
    assert _rel(x, _oracle_steps(s, seed, 2 * s.m)) <= 1e-12


def test_kernel_form_option_is_checked():
    s = synth.make_system(64, 16, 4, 9)
    with asyrk.Problem.from_system(s) as p:
        x = np.zeros(s.n)
        assert p.solve(x, kernel_form=2, raise_on_error=False)[0] == asyrk.EINVAL
        assert p.solve(x, kernel_form=asyrk.FORM_LATENCY, update=asyrk.UPDATE_SINGLE,
                       raise_on_error=False)[0] == asyrk.EINVAL
