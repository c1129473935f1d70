"""Least squares through Section 6's square consistent system, on the GPU.

  * the GPU-built system equals the oracle's: same shape and nonzero count,
    the same row sequence bit for bit (so the same row weights), and the
    single-worker FP64 iterate on it matches the oracle's to 1e-12 (so the
    same entries and right side), for F64/F32/BF16 values and phi = 1, 0.5,
    with an empty column and an empty row of A;
  * async solves reach x_LS (numpy lstsq) of an inconsistent system: FP64
    values to 1e-8, FP32 values with FP64 refinement to 1e-9;
  * a large inconsistent system (m = 200000, n = 50000, Section 5's random
    positions) reaches ||A^T(A x - b)|| <= 1e-6 ||A^T b||, re-measured on the host;
  * the GPU Lanczos estimate of lambda_min (nonzero) and lambda_max of A^T A
    lies inside the spectrum and reaches its ends (numpy SVD), skipping the
    null space of a rank-deficient A; zeta = 0 takes sigma_r/sqrt(2) from it;
  * bad arguments are refused.
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


def _stored(v64, dtype):
    """The system's values as the library stores them (BF16 through FP32)."""
    if dtype == "f64":
        return v64
    v32 = v64.astype(np.float32).astype(np.float64)
    if dtype == "f32":
        return v32
    return synth.bf16_bits_to_f64(synth.f64_to_bf16_bits(v32))


def _with_gaps(dtype):
    """An inconsistent system with an empty column (7) and an empty row (11)."""
    s = synth.make_system(700, 150, (2, 9), 44, row_norms="lognormal", value_dtype=dtype)
    A = oracle.dense(s.m, s.n, s.row_ptr, s.col, s.val64)
    A[:, 7] = 0.0
    A[11, :] = 0.0
    rp = np.zeros(s.m + 1, dtype=np.int64)
    rp[1:] = np.cumsum(np.count_nonzero(A, axis=1))
    rows, cols = np.nonzero(A)
    v64 = A[rows, cols]
    b = A @ s.x_true + 0.2 * np.random.default_rng(3).standard_normal(s.m)
    store = v64 if dtype == "f64" else (v64.astype(np.float32) if dtype == "f32"
                                        else synth.f64_to_bf16_bits(v64))
    return s.m, s.n, rp, cols.astype(np.int32), v64, store, b


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("phi", [1.0, 0.5])
def test_system_matches_oracle(dtype, phi):
    m, n, rp, col, v64, store, b = _with_gaps(dtype)
    zeta, seed = 0.3, 1234
    rows, cols, arp, acol, aval, rhs = oracle.lsq_augment(m, n, rp, col, v64, b, zeta, phi)
    aval = _stored(aval, dtype)
    assert rows == (n - 1) + m
    with asyrk.Problem.lsq(m, n, rp, col, store, dtype, b, zeta, phi=phi, seed=seed) as p:
        st = p.stats()
        assert (st["m"], st["n"], st["nnz"]) == (rows, cols, int(arp[-1]))
        samp = oracle.Sampler(rows, arp, aval)
        got = p.draw_rows(0, 200_000, 0)
        want = oracle.draw_rows(seed, 0, 0, 200_000, samp.thr, samp.alias, samp.uniform)
        np.testing.assert_array_equal(got, want)
        z = np.zeros(cols)
        s_, info = p.solve(z, tol=0.0, max_sweeps=3, mode=asyrk.MODE_SEQUENTIAL)
        assert s_ == asyrk.OK
    zo = np.zeros(cols)
    oracle.rk_steps(rows, cols, arp, acol, aval, rhs, zo, 1.0, seed, 0, 0, 3 * rows, sampler=samp)
    assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)
    assert z[7] == 0.0  # the empty column is never touched


def _inconsistent(m, n, L, seed, dtype):
    s = synth.make_system(m, n, L, seed, row_norms="unit", value_dtype=dtype)
    b = s.b + 0.3 * np.random.default_rng(seed + 7).standard_normal(m)
    A = oracle.dense(m, n, s.row_ptr, s.col, s.val64)
    x_ls = np.linalg.lstsq(A, b, rcond=None)[0]
    sr = np.linalg.svd(A, compute_uv=False).min()
    return s, b, A, x_ls, sr


def test_async_reaches_least_squares_f64():
    s, b, A, x_ls, sr = _inconsistent(3000, 1000, 12, 71, "f64")
    zeta = sr / np.sqrt(2)
    z_true = np.concatenate([zeta * x_ls, A @ x_ls])
    with asyrk.Problem.lsq(s.m, s.n, s.row_ptr, s.col, s.val_store, "f64", b, zeta, seed=9) as p:
        z = np.zeros(s.n + s.m)
        st, info = p.solve(z, tol=1e-9, max_sweeps=4000, x_true=z_true)
        assert st == asyrk.OK, info.as_dict()
        x = p.lsq_solution(z)
    assert np.linalg.norm(x - x_ls) <= 1e-8 * np.linalg.norm(x_ls)


def test_refined_f32_reaches_least_squares():
    s, b, A, x_ls, sr = _inconsistent(3000, 1000, 12, 72, "f32")
    zeta = sr / np.sqrt(2)
    with asyrk.Problem.lsq(s.m, s.n, s.row_ptr, s.col, s.val_store, "f32", b, zeta, seed=9) as p:
        z = np.zeros(s.n + s.m)
        st, info = p.solve(z, tol=1e-12, max_sweeps=6000, mode=asyrk.MODE_REFINE)
        assert st == asyrk.OK, info.as_dict()
        x = p.lsq_solution(z)
    assert np.linalg.norm(x - x_ls) <= 1e-9 * np.linalg.norm(x_ls)


def test_large_inconsistent_system_reaches_normal_equations():
    import torch
    m, n = 200_000, 50_000
    d = synth.make_system_torch(m, n, ("poisson", 40), 505, row_norms="unit", value_dtype="f32")
    g = torch.Generator(device="cuda").manual_seed(17)
    b = d["b"] + 0.3 * torch.randn(m, dtype=torch.float64, device="cuda", generator=g)
    torch.cuda.synchronize()
    # any zeta > 0 gives x_LS; Section 6's sigma_r/sqrt(2) is estimated from the spectrum
    # edge of such random unit-row matrices, sigma_r ~ sqrt(m/n) (1 - sqrt(n/m)) = 1 here
    zeta = 1.0 / np.sqrt(2)
    with asyrk.Problem.lsq(m, n, d["row_ptr"], d["col"], d["val_store"], asyrk.F32, b, zeta,
                           seed=3, device_ptrs=True) as p:
        z = torch.zeros(n + m, dtype=torch.float64, device="cuda")
        st, info = p.solve(z, tol=1e-10, max_sweeps=5000, mode=asyrk.MODE_REFINE,
                           device_ptrs=True)
        assert st == asyrk.OK, info.as_dict()
        x = p.lsq_solution(z, on_device=True)
    rp = d["row_ptr"].cpu().numpy()
    col = d["col"].cpu().numpy()
    val = d["val_store"].cpu().numpy().astype(np.float64)
    bh = b.cpu().numpy()
    gr = oracle.normal_residual(m, n, rp, col, val, bh, x.cpu().numpy())
    atb = oracle.normal_residual(m, n, rp, col, val, bh, np.zeros(n))
    assert np.linalg.norm(gr) <= 1e-6 * np.linalg.norm(atb)


@pytest.mark.parametrize("m,n,dtype", [(3000, 1000, "f64"), (1000, 300, "f32"),
                                       (2000, 1500, "bf16")])
def test_spectrum_estimate_lies_inside_and_converges(m, n, dtype):
    s = synth.make_system(m, n, 10, 31, row_norms="unit", value_dtype=dtype)
    sv = np.linalg.svd(oracle.dense(m, n, s.row_ptr, s.col, s.val64), compute_uv=False)
    st, lmin, lmax = asyrk.asyrk_spectrum_estimate(m, n, s.row_ptr, s.col, s.val_store,
                                                   asyrk.DTYPES[dtype], steps=200, seed=4)
    assert st == asyrk.OK
    # Ritz values lie inside the spectrum (Cauchy interlacing) ...
    assert lmin >= (1 - 1e-9) * sv.min() ** 2 and lmax <= (1 + 1e-9) * sv.max() ** 2
    # ... and after 200 steps sit at its ends
    assert lmin <= 1.01 * sv.min() ** 2 and lmax >= (1 - 1e-9) * sv.max() ** 2


def test_spectrum_estimate_skips_the_null_space():
    m, n = 1000, 300
    s = synth.make_system(m, n, 8, 9, row_norms="unit", value_dtype="f64")
    A = oracle.dense(m, n, s.row_ptr, s.col, s.val64)
    A[:, 5] = A[:, 9]  # rank n - 1; rows stay non-empty
    rp = np.zeros(m + 1, dtype=np.int64)
    rp[1:] = np.cumsum(np.count_nonzero(A, axis=1))
    rows, cols = np.nonzero(A)
    sv = np.linalg.svd(A, compute_uv=False)
    sr = sv[sv > 1e-10 * sv[0]].min()
    assert sv.min() < 1e-12
    st, lmin, lmax = asyrk.asyrk_spectrum_estimate(m, n, rp, cols.astype(np.int32), A[rows, cols],
                                                   asyrk.F64, steps=100)
    assert st == asyrk.OK
    assert (1 - 1e-9) * sr ** 2 <= lmin <= 1.01 * sr ** 2


def test_estimated_zeta_and_least_squares():
    s, b, A, x_ls, sr = _inconsistent(3000, 1000, 12, 73, "f64")
    with asyrk.Problem.lsq(s.m, s.n, s.row_ptr, s.col, s.val_store, "f64", b, seed=9) as p:
        zeta, phi = p.lsq_params()
        assert phi == 1.0
        assert sr / np.sqrt(2) * (1 - 1e-9) <= zeta <= 1.005 * sr / np.sqrt(2)
        z = np.zeros(s.n + s.m)
        st, info = p.solve(z, tol=1e-11, max_sweeps=4000)
        assert st == asyrk.OK, info.as_dict()
        x = p.lsq_solution(z)
    assert np.linalg.norm(x - x_ls) <= 1e-8 * np.linalg.norm(x_ls)


def test_bad_arguments_are_refused():
    m, n, rp, col, v64, store, b = _with_gaps("f64")
    for zeta, phi in [(-1.0, 1.0), (np.inf, 1.0), (0.5, -1.0), (0.5, np.nan)]:
        st, h = asyrk.asyrk_lsq_create(m, n, rp, col, store, asyrk.F64, b, zeta, phi=phi)
        assert st == asyrk.EINVAL and not h.value
    st, h = asyrk.asyrk_lsq_create(m, n, rp, col, store, asyrk.F64, b, 0.0, lanczos_steps=-1)
    assert st == asyrk.EINVAL and not h.value
    st, lo, hi = asyrk.asyrk_spectrum_estimate(m, n, rp, col, store, asyrk.F64, steps=-1)
    assert st == asyrk.EINVAL
    bad_sp = col.copy()
    bad_sp[0] = -1
    st, lo, hi = asyrk.asyrk_spectrum_estimate(m, n, rp, bad_sp, store, asyrk.F64)
    assert st == asyrk.EINVAL
    bad = col.copy()
    bad[5] = n
    st, h = asyrk.asyrk_lsq_create(m, n, rp, bad, store, asyrk.F64, b, 0.5)
    assert st == asyrk.EINVAL and not h.value
    bb = b.copy()
    bb[3] = np.nan
    st, h = asyrk.asyrk_lsq_create(m, n, rp, col, store, asyrk.F64, bb, 0.5)
    assert st == asyrk.EINVAL and not h.value
    # a plain problem has no least-squares solution to extract
    s = synth.plain_f64_system()
    with asyrk.Problem.from_system(s) as p:
        assert asyrk.asyrk_lsq_solution(p.h, np.zeros(s.n), np.zeros(s.n)) == asyrk.EINVAL


def test_bf16_values_refined_least_squares_device_pointers():
    """BF16-stored A (the stored values are A), FP64 refinement, every array on the
    device, zeta estimated: x_LS of the stored matrix to 1e-9 (numpy lstsq)."""
    import torch
    s, b, A, x_ls, sr = _inconsistent(3000, 1000, 12, 74, "bf16")
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    with asyrk.Problem.lsq(s.m, s.n, d(s.row_ptr), d(s.col), d(s.val_store), "bf16", d(b),
                           seed=11, device_ptrs=True) as p:
        zeta, _ = p.lsq_params()
        assert 0.9 * sr / np.sqrt(2) <= zeta <= 1.02 * sr / np.sqrt(2)  # BF16-rounded estimate
        z = torch.zeros(s.n + s.m, dtype=torch.float64, device="cuda")
        st, info = p.solve(z, tol=1e-12, max_sweeps=8000, mode=asyrk.MODE_REFINE,
                           device_ptrs=True)
        assert st == asyrk.OK, info.as_dict()
        x = p.lsq_solution(z, on_device=True).cpu().numpy()
    assert np.linalg.norm(x - x_ls) <= 1e-9 * np.linalg.norm(x_ls)
