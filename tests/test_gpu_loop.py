"""The graph-captured solve loop (graph_loop = 1: one CUDA-graph launch runs
sweeps, checks and the stop decision in a WHILE node) against the host-driven
loop (the default).

  * SEQUENTIAL: the same kernels in the same order, so the same iterate bit for
    bit, the same sweep count and the same final position;
  * ASYNC, each check measure (error, residual, Table 2's normal residual), fixed
    and adaptive check intervals: both loops reach the tolerance, within a few
    sweeps of each other;
  * max_sweeps reached: NOT_CONVERGED after exactly max_sweeps; tol <= 0 runs
    exactly max_sweeps; max_sweeps = 0 does nothing.
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


def _solve(p, s, graph_loop, **kw):
    p.position = 0
    x = np.zeros(s.n)
    st, info = p.solve(x, graph_loop=graph_loop, **kw)
    return st, info, x, p.position


def test_sequential_is_identical_in_both_loops():
    s = synth.plain_f64_system()
    with asyrk.Problem.from_system(s) as p:
        a = _solve(p, s, True, tol=1e-6, max_sweeps=50, mode=asyrk.MODE_SEQUENTIAL,
                   x_true=s.x_true)
        b = _solve(p, s, False, tol=1e-6, max_sweeps=50, mode=asyrk.MODE_SEQUENTIAL,
                   x_true=s.x_true)
    assert a[0] == b[0] == asyrk.OK
    assert a[1].sweeps == b[1].sweeps and a[3] == b[3]
    np.testing.assert_array_equal(a[2], b[2])


@pytest.mark.parametrize("measure", ["error", "residual", "normal"])
@pytest.mark.parametrize("every", [1, 3, 0])
def test_async_reaches_tolerance_in_both_loops(measure, every):
    if measure == "normal":
        s = synth.make_system(8000, 10000, ("poisson", 10), 41, row_norms="unit",
                              value_dtype="f32")
        kw = dict(tol=1e-5, measure=asyrk.MEASURE_NORMAL_RESIDUAL)
    else:
        s = synth.make_system(1 << 15, 1 << 13, 16, 21, row_norms="lognormal", value_dtype="f32")
        kw = dict(tol=1e-5, x_true=s.x_true if measure == "error" else None,
                  measure=asyrk.MEASURE_RESIDUAL if measure == "residual" else asyrk.MEASURE_AUTO)
    with asyrk.Problem.from_system(s) as p:
        dev = _solve(p, s, True, max_sweeps=3000, check_every=every, **kw)
        host = _solve(p, s, False, max_sweeps=3000, check_every=every, **kw)
    for st, info, x, pos in (dev, host):
        assert st == asyrk.OK, info.as_dict()
        assert pos == info.projections
        if measure == "normal":
            g = oracle.normal_residual(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x)
            assert float(g @ g) <= 1.0001e-5
        elif measure == "error":
            assert np.linalg.norm(x - s.x_true) <= 1.0001e-5 * np.linalg.norm(s.x_true)
        else:
            rn = oracle.residual(s.m, s.row_ptr, s.col, s.val64, s.b, x)[0]
            assert rn <= 1.0001e-5 * np.linalg.norm(s.b)
    assert abs(dev[1].sweeps - host[1].sweeps) <= 0.12 * host[1].sweeps + 3


def test_sweep_limits_in_the_graph_loop():
    s = synth.plain_f64_system()
    with asyrk.Problem.from_system(s) as p:
        st, info, x, pos = _solve(p, s, True, tol=1e-30, max_sweeps=7, x_true=s.x_true)
        assert st == asyrk.NOT_CONVERGED and info.sweeps == 7 and pos == 7 * s.m
        st, info, x, pos = _solve(p, s, True, tol=0.0, max_sweeps=5, check_every=2)
        assert st == asyrk.OK and info.sweeps == 5 and pos == 5 * s.m
        st, info, x, pos = _solve(p, s, True, tol=1e-8, max_sweeps=0)
        assert info.sweeps == 0 and pos == 0 and not np.any(x)
