"""Served solves (continuous batching) on the GPU.

  * a mix of requests -- FP32 plain to 1e-6, BF16 with FP64 refinement to
    1e-10, of several sizes, several requests per problem -- all reach their
    tolerance, checked on the host against x*;
  * each request's result is the same alone and in the mix, within its
    tolerance (both within tol of x*);
  * requests that arrive while others run are admitted as slots free up;
  * the memory budget limits how many run at once, a request bigger than the
    budget is refused, cancelling and timeouts behave as documented;
  * requests for problems that fit a CTA's shared memory run on-chip (one CTA
    launch each, plain or refined) and give the results the shared engine step
    gives; a running on-chip request that is cancelled ends as cancelled.
"""
import time

import numpy as np
import pytest

from paper_1401_4780_gb300 import asyrk, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    asyrk.load()


@pytest.fixture(scope="module")
def pool():
    """Two small BF16 systems, two small FP32 ones, one larger FP32 one."""
    systems = [synth.make_system(4096, 1024, 16, 9000 + k, row_norms="unit",
                                 value_dtype="bf16" if k < 2 else "f32") for k in range(4)]
    systems.append(synth.make_system(1 << 16, 1 << 14, 32, 9100, row_norms="unit",
                                     value_dtype="f32"))
    probs = [asyrk.Problem.from_system(s) for s in systems]
    yield systems, probs
    for p in probs:
        p.close()


def _err(x, s):
    return np.linalg.norm(x - s.x_true) / np.linalg.norm(s.x_true)


def _jobs():
    # (system index, mode, tol)
    jobs = []
    for k in range(24):
        idx = k % 5
        if idx < 2 and k % 2 == 0:
            jobs.append((idx, asyrk.MODE_REFINE, 1e-10))
        else:
            jobs.append((idx, asyrk.MODE_ASYNC, 1e-6))
    return jobs


def test_mixed_requests_all_reach_their_tolerance(pool):
    systems, probs = pool
    with asyrk.Server(8 << 30, max_slots=16) as sv:
        tickets = []
        for idx, mode, tol in _jobs():
            tickets.append(sv.submit(probs[idx], x_true=systems[idx].x_true, tol=tol, mode=mode,
                                     max_sweeps=2000))
        for (idx, mode, tol), t in zip(_jobs(), tickets):
            st, x, info = sv.wait(t, systems[idx].n, timeout_us=120_000_000)
            assert st == asyrk.OK, (idx, mode, st, info.as_dict())
            assert _err(x, systems[idx]) <= tol * 1.0001
            assert abs(info.rel_err - _err(x, systems[idx])) <= 1e-3 * _err(x, systems[idx]) + 1e-15
            assert info.seconds > 0 and info.sweeps > 0
            if mode == asyrk.MODE_REFINE:
                assert info.refine_steps >= 2 and info.rel_res < 1e-8
        stt = sv.stats()
        assert stt["completed"] == len(tickets) and stt["active"] == 0 and stt["queued"] == 0
        assert stt["max_active"] > 1 and stt["mem_used"] == 0 and stt["fatal"] == 0


def test_same_result_alone_and_in_the_mix(pool):
    systems, probs = pool
    jobs = [(0, asyrk.MODE_REFINE, 1e-10), (2, asyrk.MODE_ASYNC, 1e-6), (4, asyrk.MODE_ASYNC, 1e-6)]
    alone = []
    for idx, mode, tol in jobs:
        with asyrk.Server(8 << 30) as sv:
            t = sv.submit(probs[idx], x_true=systems[idx].x_true, tol=tol, mode=mode)
            st, x, _ = sv.wait(t, systems[idx].n, timeout_us=60_000_000)
            assert st == asyrk.OK
            alone.append(x)
    with asyrk.Server(8 << 30) as sv:
        filler = [sv.submit(probs[k % 5], x_true=systems[k % 5].x_true, tol=1e-6)
                  for k in range(10)]
        ts = [sv.submit(probs[idx], x_true=systems[idx].x_true, tol=tol, mode=mode)
              for idx, mode, tol in jobs]
        mixed = []
        for (idx, _, _), t in zip(jobs, ts):
            st, x, _ = sv.wait(t, systems[idx].n, timeout_us=60_000_000)
            assert st == asyrk.OK
            mixed.append(x)
        for k, t in enumerate(filler):
            assert sv.wait(t, systems[k % 5].n, timeout_us=60_000_000)[0] == asyrk.OK
    for (idx, _, tol), xa, xm in zip(jobs, alone, mixed):
        s = systems[idx]
        assert _err(xa, s) <= tol * 1.0001 and _err(xm, s) <= tol * 1.0001
        assert np.linalg.norm(xa - xm) / np.linalg.norm(s.x_true) <= 2 * tol * 1.0001


def test_late_arrivals_join_while_others_run(pool):
    systems, probs = pool
    with asyrk.Server(8 << 30, max_slots=4) as sv:
        first = sv.submit(probs[4], x_true=systems[4].x_true, tol=1e-6)
        time.sleep(0.002)
        later = [sv.submit(probs[k], x_true=systems[k].x_true, tol=1e-6) for k in (2, 3, 2, 3)]
        st, _, info_first = sv.wait(first, systems[4].n, timeout_us=60_000_000)
        assert st == asyrk.OK
        for k, t in zip((2, 3, 2, 3), later):
            st, x, info = sv.wait(t, systems[k].n, timeout_us=60_000_000)
            assert st == asyrk.OK and _err(x, systems[k]) <= 1e-6
        assert sv.stats()["max_active"] >= 2


def test_budget_limits_concurrency_and_oversized_requests_are_refused(pool):
    systems, probs = pool
    small = probs[2]
    per_problem = small.stats()["device_bytes"]
    slot = 1024 * (4 + 8 + 8) + 4096 // 8 + 5 * 256 + 4096 * 0
    budget = per_problem + 2 * slot + 4096  # the problem once and two slots
    with asyrk.Server(budget, max_slots=8) as sv:
        ts = [sv.submit(small, x_true=systems[2].x_true, tol=1e-6) for _ in range(6)]
        for t in ts:
            st, x, _ = sv.wait(t, systems[2].n, timeout_us=60_000_000)
            assert st == asyrk.OK and _err(x, systems[2]) <= 1e-6
        stt = sv.stats()
        assert stt["max_active"] <= 2 and stt["completed"] == 6
        with pytest.raises(asyrk.AsyrkError) as e:
            sv.submit(probs[4], tol=1e-6)  # needs more than the whole budget
        assert e.value.status == asyrk.ENOMEM


def test_cancel_and_timeout(pool):
    systems, probs = pool
    with asyrk.Server(8 << 30, max_slots=1, onchip=False) as sv:  # the queued one stays queued
        running = sv.submit(probs[4], x_true=systems[4].x_true, tol=1e-14, max_sweeps=10**6)
        queued = sv.submit(probs[2], x_true=systems[2].x_true, tol=1e-6)
        st, x, _ = sv.wait(running, systems[4].n, timeout_us=1000)
        assert st == asyrk.ETIMEOUT and x is None
        assert sv.cancel(queued) == asyrk.OK
        st, _, _ = sv.wait(queued, systems[2].n, timeout_us=10_000_000)
        assert st == asyrk.ECANCELED
        assert sv.cancel(running) == asyrk.OK
        st, x, info = sv.wait(running, systems[4].n, timeout_us=30_000_000)
        assert st == asyrk.ECANCELED and info.sweeps >= 1
        st, _, _ = sv.wait(12345, 1, timeout_us=0)
        assert st == asyrk.EINVAL


def test_destroy_with_pending_work_returns(pool):
    systems, probs = pool
    sv = asyrk.Server(8 << 30, max_slots=2)
    for _ in range(5):
        sv.submit(probs[4], x_true=systems[4].x_true, tol=1e-14, max_sweeps=10**6)
    t0 = time.time()
    sv.close()
    assert time.time() - t0 < 30.0


def test_onchip_requests_match_the_shared_step(pool):
    systems, probs = pool
    jobs = [(0, asyrk.MODE_REFINE, 1e-10), (1, asyrk.MODE_ASYNC, 1e-6), (2, asyrk.MODE_REFINE, 1e-10),
            (3, asyrk.MODE_ASYNC, 1e-6)]
    results = {}
    for onchip in (True, False):
        with asyrk.Server(8 << 30, onchip=onchip) as sv:
            ts = [sv.submit(probs[idx], x_true=systems[idx].x_true, tol=tol, mode=mode)
                  for idx, mode, tol in jobs]
            out = []
            for (idx, mode, tol), t in zip(jobs, ts):
                st, x, info = sv.wait(t, systems[idx].n, timeout_us=60_000_000)
                assert st == asyrk.OK, (onchip, idx, info.as_dict())
                assert _err(x, systems[idx]) <= tol * 1.0001
                assert abs(info.rel_err - _err(x, systems[idx])) <= 1e-3 * _err(x, systems[idx]) + 1e-15
                if mode == asyrk.MODE_REFINE:
                    assert info.refine_steps >= 2 and info.rel_res < 1e-8
                assert info.j_end == info.sweeps * systems[idx].m
                out.append(x)
            stt = sv.stats()
            assert stt["onchip_completed"] == (len(jobs) if onchip else 0)
            assert stt["mem_used"] == 0 and stt["fatal"] == 0
            results[onchip] = out
    for (idx, _, tol), xa, xb in zip(jobs, results[True], results[False]):
        assert np.linalg.norm(xa - xb) / np.linalg.norm(systems[idx].x_true) <= 2 * tol * 1.0001


def test_cancel_a_running_onchip_request(pool):
    systems, probs = pool
    with asyrk.Server(8 << 30) as sv:
        t = sv.submit(probs[2], x_true=systems[2].x_true, tol=1e-14, max_sweeps=20000)
        time.sleep(0.05)
        assert sv.cancel(t) == asyrk.OK
        st, _, info = sv.wait(t, systems[2].n, timeout_us=60_000_000)
        assert st == asyrk.ECANCELED and info.sweeps >= 1
        assert sv.stats()["onchip_completed"] == 1


def test_admission_caps_the_warp_demand_of_the_shared_step(pool):
    # the 65536 x 16384 system's Cor. 2 worker cap is ~1340 workers, ~335 warps;
    # with admit_load 0.1 (a tenth of the resident warps) two of them exceed
    # the limit, so the shared step runs them one after another; with no limit
    # they run together; the results reach the tolerance either way
    systems, probs = pool
    s, p = systems[4], probs[4]
    for load, one_at_a_time in ((0.1, True), (-1.0, False)):
        with asyrk.Server(8 << 30, max_slots=8, onchip=False, admit_load=load) as sv:
            ts = [sv.submit(p, x_true=s.x_true, tol=1e-6) for _ in range(4)]
            for t in ts:
                st, x, _ = sv.wait(t, s.n, timeout_us=60_000_000)
                assert st == asyrk.OK and _err(x, s) <= 1e-6
            stt = sv.stats()
            assert stt["completed"] == 4 and stt["fatal"] == 0
            if one_at_a_time:
                assert stt["max_active_shared"] == 1
            else:
                assert stt["max_active_shared"] >= 2


@pytest.mark.parametrize("partition", [0, -1])
def test_onchip_requests_and_the_shared_step_on_split_sms(pool, partition):
    # by default the on-chip requests get 16 SMs of their own and the shared
    # step the rest (green contexts); -1 keeps one pool; results are the same
    # either way: every request within its tolerance
    import torch
    systems, probs = pool
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    with asyrk.Server(8 << 30, max_slots=8, partition=partition) as sv:
        jobs = [(2, asyrk.MODE_ASYNC, 1e-6), (0, asyrk.MODE_REFINE, 1e-10), (4, asyrk.MODE_ASYNC, 1e-6),
                (3, asyrk.MODE_ASYNC, 1e-6), (1, asyrk.MODE_REFINE, 1e-10)]
        ts = [sv.submit(probs[i], x_true=systems[i].x_true, tol=tol, mode=mode)
              for i, mode, tol in jobs]
        for (i, _, tol), t in zip(jobs, ts):
            st, x, _ = sv.wait(t, systems[i].n, timeout_us=60_000_000)
            assert st == asyrk.OK and _err(x, systems[i]) <= tol * 1.0001
        stt = sv.stats()
        if partition == 0:
            assert stt["onchip_sms"] >= 16 and stt["step_sms"] + stt["onchip_sms"] == sms
            assert stt["onchip_completed"] >= 3
        else:
            assert stt["onchip_sms"] == 0 and stt["step_sms"] == 0
