"""The on-chip batched engine: each member is solved by one thread-block cluster
whose shared memory holds the member's FP32 iterate and row-claim bits.

  * with one worker per member the projections run strictly in order, and the
    iterate after two sweeps matches the FP64 oracle's sequential RK iterate on
    the same row sequence (Eq. (2), rows drawn with probability ||a_i||^2/||A||_F^2)
    to FP32 accuracy -- for members held by one CTA and by a cluster of two;
  * many workers reach ||x - x*||/||x*|| <= 1e-6 on every member within 1.5x the
    oracle's median sweep count, with cluster sizes 1, 4 and 8;
  * each result is the same alone (the single-system solver) and in the mix;
  * the residual measure, the sweep budget, shuffled sweeps, the row sequence's
    position, the host-launched form, and the engine selection (AUTO puts the
    members that fit on-chip and the others in the global-iterate engine, both
    at once; ONCHIP refuses a member that does not fit or the single-coordinate
    update);
  * a hybrid batch of small members and members too large for a CTA reaches the
    tolerance on all of them, graph-launched and host-launched.
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


def _systems():
    shapes = [(2048, 512, 8), (3000, 750, 64), (4096, 1024, 16), (6000, 1500, 33),
              (8192, 2048, 40), (12000, 3000, 12), (16384, 4096, 24), (2500, 625, 57)]
    out = []
    for k, (m, n, L) in enumerate(shapes):
        dt = "bf16" if k % 4 == 3 else "f32"
        out.append(synth.make_system(m, n, L, 700 + k, row_norms="unit", value_dtype=dt))
    return out


def _err(x, s):
    return np.linalg.norm(x - s.x_true) / np.linalg.norm(s.x_true)


def _close(probs):
    for p in probs:
        p.close()


def test_one_worker_matches_the_sequential_oracle_iterate():
    # the last member's iterate and claim bits (51200 + 1600 words) exceed one
    # CTA's 200 KiB: it is spread over a cluster of two
    systems = [synth.make_system(2048, 512, 8, 31, row_norms="lognormal", value_dtype="f32"),
               synth.make_system(3000, 750, 40, 32, row_norms="unit", value_dtype="bf16"),
               synth.make_system(204800, 51200, 8, 33, row_norms="lognormal", value_dtype="f32")]
    probs = [asyrk.Problem.from_system(s) for s in systems]
    try:
        with asyrk.Batch(probs, engine=asyrk.ENGINE_ONCHIP, workers=1, cluster_max=2) as b:
            xs = [np.zeros(s.n) for s in systems]
            st, infos, bi = b.solve(xs, tols=[0.0] * 3, max_sweeps=2)
            assert bi.engine == asyrk.ENGINE_ONCHIP
            assert st == asyrk.NOT_CONVERGED and all(i.sweeps == 2 for i in infos)
            assert all(i.workers == 1 for i in infos)
        for s, x, p in zip(systems, xs, probs):
            xo = np.zeros(s.n)
            oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, xo, 1.0,
                            synth.solver_seed(s.seed), 0, 0, 2 * s.m)
            rel = np.linalg.norm(x - xo) / np.linalg.norm(xo)
            # FP32 iterate, values and atomics against the FP64 oracle
            assert rel <= 2e-5, (s.m, rel)
            assert p.position == 2 * s.m
    finally:
        _close(probs)


@pytest.mark.parametrize("cluster_max", [1, 4, 8])
def test_members_reach_tolerance_within_oracle_sweeps(cluster_max):
    systems = _systems()
    probs = [asyrk.Problem.from_system(s) for s in systems]
    try:
        with asyrk.Batch(probs, engine=asyrk.ENGINE_ONCHIP, cluster_max=cluster_max) as b:
            xs = [np.zeros(s.n) for s in systems]
            st, infos, bi = b.solve(xs, tols=[1e-6] * len(systems), max_sweeps=400,
                                    x_trues=[s.x_true for s in systems])
            assert st == asyrk.OK, [i.status for i in infos]
            assert bi.engine == asyrk.ENGINE_ONCHIP and bi.graph == 1
            assert bi.converged == len(systems)
            assert bi.iterations == max(i.sweeps for i in infos)
        for s, x, info in zip(systems, xs, infos):
            assert _err(x, s) <= 1e-6 and abs(info.rel_err - _err(x, s)) <= 1e-3 * _err(x, s)
            assert info.rel_res < 1e-5 and info.workers >= 1
            sweeps = []
            for k in range(3):
                xo = np.zeros(s.n)
                r = oracle.rk_solve(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, xo, 1.0,
                                    synth.solver_seed(s.seed) + k, 1e-6, 400, x_true=s.x_true)
                sweeps.append(r.sweeps)
            assert info.sweeps <= 1.5 * np.median(sweeps), (s.m, info.sweeps, sweeps)
    finally:
        _close(probs)


def test_each_result_is_the_same_alone_and_in_the_mix():
    systems = _systems()
    probs = [asyrk.Problem.from_system(s) for s in systems]
    try:
        alone = []
        for s, p in zip(systems, probs):
            x = np.zeros(s.n)
            st, _ = p.solve(x, tol=1e-6, max_sweeps=400, x_true=s.x_true)
            assert st == asyrk.OK
            alone.append(x)
        with asyrk.Batch(probs) as b:  # AUTO: every member fits, so on-chip
            mix = [np.zeros(s.n) for s in systems]
            st, _, bi = b.solve(mix, tols=[1e-6] * len(systems), max_sweeps=400,
                                x_trues=[s.x_true for s in systems])
            assert st == asyrk.OK and bi.engine == asyrk.ENGINE_ONCHIP
        for s, xa, xm in zip(systems, alone, mix):
            assert _err(xa, s) <= 1e-6 and _err(xm, s) <= 1e-6
            assert np.linalg.norm(xa - xm) / np.linalg.norm(s.x_true) <= 2e-6
    finally:
        _close(probs)


def test_residual_measure_budget_and_position():
    systems = _systems()[:4]
    probs = [asyrk.Problem.from_system(s) for s in systems]
    try:
        with asyrk.Batch(probs, engine=asyrk.ENGINE_ONCHIP) as b:
            xs = [np.zeros(s.n) for s in systems]
            st, infos, _ = b.solve(xs, tols=[1e-5] * 4, max_sweeps=400)  # ||b - Ax||/||b||
            assert st == asyrk.OK
            for s, x, info, p in zip(systems, xs, infos, probs):
                assert info.rel_err == -1.0 and info.rel_res <= 1.2e-5
                r = np.linalg.norm(s.b - synth.spmv_f64(s.m, s.row_ptr, s.col, s.val64, x))
                assert r / np.linalg.norm(s.b) <= 1.2e-5
                assert p.position == info.sweeps * s.m == info.j_end
            xs = [np.zeros(s.n) for s in systems]
            st, infos, bi = b.solve(xs, tols=[1e-12] * 4, max_sweeps=3,
                                    x_trues=[s.x_true for s in systems])
            assert st == asyrk.NOT_CONVERGED and bi.converged == 0
            assert all(i.sweeps == 3 and i.status == asyrk.NOT_CONVERGED for i in infos)
            # a member that starts at its solution does no sweep
            xs = [s.x_true.copy() for s in systems]
            st, infos, _ = b.solve(xs, tols=[1e-6] * 4, max_sweeps=10,
                                   x_trues=[s.x_true for s in systems])
            assert st == asyrk.OK and all(i.sweeps == 0 for i in infos)
    finally:
        _close(probs)


def test_shuffled_sweeps_and_host_launches():
    systems = [synth.make_system(2000 + 500 * k, 400, 8, 60 + k, row_norms="unit",
                                 value_dtype="f32") for k in range(3)]
    probs = [asyrk.Problem.from_system(s) for s in systems]
    try:
        for graph in (True, False):
            with asyrk.Batch(probs, engine=asyrk.ENGINE_ONCHIP, sampling=asyrk.SAMPLE_SHUFFLED,
                             graph=graph) as b:
                xs = [np.zeros(s.n) for s in systems]
                st, infos, bi = b.solve(xs, tols=[1e-6] * 3, max_sweeps=3000,
                                        x_trues=[s.x_true for s in systems])
                assert st == asyrk.OK, [i.as_dict() for i in infos]
                assert bi.graph == (1 if graph else 0)
            for x, s in zip(xs, systems):
                assert _err(x, s) <= 1e-6
    finally:
        _close(probs)


def test_engine_selection():
    small = synth.make_system(2048, 512, 8, 41, value_dtype="f32")
    wide = synth.make_system(65536, 1 << 20, 4, 42, value_dtype="f32")  # x alone is 4 MiB
    with asyrk.Problem.from_system(small) as ps, asyrk.Problem.from_system(wide) as pw:
        assert asyrk.asyrk_batch_create([ps.h, pw.h], engine=asyrk.ENGINE_ONCHIP)[0] == asyrk.EINVAL
        assert "does not fit" in asyrk.asyrk_last_error()
        assert asyrk.asyrk_batch_create([ps.h], engine=asyrk.ENGINE_ONCHIP,
                                        update=asyrk.UPDATE_SINGLE)[0] == asyrk.EINVAL
        assert asyrk.asyrk_batch_create([ps.h], engine=3)[0] == asyrk.EINVAL
        assert asyrk.asyrk_batch_create([ps.h], cluster_max=3)[0] == asyrk.EINVAL
        # AUTO: the member that fits runs on-chip, the other one in the global engine
        for members, want, n_on in (([ps], asyrk.ENGINE_ONCHIP, 1),
                                    ([ps, pw], asyrk.ENGINE_ONCHIP | asyrk.ENGINE_GLOBAL, 1)):
            with asyrk.Batch(members) as b:
                xs = [np.zeros(p.n) for p in members]
                _, infos, bi = b.solve(xs, tols=[1e-3] * len(members), max_sweeps=2)
                assert bi.engine == want and bi.onchip_members == n_on
                assert all(i.sweeps == 2 for i in infos)
        with asyrk.Batch([ps], engine=asyrk.ENGINE_GLOBAL) as b:
            _, _, bi = b.solve([np.zeros(ps.n)], tols=[1e-3], max_sweeps=2)
            assert bi.engine == asyrk.ENGINE_GLOBAL


@pytest.mark.parametrize("graph,partition", [(True, True), (True, False), (False, True), (True, 24)])
def test_hybrid_batch_reaches_tolerance(graph, partition):
    # two members exceed a CTA's shared memory (x alone 256 KiB): global engine.
    # Graph-launched, the two engines run at once, by default each on its own
    # share of the SMs (green contexts); without the split they share every SM;
    # the host-driven loop runs the engines one after the other, unsplit
    systems = _systems()[:5] + [synth.make_system(4 * 65536, 65536, 12, 50 + k, row_norms="unit",
                                                  value_dtype="f32") for k in range(2)]
    probs = [asyrk.Problem.from_system(s) for s in systems]
    try:
        with asyrk.Batch(probs, graph=graph, partition=partition) as b:
            xs = [np.zeros(s.n) for s in systems]
            st, infos, bi = b.solve(xs, tols=[1e-6] * len(systems), max_sweeps=400,
                                    x_trues=[s.x_true for s in systems])
            assert st == asyrk.OK, [i.status for i in infos]
            assert bi.engine == asyrk.ENGINE_ONCHIP | asyrk.ENGINE_GLOBAL
            assert 1 <= bi.onchip_members <= 5 and bi.converged == len(systems)
            assert bi.iterations == max(i.sweeps for i in infos)
            # each engine's part ends within the timed loop
            assert 0 < bi.global_ms <= bi.device_ms * (1 + 1e-6)
            assert 0 < bi.onchip_ms <= bi.device_ms * (1 + 1e-6)
            assert max(bi.global_ms, bi.onchip_ms) >= 0.5 * bi.device_ms
            if graph and partition:
                import torch
                sms = torch.cuda.get_device_properties(0).multi_processor_count
                assert 8 <= bi.global_sms <= sms - 8
                if partition is not True:  # the on-chip engine's SMs, asked for
                    assert abs((sms - bi.global_sms) - partition) <= 8
            else:
                assert bi.global_sms == 0
        for s, x, info, p in zip(systems, xs, infos, probs):
            assert _err(x, s) <= 1e-6 and abs(info.rel_err - _err(x, s)) <= 1e-3 * _err(x, s)
            assert info.rel_res < 1e-5
            assert p.position == info.sweeps * s.m
    finally:
        _close(probs)


def test_grouped_onchip_launches_match_the_sequential_oracle_iterate():
    # in a hybrid batch on split SMs the on-chip members run grouped, several
    # per launch (one CTA each); with one worker each, every on-chip member's
    # iterate after two sweeps is the oracle's sequential RK iterate to FP32
    # accuracy, as it is with one launch per member
    # (the global member, 2^21 x 4096, does not fit a CTA and its Corollary 2
    # cap keeps its sweep long, so the one-worker on-chip members stay on-chip)
    small = [synth.make_system(512 + 256 * k, 128 + 64 * k, 8 + 4 * k, 60 + k,
                               row_norms="lognormal", value_dtype="f32") for k in range(6)]
    big = synth.make_system(1 << 21, 4096, 8, 66, row_norms="unit", value_dtype="f32")
    systems = small + [big]
    probs = [asyrk.Problem.from_system(s) for s in systems]
    try:
        with asyrk.Batch(probs, workers=1) as b:
            xs = [np.zeros(s.n) for s in systems]
            _, infos, bi = b.solve(xs, tols=[0.0] * len(systems), max_sweeps=2)
            assert bi.engine == asyrk.ENGINE_ONCHIP | asyrk.ENGINE_GLOBAL
            assert bi.onchip_members == len(small) and bi.global_sms > 0
        for s, x, info in zip(small, xs, infos):
            assert info.workers == 1 and info.sweeps == 2
            xo = np.zeros(s.n)
            oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, xo, 1.0,
                            synth.solver_seed(s.seed), 0, 0, 2 * s.m)
            assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 2e-5, s.m
    finally:
        _close(probs)
