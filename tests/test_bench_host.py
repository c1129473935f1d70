"""Host-side logic of bench.py on the CPU: the replica aggregation over ranks
(world size 2, gloo), the clock-record parser, the traffic-record check and the
reference arm's JSON line (the oracle timed on the host)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

WORKER = r"""
import json, os, sys
sys.path.insert(0, %r)
import bench
d = bench.Dist(backend="gloo")
d.barrier()
mx = d.reduce(10.0 * (d.rank + 1), "max")
sm = d.reduce(3.0 + d.rank, "sum")
print(json.dumps({"rank": d.rank, "world": d.world, "max": mx, "sum": sm}))
d.close()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_max_and_sum_over_gloo(tmp_path):
    port = _free_port()
    script = tmp_path / "w.py"
    script.write_text(WORKER % ROOT)
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for o in outs:
        assert o["world"] == 2 and o["max"] == 20.0 and o["sum"] == 7.0


def test_single_process_dist_is_identity():
    d = bench.Dist()
    assert d.world == 1 and d.reduce(4.5, "max") == 4.5 and d.reduce(4.5, "sum") == 4.5


def test_clock_parser_flags_slowdowns():
    c = bench.ClockSampler(0)
    c.proc = None
    c.lines = ["0, 1965, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1800, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 1900, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active"]

    class _P:
        stdout = []

        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    class _T:
        def join(self, timeout=None):
            pass

    c.proc, c.t = _P(), _T()
    out = c.stop()
    assert out["sm_mhz"] == 1900 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"]


def test_traffic_record_requires_matching_kernel_sources(tmp_path, monkeypatch):
    f = tmp_path / "k.txt"
    f.write_text("source_sha256: %s\ndram_bytes_per_launch: 1234.5\n" % bench.kernel_source_hash())
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(f))
    assert bench.recorded_traffic() == 1234.5
    f.write_text("source_sha256: 0000\ndram_bytes_per_launch: 1234.5\n")
    assert bench.recorded_traffic() is None


def test_reference_arm_prints_the_contract_line():
    # bench.py --impl reference times the FP64 oracle on the host cores on the
    # GPU arm's workload and metric; its one JSON line carries impl, the
    # metric's value and unit, a cpu_baseline describing the run, and an e2e
    # record of the same value with no host-device traffic
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["unit"] == "row projections/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["m"] == 1 << 22 and d["config"]["nnz_per_row"] == 32
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
