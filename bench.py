#!/usr/bin/env python
"""Benchmark: asynchronous randomized Kaczmarz row projections per second on one GB300.

Workload (default): the large async system -- m = 2^22, n = 2^20, 32 distinct
uniformly random columns per row, N(0,1) values, row norms lognormal(0,1) (so
rows are drawn through the alias table), FP32 values and iterate, int32 columns,
x* ~ N(0,1), b = A x* in FP64, gamma = 1, tolerance ||x-x*||/||x*|| <= 1e-5.

A step is one solve of that system from x0 = 0 to the tolerance through the C
ABI (asyrk_solve, ASYNC mode): projection launches of one sweep each, an FP64
check after each.  `value` = projections of all timed steps / their device time
(CUDA events on the launch stream; inputs resident in HBM).  The matrix stream
(1.07 GB of columns and values) is larger than the 129 MB L2, so no flush is
needed between steps.

`e2e` runs the same solve through the public API from pinned HOST buffers:
asyrk_create (CSR and b copied to the device, row records and alias table
built), asyrk_solve with x0/x in host memory, asyrk_destroy, all timed.

`--impl reference` times the FP64 CPU oracle (test infrastructure, one thread)
on the same workload: each step a bounded number of projections.

Multi-GPU: one independent replica per rank (a single system does not shard:
every row updates the shared x); `value` sums the replicas' projections over the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "row projections/s and time to 1e-8 rel. error vs plain FP32 kernel; p50/p99 served"
UNIT = "row projections/s"
# algorithmic bytes per projection of the large async workload: 32 x (4 B column
# + 4 B value) + a 16 B row record (start, length, b_i, 1/||a_i||^2) + an 8 B
# alias entry (threshold, alias row)
BYTES_PER_PROJECTION = 32 * 8 + 16 + 8
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "k_project_large_async.txt")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1401_4780_gb300", "csrc", f)
                  for f in ("project.cu", "worker.cuh", "common.cuh")]


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["asyrk", "reference"], default="asyrk")
    ap.add_argument("--gamma", type=float, default=1.0)
    ap.add_argument("--tol", type=float, default=1e-5)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="target CPU time of the oracle sample")
    ap.add_argument("--scale", type=int, default=0,
                    help="shrink m and n by 2^scale (testing only; not a bench number)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the plain/refine, batched and served measurements")
    ap.add_argument("--served-seconds", type=float, default=30.0,
                    help="length of the Poisson arrival window of the served measurement")
    ap.add_argument("--served-seconds2", type=float, default=10.0,
                    help="arrival window of the second, lower-rate served measurement")
    ap.add_argument("--admit-load", type=float, default=0.0,
                    help="server admission limit (warp demand / resident warps; 0: default)")
    ap.add_argument("--server-partition", type=int, default=0,
                    help="server: SMs of the on-chip requests (0: default, -1: no split)")
    ap.add_argument("--served-rate", type=float, default=2000.0, help="requests per second")
    ap.add_argument("--served-rate2", type=float, default=1000.0,
                    help="a second, lower offered rate (0: skip)")
    ap.add_argument("--batched-only", action="store_true",
                    help="profiling aid: run only the 256-system batched case, print its JSON")
    ap.add_argument("--batched-systems", type=int, default=0,
                    help="with --batched-only: the first N systems only (a reduced case for ncu)")
    ap.add_argument("--served-only", action="store_true",
                    help="tuning aid: run only the served measurement(s), print their JSON")
    ap.add_argument("--batch-host-loop", action="store_true",
                    help="with --batched-only: host-driven engine loop (separate launches)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU; replicas)
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self, backend=None):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            if backend is None:
                import torch
                backend = "nccl" if torch.cuda.is_available() else "gloo"
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()

    def reduce(self, value, op):
        """All-reduce a float (op: "max" or "sum")."""
        if self.pg is None:
            return value
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX if op == "max" else self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg is not None:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_numa_node(dev):
    """The NUMA node sysfs gives for the GPU's PCI device (None when unknown)."""
    import torch
    try:
        pr = torch.cuda.get_device_properties(dev)
        bus = "%04x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        with open("/sys/bus/pci/devices/%s/numa_node" % bus) as f:
            node = int(f.read().strip())
        return node if node >= 0 else None
    except (AttributeError, OSError, RuntimeError, ValueError):
        return None


def cpu_numa_nodes(cpus):
    """The NUMA nodes of the given CPUs (from sysfs), as a sorted list."""
    nodes = set()
    for c in cpus:
        try:
            for name in os.listdir("/sys/devices/system/cpu/cpu%d" % c):
                if name.startswith("node") and name[4:].isdigit():
                    nodes.add(int(name[4:]))
        except OSError:
            pass
    return sorted(nodes)


_NODE_PINNED = []  # (address, size) of host buffers bound to a NUMA node and registered


def pinned_on_node(arr, node):
    """A page-locked host copy of arr whose pages live on NUMA node `node` (the GPU's):
    anonymous memory bound to the node with mbind, filled, then registered with
    CUDA.  Falls back to torch's pinned allocation when any step is unavailable."""
    import platform
    import torch
    arr = np.ascontiguousarray(arr)
    nr = {"aarch64": 235, "x86_64": 237}.get(platform.machine())
    if node is None or nr is None or arr.nbytes == 0:
        return torch.from_numpy(arr).pin_memory()
    libc = ctypes.CDLL(None, use_errno=True)
    libc.mmap.restype = ctypes.c_void_p
    libc.mmap.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                          ctypes.c_int, ctypes.c_long]
    libc.munmap.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
    page = os.sysconf("SC_PAGE_SIZE")
    size = (arr.nbytes + page - 1) // page * page
    addr = libc.mmap(None, size, 3, 0x22, -1, 0)  # PROT_READ|WRITE, MAP_PRIVATE|ANONYMOUS
    if not addr or addr == ctypes.c_void_p(-1).value:
        return torch.from_numpy(arr).pin_memory()
    mask = (ctypes.c_ulong * 16)()
    mask[node // 64] = 1 << (node % 64)
    rc = libc.syscall(ctypes.c_long(nr), ctypes.c_void_p(addr), ctypes.c_ulong(size),
                      ctypes.c_int(2), mask, ctypes.c_ulong(16 * 64 + 1), ctypes.c_uint(0))
    if rc != 0:  # MPOL_BIND refused
        libc.munmap(addr, size)
        return torch.from_numpy(arr).pin_memory()
    ctypes.memmove(addr, arr.ctypes.data, arr.nbytes)  # first touch, on the node
    try:
        ok = int(torch.cuda.cudart().cudaHostRegister(addr, size, 0)) == 0
    except (AttributeError, RuntimeError, TypeError):
        ok = False
    if not ok:
        libc.munmap(addr, size)
        return torch.from_numpy(arr).pin_memory()
    _NODE_PINNED.append((addr, size))
    buf = (ctypes.c_char * arr.nbytes).from_address(addr)
    return torch.frombuffer(buf, dtype=torch.from_numpy(arr[:0]).dtype)


def gpu_local_cpus(dev):
    """The CPUs sysfs lists as local to the GPU's PCI device, among those this
    process may use (None when unknown)."""
    import torch
    try:
        pr = torch.cuda.get_device_properties(dev)
        bus = "%04x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        with open("/sys/bus/pci/devices/%s/local_cpulist" % bus) as f:
            text = f.read().strip()
    except (AttributeError, OSError, RuntimeError):
        return None
    cpus = set()
    for part in text.split(","):
        if "-" in part:
            lo, hi = part.split("-")
            cpus.update(range(int(lo), int(hi) + 1))
        elif part:
            cpus.add(int(part))
    local = cpus & os.sched_getaffinity(0)
    return local or None


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per projection launch from the committed ncu summary, or None
    when the kernel sources changed since the capture."""
    try:
        kv = {}
        with open(PROFILE_SUMMARY) as f:
            for ln in f:
                if ":" in ln and not ln.startswith(" "):
                    k, v = ln.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("source_sha256") != kernel_source_hash():
            return None
        return float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def make_workload(rank, scale):
    from paper_1401_4780_gb300 import synth
    m, n = (1 << 22) >> scale, (1 << 20) >> scale
    return synth.large_async_system(rep=rank, m=m, n=n)


def workload_config(s, args):
    return {"workload": "large async system: m=2^22, n=2^20, 32 nnz/row, N(0,1) values, "
                        "lognormal(0,1) row norms, FP32 values and x, int32 columns"
                        if args.scale == 0 else "reduced large async system (testing)",
            "m": s.m, "n": s.n, "nnz_per_row": 32, "nnz": s.nnz, "gamma": args.gamma,
            "tol": args.tol, "x0": "zeros", "step": "one solve to tol from x0",
            "check_interval": "adaptive (check_every=0)",
            "l2_flush": "none: 1.07 GB column/value stream > 129 MB L2 per sweep",
            "parallelism": "replicas (one independent system per GPU)"}


def cpu_oracle_sample(s, gamma, target_s, seed):
    """Projections/s of the FP64 oracle (one thread) on a bounded sample of the workload."""
    import oracle
    from paper_1401_4780_gb300 import synth  # noqa: F401
    val64 = s.val64
    samp = oracle.Sampler(s.m, s.row_ptr, val64)
    x = np.zeros(s.n)
    t0 = time.perf_counter()
    calib = 200_000
    oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, val64, s.b, x, gamma, seed, 0, 0, calib,
                    sampler=samp)
    dt = time.perf_counter() - t0
    rate = calib / dt
    nsteps = int(max(calib, min(rate * target_s, 50 * s.m)))
    t0 = time.perf_counter()
    oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, val64, s.b, x, gamma, seed, 0, calib, nsteps,
                    sampler=samp)
    dt = time.perf_counter() - t0
    return nsteps / dt, nsteps, dt


def cpu_multicore_sample(s, gamma, seed):
    """The paper's own multicore scheme (Section 5: per-thread row slices scanned in a
    fresh random order, lock-free atomic FP32 updates) on all host cores: 2 scans of the
    same system from x0 = 0."""
    from oracle import cpu_baseline
    x = np.zeros(s.n, dtype=np.float32)
    val32 = s.val64.astype(np.float32)
    done, secs, threads = cpu_baseline.run(s.m, s.row_ptr, s.col, val32, s.b, x, gamma=gamma,
                                           scans=2, seed=seed)
    return {"value": done / secs, "unit": UNIT, "cores": threads,
            "kind": "the paper's multicore scheme (Section 5), pthreads, FP32",
            "sample": "%d projections (2 scans of every thread's slice) of the same system "
                      "from x0=0, %.2f s" % (done, secs)}


def run_reference(args, dist):
    if dist.rank != 0:
        return
    from paper_1401_4780_gb300 import synth
    s = make_workload(0, args.scale)
    seed = synth.solver_seed(s.seed)
    import oracle
    val64 = s.val64
    samp = oracle.Sampler(s.m, s.row_ptr, val64)
    x = np.zeros(s.n)
    # size each step to about 5 s of single-thread oracle work
    t0 = time.perf_counter()
    oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, val64, s.b, x, args.gamma, seed, 0, 0, 100_000,
                    sampler=samp)
    per_step = int(max(100_000, 100_000 / (time.perf_counter() - t0) * 5.0))
    j = 100_000
    for _ in range(args.warmup):
        oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, val64, s.b, x, args.gamma, seed, 0, j,
                        per_step, sampler=samp)
        j += per_step
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, val64, s.b, x, args.gamma, seed, 0, j,
                        per_step, sampler=samp)
        times.append(time.perf_counter() - t0)
        j += per_step
    total = sum(times)
    value = per_step * args.steps / total
    sample = "%d projections per step (%.2f sweeps) of the workload, FP64 oracle, 1 thread" % (
        per_step, per_step / s.m)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(s, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the other workloads: FP64 plain, BF16 refinement, batched, served
# ---------------------------------------------------------------------------
def _timed_solve(p, x, reps=3, **kw):
    best = None
    for _ in range(reps):
        p.position = 0
        x[:] = 0.0
        st, info = p.solve(x, **kw)
        if best is None or info.seconds < best[1].seconds:
            best = (st, info)
    return best


def extras_plain_refine(asyrk, synth):
    out = {}
    s1 = synth.plain_f64_system()
    with asyrk.Problem.from_system(s1) as p:
        x = np.zeros(s1.n)
        st, i = _timed_solve(p, x, tol=1e-8, max_sweeps=400, x_true=s1.x_true)
        out["plain_f64_async_to_1e-8"] = {"status": st, "ms": 1e3 * i.seconds, "sweeps": i.sweeps,
                                          "rel_err": i.rel_err, "workers": i.workers}
        # the same FP64 system through refinement: FP32 inner sweeps on the FP64
        # values, the residual, norms and update in FP64 (this GPU's FP64 rate is low)
        for tol in (1e-8, 1e-10):
            st, i = _timed_solve(p, x, tol=tol, max_sweeps=2000, x_true=s1.x_true,
                                 mode=asyrk.MODE_REFINE)
            out["f64_values_refine_to_%g" % tol] = {"status": st, "ms": 1e3 * i.seconds,
                                                    "sweeps": i.sweeps,
                                                    "refine_steps": i.refine_steps,
                                                    "rel_err": i.rel_err}
    s3 = synth.bf16_refine_system()
    s3f = synth.make_system(s3.m, s3.n, 16, s3.seed, row_norms="unit", value_dtype="f32")
    with asyrk.Problem.from_system(s3) as p:
        x = np.zeros(s3.n)
        for tol in (1e-8, 1e-10):
            st, i = _timed_solve(p, x, tol=tol, max_sweeps=2000, x_true=s3.x_true,
                                 mode=asyrk.MODE_REFINE)
            out["bf16_refine_to_%g" % tol] = {"status": st, "ms": 1e3 * i.seconds,
                                               "sweeps": i.sweeps, "refine_steps": i.refine_steps,
                                               "rel_err": i.rel_err, "rel_res": i.rel_res}
    with asyrk.Problem.from_system(s3f) as p:
        x = np.zeros(s3f.n)
        st, i = _timed_solve(p, x, tol=1e-6, max_sweeps=400, x_true=s3f.x_true)
        out["plain_fp32_kernel_to_1e-6"] = {"status": st, "ms": 1e3 * i.seconds,
                                            "sweeps": i.sweeps, "rel_err": i.rel_err}
        st, i = _timed_solve(p, x, reps=1, tol=1e-8, max_sweeps=300, x_true=s3f.x_true)
        out["plain_fp32_kernel_to_1e-8"] = {"status": st, "reached_rel_err": i.rel_err,
                                            "sweeps": i.sweeps,
                                            "note": "FP32 iterate floor; 1e-8 needs refinement"}
    out["workload"] = ("plain FP64: m=4096, n=1024, 16 nnz/row, unit rows; refine: same shape, "
                       "BF16 values, FP32 inner, FP64 outer")
    return out


# Table 2 (AsyRK columns): (m, n, delta, seconds on 10 cores, epochs of n iterations)
TABLE2 = [(80000, 100000, 0.0005, 3.6, 195), (80000, 100000, 0.001, 7.6, 284),
          (80000, 100000, 0.003, 18.4, 232), (500000, 1000000, 0.00005, 5.8, 19),
          (500000, 1000000, 0.0001, 10.4, 30), (500000, 1000000, 0.0002, 15.0, 31)]


def extras_table2(asyrk, synth, torch):
    """Table 2's shapes: Section 5's generator (delta*m*n random positions, so
    Poisson(delta*n) row lengths; unit rows), FP32 async, stop on
    ||A^T(Ax - b)||^2 <= 1e-5 checked at adaptive intervals (half the sweeps the
    measured contraction still needs); with i.i.d. weighted draws
    and with Section 5's shuffled sweeps (rows without replacement)."""
    rows = []
    for k, (m, n, delta, t_paper, ep_paper) in enumerate(TABLE2):
        d = synth.make_system_torch(m, n, ("poisson", delta * n), 7000 + k, row_norms="unit",
                                    value_dtype="f32")
        torch.cuda.synchronize()
        p = asyrk.Problem(m, n, d["row_ptr"], d["col"], d["val_store"], asyrk.F32, d["b"],
                          seed=synth.solver_seed(7000 + k), device_ptrs=True)
        nnz = int(d["row_ptr"][-1].item())
        del d
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        for sampling, sname in ((asyrk.SAMPLE_WEIGHTED, "weighted i.i.d."),
                                (asyrk.SAMPLE_SHUFFLED, "shuffled sweeps")):
            best = None
            for rep in range(2):
                x.zero_()
                p.position = 0
                torch.cuda.synchronize()
                st, info = p.solve(x, tol=1e-5, max_sweeps=3000, device_ptrs=True, profile=True,
                                   measure=asyrk.MEASURE_NORMAL_RESIDUAL, sampling=sampling,
                                   check_every=0)
                if best is None or info.seconds < best[1].seconds:
                    best = (st, info)
            st, info = best
            final = p.normal_residual(x, x_on_device=True)
            rows.append({"m": m, "n": n, "delta": delta, "nnz": nnz, "sampling": sname,
                         "status": st, "ms": 1e3 * info.seconds,
                         "projection_ms": info.project_ms, "sweeps": info.sweeps,
                         "epochs_n_iterations": info.projections / n,
                         "epochs_m_iterations": info.projections / m,
                         "normal_residual2": final,
                         "paper_10_cores": {"seconds": t_paper, "epochs": ep_paper},
                         "speedup_vs_paper_time": t_paper / info.seconds})
        p.close()
    return {"workload": "Table 2 shapes; Section 5's generator with unit rows, FP32 values and "
                        "iterate; stop ||A^T(Ax-b)||^2 <= 1e-5 (absolute), checked at adaptive "
                        "intervals (check_every=0); "
                        "the paper's numbers are 10 cores of an unnamed Intel Xeon (context)",
            "rows": rows}


def extras_tau_threshold(asyrk, synth):
    """Corollary 2's delay bound on a small system (m=4096, n=1024, 16 nnz/row, unit
    rows, FP32; to ||x-x*||/||x*|| <= 1e-6): the automatic worker count is the
    bound's estimate m/(2e(1+sqrt(m/n))^2) - 1; multiples of it show where the
    asynchronous iteration stops converging."""
    s = synth.make_system(4096, 1024, 16, synth.config_seed(3), row_norms="unit",
                          value_dtype="f32")
    rows = []
    with asyrk.Problem.from_system(s) as p:
        x = np.zeros(s.n)
        st, info = p.solve(x, tol=1e-6, max_sweeps=2000, x_true=s.x_true)
        w0 = info.workers
        for mult in (1, 2, 3, 6, 12, 48):
            best = None
            for rep in range(3):
                p.position = 0
                x = np.zeros(s.n)
                st, info = p.solve(x, tol=1e-6, max_sweeps=2000, x_true=s.x_true,
                                   workers=w0 * mult)
                if best is None or info.seconds < best[1].seconds:
                    best = (st, info)
            st, info = best
            rows.append({"workers": info.workers, "multiple_of_bound": mult, "status": st,
                         "sweeps": info.sweeps, "ms": 1e3 * info.seconds,
                         "skipped_fraction": info.skipped / max(1, info.projections)})
    return {"workload": "m=4096, n=1024, 16 nnz/row, unit rows, FP32, tol 1e-6; workers as "
                        "multiples of Corollary 2's estimate (the automatic count); status 0 "
                        "converged, 2 diverged", "rows": rows}


def extras_tau_study(asyrk, synth, torch):
    """Figures 1-2 on the GPU: m=80000, n=100000, delta = 0.001 and 0.003, gamma = 1;
    epochs (n projections) to ||Ax - b||/||b|| <= 1e-4 and time, for a range of worker
    counts W (the delay tau grows with W, and with row density under full-row
    updates, Section 5); speedup against the smallest W's time."""
    out = []
    for k, delta in enumerate((0.001, 0.003)):
        m, n = 80000, 100000
        d = synth.make_system_torch(m, n, ("poisson", delta * n), 7100 + k, row_norms="unit",
                                    value_dtype="f32")
        torch.cuda.synchronize()
        p = asyrk.Problem(m, n, d["row_ptr"], d["col"], d["val_store"], asyrk.F32, d["b"],
                          seed=synth.solver_seed(7100 + k), device_ptrs=True)
        del d
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        rows = []
        for W in (32, 128, 512, 2048, 8192, 32768, 0):
            x.zero_()
            p.position = 0
            torch.cuda.synchronize()
            st, info = p.solve(x, tol=1e-4, max_sweeps=3000, workers=W, device_ptrs=True,
                               measure=asyrk.MEASURE_RESIDUAL, sampling=asyrk.SAMPLE_SHUFFLED,
                               check_every=0)
            rows.append({"workers": info.workers, "status": st, "ms": 1e3 * info.seconds,
                         "epochs_n_iterations": info.projections / n,
                         "skipped_fraction": info.skipped / max(1, info.projections + info.skipped),
                         "projections_per_s": info.projections / info.seconds})
        p.close()
        t0 = rows[0]["ms"]
        for r in rows:
            r["speedup_vs_fewest_workers"] = t0 / r["ms"]
        out.append({"delta": delta, "rows": rows})
    return {"workload": "Figures 1-2 shapes: m=80000, n=100000, Section 5's generator (unit rows, "
                        "Poisson(delta n) per row), FP32, gamma=1, shuffled sweeps as in the "
                        "paper's implementation; stop ||Ax-b||/||b|| <= 1e-4; workers=0 is the "
                        "automatic count", "deltas": out}


def extras_lsq(asyrk, synth, torch):
    """Section 6: least squares of an inconsistent system through the square
    consistent system [[0, A^T], [A, -zeta I]] (phi = 1), built on the GPU,
    solved with FP32 values and FP64 refinement."""
    m, n = 1 << 20, 1 << 18
    d = synth.make_system_torch(m, n, ("poisson", 32), 9100, row_norms="unit", value_dtype="f32")
    g = torch.Generator(device="cuda").manual_seed(9101)
    b = d["b"] + 0.3 * torch.randn(m, dtype=torch.float64, device="cuda", generator=g)
    torch.cuda.synchronize()
    # zeta = 0: Section 6's sigma_r/sqrt(2), sigma_r from 100 Lanczos steps on the GPU
    t0 = time.perf_counter()
    p = asyrk.Problem.lsq(m, n, d["row_ptr"], d["col"], d["val_store"], asyrk.F32, b, 0.0,
                          seed=synth.solver_seed(9100), device_ptrs=True)
    torch.cuda.synchronize()
    build_ms = 1e3 * (time.perf_counter() - t0)
    zeta, _ = p.lsq_params()
    st_ = p.stats()
    z = torch.zeros(n + m, dtype=torch.float64, device="cuda")

    def timed(reps=2):
        best = None
        for rep in range(reps):
            z.zero_()
            p.position = 0
            torch.cuda.synchronize()
            r = p.solve(z, tol=1e-10, max_sweeps=5000, mode=asyrk.MODE_REFINE, device_ptrs=True)
            if best is None or r[1].seconds < best[1].seconds:
                best = r
        return best

    # the system mixes rows of ~4x the mean length (A^T) with rows of ~1.03x (A):
    # the default sub-warp width fits the longest rows; the autotuner measures
    st0, info0 = timed()
    t0 = time.perf_counter()
    tune = p.autotune()
    tune_ms = 1e3 * (time.perf_counter() - t0)
    st, info = timed()
    x = p.lsq_solution(z, on_device=True)
    p.close()
    # optimality ||A^T(A x - b)|| / ||A^T b|| in FP64 on the GPU, through a plain problem on A
    pa = asyrk.Problem(m, n, d["row_ptr"], d["col"], d["val_store"], asyrk.F32, b, seed=1,
                       device_ptrs=True)
    opt = (pa.normal_residual(x, x_on_device=True)
           / pa.normal_residual(torch.zeros(n, dtype=torch.float64, device="cuda"),
                                x_on_device=True)) ** 0.5
    pa.close()
    return {"workload": "inconsistent A x = b: m=2^20, n=2^18, Section 5's random positions "
                        "(Poisson(32) per row), unit rows, FP32 values, b = A x* + N(0, 0.3^2); "
                        "system of Section 6 with phi=1, zeta=sigma_r/sqrt(2), sigma_r estimated "
                        "by 100 Lanczos steps on the GPU (random-matrix edge: ~1); FP64-refined "
                        "solve to relative residual 1e-10 of that system",
            "zeta": zeta,
            "system_rows": st_["m"], "system_cols": st_["n"], "system_nnz": st_["nnz"],
            "build_ms_incl_sigma_estimate": build_ms,
            "default_shape": {"status": st0, "solve_ms": 1e3 * info0.seconds,
                              "subwarp": info0.subwarp, "workers": info0.workers,
                              "projections_per_s": info0.projections / info0.seconds},
            "autotune": {"ms": tune_ms, "subwarp": tune.subwarp, "workers": tune.workers},
            "status": st, "subwarp": info.subwarp, "workers": info.workers, "solve_ms": 1e3 * info.seconds,
            "sweeps": info.sweeps, "projections": info.projections,
            "projections_per_s": info.projections / info.seconds,
            "normal_eq_rel_residual": opt}


def extras_batched(asyrk, synth, torch, graph=True, systems=0):
    shapes = synth.batch_shapes()
    if systems > 0:  # profiling aid: the first `systems` members only
        shapes = shapes[:systems]
    base = synth.config_seed(4) * 1000
    probs, x_trues = [], []
    for k, (m, n, L) in enumerate(shapes):
        d = synth.make_system_torch(m, n, L, base + k, row_norms="unit", value_dtype="f32")
        torch.cuda.synchronize()
        probs.append(asyrk.Problem(m, n, d["row_ptr"], d["col"], d["val_store"], asyrk.F32, d["b"],
                                   seed=synth.solver_seed(base + k), device_ptrs=True))
        x_trues.append(d["x_true"])
        del d
    # the autotuner, once per row-length class (the largest system of each)
    tuned = {}
    by_class = {}
    for p, (m, n, L) in zip(probs, shapes):
        c = 1 << (L - 1).bit_length()
        if c not in by_class or m > by_class[c][1]:
            by_class[c] = (p, m)
    for c, (p, _) in sorted(by_class.items()):
        r = p.autotune()
        tuned[str(c)] = {"subwarp": r.subwarp, "workers_at_that_m": r.workers,
                         "projections_per_s": r.projections_per_s, "trials": r.trials}
    xs = [torch.zeros(n, dtype=torch.float64, device="cuda") for (_, n, _) in shapes]
    tols = [1e-6] * len(shapes)

    def run(engine):
        with asyrk.Batch(probs, graph=graph, engine=engine) as b:
            b.solve(xs, tols=tols, max_sweeps=400, x_trues=x_trues, device_ptrs=True)  # warm-up
            for x in xs:
                x.zero_()
            torch.cuda.synchronize()
            return b.solve(xs, tols=tols, max_sweeps=400, x_trues=x_trues, device_ptrs=True)

    # the global-iterate engine first, then the default (on-chip when every member fits)
    st_g, infos_g, bi_g = run(asyrk.ENGINE_GLOBAL)
    errs_g = [float(torch.linalg.norm(x - xt) / torch.linalg.norm(xt)) for x, xt in zip(xs, x_trues)]
    global_engine = {"status": st_g, "converged": bi_g.converged, "device_ms": bi_g.device_ms,
                     "wall_ms": 1e3 * bi_g.seconds, "iterations": bi_g.iterations,
                     "projections_per_s": bi_g.projections / (bi_g.device_ms / 1e3),
                     "max_rel_err_host": max(errs_g), "kernel_launches": bi_g.kernel_launches,
                     "resident_warps": bi_g.resident_warps}
    for x in xs:
        x.zero_()
    st, infos, bi = run(asyrk.ENGINE_AUTO)
    errs = [float(torch.linalg.norm(x - xt) / torch.linalg.norm(xt)) for x, xt in zip(xs, x_trues)]
    # the plain single-system FP32 kernel, one system after another, same tolerance
    t_plain, proj_plain, ok_plain = 0.0, 0, 0
    for p, x, xt in zip(probs, xs, x_trues):
        x.zero_()
        stp, ip = p.solve(x, tol=1e-6, max_sweeps=400, x_true=xt, device_ptrs=True)
        t_plain += ip.seconds
        proj_plain += ip.projections - ip.skipped
        ok_plain += stp == asyrk.OK
    sweeps = [i.sweeps for i in infos]
    # algorithmic bytes: each projection streams its row (4 B column + 4 B value per
    # nonzero) and its 32 B record; per system, its projections x its row length
    alg_bytes = sum(i.projections * (8 * L + 32) for i, (m, n, L) in zip(infos, shapes))
    peak, peak_kind = read_peaks()
    out = {"workload": "%d systems: m = floor(2^U(11,18)), n = m/4, nnz/row U{8..64} per system, "
                       "N(0,1) values, unit rows, FP32; each to ||x-x*||/||x*|| <= 1e-6" % len(shapes),
           "systems": len(shapes), "sum_m": int(sum(m for m, _, _ in shapes)),
           "sum_nnz": int(sum(m * L for m, _, L in shapes)), "status": st,
           "converged": bi.converged, "iterations": bi.iterations, "graph_launch": bool(bi.graph),
           "engine": {1: "global iterate (L2 atomics)",
                      2: "on-chip: one CTA per system, x in its shared memory",
                      3: "both at once on split SMs: on-chip CTAs for the members that fit, "
                         "the global iterate for the rest"}.get(bi.engine, bi.engine),
           "onchip_members": bi.onchip_members,
           "global_part_ms": bi.global_ms, "onchip_part_ms": bi.onchip_ms,
           "workers_per_system_median": float(np.median([i.workers for i in infos])),
           "device_ms": bi.device_ms, "wall_ms": 1e3 * bi.seconds,
           "projections_per_s": bi.projections / (bi.device_ms / 1e3),
           "row_stream_gbs": alg_bytes / (bi.device_ms / 1e3) / 1e9,
           "row_stream_frac_of_hbm": alg_bytes / (bi.device_ms / 1e3) / 1e9 / peak,
           "hbm_peak_source": peak_kind,
           "max_rel_err_host": max(errs), "sweeps_median": float(np.median(sweeps)),
           "sweeps_max": int(max(sweeps)), "kernel_launches": bi.kernel_launches,
           "resident_warps": bi.resident_warps, "autotuned_by_row_length_class": tuned,
           "global_engine_sms": bi.global_sms,
           "plain_fp32_one_at_a_time": {"wall_ms": 1e3 * t_plain, "converged": ok_plain,
                                        "projections_per_s": proj_plain / t_plain},
           "speedup_vs_one_at_a_time": t_plain / bi.seconds,
           "global_engine": global_engine,
           "speedup_vs_global_engine": bi_g.device_ms / bi.device_ms}
    for p in probs:
        p.close()
    return out


def extras_served(asyrk, synth, torch, seconds, rate, admit_load=0.0, partition=0):
    import threading
    pool = {"small_bf16": [], "small_f32": [], "large_bf16": [], "large_f32": []}
    xts = {}
    seed0 = synth.config_seed(5) * 1000
    k = 0
    for cls, (m, n, L, dt, count) in {"small_bf16": (4096, 1024, 16, "bf16", 32),
                                      "small_f32": (4096, 1024, 16, "f32", 32),
                                      "large_bf16": (1 << 20, 1 << 18, 32, "bf16", 2),
                                      "large_f32": (1 << 20, 1 << 18, 32, "f32", 2)}.items():
        for _ in range(count):
            d = synth.make_system_torch(m, n, L, seed0 + k, row_norms="unit", value_dtype=dt)
            torch.cuda.synchronize()
            vd = asyrk.BF16 if dt == "bf16" else asyrk.F32
            p = asyrk.Problem(m, n, d["row_ptr"], d["col"], d["val_store"], vd, d["b"],
                              seed=synth.solver_seed(seed0 + k), device_ptrs=True)
            pool[cls].append(p)
            xts[id(p)] = d["x_true"].cpu().numpy()
            del d
            k += 1
    rng = np.random.default_rng(synth.config_seed(5))
    t, reqs = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > seconds:
            break
        large = rng.random() < 0.05
        bf16 = rng.random() < 0.5
        tol = 1e-6 if rng.random() < 0.5 else 1e-10
        refine = bf16 or tol < 1e-8  # 1e-10 needs FP64 refinement
        cls = ("large_" if large else "small_") + ("bf16" if refine else "f32")
        p = pool[cls][int(rng.integers(len(pool[cls])))]
        reqs.append((t, p, tol, asyrk.MODE_REFINE if refine else asyrk.MODE_ASYNC, cls))
    tickets = [None] * len(reqs)
    sv = asyrk.Server(120 << 30, max_slots=512, admit_load=admit_load, partition=partition)
    # warm-up: one request of each class
    for cls in pool:
        p = pool[cls][0]
        tt = sv.submit(p, x_true=xts[id(p)], tol=1e-6,
                       mode=asyrk.MODE_REFINE if cls.endswith("bf16") else asyrk.MODE_ASYNC)
        sv.wait(tt, p.n)
    t0 = time.perf_counter()

    def submitter():
        for q, (ta, p, tol, mode, _) in enumerate(reqs):
            dt = t0 + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets[q] = sv.submit(p, x_true=xts[id(p)], tol=tol, mode=mode, max_sweeps=3000)

    th = threading.Thread(target=submitter)
    th.start()
    # latency percentiles count the requests that arrive after a warm-up of
    # 2 s (a fifth of shorter windows); throughput counts every request
    warm_s = min(2.0, 0.2 * seconds)
    lat, lat_all, ok, errs_ok = {}, [], 0, True
    for q, (ta, p, tol, mode, cls) in enumerate(reqs):
        while tickets[q] is None:
            time.sleep(0.0005)
        st, x, info = sv.wait(tickets[q], p.n)
        ok += st == asyrk.OK
        lat_all.append(info.seconds)
        if ta >= warm_s:
            lat.setdefault(cls, []).append(info.seconds)
        if st == asyrk.OK and not (info.rel_err <= tol * 1.0001):
            errs_ok = False
    t_end = time.perf_counter()
    th.join()
    stats = sv.stats()
    sv.close()
    allv = np.concatenate([np.array(v) for v in lat.values()])
    out = {"workload": "Poisson arrivals; 95%% m=4096, n=1024, 16 nnz/row, 5%% m=2^20, n=2^18, "
                       "32 nnz/row (unit rows); mode FP32 or BF16+FP64 refinement, tol 1e-6 or "
                       "1e-10 (1e-10 always refined); budget 120 GB; pool of 68 resident problems",
           "offered_rate_per_s": rate, "window_s": seconds, "requests": len(reqs),
           "converged": ok, "all_errors_within_tol": errs_ok,
           "solves_per_s": len(reqs) / (t_end - t0),
           "latency_after_warmup_s": warm_s, "latency_requests": int(allv.size),
           "p50_ms": 1e3 * float(np.percentile(allv, 50)),
           "p99_ms": 1e3 * float(np.percentile(allv, 99)),
           "p50_ms_all_requests": 1e3 * float(np.percentile(lat_all, 50)),
           "p99_ms_all_requests": 1e3 * float(np.percentile(lat_all, 99)),
           "per_class": {c: {"n": len(v), "p50_ms": 1e3 * float(np.percentile(v, 50)),
                             "p99_ms": 1e3 * float(np.percentile(v, 99))}
                         for c, v in sorted(lat.items())},
           "engine_steps": stats["iterations"], "max_in_flight": stats["max_active"],
           "max_in_shared_step": stats["max_active_shared"], "admit_load": admit_load,
           "sm_split": {"shared_step": stats["step_sms"], "on_chip": stats["onchip_sms"]},
           "solved_on_chip": stats["onchip_completed"]}
    # the plain single-system FP32 kernel, one request at a time, at 1e-6
    times = {}
    for cls, count in (("small_f32", 16), ("large_f32", 2)):
        ts = []
        for q in range(count):
            p = pool[cls][q % len(pool[cls])]
            x = np.zeros(p.n)
            p.position = 0
            stp, ip = p.solve(x, tol=1e-6, max_sweeps=400, x_true=xts[id(p)])
            ts.append(ip.seconds)
        times[cls] = float(np.median(ts))
    per_solve = 0.95 * times["small_f32"] + 0.05 * times["large_f32"]
    out["plain_fp32_one_at_a_time"] = {"small_ms": 1e3 * times["small_f32"],
                                       "large_ms": 1e3 * times["large_f32"],
                                       "solves_per_s_at_the_mix": 1.0 / per_solve}
    for v in pool.values():
        for p in v:
            p.close()
    return out


def run_asyrk(args, dist):
    import torch

    from paper_1401_4780_gb300 import asyrk, synth

    assert torch.cuda.is_available(), "bench.py needs a GPU"
    torch.cuda.set_device(dist.local_rank)
    # host buffers (pinned inputs of the end-to-end leg) on the GPU's side of the
    # host: run on the CPUs local to it while the GPU legs run
    all_cpus = os.sched_getaffinity(0)
    local = gpu_local_cpus(dist.local_rank)
    if local and local != all_cpus:
        os.sched_setaffinity(0, local)
    affinity = {"gpu_local_cpus": len(local) if local else None, "cpus": len(all_cpus),
                "pinned_to_local": bool(local and local != all_cpus),
                "gpu_numa_node": gpu_numa_node(dist.local_rank),
                "cpu_numa_nodes": cpu_numa_nodes(all_cpus)}
    asyrk.load()
    s = make_workload(dist.rank, args.scale)
    seed = synth.solver_seed(s.seed)
    stream = torch.cuda.current_stream()
    max_sweeps = 1000

    # ---------------- device-resident timed steps ----------------
    p = asyrk.Problem.from_system(s, seed=seed)
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    xt = torch.from_numpy(s.x_true).cuda()
    torch.cuda.synchronize()

    def step():
        x.zero_()
        # check_every = 0: the solve's adaptive check interval (next check after
        # half the sweeps the measured contraction still needs); it stops at
        # most 10 % past the sweep that meets the tolerance
        st, info = p.solve(x, gamma=args.gamma, tol=args.tol, max_sweeps=max_sweeps, x_true=xt,
                           device_ptrs=True, stream=stream, profile=True, check_every=0)
        if st != asyrk.OK:
            raise RuntimeError("solve status %d: %s" % (st, asyrk.asyrk_last_error()))
        return info

    for _ in range(args.warmup):
        step()
    dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dist.local_rank)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos = [step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clock = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max = dist.reduce(ms, "max")
    # skipped projections (row exclusion) do no update: only applied ones count
    proj = sum(i.projections - i.skipped for i in infos)
    skipped = sum(i.skipped for i in infos)
    proj_all = dist.reduce(proj, "sum")
    launches_all = dist.reduce(sum(i.kernel_launches for i in infos), "sum")
    value = proj_all / (ms_max / 1e3)

    # dominant kernel: the projection launches, event-timed on their stream
    proj_ms = sum(i.project_ms for i in infos)
    proj_launches = sum(i.project_launches for i in infos)
    per_launch_s = proj_ms / 1e3 / proj_launches
    per_launch_proj = proj / proj_launches
    achieved = BYTES_PER_PROJECTION * per_launch_proj / per_launch_s / 1e9
    peak, peak_kind = read_peaks()
    # the committed ncu summary holds DRAM bytes for a launch of one sweep
    # (4,194,304 drawn projections); a launch here may run several sweeps (the
    # adaptive check interval), so the bytes are scaled by the drawn
    # projections per launch (the stream is read once per projection)
    traffic = recorded_traffic()
    if traffic is not None:
        drawn_per_launch = (proj + skipped) / proj_launches
        traffic = traffic * drawn_per_launch / float(1 << 22) if args.scale == 0 else None
    sweeps = [i.sweeps for i in infos]
    # L2 denominators measured now on this GPU: random red.add.f32 and gathers
    # on an array the size of x (the kernel does 32 of each per projection)
    probe = {}
    for name, kind in (("red_f32_per_s", asyrk.PROBE_RED_F32),
                       ("gather_f32_per_s", asyrk.PROBE_GATHER_F32),
                       ("gather_red_pairs_per_s", asyrk.PROBE_GATHER_RED)):
        ops = 1 << 28
        st_, pms = asyrk.asyrk_probe(kind, s.n, ops)
        probe[name] = ops / (pms / 1e3) if st_ == asyrk.OK and pms > 0 else None
    # the bound of the row-projection kernel: min(HBM / 280 B, red-rate / 32,
    # gather+red pair rate / 32) projections/s.  x (n FP32 = 4 MB) is L2-resident,
    # so the binding resource is the L2 atomic rate: the line reports the kernel's
    # red.add.f32 rate (32 per applied projection) against the probe's rate of
    # random red.add.f32 on an array of x's size, measured now on this GPU, with
    # the HBM fraction of the row stream beside it
    reds_per_s = 32 * per_launch_proj / per_launch_s
    red_peak = probe.get("red_f32_per_s")
    pair_peak = probe.get("gather_red_pairs_per_s")
    hbm = {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"
           if peak_kind == "measured" else "fallback 6.8 TB/s",
           "bytes_per_projection": BYTES_PER_PROJECTION}
    gather_peak = probe.get("gather_f32_per_s")
    bounds = {"hbm_projections_per_s": peak * 1e9 / BYTES_PER_PROJECTION,
              "l2_red_projections_per_s": red_peak / 32 if red_peak else None,
              "l2_gather_red_projections_per_s": pair_peak / 32 if pair_peak else None,
              # the bound as the method's scope defines it: min(HBM / 280 B,
              # atomic rate / 32, L2 read-sector rate / (2 x 32 sectors)), with
              # the gather probe's rate as the L2 read-sector rate
              "min_of_hbm_atomic_l2sector": min(
                  [v for v in (peak * 1e9 / BYTES_PER_PROJECTION,
                               red_peak / 32 if red_peak else None,
                               gather_peak / 64 if gather_peak else None) if v])}
    l2_resident = 4 * s.n <= (64 << 20)
    if l2_resident and red_peak:
        roofline = {"bound": "l2_atomic", "achieved": reds_per_s / 1e9, "peak": red_peak / 1e9,
                    "unit": "G red.add.f32/s", "frac": reds_per_s / red_peak,
                    "peak_source": "measured in this run on this GPU: asyrk_probe "
                                   "PROBE_RED_F32, 2^28 random red.add.f32 on an n-float array "
                                   "(the size of x), 8 in flight per thread, CUDA events",
                    "traffic": traffic, "hbm": hbm}
    else:
        roofline = dict(bound="hbm", traffic=traffic, **hbm)
    roofline.update({
        "kernel": "k_project<float,float,8> (one sweep per launch)",
        "binding": "L2: ~64 random 4-byte gathers/red.adds per projection on the "
                   "L2-resident x, and their latency (ncu: L2 tag requests ~75% of "
                   "peak, DRAM ~9%, long-scoreboard stalls)",
        "traffic_unit": "DRAM bytes per launch (ncu dram__bytes_read.sum + write.sum)",
        "projections_per_launch": per_launch_proj,
        "launch_ms": per_launch_s * 1e3,
        "kernel_share_of_step": proj_ms / ms,
        "bounds_projections_per_s": bounds,
        "achieved_projections_per_s": per_launch_proj / per_launch_s,
        "frac_of_min_bound": (per_launch_proj / per_launch_s) / bounds["min_of_hbm_atomic_l2sector"],
        # the L2 pipe's time per second if gathers and red.adds take turns in it:
        # reds at the red-only rate plus gathers at the gather-only rate
        "l2_op_time_frac": (reds_per_s / red_peak + reds_per_s / gather_peak)
        if red_peak and gather_peak else None,
        "l2": {"achieved_red_f32_per_s": reds_per_s,
               "achieved_gather_red_pairs_per_s": reds_per_s,
               "probe": probe,
               "frac_of_probe_red": reds_per_s / red_peak if red_peak else None,
               "frac_of_probe_pairs": reds_per_s / pair_peak if pair_peak else None}})
    # the workload's gamma sweep {0.5, 1}: time to tol and sweeps for each
    gamma_sweep = None
    if dist.rank == 0 and not args.no_extras:
        gamma_sweep = []
        for g in (0.5, 1.0):
            x.zero_()
            torch.cuda.synchronize()
            st, info = p.solve(x, gamma=g, tol=args.tol, max_sweeps=max_sweeps, x_true=xt,
                               device_ptrs=True, stream=stream, profile=True, check_every=0)
            gamma_sweep.append({"gamma": g, "status": st, "ms": 1e3 * info.seconds,
                                "sweeps": info.sweeps, "rel_err": info.rel_err,
                                "applied_projections_per_s":
                                    (info.projections - info.skipped) / info.seconds})
        # time to 1e-8 on the same system: FP32 values and FP32 inner solves
        # with FP64 refinement (the plain FP32 kernel stalls near 1e-7)
        x.zero_()
        torch.cuda.synchronize()
        st, info = p.solve(x, gamma=1.0, tol=1e-8, max_sweeps=max_sweeps, x_true=xt,
                           device_ptrs=True, stream=stream, mode=asyrk.MODE_REFINE)
        gamma_sweep.append({"mode": "refine", "tol": 1e-8, "status": st,
                            "ms": 1e3 * info.seconds, "sweeps": info.sweeps,
                            "refine_steps": info.refine_steps, "rel_err": info.rel_err,
                            "rel_res": info.rel_res})
    p.close()

    # ---------------- end to end from host buffers ----------------
    node = gpu_numa_node(dist.local_rank)
    pin = lambda a: pinned_on_node(a, node)
    h_rp, h_col, h_val, h_b, h_xt = (pin(s.row_ptr), pin(s.col), pin(s.val_store), pin(s.b),
                                     pin(s.x_true))
    h_x = torch.zeros(s.n, dtype=torch.float64).pin_memory()
    # the host link as this machine gives it: the column array from its page-locked
    # buffer to the device, event-timed (best of 3), before the end-to-end steps
    h2d_gbs = None
    if args.e2e_steps > 0:
        d_col = torch.empty(h_col.numel(), dtype=h_col.dtype, device="cuda")
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            d_col.copy_(h_col, non_blocking=True)
            e1.record()
            torch.cuda.synchronize()
            ms_c = e0.elapsed_time(e1)
            best = ms_c if best is None else min(best, ms_c)
        h2d_gbs = h_col.numel() * h_col.element_size() / (best / 1e3) / 1e9
        del d_col
    e2e_t, e2e_proj, e2e_sweeps = 0.0, 0, 0
    split = {"create_s": 0.0, "solve_s": 0.0, "destroy_s": 0.0}
    create_ms = []
    for k in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):  # first round warms up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with asyrk.Problem(s.m, s.n, h_rp, h_col, h_val, asyrk.F32, h_b, seed=seed) as q:
            t1 = time.perf_counter()
            h_x.zero_()
            st, info = q.solve(h_x, gamma=args.gamma, tol=args.tol, max_sweeps=max_sweeps,
                               x_true=h_xt, check_every=0)
            t2 = time.perf_counter()
        dt = time.perf_counter() - t0
        if k > 0:
            create_ms.append(1e3 * (t1 - t0))
            split["create_s"] += t1 - t0
            split["solve_s"] += t2 - t1
            split["destroy_s"] += t0 + dt - t2
        if st != asyrk.OK:
            raise RuntimeError("e2e solve status %d" % st)
        if k > 0:
            e2e_t += dt
            e2e_proj += info.projections - info.skipped
            e2e_sweeps += info.sweeps
    e2e_t = dist.reduce(e2e_t, "max")
    e2e_proj = dist.reduce(e2e_proj, "sum")
    # what crosses the host link per step: asyrk_create copies the CSR arrays and
    # b (the row records and the alias table are built on the GPU); the solve
    # copies x0 and x* in and x out, and reads one 8-byte measure per check (at
    # most one per sweep with the adaptive interval, plus the initial one: counted
    # as one per sweep) and a few status words
    h2d = (s.row_ptr.nbytes + s.col.nbytes + s.val_store.nbytes + s.b.nbytes
           + 2 * 8 * s.n)
    checks = e2e_sweeps / max(1, args.e2e_steps) + 1
    d2h = 8 * s.n + 8 * checks + 64
    e2e = None if args.e2e_steps <= 0 else {"value": e2e_proj / e2e_t, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h),
           "what": "asyrk_create from pinned host CSR + asyrk_solve (host x0 -> host x) + destroy",
           "ms_per_step_split": {k: 1e3 * v / max(1, args.e2e_steps) for k, v in split.items()},
           "create_ms_each_step": create_ms,
           "host_affinity": affinity, "h2d_probe_gbs": h2d_gbs,
           "note": "create copies 1.1 GB over the host link (~210 GB/s: ~5.2 ms of its ~6.3 ms); "
                   "on some boxes the link stalls for 10-60 ms about every 0.5 s whatever the "
                   "process runs, which slows the creates that meet a stall to 16-240 ms"}

    cpu = None
    cpu_mt = None
    if dist.rank == 0 and dist.world == 1 and args.cpu_seconds > 0:
        os.sched_setaffinity(0, all_cpus)  # the CPU baselines get every core again
        rate, nsteps, dt = cpu_oracle_sample(s, args.gamma, args.cpu_seconds, seed)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "%d projections (%.2f sweeps) of the same system from x0=0, FP64 "
                         "oracle, single thread, %.1f s" % (nsteps, nsteps / s.m, dt)}
        cpu_mt = cpu_multicore_sample(s, args.gamma, seed)

    extras = None
    if dist.rank == 0 and not args.no_extras:
        # each extra measurement is reported on its own: one that fails records its
        # error instead of taking the benchmark line down with it.  Each starts with
        # the problem memory pool trimmed, so that it does not inherit the memory the
        # previous one freed (measured: 50.5 against 49.9 ms on the batched workload)
        def guarded(fn, *a):
            try:
                asyrk.asyrk_trim_memory()
                return fn(*a)
            except Exception as exc:  # noqa: BLE001 -- reported, not swallowed
                try:
                    torch.cuda.synchronize()
                except Exception:  # noqa: BLE001 -- the error above is the one reported
                    pass
                return {"error": "%s: %s" % (type(exc).__name__, exc)}

        extras = {"gamma_sweep": gamma_sweep,
                  "plain_and_refine": guarded(extras_plain_refine, asyrk, synth),
                  "table2": guarded(extras_table2, asyrk, synth, torch),
                  "least_squares": guarded(extras_lsq, asyrk, synth, torch),
                  "tau_study": guarded(extras_tau_study, asyrk, synth, torch),
                  "tau_threshold": guarded(extras_tau_threshold, asyrk, synth),
                  "batched": guarded(extras_batched, asyrk, synth, torch),
                  "served": guarded(extras_served, asyrk, synth, torch, args.served_seconds,
                                    args.served_rate, args.admit_load)}
        if args.served_rate2 > 0:
            extras["served_lower_rate"] = guarded(extras_served, asyrk, synth, torch,
                                                  args.served_seconds2, args.served_rate2,
                                                  args.admit_load)

    if dist.rank == 0:
        cfg = workload_config(s, args)
        cfg.update({"sweeps_per_step": sweeps, "workers": infos[0].workers,
                    "skipped_fraction": skipped / max(1, skipped + proj),
                    "row_exclusion": "on (a row held by another worker is skipped)",
                    "subwarp": infos[0].subwarp, "time_to_tol_ms_median":
                    statistics.median([1e3 * i.seconds for i in infos])})
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": cfg, "clocks": clock, "e2e": e2e, "gpu_launches": int(launches_all),
                "roofline": roofline, "cpu_baseline": cpu, "cpu_multicore": cpu_mt,
                "kernel_source_sha256": kernel_source_hash(), "extras": extras}
        print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    dist = Dist()
    try:
        if args.impl == "reference":
            run_reference(args, dist)
        elif args.served_only:
            import torch
            from paper_1401_4780_gb300 import asyrk, synth
            torch.cuda.set_device(dist.local_rank)
            asyrk.load()
            out = {"served": extras_served(asyrk, synth, torch, args.served_seconds,
                                           args.served_rate, args.admit_load,
                                           args.server_partition)}
            if args.served_rate2 > 0:
                out["served_lower_rate"] = extras_served(asyrk, synth, torch,
                                                         args.served_seconds2,
                                                         args.served_rate2, args.admit_load,
                                                         args.server_partition)
            print(json.dumps(out), flush=True)
        elif args.batched_only:
            import torch
            from paper_1401_4780_gb300 import asyrk, synth
            torch.cuda.set_device(dist.local_rank)
            asyrk.load()
            print(json.dumps(extras_batched(asyrk, synth, torch, graph=not args.batch_host_loop,
                                            systems=args.batched_systems)),
                  flush=True)
        else:
            run_asyrk(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
