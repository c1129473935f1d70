"""ctypes binding of the C ABI in ``include/asyrk.h`` (libasyrk.so).

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels.  The functions carry the C names; ``Problem`` is a small owner object
around a handle.  Arrays may be numpy arrays (host) or CUDA ``torch.Tensor``s
(device; pass ``device_ptrs=True``).  Loading fails loudly when the library has
not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libasyrk.so")

F64, F32, BF16 = 0, 1, 2
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, NOT_CONVERGED, DIVERGED = 0, -1, -2, -3, -4, 1, 2
ECANCELED = -5
MODE_SEQUENTIAL, MODE_ASYNC, MODE_REFINE = 0, 1, 2
MEASURE_AUTO, MEASURE_RESIDUAL, MEASURE_NORMAL_RESIDUAL = 0, 1, 2
FORM_AUTO, FORM_LATENCY, FORM_THROUGHPUT = 0, 1, -1
SAMPLE_WEIGHTED, SAMPLE_SHUFFLED = 0, 1
UPDATE_ROW, UPDATE_SINGLE = 0, 1
ENGINE_AUTO, ENGINE_GLOBAL, ENGINE_ONCHIP = 0, 1, 2
DTYPES = {"f64": F64, "f32": F32, "bf16": BF16}


class AsyrkError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s (%d): %s" % (where, asyrk_strerror(status), status,
                                               asyrk_last_error()))


class CreateOpts(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("device_ptrs", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("stream", ctypes.c_void_p)]


class LsqOpts(ctypes.Structure):
    _fields_ = [("zeta", ctypes.c_double), ("phi", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("device_ptrs", ctypes.c_int32), ("lanczos_steps", ctypes.c_int32),
                ("stream", ctypes.c_void_p)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("device_ptrs", ctypes.c_int32),
                ("workers", ctypes.c_int32), ("subwarp", ctypes.c_int32),
                ("check_every", ctypes.c_int64), ("x_true", ctypes.c_void_p),
                ("stream", ctypes.c_void_p), ("inner_tol", ctypes.c_double),
                ("inner_sweeps", ctypes.c_int64), ("profile", ctypes.c_int32),
                ("row_exclusion", ctypes.c_int32), ("measure", ctypes.c_int32),
                ("sampling", ctypes.c_int32), ("update", ctypes.c_int32),
                ("graph_loop", ctypes.c_int32), ("kernel_form", ctypes.c_int32)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("workers", ctypes.c_int32),
                ("subwarp", ctypes.c_int32), ("refine_steps", ctypes.c_int32),
                ("sweeps", ctypes.c_int64), ("projections", ctypes.c_int64),
                ("seconds", ctypes.c_double), ("rel_err", ctypes.c_double),
                ("rel_res", ctypes.c_double), ("project_ms", ctypes.c_double),
                ("project_launches", ctypes.c_int64), ("j_end", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_int64), ("skipped", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ProblemStats(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("nnz_padded", ctypes.c_int64), ("max_row_len", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("frob2", ctypes.c_double),
                ("dtype", ctypes.c_int32), ("uniform", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("j_next", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ["asyrk_create", "asyrk_destroy", "asyrk_solve", "asyrk_residual", "asyrk_draw_rows",
           "asyrk_get_position", "asyrk_set_position", "asyrk_problem_get_stats",
           "asyrk_strerror", "asyrk_last_error", "asyrk_abi_version", "asyrk_probe",
           "asyrk_residual_noalloc", "asyrk_normal_residual", "asyrk_autotune", "asyrk_batch_create", "asyrk_batch_solve",
           "asyrk_batch_destroy", "asyrk_server_create", "asyrk_server_submit",
           "asyrk_server_wait", "asyrk_server_cancel", "asyrk_server_get_stats",
           "asyrk_server_destroy", "asyrk_lsq_create", "asyrk_lsq_solution",
           "asyrk_lsq_params", "asyrk_spectrum_estimate", "asyrk_trim_memory"]
NOALLOC_MAX_ROWS = 16777216
PROBE_RED_F32, PROBE_GATHER_F32, PROBE_GATHER_RED, PROBE_STREAM = 0, 1, 2, 3

_lib = None


def load(path: str = LIB_PATH):
    """Load libasyrk.so (built by ``__graft_entry__.build()``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libasyrk.so is not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    P, i64, u64, i32, u32, f64 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64,
                                  ctypes.c_int32, ctypes.c_uint32, ctypes.c_double)
    lib.asyrk_create.argtypes = [ctypes.POINTER(P), i64, i64, P, P, P, ctypes.c_int, P,
                                 ctypes.POINTER(CreateOpts)]
    lib.asyrk_create.restype = ctypes.c_int
    lib.asyrk_lsq_create.argtypes = [ctypes.POINTER(P), i64, i64, P, P, P, ctypes.c_int, P,
                                     ctypes.POINTER(LsqOpts)]
    lib.asyrk_lsq_create.restype = ctypes.c_int
    lib.asyrk_lsq_solution.argtypes = [P, P, ctypes.c_int, P]
    lib.asyrk_lsq_solution.restype = ctypes.c_int
    lib.asyrk_lsq_params.argtypes = [P, ctypes.POINTER(f64), ctypes.POINTER(f64)]
    lib.asyrk_lsq_params.restype = ctypes.c_int
    lib.asyrk_spectrum_estimate.argtypes = [i64, i64, P, P, P, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int32, ctypes.c_uint64, P,
                                            ctypes.POINTER(f64), ctypes.POINTER(f64)]
    lib.asyrk_spectrum_estimate.restype = ctypes.c_int
    lib.asyrk_destroy.argtypes = [P]
    lib.asyrk_destroy.restype = None
    lib.asyrk_trim_memory.argtypes = []
    lib.asyrk_trim_memory.restype = ctypes.c_int
    lib.asyrk_solve.argtypes = [P, P, f64, f64, i64, ctypes.POINTER(SolveOpts),
                                ctypes.POINTER(SolveInfo)]
    lib.asyrk_solve.restype = ctypes.c_int
    lib.asyrk_residual.argtypes = [P, P, ctypes.c_int, ctypes.POINTER(f64)]
    lib.asyrk_residual.restype = ctypes.c_int
    lib.asyrk_normal_residual.argtypes = [P, P, ctypes.c_int, ctypes.POINTER(f64)]
    lib.asyrk_normal_residual.restype = ctypes.c_int
    lib.asyrk_draw_rows.argtypes = [P, u64, i64, u32, ctypes.c_int, P]
    lib.asyrk_draw_rows.restype = ctypes.c_int
    lib.asyrk_get_position.argtypes = [P, ctypes.POINTER(u64)]
    lib.asyrk_get_position.restype = ctypes.c_int
    lib.asyrk_set_position.argtypes = [P, u64]
    lib.asyrk_set_position.restype = ctypes.c_int
    lib.asyrk_problem_get_stats.argtypes = [P, ctypes.POINTER(ProblemStats)]
    lib.asyrk_problem_get_stats.restype = ctypes.c_int
    lib.asyrk_strerror.argtypes = [ctypes.c_int]
    lib.asyrk_strerror.restype = ctypes.c_char_p
    lib.asyrk_last_error.argtypes = []
    lib.asyrk_last_error.restype = ctypes.c_char_p
    lib.asyrk_abi_version.argtypes = []
    lib.asyrk_abi_version.restype = ctypes.c_int
    lib.asyrk_probe.argtypes = [ctypes.c_int, i64, i64, ctypes.POINTER(ctypes.c_float)]
    lib.asyrk_probe.restype = ctypes.c_int
    lib.asyrk_residual_noalloc.argtypes = [i64, i64, i64, P, P, P, ctypes.c_int, P, P, P, P]
    lib.asyrk_residual_noalloc.restype = ctypes.c_int
    lib.asyrk_autotune.argtypes = [P, i64, ctypes.c_int, ctypes.POINTER(TuneResult)]
    lib.asyrk_autotune.restype = ctypes.c_int
    lib.asyrk_batch_create.argtypes = [ctypes.POINTER(P), P, ctypes.c_int,
                                       ctypes.POINTER(BatchOpts)]
    lib.asyrk_batch_create.restype = ctypes.c_int
    lib.asyrk_batch_solve.argtypes = [P, P, P, P, i64, P, ctypes.c_int, P,
                                      ctypes.POINTER(BatchInfo)]
    lib.asyrk_batch_solve.restype = ctypes.c_int
    lib.asyrk_batch_destroy.argtypes = [P]
    lib.asyrk_batch_destroy.restype = None
    lib.asyrk_server_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(ServerOpts)]
    lib.asyrk_server_create.restype = ctypes.c_int
    lib.asyrk_server_submit.argtypes = [P, P, P, P, f64, f64, ctypes.c_int, i64,
                                        ctypes.POINTER(u64)]
    lib.asyrk_server_submit.restype = ctypes.c_int
    lib.asyrk_server_wait.argtypes = [P, u64, P, ctypes.POINTER(SolveInfo), i64]
    lib.asyrk_server_wait.restype = ctypes.c_int
    lib.asyrk_server_cancel.argtypes = [P, u64]
    lib.asyrk_server_cancel.restype = ctypes.c_int
    lib.asyrk_server_get_stats.argtypes = [P, ctypes.POINTER(ServerStats)]
    lib.asyrk_server_get_stats.restype = ctypes.c_int
    lib.asyrk_server_destroy.argtypes = [P]
    lib.asyrk_server_destroy.restype = None
    _lib = lib
    return lib


class TuneResult(ctypes.Structure):
    _fields_ = [("subwarp", ctypes.c_int32), ("workers", ctypes.c_int32),
                ("projections_per_s", ctypes.c_double), ("trials", ctypes.c_int32),
                ("from_cache", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchOpts(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("graph", ctypes.c_int32),
                ("row_exclusion", ctypes.c_int32), ("sampling", ctypes.c_int32),
                ("update", ctypes.c_int32), ("engine", ctypes.c_int32),
                ("cluster_max", ctypes.c_int32), ("workers", ctypes.c_int32),
                ("partition", ctypes.c_int32)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("iterations", ctypes.c_int64), ("projections", ctypes.c_int64),
                ("seconds", ctypes.c_double), ("device_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("resident_warps", ctypes.c_int32),
                ("graph", ctypes.c_int32), ("engine", ctypes.c_int32),
                ("onchip_members", ctypes.c_int32), ("global_sms", ctypes.c_int32),
                ("global_ms", ctypes.c_float), ("onchip_ms", ctypes.c_float),
                ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerOpts(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_int64), ("max_slots", ctypes.c_int32),
                ("row_exclusion", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("max_inner_sweeps", ctypes.c_int64), ("onchip", ctypes.c_int32),
                ("partition", ctypes.c_int32), ("admit_load", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("active", ctypes.c_int64),
                ("iterations", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("mem_used", ctypes.c_int64), ("mem_budget", ctypes.c_int64),
                ("arena_reserved", ctypes.c_int64), ("max_slots", ctypes.c_int32),
                ("max_active", ctypes.c_int32), ("fatal", ctypes.c_int32),
                ("max_active_shared", ctypes.c_int32), ("onchip_completed", ctypes.c_int64),
                ("step_sms", ctypes.c_int32), ("onchip_sms", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _ptr(a):
    """Data pointer of a numpy array or a torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data_as(ctypes.c_void_p)
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    raise TypeError(type(a))


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(s.cuda_stream)
    return ctypes.c_void_p(int(s))


# ---------------------------------------------------------------------------
# C-named wrappers
# ---------------------------------------------------------------------------
def asyrk_strerror(status: int) -> str:
    return load().asyrk_strerror(status).decode()


def asyrk_last_error() -> str:
    return load().asyrk_last_error().decode()


def asyrk_abi_version() -> int:
    return load().asyrk_abi_version()


def asyrk_create(m, n, row_ptr, col_idx, values, vdtype, b, seed=0, device_ptrs=False,
                 stream=None):
    """Returns (status, handle)."""
    h = ctypes.c_void_p()
    o = CreateOpts(seed=seed, device_ptrs=1 if device_ptrs else 0, reserved=0,
                   stream=_stream(stream))
    st = load().asyrk_create(ctypes.byref(h), m, n, _ptr(row_ptr), _ptr(col_idx), _ptr(values),
                             vdtype, _ptr(b), ctypes.byref(o))
    return st, h


def asyrk_lsq_create(m, n, row_ptr, col_idx, values, vdtype, b, zeta, phi=1.0, seed=0,
                     device_ptrs=False, stream=None, lanczos_steps=0):
    """Section 6's least-squares system (zeta = 0: estimated); returns (status, handle)."""
    h = ctypes.c_void_p()
    o = LsqOpts(zeta=float(zeta), phi=float(phi), seed=seed, device_ptrs=1 if device_ptrs else 0,
                lanczos_steps=lanczos_steps, stream=_stream(stream))
    st = load().asyrk_lsq_create(ctypes.byref(h), m, n, _ptr(row_ptr), _ptr(col_idx),
                                 _ptr(values), vdtype, _ptr(b), ctypes.byref(o))
    return st, h


def asyrk_lsq_solution(h, z, x_out, on_device=False):
    return load().asyrk_lsq_solution(h, _ptr(z), 1 if on_device else 0, _ptr(x_out))


def asyrk_lsq_params(h):
    z, f = ctypes.c_double(), ctypes.c_double()
    st = load().asyrk_lsq_params(h, ctypes.byref(z), ctypes.byref(f))
    return st, z.value, f.value


def asyrk_spectrum_estimate(m, n, row_ptr, col_idx, values, vdtype, steps=0, seed=0,
                            device_ptrs=False, stream=None):
    """(status, lambda_min nonzero, lambda_max) of A^T A by Lanczos on the GPU."""
    lo, hi = ctypes.c_double(), ctypes.c_double()
    st = load().asyrk_spectrum_estimate(m, n, _ptr(row_ptr), _ptr(col_idx), _ptr(values), vdtype,
                                        1 if device_ptrs else 0, steps, seed, _stream(stream),
                                        ctypes.byref(lo), ctypes.byref(hi))
    return st, lo.value, hi.value


def asyrk_destroy(h):
    load().asyrk_destroy(h)


def asyrk_trim_memory() -> int:
    """Return the unused memory of the current device's problem memory pool to the driver."""
    return load().asyrk_trim_memory()


def asyrk_solve(h, x, gamma, tol, max_sweeps, opts: SolveOpts = None):
    """x is updated in place; returns (status, SolveInfo)."""
    info = SolveInfo()
    st = load().asyrk_solve(h, _ptr(x), float(gamma), float(tol), int(max_sweeps),
                            ctypes.byref(opts) if opts is not None else None, ctypes.byref(info))
    return st, info


def asyrk_residual(h, x, x_on_device=False):
    out = ctypes.c_double()
    st = load().asyrk_residual(h, _ptr(x), 1 if x_on_device else 0, ctypes.byref(out))
    return st, out.value


def asyrk_normal_residual(h, x, x_on_device=False):
    out = ctypes.c_double()
    st = load().asyrk_normal_residual(h, _ptr(x), 1 if x_on_device else 0, ctypes.byref(out))
    return st, out.value


def asyrk_draw_rows(h, j0, count, stream_id=0, sampling=SAMPLE_WEIGHTED):
    rows = np.zeros(count, dtype=np.int32)
    st = load().asyrk_draw_rows(h, j0, count, stream_id, sampling, _ptr(rows))
    return st, rows


def asyrk_probe(kind, n, ops):
    """Returns (status, kernel milliseconds) of one memory-operation probe."""
    ms = ctypes.c_float()
    st = load().asyrk_probe(kind, n, ops, ctypes.byref(ms))
    return st, ms.value


def asyrk_residual_noalloc(m, n, nnz, row_ptr, col_idx, values, vdtype, b, x, out, stream=None):
    """Enqueue ||b - A x|| -> out[0], ||b|| -> out[1] (all device arrays); returns the status.

    Allocates nothing: for callers that cannot call cudaMalloc (see asyrk.h)."""
    return load().asyrk_residual_noalloc(m, n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(values),
                                         vdtype, _ptr(b), _ptr(x), _ptr(out), _stream(stream))


def asyrk_autotune(h, trial_projections=0, force=False):
    r = TuneResult()
    st = load().asyrk_autotune(h, trial_projections, 1 if force else 0, ctypes.byref(r))
    return st, r


def _ptr_array(items):
    arr = (ctypes.c_void_p * len(items))()
    for k, a in enumerate(items):
        p = _ptr(a)
        arr[k] = None if p is None else (p.value if isinstance(p, ctypes.c_void_p) else p)
    return arr


def asyrk_batch_create(handles, stream=None, graph=True, row_exclusion=0,
                       sampling=SAMPLE_WEIGHTED, update=UPDATE_ROW, engine=0, cluster_max=0,
                       workers=0, partition=True):
    b = ctypes.c_void_p()
    hs = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    o = BatchOpts(stream=_stream(stream), graph=0 if graph else -1, row_exclusion=row_exclusion,
                  sampling=sampling, update=update, engine=engine, cluster_max=cluster_max,
                  workers=workers,
                  partition=(partition if not isinstance(partition, bool) else (0 if partition else -1)))
    st = load().asyrk_batch_create(ctypes.byref(b), hs, len(handles), ctypes.byref(o))
    return st, b


def asyrk_batch_solve(b, xs, gammas=None, tols=None, max_sweeps=1000, x_trues=None,
                      device_ptrs=False):
    """xs updated in place; returns (status, [SolveInfo], BatchInfo)."""
    n = len(xs)
    xa = _ptr_array(xs)
    ga = None if gammas is None else np.ascontiguousarray(gammas, dtype=np.float64)
    ta = None if tols is None else np.ascontiguousarray(tols, dtype=np.float64)
    xt = None if x_trues is None else _ptr_array(x_trues)
    infos = (SolveInfo * n)()
    bi = BatchInfo()
    st = load().asyrk_batch_solve(b, xa, _ptr(ga), _ptr(ta), int(max_sweeps), xt,
                                  1 if device_ptrs else 0, infos, ctypes.byref(bi))
    return st, list(infos), bi


def asyrk_batch_destroy(b):
    load().asyrk_batch_destroy(b)


def asyrk_server_create(mem_budget_bytes, max_slots=0, row_exclusion=0, inner_tol=0.0,
                        max_inner_sweeps=0, onchip=True, admit_load=0.0, partition=0):
    h = ctypes.c_void_p()
    o = ServerOpts(mem_budget_bytes=int(mem_budget_bytes), max_slots=max_slots,
                   row_exclusion=row_exclusion, inner_tol=inner_tol,
                   max_inner_sweeps=max_inner_sweeps, onchip=0 if onchip else -1,
                   admit_load=float(admit_load), partition=int(partition))
    st = load().asyrk_server_create(ctypes.byref(h), ctypes.byref(o))
    return st, h


def asyrk_server_submit(sv, problem_h, x0=None, x_true=None, gamma=1.0, tol=1e-6,
                        mode=MODE_ASYNC, max_sweeps=1000):
    t = ctypes.c_uint64()
    x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
    xt = None if x_true is None else np.ascontiguousarray(x_true, dtype=np.float64)
    st = load().asyrk_server_submit(sv, problem_h, _ptr(x0), _ptr(xt), float(gamma), float(tol),
                                    mode, int(max_sweeps), ctypes.byref(t))
    return st, t.value


def asyrk_server_wait(sv, ticket, n, timeout_us=-1):
    """Returns (status, x (n doubles) or None on timeout, SolveInfo)."""
    x = np.zeros(n)
    info = SolveInfo()
    st = load().asyrk_server_wait(sv, ticket, _ptr(x), ctypes.byref(info), int(timeout_us))
    return st, (None if st == ETIMEOUT else x), info


def asyrk_server_cancel(sv, ticket):
    return load().asyrk_server_cancel(sv, ticket)


def asyrk_server_get_stats(sv):
    s = ServerStats()
    st = load().asyrk_server_get_stats(sv, ctypes.byref(s))
    return st, s


def asyrk_server_destroy(sv):
    load().asyrk_server_destroy(sv)


def asyrk_get_position(h):
    j = ctypes.c_uint64()
    st = load().asyrk_get_position(h, ctypes.byref(j))
    return st, j.value


def asyrk_set_position(h, j):
    return load().asyrk_set_position(h, j)


def asyrk_problem_get_stats(h):
    s = ProblemStats()
    st = load().asyrk_problem_get_stats(h, ctypes.byref(s))
    return st, s


# ---------------------------------------------------------------------------
# owner object
# ---------------------------------------------------------------------------
def solve_opts(mode=MODE_ASYNC, workers=0, subwarp=0, check_every=1, x_true=None, stream=None,
               inner_tol=0.0, inner_sweeps=0, profile=False, device_ptrs=False, row_exclusion=0,
               measure=MEASURE_AUTO, sampling=SAMPLE_WEIGHTED, update=UPDATE_ROW, graph_loop=False,
               kernel_form=0):
    return SolveOpts(mode=mode, device_ptrs=1 if device_ptrs else 0, workers=workers,
                     subwarp=subwarp, check_every=check_every, x_true=_ptr(x_true),
                     stream=_stream(stream), inner_tol=inner_tol, inner_sweeps=inner_sweeps,
                     profile=1 if profile else 0, row_exclusion=row_exclusion, measure=measure,
                     sampling=sampling, update=update, graph_loop=1 if graph_loop else 0,
                     kernel_form=kernel_form)


class Problem:
    """Owns one asyrk_problem handle."""

    def __init__(self, m, n, row_ptr, col_idx, values, vdtype, b, seed=0, device_ptrs=False,
                 stream=None):
        if isinstance(vdtype, str):
            vdtype = DTYPES[vdtype]
        st, h = asyrk_create(m, n, row_ptr, col_idx, values, vdtype, b, seed=seed,
                             device_ptrs=device_ptrs, stream=stream)
        if st != OK:
            raise AsyrkError(st, "asyrk_create")
        self.h = h
        self.m, self.n = m, n

    @classmethod
    def from_system(cls, s, seed=None, **kw):
        """From a ``synth.System`` (stored values as generated)."""
        from . import synth
        if seed is None:
            seed = synth.solver_seed(s.seed)
        return cls(s.m, s.n, s.row_ptr, s.col, s.val_store, DTYPES[s.value_dtype], s.b, seed=seed,
                   **kw)

    @classmethod
    def lsq(cls, m, n, row_ptr, col_idx, values, vdtype, b, zeta=0.0, phi=1.0, seed=0,
            device_ptrs=False, stream=None, lanczos_steps=0):
        """Section 6's square consistent system for min ||A x - b|| (A: m x n).

        zeta = 0 takes Section 6's sigma_r/sqrt(2) with sigma_r estimated on the GPU.
        The problem's iterate has n + m entries; ``lsq_solution`` maps it to x_LS."""
        if isinstance(vdtype, str):
            vdtype = DTYPES[vdtype]
        st, h = asyrk_lsq_create(m, n, row_ptr, col_idx, values, vdtype, b, zeta, phi=phi,
                                 seed=seed, device_ptrs=device_ptrs, stream=stream,
                                 lanczos_steps=lanczos_steps)
        if st != OK:
            raise AsyrkError(st, "asyrk_lsq_create")
        self = cls.__new__(cls)
        self.h = h
        st, stats = asyrk_problem_get_stats(h)
        self.m, self.n = stats.m, stats.n
        self.lsq_n = n
        return self

    def lsq_params(self):
        """(zeta as stored, phi) of a least-squares problem."""
        st, z, f = asyrk_lsq_params(self.h)
        if st != OK:
            raise AsyrkError(st, "asyrk_lsq_params")
        return z, f

    def lsq_solution(self, z, on_device=False):
        """x_LS from the iterate z of a least-squares problem (numpy or torch like z)."""
        if on_device:
            import torch
            x = torch.empty(self.lsq_n, dtype=torch.float64, device=z.device)
        else:
            x = np.empty(self.lsq_n, dtype=np.float64)
        st = asyrk_lsq_solution(self.h, z, x, on_device)
        if st != OK:
            raise AsyrkError(st, "asyrk_lsq_solution")
        return x

    def close(self):
        if self.h is not None and self.h.value:
            asyrk_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, x, gamma=1.0, tol=1e-8, max_sweeps=1000, raise_on_error=True, **kw):
        st, info = asyrk_solve(self.h, x, gamma, tol, max_sweeps, solve_opts(**kw))
        if st < 0 and raise_on_error:
            raise AsyrkError(st, "asyrk_solve")
        return st, info

    def residual(self, x, x_on_device=False):
        st, r = asyrk_residual(self.h, x, x_on_device)
        if st != OK:
            raise AsyrkError(st, "asyrk_residual")
        return r

    def normal_residual(self, x, x_on_device=False):
        """||A^T (A x - b)||^2 (Table 2's measure), FP64 on the GPU."""
        st, r = asyrk_normal_residual(self.h, x, x_on_device)
        if st != OK:
            raise AsyrkError(st, "asyrk_normal_residual")
        return r

    def draw_rows(self, j0, count, stream_id=0, sampling=SAMPLE_WEIGHTED):
        st, rows = asyrk_draw_rows(self.h, j0, count, stream_id, sampling)
        if st != OK:
            raise AsyrkError(st, "asyrk_draw_rows")
        return rows

    @property
    def position(self):
        return asyrk_get_position(self.h)[1]

    @position.setter
    def position(self, j):
        asyrk_set_position(self.h, j)

    def stats(self):
        return asyrk_problem_get_stats(self.h)[1].as_dict()

    def autotune(self, trial_projections=0, force=False):
        st, r = asyrk_autotune(self.h, trial_projections, force)
        if st != OK:
            raise AsyrkError(st, "asyrk_autotune")
        return r


class Batch:
    """Owns one asyrk_batch handle over a list of Problem objects.

    engine: ENGINE_AUTO (members that fit a CTA's shared memory on-chip, the rest in
    the global-iterate engine, both at once), ENGINE_GLOBAL or ENGINE_ONCHIP (every
    member on-chip, else EINVAL); cluster_max: CTAs per on-chip cluster at most
    (0: one); workers: on-chip workers per member at most (0: the Cor. 2 estimate);
    partition: with both engines at once, split the SMs between them (False: share).
    """

    def __init__(self, problems, stream=None, graph=True, row_exclusion=0,
                 sampling=SAMPLE_WEIGHTED, update=UPDATE_ROW, engine=0, cluster_max=0,
                 workers=0, partition=True):
        self.problems = list(problems)
        st, b = asyrk_batch_create([p.h for p in self.problems], stream=stream, graph=graph,
                                   row_exclusion=row_exclusion, sampling=sampling, update=update,
                                   engine=engine, cluster_max=cluster_max, workers=workers,
                                   partition=partition)
        if st != OK:
            raise AsyrkError(st, "asyrk_batch_create")
        self.b = b

    def solve(self, xs, gammas=None, tols=None, max_sweeps=1000, x_trues=None,
              device_ptrs=False, raise_on_error=True):
        st, infos, bi = asyrk_batch_solve(self.b, xs, gammas, tols, max_sweeps, x_trues,
                                          device_ptrs)
        if st < 0 and raise_on_error:
            raise AsyrkError(st, "asyrk_batch_solve")
        return st, infos, bi

    def close(self):
        if self.b is not None and self.b.value:
            asyrk_batch_destroy(self.b)
        self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Owns one asyrk_server (continuous batching of solve requests).

    onchip: requests whose problem fits a CTA's shared memory are solved on-chip,
    one CTA launch each, beside the shared engine step (False: all in the step).
    admit_load: the shared step admits queued requests in arrival order while the
    warp demands of those in the step add up to at most admit_load x the resident
    warps (0: 1.0; < 0: no limit).
    partition: SMs for the on-chip requests, the shared step on the others (0: 16;
    -1: no split, both on every SM).
    """

    def __init__(self, mem_budget_bytes, max_slots=0, row_exclusion=0, inner_tol=0.0,
                 max_inner_sweeps=0, onchip=True, admit_load=0.0, partition=0):
        st, h = asyrk_server_create(mem_budget_bytes, max_slots, row_exclusion, inner_tol,
                                    max_inner_sweeps, onchip, admit_load, partition)
        if st != OK:
            raise AsyrkError(st, "asyrk_server_create")
        self.h = h

    def submit(self, problem, x0=None, x_true=None, gamma=1.0, tol=1e-6, mode=MODE_ASYNC,
               max_sweeps=1000):
        st, t = asyrk_server_submit(self.h, problem.h, x0, x_true, gamma, tol, mode, max_sweeps)
        if st != OK:
            raise AsyrkError(st, "asyrk_server_submit")
        return t

    def wait(self, ticket, n, timeout_us=-1):
        return asyrk_server_wait(self.h, ticket, n, timeout_us)

    def cancel(self, ticket):
        return asyrk_server_cancel(self.h, ticket)

    def stats(self):
        return asyrk_server_get_stats(self.h)[1].as_dict()

    def close(self):
        if self.h is not None and self.h.value:
            asyrk_server_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
