"""Seeded synthetic sparse systems shaped like the AsyRK paper's experiments.

Section 5 of the paper builds A by choosing delta*m*n random positions, filling
them with N(0,1) values and normalizing the rows.  This module generates such
systems (with a fixed number of distinct, uniformly random columns per row),
picks x* ~ N(0,1) and sets b = A x* in FP64 from the values as stored, so that
A x = b is consistent in FP64 for the stored matrix.

This module is the only code that both the CUDA path (through its callers) and
the CPU oracle receive inputs from.  It holds none of the method's arithmetic:
no row sampling, no projection, no error measure.

Value storage:
  * ``"f64"``  values kept in FP64;
  * ``"f32"``  values rounded to FP32 (round to nearest even);
  * ``"bf16"`` values rounded from FP64 straight to BF16 (round to nearest
    even, no double rounding); ``val_store`` then holds the 16-bit patterns.
``val64`` always holds the exact stored values widened to FP64, which is the
matrix both sides solve.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

VALUE_DTYPES = ("f64", "f32", "bf16")


@dataclass
class System:
    m: int
    n: int
    row_ptr: np.ndarray          # int64, m+1
    col: np.ndarray              # int32, nnz, strictly ascending within a row
    val_store: np.ndarray        # float64 / float32 / uint16 (bf16 bits)
    value_dtype: str
    x_true: np.ndarray           # float64, n
    b: np.ndarray                # float64, m  (= A x* in FP64)
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def val64(self) -> np.ndarray:
        return stored_to_f64(self.val_store, self.value_dtype)


def solver_seed(gen_seed: int) -> int:
    """Philox key used for a system generated with ``gen_seed``."""
    return int(gen_seed) ^ 0x5EED


def config_seed(config_id: int, rep: int = 0) -> int:
    return 1234 + 1000 * int(config_id) + int(rep)


# ---------------------------------------------------------------------------
# value rounding
# ---------------------------------------------------------------------------
def f64_to_bf16_bits(v: np.ndarray) -> np.ndarray:
    """Round FP64 to BF16 (nearest, ties to even) in one step; 16-bit patterns."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    bits = v.view(np.uint64)
    drop = np.uint64(45)  # 52 - 7 mantissa bits
    lsb = (bits >> drop) & np.uint64(1)
    rounded = (bits + (np.uint64((1 << 44) - 1) + lsb)) & ~np.uint64((1 << 45) - 1)
    as32 = rounded.view(np.float64).astype(np.float32)  # exact: 8 significant bits
    return (as32.view(np.uint32) >> np.uint32(16)).astype(np.uint16)


def bf16_bits_to_f64(h: np.ndarray) -> np.ndarray:
    u = (np.asarray(h, dtype=np.uint16).astype(np.uint32) << np.uint32(16))
    return u.view(np.float32).astype(np.float64)


def stored_to_f64(val_store: np.ndarray, value_dtype: str) -> np.ndarray:
    if value_dtype == "f64":
        return np.asarray(val_store, dtype=np.float64)
    if value_dtype == "f32":
        return np.asarray(val_store, dtype=np.float32).astype(np.float64)
    if value_dtype == "bf16":
        return bf16_bits_to_f64(val_store)
    raise ValueError(value_dtype)


def _store(v64: np.ndarray, value_dtype: str) -> np.ndarray:
    if value_dtype == "f64":
        return np.ascontiguousarray(v64, dtype=np.float64)
    if value_dtype == "f32":
        return np.ascontiguousarray(v64.astype(np.float32))
    if value_dtype == "bf16":
        return f64_to_bf16_bits(v64)
    raise ValueError(value_dtype)


# ---------------------------------------------------------------------------
# structure
# ---------------------------------------------------------------------------
def _distinct_sorted_columns(rng: np.random.Generator, m: int, n: int, L: int) -> np.ndarray:
    """(m, L) int32, each row L distinct columns drawn uniformly, ascending."""
    if L > n:
        raise ValueError("row length exceeds n")
    if 4 * L > n:  # dense rows: sample without replacement directly
        out = np.empty((m, L), dtype=np.int32)
        for i in range(m):
            out[i] = np.sort(rng.choice(n, size=L, replace=False))
        return out
    cols = rng.integers(0, n, size=(m, L), dtype=np.int32)
    cols.sort(axis=1)
    while True:
        bad = np.nonzero((np.diff(cols, axis=1) == 0).any(axis=1))[0]
        if bad.size == 0:
            return cols
        redo = rng.integers(0, n, size=(bad.size, L), dtype=np.int32)
        redo.sort(axis=1)
        cols[bad] = redo


def make_system(m: int, n: int, nnz_per_row, seed: int, *, row_norms: str = "unit",
                value_dtype: str = "f64", x_true=None) -> System:
    """Random sparse consistent system.

    ``nnz_per_row``: an int (every row), a (lo, hi) pair (each row's length
    drawn uniformly in [lo, hi]) or ("poisson", mean): each row's length drawn
    from Poisson(mean), at least 1 -- the row counts of Section 5's generator,
    which places delta*m*n nonzeros at random positions (mean = delta*n).  ``row_norms``: ``"unit"`` (rows normalized,
    Section 5) or ``"lognormal"`` (row 2-norms exp(N(0,1)), so rows are not
    equally likely).
    """
    if value_dtype not in VALUE_DTYPES:
        raise ValueError(value_dtype)
    rng = np.random.default_rng(seed)
    if np.isscalar(nnz_per_row):
        L = int(nnz_per_row)
        cols = _distinct_sorted_columns(rng, m, n, L)
        lengths = np.full(m, L, dtype=np.int64)
        col = cols.reshape(-1)
        del cols
    else:
        if nnz_per_row[0] == "poisson":
            lengths = np.clip(rng.poisson(float(nnz_per_row[1]), size=m), 1, n).astype(np.int64)
        else:
            lo, hi = int(nnz_per_row[0]), int(nnz_per_row[1])
            lengths = rng.integers(lo, hi + 1, size=m).astype(np.int64)
        parts = []
        for L in np.unique(lengths):
            idx = np.nonzero(lengths == L)[0]
            parts.append((idx, _distinct_sorted_columns(rng, idx.size, n, int(L))))
        row_ptr_tmp = np.zeros(m + 1, dtype=np.int64)
        np.cumsum(lengths, out=row_ptr_tmp[1:])
        col = np.empty(int(row_ptr_tmp[-1]), dtype=np.int32)
        for idx, c in parts:
            L = c.shape[1]
            pos = row_ptr_tmp[idx][:, None] + np.arange(L)[None, :]
            col[pos.reshape(-1)] = c.reshape(-1)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lengths, out=row_ptr[1:])
    nnz = int(row_ptr[-1])

    v = rng.standard_normal(nnz)
    row_id = np.repeat(np.arange(m, dtype=np.int64), lengths)
    ss = np.bincount(row_id, weights=v * v, minlength=m)
    scale = 1.0 / np.sqrt(ss)
    if row_norms == "lognormal":
        scale = scale * np.exp(rng.standard_normal(m))
    elif row_norms != "unit":
        raise ValueError(row_norms)
    v *= scale[row_id]
    del row_id
    val_store = _store(v, value_dtype)
    del v
    val64 = stored_to_f64(val_store, value_dtype)

    if x_true is None:
        x_true = rng.standard_normal(n)
    x_true = np.ascontiguousarray(x_true, dtype=np.float64)
    b = spmv_f64(m, row_ptr, col, val64, x_true)
    return System(m=m, n=n, row_ptr=row_ptr, col=col, val_store=val_store,
                  value_dtype=value_dtype, x_true=x_true, b=b, seed=int(seed),
                  meta={"nnz_per_row": nnz_per_row, "row_norms": row_norms})


def spmv_f64(m, row_ptr, col, val64, x) -> np.ndarray:
    """A x in FP64 (used only to construct b = A x*)."""
    prod = val64 * x[col]
    out = np.add.reduceat(prod, row_ptr[:-1]) if prod.size else np.zeros(m)
    return np.ascontiguousarray(out, dtype=np.float64)


# ---------------------------------------------------------------------------
# the five workloads (sizes as stated; ``scale`` shrinks the large ones for tests)
# ---------------------------------------------------------------------------
def plain_f64_system(rep: int = 0, m: int = 4096, n: int = 1024, L: int = 16) -> System:
    """m=4096, n=1024, 16 nnz/row, N(0,1), unit rows, FP64 values."""
    return make_system(m, n, L, config_seed(1, rep), row_norms="unit", value_dtype="f64")


def large_async_system(rep: int = 0, m: int = 1 << 22, n: int = 1 << 20, L: int = 32) -> System:
    """m=2^22, n=2^20, 32 nnz/row, N(0,1), row norms lognormal(0,1), FP32 values."""
    return make_system(m, n, L, config_seed(2, rep), row_norms="lognormal", value_dtype="f32")


def bf16_refine_system(rep: int = 0, m: int = 4096, n: int = 1024, L: int = 16) -> System:
    """Plain-system shape, unit rows, values rounded to BF16 (the BF16 matrix is A)."""
    return make_system(m, n, L, config_seed(3, rep), row_norms="unit", value_dtype="bf16")


def batch_shapes(count: int = 256, seed: int = None, m_lo_log2: int = 11, m_hi_log2: int = 18,
                 nnz_lo: int = 8, nnz_hi: int = 64):
    """(m, n, nnz_per_row) per system: m = floor(2^U(lo,hi)), n = m/4,
    nnz/row uniform in [nnz_lo, nnz_hi] per system."""
    rng = np.random.default_rng(config_seed(4) if seed is None else seed)
    e = rng.uniform(m_lo_log2, m_hi_log2, size=count)
    ms = np.floor(2.0 ** e).astype(np.int64)
    Ls = rng.integers(nnz_lo, nnz_hi + 1, size=count)
    return [(int(mm), int(mm // 4), int(L)) for mm, L in zip(ms, Ls)]


def batch_systems(count: int = 256, rep: int = 0, value_dtype: str = "f32", **shape_kw):
    shapes = batch_shapes(count, **shape_kw)
    base = config_seed(4, rep) * 1000
    return [make_system(m, n, L, base + k, row_norms="unit", value_dtype=value_dtype)
            for k, (m, n, L) in enumerate(shapes)]


# ---------------------------------------------------------------------------
# the same construction on the GPU (for benchmark inputs too large to build
# quickly on the host); seeded with a torch generator, so it reproduces itself
# but not the numpy systems above
# ---------------------------------------------------------------------------
def make_system_torch(m: int, n: int, L, seed: int, *, row_norms: str = "unit",
                      value_dtype: str = "f32", device: str = "cuda"):
    """Dict of device tensors: row_ptr (int64), col (int32), val_store (float64 /
    float32 / int16 BF16 bits), x_true and b (float64); L distinct uniformly
    random columns per row (ascending) -- L an int, or ("poisson", mean) for
    Poisson(mean) row lengths (at least 1) --, N(0,1) values, rows normalized (or
    lognormal(0,1) norms), rounded to the storage type, b = A x* in FP64 from
    the stored values."""
    import torch
    if value_dtype not in VALUE_DTYPES:
        raise ValueError(value_dtype)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    if isinstance(L, (tuple, list)):
        if L[0] != "poisson":
            raise ValueError(L)
        lengths = torch.poisson(torch.full((m,), float(L[1]), device=device, dtype=torch.float64),
                                generator=g).clamp(1, n).to(torch.int64)
    else:
        lengths = torch.full((m,), int(L), device=device, dtype=torch.int64)
    Lmax = int(lengths.max().item())
    if Lmax > n:
        raise ValueError("row length exceeds n")
    cols = torch.randint(0, n, (m, Lmax), generator=g, device=device, dtype=torch.int64)
    srt = torch.sort(cols, dim=1)[0]
    for _ in range(1000):
        bad = (srt[:, 1:] == srt[:, :-1]).any(dim=1).nonzero().flatten()
        if bad.numel() == 0:
            break
        cols[bad] = torch.randint(0, n, (bad.numel(), Lmax), generator=g, device=device,
                                  dtype=torch.int64)
        srt[bad] = torch.sort(cols[bad], dim=1)[0]
    else:
        raise RuntimeError("could not draw distinct columns")
    # each row keeps its first L_i draws (a uniform subset), ascending; the rest
    # become a sentinel that sorts last
    keep = torch.arange(Lmax, device=device)[None, :] < lengths[:, None]
    cols = torch.where(keep, cols, torch.full_like(cols, n))
    cols, order = torch.sort(cols, dim=1)
    keep = cols < n
    v = torch.randn((m, Lmax), generator=g, device=device, dtype=torch.float64) * keep
    scale = 1.0 / torch.sqrt((v * v).sum(dim=1, keepdim=True))
    if row_norms == "lognormal":
        scale = scale * torch.exp(torch.randn((m, 1), generator=g, device=device,
                                              dtype=torch.float64))
    elif row_norms != "unit":
        raise ValueError(row_norms)
    v = v * scale
    if value_dtype == "f64":
        store, v64 = v, v
    elif value_dtype == "f32":
        store = v.to(torch.float32)
        v64 = store.to(torch.float64)
    else:
        store32 = v.to(torch.bfloat16)  # round to nearest even from FP64
        v64 = store32.to(torch.float64)
        store = store32.view(torch.int16)
    x_true = torch.randn(n, generator=g, device=device, dtype=torch.float64)
    b = (v64 * x_true[cols.clamp(max=n - 1)]).sum(dim=1)
    row_ptr = torch.zeros(m + 1, device=device, dtype=torch.int64)
    row_ptr[1:] = torch.cumsum(lengths, 0)
    return {"m": m, "n": n, "L": L, "row_ptr": row_ptr, "col": cols[keep].to(torch.int32),
            "val_store": store[keep].contiguous(), "x_true": x_true, "b": b,
            "value_dtype": value_dtype, "seed": int(seed)}
