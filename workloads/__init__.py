"""Seeded synthetic inputs for CSR-dtANS (shared by tests, bench.py and the oracle).

This module holds input generators only: it contains none of the method's
arithmetic (no coding tables, no encoding, no products).  Every generator
returns plain CSR arrays (row_ptr int64, cols uint32 sorted ascending within
each row and distinct, vals float64/float32) and dense right-hand sides;
``unsorted_duplicates`` turns such a matrix into one whose rows are in random
column order and hold repeated columns.

The five workloads stand in for the SuiteSparse matrices the paper measures
on (Sec. V), with the shapes, sizes and value distributions listed with each
function.  Small ``scale`` arguments give the same construction at sizes the
CPU oracle finishes in seconds.
"""
from __future__ import annotations

import numpy as np


def _csr_from_rows(m: int, rows: np.ndarray, cols: np.ndarray, n: int):
    """Builds sorted, duplicate-free CSR from (row, col) pairs (int64)."""
    key = np.sort(rows.astype(np.int64) * np.int64(n) + cols.astype(np.int64))
    if len(key) > 1:  # sorted distinct keys (a sort + mask; np.unique is far slower here on 10^8 keys)
        keep = np.empty(len(key), bool)
        keep[0] = True
        np.not_equal(key[1:], key[:-1], out=keep[1:])
        key = key[keep]
    r = key // n
    c = (key % n).astype(np.uint32)
    counts = np.bincount(r, minlength=m)
    row_ptr = np.zeros(m + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, c


def _zipf_probs(k: int, s: float) -> np.ndarray:
    w = 1.0 / np.arange(1, k + 1, dtype=np.float64) ** s
    return w / w.sum()


def pr1(seed: int = 0, n: int = 4096, mean_len: float = 10.0, band: int = 512, nvals: int = 16,
        zipf_s: float = 1.2):
    """Square n x n, row lengths Poisson(mean_len), distinct columns uniform in
    [i - band, i + band] clipped to [0, n), FP64 values from `nvals` constants
    (uniform in [-1, 1]) with Zipf(s) frequencies over their rank; x ~ U[-1, 1]."""
    rng = np.random.default_rng(seed)
    lens = rng.poisson(mean_len, n)
    rows, cols = [], []
    for i in range(n):
        lo, hi = max(0, i - band), min(n - 1, i + band)
        L = min(int(lens[i]), hi - lo + 1)
        c = rng.choice(hi - lo + 1, size=L, replace=False) + lo
        rows.append(np.full(L, i, np.int64))
        cols.append(c.astype(np.int64))
    rows = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    cols = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    row_ptr, c = _csr_from_rows(n, rows, cols, n)
    consts = rng.uniform(-1.0, 1.0, nvals)
    vals = consts[rng.choice(nvals, size=len(c), p=_zipf_probs(nvals, zipf_s))]
    x = rng.uniform(-1.0, 1.0, n)
    return dict(name=f"pr1_n{n}", m=n, n=n, row_ptr=row_ptr, cols=c, vals=vals.astype(np.float64), x=x)


def stencil27(grid: int = 128, seed: int = 1):
    """27-point 3-D stencil on a periodic grid^3 (every row has 27 entries):
    26 on the diagonal and -1 elsewhere, FP64; x ~ U[-1, 1]."""
    g = grid
    m = g * g * g
    idx = np.arange(m, dtype=np.int64)
    z, y, xx = idx // (g * g), (idx // g) % g, idx % g
    offs = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    cols = np.empty((m, len(offs)), np.int64)
    for t, (dz, dy, dx) in enumerate(offs):
        cols[:, t] = (((z + dz) % g) * g + ((y + dy) % g)) * g + ((xx + dx) % g)
    if g < 3:  # wrap-around aliases: keep distinct columns only
        rows = np.repeat(idx, len(offs))
        row_ptr, c = _csr_from_rows(m, rows, cols.reshape(-1), m)
    else:
        cols.sort(axis=1)
        c = cols.reshape(-1).astype(np.uint32)
        row_ptr = np.arange(0, 27 * m + 1, 27, dtype=np.int64)
    rows_of = np.repeat(np.arange(m, dtype=np.int64), np.diff(row_ptr))
    vals = np.where(c.astype(np.int64) == rows_of, 26.0, -1.0)
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1.0, 1.0, m)
    return dict(name=f"stencil27_{g}^3", m=m, n=m, row_ptr=row_ptr, cols=c, vals=vals, x=x)


def power_law(rows: int = 4_194_304, seed: int = 2, mu: float = 2.5, sigma: float = 1.0, max_len: int = 4096,
              near: int = 2048, near_frac: float = 0.7, levels: int = 256):
    """Square, row lengths round(exp(N(mu, sigma))) clipped to [1, max_len];
    columns 70% uniform within +-near of the diagonal (clipped) and 30% uniform
    in [0, n), duplicates removed; FP32 values N(0, 1) quantised to `levels`
    levels of step 1/32 (clamped to [-4, 4)); x ~ U[-1, 1] FP32."""
    rng = np.random.default_rng(seed)
    n = rows
    lens = np.clip(np.rint(np.exp(rng.normal(mu, sigma, n))), 1, max_len).astype(np.int64)
    total = int(lens.sum())
    r = np.repeat(np.arange(n, dtype=np.int64), lens)
    is_near = rng.random(total) < near_frac
    c = np.empty(total, np.int64)
    nn = int(is_near.sum())
    c[is_near] = np.clip(r[is_near] + rng.integers(-near, near + 1, nn), 0, n - 1)
    c[~is_near] = rng.integers(0, n, total - nn)
    del is_near
    row_ptr, cols = _csr_from_rows(n, r, c, n)
    del r, c
    half = levels // 2
    q = np.clip(np.rint(rng.normal(0.0, 1.0, len(cols)) * 32.0), -half, half - 1)
    vals = (q / 32.0).astype(np.float32)
    x = rng.uniform(-1.0, 1.0, n).astype(np.float32)
    return dict(name=f"power_law_{n}", m=n, n=n, row_ptr=row_ptr, cols=cols, vals=vals, x=x)


def random_uniform(rows: int, rng: np.random.Generator, mean_len: float, consts: np.ndarray, zipf_s: float,
                   dtype=np.float64):
    """Square, Poisson(mean_len) row lengths, distinct uniform columns, values
    drawn from `consts` with Zipf(s) frequencies."""
    n = rows
    lens = rng.poisson(mean_len, n).astype(np.int64)
    total = int(lens.sum())
    r = np.repeat(np.arange(n, dtype=np.int64), lens)
    c = rng.integers(0, n, total)
    row_ptr, cols = _csr_from_rows(n, r, c, n)
    vals = consts[rng.choice(len(consts), size=len(cols), p=_zipf_probs(len(consts), zipf_s))].astype(dtype)
    return dict(m=n, n=n, row_ptr=row_ptr, cols=cols, vals=vals)


def batched(seed: int = 3, count: int = 64, lo_log2: int = 12, hi_log2: int = 18, mean_len: float = 16.0,
            nvals: int = 64, zipf_s: float = 1.0):
    """`count` independent square matrices with rows log-uniform in
    [2^lo, 2^hi], Poisson(16) row lengths, distinct uniform columns, FP64 values
    from 64 constants (uniform in [-1, 1]) with Zipf(1.0) frequencies."""
    rng = np.random.default_rng(seed)
    consts = rng.uniform(-1.0, 1.0, nvals)
    sizes = np.rint(2.0 ** rng.uniform(lo_log2, hi_log2, count)).astype(np.int64)
    mats = []
    for t, sz in enumerate(sizes):
        A = random_uniform(int(sz), rng, mean_len, consts, zipf_s)
        A["x"] = rng.uniform(-1.0, 1.0, int(sz))
        A["name"] = f"batch{t}_{sz}"
        mats.append(A)
    return mats


def multi_rhs(seed: int = 3, rows: int = 1 << 20, k: int = 8, mean_len: float = 16.0, nvals: int = 64,
              zipf_s: float = 1.0):
    """One 2^20-row matrix of the batched kind with k right-hand sides
    (row-major n x k, FP64, U[-1, 1])."""
    rng = np.random.default_rng(seed + 1000)
    consts = rng.uniform(-1.0, 1.0, nvals)
    A = random_uniform(rows, rng, mean_len, consts, zipf_s)
    A["X"] = rng.uniform(-1.0, 1.0, (rows, k))
    A["name"] = f"multi_rhs_{rows}_k{k}"
    return A


def pruned_linear(seed: int = 4, dim: int = 8192, density: float = 0.1, codebook: int = 16, sd: float = 0.02,
                  batch: int = 32, dtype=np.float32):
    """dim x dim, each entry kept with probability `density` (unstructured),
    values from a `codebook`-entry codebook drawn from N(0, sd^2) with uniform
    assignment; X and G are dim x batch, N(0, 1)."""
    rng = np.random.default_rng(seed)
    total = int(rng.binomial(dim * dim, density))
    flat = rng.choice(dim * dim, size=total, replace=False)
    flat.sort()
    r, c = flat // dim, flat % dim
    counts = np.bincount(r, minlength=dim)
    row_ptr = np.zeros(dim + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    cb = rng.normal(0.0, sd, codebook).astype(dtype)
    vals = cb[rng.integers(0, codebook, total)]
    X = rng.normal(0.0, 1.0, (dim, batch)).astype(dtype)
    G = rng.normal(0.0, 1.0, (dim, batch)).astype(dtype)
    return dict(name=f"pruned_{dim}_b{batch}", m=dim, n=dim, row_ptr=row_ptr, cols=c.astype(np.uint32),
                vals=vals, X=X, G=G, codebook=cb)


def random_csr(seed: int, m: int, n: int, mean_len: float, nvals: int | None = None, dtype=np.float64,
               empty_frac: float = 0.0, max_len: int | None = None, integer_valued: bool = False):
    """General small test matrices: Poisson row lengths (optionally some empty
    rows), distinct uniform columns, values either continuous U[-1, 1], from
    `nvals` constants, or small integers."""
    rng = np.random.default_rng(seed)
    lens = rng.poisson(mean_len, m).astype(np.int64)
    if empty_frac > 0:
        lens[rng.random(m) < empty_frac] = 0
    lens = np.minimum(lens, n if max_len is None else min(n, max_len))
    total = int(lens.sum())
    r = np.repeat(np.arange(m, dtype=np.int64), lens)
    c = rng.integers(0, n, total)
    row_ptr, cols = _csr_from_rows(m, r, c, n)
    nz = len(cols)
    if integer_valued:
        vals = rng.integers(-8, 9, nz).astype(dtype)
    elif nvals:
        vals = rng.uniform(-1, 1, nvals).astype(dtype)[rng.integers(0, nvals, nz)]
    else:
        vals = rng.uniform(-1, 1, nz).astype(dtype)
    return dict(name=f"rand_{m}x{n}", m=m, n=n, row_ptr=row_ptr, cols=cols, vals=vals)


def unsorted_duplicates(A: dict, seed: int, dup_frac: float = 0.15):
    """The matrix A with about dup_frac * nnz extra entries that repeat a
    column of their row (each with a value drawn from A's values, so a
    repeated column may carry a different value), and every row's entries in
    random order.  The result is valid CSR input that is neither sorted nor
    duplicate-free; x and the other keys of A are kept."""
    rng = np.random.default_rng(seed)
    rp = np.asarray(A["row_ptr"], np.int64)
    m = len(rp) - 1
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(rp))
    cols = np.asarray(A["cols"]).astype(np.int64)
    vals = np.asarray(A["vals"])
    nz = len(cols)
    nd = int(rng.binomial(nz, dup_frac)) if nz else 0
    pick = rng.integers(0, nz, nd) if nd else np.zeros(0, np.int64)
    rows = np.concatenate([rows, rows[pick]])
    cols = np.concatenate([cols, cols[pick]])
    dv = vals[rng.integers(0, nz, nd)] if nd else vals[:0]
    vals = np.concatenate([vals, dv])
    order = np.lexsort((rng.random(len(rows)), rows))  # by row, random order within a row
    out = dict(A)
    out["row_ptr"] = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=m))]).astype(np.int64)
    out["cols"] = cols[order].astype(np.uint32)
    out["vals"] = vals[order]
    out["name"] = A.get("name", "matrix") + "_unsorted_dups"
    return out
