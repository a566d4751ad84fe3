"""Round trips of the oracle: decode(encode(A)) == A (rows sorted by column,
values bit-identical) over every shape the format has to handle.  No GPU."""
import numpy as np
import pytest

import oracle as O
import workloads as WL


def _sorted_csr(A):
    cs, vs = O.sort_rows(A["row_ptr"], A["cols"], A["vals"])
    return A["row_ptr"], cs, vs


def _check(A, **kw):
    E = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], A["n"], **kw)
    rp, c, v = O.decode_matrix(E)
    rp0, c0, v0 = _sorted_csr(A)
    assert np.array_equal(rp, rp0)
    assert np.array_equal(c, c0)
    assert np.array_equal(O.value_keys(v), O.value_keys(v0))
    return E


def _mk(m, n, lens, rng, vals_fn, dtype=np.float64):
    rp = np.zeros(m + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    cols = np.concatenate([np.sort(rng.choice(n, size=L, replace=False)) for L in lens] or [np.zeros(0)])
    return dict(m=m, n=n, row_ptr=rp, cols=cols.astype(np.uint32), vals=vals_fn(int(rp[-1])).astype(dtype))


@pytest.mark.parametrize("L", [0, 1, 3, 4, 5, 8, 9, 31, 4097])
def test_row_lengths(L):
    rng = np.random.default_rng(L)
    m, n = 40, 5000
    lens = np.full(m, L)
    lens[::3] = rng.integers(0, L + 1, len(lens[::3]))
    A = _mk(m, n, lens, rng, lambda k: rng.choice([0.5, -2.0, 3.25], size=k))
    _check(A)


def test_empty_matrix_and_empty_rows():
    rng = np.random.default_rng(0)
    A = _mk(70, 10, np.zeros(70, np.int64), rng, lambda k: rng.uniform(size=k))
    E = _check(A)
    assert E.nwords == 70  # one n word per unit
    A = _mk(0, 10, np.zeros(0, np.int64), rng, lambda k: rng.uniform(size=k))
    E = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], 10)
    assert E.nwords == 0 and E.nslices == 0


def test_single_symbol_domains():
    rng = np.random.default_rng(1)
    m = 33
    rp = np.arange(0, 7 * m + 1, 7)
    cols = np.tile(np.arange(0, 14, 2), m).astype(np.uint32)  # deltas: 0 then 2s
    A = dict(m=m, n=14, row_ptr=rp, cols=cols, vals=np.full(7 * m, 1.5))
    E = _check(A)
    assert E.tabV.nkept == 1 and not E.tabV.has_esc
    assert E.tabV.multiplicities()[O.value_keys(np.array([1.5]))[0]] == 256


def test_many_symbols_force_escapes():
    """More than K distinct values and columns: escapes in both domains."""
    rng = np.random.default_rng(2)
    A = WL.random_csr(2, 600, 200000, 12.0)  # continuous values: ~7200 distinct
    E = _check(A)
    assert E.tabV.has_esc and E.tabD.has_esc
    assert E.unit_raw.sum() > 0


def test_all_escape_domain():
    """Every value distinct and rare: the table may keep nothing (ESC only)."""
    rng = np.random.default_rng(3)
    A = WL.random_csr(3, 50, 100, 3.0)
    E = _check(A)
    if E.tabV.nkept == 0:
        assert E.tabV.pad_esc


def test_special_values_bit_preserved():
    rng = np.random.default_rng(4)
    specials = np.array([0.0, -0.0, np.nan, -np.inf, np.inf, 5e-324, np.float64(np.nan) * -1], np.float64)
    bits = specials.view(np.uint64).copy()
    bits[2] = np.uint64(0x7FF8DEADBEEF0001)  # NaN payload
    specials = bits.view(np.float64)
    A = WL.random_csr(4, 64, 64, 6.0)
    A["vals"] = specials[rng.integers(0, len(specials), len(A["vals"]))]
    _check(A)
    A32 = WL.random_csr(5, 64, 64, 6.0, dtype=np.float32)
    s32 = np.array([0.0, -0.0, np.nan, np.inf, -np.inf, 1e-45], np.float32)
    A32["vals"] = s32[rng.integers(0, len(s32), len(A32["vals"]))]
    _check(A32)


def test_duplicates_and_unsorted_columns():
    rng = np.random.default_rng(6)
    m, n = 20, 50
    lens = rng.integers(0, 12, m)
    rp = np.zeros(m + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    cols = rng.integers(0, n, int(rp[-1])).astype(np.uint32)  # unsorted, with duplicates
    vals = rng.uniform(-1, 1, int(rp[-1]))
    A = dict(m=m, n=n, row_ptr=rp, cols=cols, vals=vals)
    _check(A)


@pytest.mark.parametrize("gen", ["pr1", "stencil", "powerlaw", "pruned", "f32"])
def test_workload_constructions(gen):
    if gen == "pr1":
        A = WL.pr1(seed=0, n=1024)
    elif gen == "stencil":
        A = WL.stencil27(grid=6)
    elif gen == "powerlaw":
        A = WL.power_law(rows=3000, seed=2)
    elif gen == "pruned":
        A = WL.pruned_linear(dim=256, batch=4)
    else:
        A = WL.random_csr(8, 500, 700, 9.0, nvals=40, dtype=np.float32)
    _check(A)


@pytest.mark.parametrize("U,order", [(4, 0), (4, 1), (7, 1), (32, 1), (1, 0), (0, 1)])
def test_split_units_layout(U, order):
    A = WL.power_law(rows=1500, seed=11, max_len=300)
    E = _check(A, unit_max_nnz=U, row_order=order)
    assert (E.unit_len <= U).all() or U == 0
    # units cover every row exactly once, in row order within a row
    cov = np.zeros(A["m"], np.int64)
    np.add.at(cov, E.unit_row, E.unit_len)
    assert np.array_equal(cov, np.diff(A["row_ptr"]))
    if order == 1:
        lens = np.diff(A["row_ptr"])
        ul = np.array([int(lens[r]) if U == 0 else -(-int(lens[r]) // max(1, -(-int(lens[r]) // U)))
                       for r in E.unit_row])
        first = np.r_[True, E.unit_row[1:] != E.unit_row[:-1]]
        assert (np.diff(ul[first]) <= 0).all()


@pytest.mark.parametrize("U,window", [(0, 64), (8, 100), (32, 1), (16, 5000), (4, 333)])
def test_windowed_order_layout(U, window):
    """row_order = 1 within blocks of `window` rows: the units' rows, read in
    stream order, are each block's rows sorted by (longest unit descending,
    row), blocks in natural order -- rebuilt here by brute force."""
    A = WL.power_law(rows=1200, seed=13, max_len=200)
    E = _check(A, unit_max_nnz=U, row_order=1, order_window=window)
    lens = np.diff(A["row_ptr"])

    def longest(L):
        return L if U == 0 or L <= U else -(-L // (-(-L // U)))

    want = []
    for b in range(0, A["m"], window):
        rows = range(b, min(A["m"], b + window))
        want += sorted(rows, key=lambda r: (-longest(int(lens[r])), r))
    first = np.r_[True, E.unit_row[1:] != E.unit_row[:-1]]
    assert E.unit_row[first].tolist() == want
    ur, _, ul = O.layout(A["row_ptr"], U, 1, window)
    assert np.array_equal(ur, E.unit_row) and np.array_equal(ul, E.unit_len)
    if window >= A["m"]:  # one block: the same layout as the global order
        ur0, _, _ = O.layout(A["row_ptr"], U, 1, 0)
        assert np.array_equal(ur0, ur)


@pytest.mark.parametrize("sw", [1, 5, 32])
def test_slice_widths(sw):
    A = WL.pr1(seed=3, n=300)
    _check(A, slice_width=sw)


def test_slot_permutation_round_trip():
    A = WL.pr1(seed=4, n=800)
    E0 = _check(A)
    E1 = _check(A, perm_seeds=(12345, 678))
    assert E1.permD is not None and not np.array_equal(E1.words, E0.words)
    assert E1.nwords == E0.nwords  # permuting slots moves digits, not sizes


def test_corrupt_stream_is_rejected():
    A = WL.pr1(seed=5, n=256)
    E = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], A["n"])
    with pytest.raises(RuntimeError):
        O.decode_units(E, words=E.words[:-1], slice_off=np.minimum(E.slice_off, len(E.words) - 1))


@pytest.mark.parametrize("gen", ["pr1", "stencil", "powerlaw_split", "escapes", "empty_rows", "f32"])
def test_row_relative_first_delta_round_trip(gen):
    """first_delta = 1 (first delta = column - row, modulo 2^32): the decoder
    that starts each unit's running column at its row recovers the matrix;
    columns below the row (negative first deltas) and split, reordered units
    (each unit relative to its own row) included."""
    kw = dict(first_delta=1)
    if gen == "pr1":
        A = WL.pr1(seed=0, n=1024)
    elif gen == "stencil":
        A = WL.stencil27(grid=6)
    elif gen == "powerlaw_split":
        A = WL.power_law(rows=3000, seed=2, max_len=300)
        kw.update(unit_max_nnz=8, row_order=1)
    elif gen == "escapes":
        A = WL.random_csr(2, 500, 100000, 12.0)
    elif gen == "empty_rows":
        A = WL.random_csr(9, 333, 50, 2.0, empty_frac=0.5)
    else:
        A = WL.random_csr(8, 500, 700, 9.0, nvals=40, dtype=np.float32)
    _check(A, **kw)


@pytest.mark.parametrize("chain", [2, 3, 8, 64])
@pytest.mark.parametrize("gen", ["pr1", "stencil", "powerlaw_split", "escapes", "empty_rows", "ragged", "f32"])
def test_chained_units_round_trip(chain, gen):
    """Chains of units (each lane's units of `chain` consecutive slices as one
    dtANS sequence): decode(encode(A)) == A, also with row-relative first
    deltas, split and reordered units, empty units inside and at the end of a
    lane's chain, and a final slice with fewer than 32 units."""
    kw = dict(chain=chain)
    if gen == "pr1":
        A = WL.pr1(seed=0, n=1024)
        kw["first_delta"] = 1
    elif gen == "stencil":
        A = WL.stencil27(grid=6)
    elif gen == "powerlaw_split":
        A = WL.power_law(rows=3000, seed=2, max_len=300)
        kw.update(unit_max_nnz=8, row_order=1)
    elif gen == "escapes":
        A = WL.random_csr(2, 500, 100000, 12.0)
    elif gen == "empty_rows":
        A = WL.random_csr(9, 333, 50, 2.0, empty_frac=0.5)
    elif gen == "ragged":
        A = WL.random_csr(10, 32 * 7 + 5, 900, 30.0, nvals=6)
    else:
        A = WL.random_csr(8, 500, 700, 9.0, nvals=40, dtype=np.float32)
    _check(A, **kw)


@pytest.mark.parametrize("chain", [1, 4])
@pytest.mark.parametrize("gen", ["pr1", "escapes", "special", "powerlaw_split"])
def test_separate_escape_stream_round_trip(chain, gen):
    """Escaped raw words in their own array (Sec. IV-F's alternative): the main
    stream loses exactly the raw words, which the escape array holds slice by
    slice, and decode(encode(A)) == A."""
    kw = dict(chain=chain)
    if gen == "pr1":
        A = WL.pr1(seed=0, n=1024)
    elif gen == "escapes":
        A = WL.random_csr(2, 500, 100000, 12.0)
    elif gen == "special":
        A = WL.random_csr(4, 640, 64, 6.0)
        bits = np.array([0, 0x8000000000000000, 0x7FF8DEADBEEF0001, 0xFFF0000000000000, 1], np.uint64)
        A["vals"] = bits[np.random.default_rng(0).integers(0, len(bits), len(A["vals"]))].view(np.float64)
    else:
        A = WL.power_law(rows=3000, seed=2, max_len=300)
        kw.update(unit_max_nnz=8, row_order=1)
    E0 = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], A["n"], **kw)
    E = _check(A, escape_stream=1, **kw)
    assert len(E0.esc_words) == 0
    assert E.nwords + len(E.esc_words) == E0.nwords
    assert len(E.esc_words) == int(E0.unit_raw.sum())
    assert E.esc_off[-1] == len(E.esc_words) and (np.diff(E.esc_off) >= 0).all()
