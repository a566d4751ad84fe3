"""Pins of the CPU oracle against what the paper and the mathematics fix.

Worked examples (Sec. III-D/E tANS, Sec. IV-D dtANS), parameter identities,
closed forms, size bounds and brute force.  No GPU.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as WL

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dtans_worked_example.txt")


def _golden():
    g = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        g[k] = v
    return g


SYM = {"a": 0, "b": 1, "c": 2}


def _toy_table():
    g = _golden()
    P = O.toy_params()
    lay = [(SYM[e.split(":")[0]], int(e.split(":")[1])) for e in g["table"]]
    return P, O.Table.explicit(P, lay), g


def test_worked_example_encode_matches_printed_stream():
    P, T, g = _toy_table()
    u = [SYM[s] for s in g["input"]]
    body, flags = O.encode_string(P, T, u)
    printed = [int(v) for v in g["printed_stream"]]
    # stored words = printed stream without the two trailing known-zero words
    assert body.tolist() == printed[:-2]
    assert printed[-2:] == [0, 0]
    # first segment: check 1 reads (r = 3 < W), check 2 extracts (r = 12 >= W)
    assert flags[0].tolist() == [1, 0]
    # the words read for segment 1 are w1 = 2 (conditional) and w3 = 3 (unconditional)
    nxt = [int(v) for v in g["next_words"]]
    assert body[3] == nxt[0] and body[4] == nxt[2]


def test_worked_example_first_segment_slots():
    P, T, g = _toy_table()
    # (1,1,1)_4 = 21 = (2)_8 (5)_8: i1 = 5 (c, 0_3), i2 = 2 (b, 1_4)
    w = [1, 1, 1]
    N = (w[0] * 4 + w[1]) * 4 + w[2]
    assert N == 21
    i1, i2 = N % 8, N // 8
    assert [i1, i2] == [int(v) for v in g["first_slots"]]
    for slot, pair in zip((i1, i2), g["first_pairs"]):
        sym, db = pair.split(":")
        dg, base = (int(t) for t in db.split("/"))
        assert T.slot_key[slot] == SYM[sym] and T.slot_digit[slot] == dg and T.slot_base[slot] == base
    # Sec. III-E: state 23 = 2_inf 7_8 -> slot 7 holds (c, digit 2, base 3)
    s, dg, base = g["decode_slot7"]
    assert T.slot_key[7] == SYM[s] and T.slot_digit[7] == int(dg) and T.slot_base[7] == int(base)


def test_worked_example_decodes_printed_stream():
    P, T, g = _toy_table()
    printed = np.array([int(v) for v in g["printed_stream"]], np.uint32)
    n = len(g["input"])
    stream = np.concatenate([[n], printed]).astype(np.uint32)
    dec, used = O.decode_string(P, T, stream, n)
    assert [int(v) for v in dec] == [SYM[s] for s in g["input"]]
    assert used == 1 + len(printed) - 2  # the two trailing zeros are never read


def test_entropy_values_of_tans_example():
    g = _golden()
    counts = [1, 5, 4]  # a, b, c in u = cbcbccbbba
    assert O.entropy(counts) == pytest.approx(float(g["entropy"][0]), abs=5e-4)
    assert O.cross_entropy(counts, [1 / 8, 4 / 8, 3 / 8]) == pytest.approx(float(g["cross_entropy"][0]), abs=5e-4)
    assert O.cross_entropy(counts, [1 / 4, 2 / 4, 1 / 4]) == pytest.approx(float(g["cross_entropy_pp"][0]), abs=1e-12)
    # H(P) = H(P, P) and H(P, P') >= H(P)
    p = np.array(counts) / 10
    assert O.cross_entropy(counts, p) == pytest.approx(O.entropy(counts), abs=1e-12)


@pytest.mark.parametrize("M", [8, 4])
def test_build_table_reproduces_paper_p_prime(M):
    """Counts (a 1, b 5, c 4) over K = 8 slots give P' = (1/8, 4/8, 3/8) (Sec. III-D),
    with tANS (M = K) and with the dtANS example's cap M = 4 (Sec. IV-D)."""
    P = O.toy_params()
    P.M = M
    t = O.build_table(P, 0, [0, 1, 2], [1, 5, 4])
    assert t.multiplicities() == {0: 1, 1: 4, 2: 3}
    # cost = n * H(P, P') = 10 * 1.366 bits
    assert t.cost_bits == pytest.approx(10 * O.cross_entropy([1, 5, 4], [1 / 8, 4 / 8, 3 / 8]), rel=1e-12)


def test_build_table_brute_force_optimum():
    """Over all integer allocations of K = 8 slots with m <= M the greedy attains
    the minimum of sum c log2(K/m) (exhaustive search on tiny cases)."""
    import itertools
    P = O.toy_params()
    rng = np.random.default_rng(7)
    for trial in range(30):
        S = int(rng.integers(1, 5))
        counts = rng.integers(1, 20, S)
        P.M = int(rng.integers(2, 9))
        if S * 1 > 8:
            continue
        t = O.build_table(P, 0, np.arange(S), counts)
        best = math.inf
        for ms in itertools.product(range(1, P.M + 1), repeat=S):
            if sum(ms) <= 8:
                best = min(best, sum(c * math.log2(8 / m) for c, m in zip(counts, ms)))
        if t.has_esc:  # escapes priced at 64 raw bits are never cheaper here
            pytest.fail("unexpected escape")
        got = sum(int(c) * math.log2(8 / t.multiplicities()[s]) for s, c in enumerate(counts))
        assert got == pytest.approx(best, abs=1e-9)


def test_parameter_identities():
    P = O.csr_params(64)
    K, W, M = 1 << P.logK, 1 << P.logW, P.M
    g = P.l // P.f
    assert K ** P.l == W ** P.o == 2 ** 96          # unpack is a bijection (Sec. IV-D)
    assert M ** P.l <= W ** P.f                       # conditional loads suffice (Sec. IV-D)
    assert M ** g == W                                # 4 digits fill one word (Sec. IV-F)
    T = O.toy_params()
    assert (1 << T.logK) ** T.l == (1 << T.logW) ** T.o
    assert T.M ** T.l <= (1 << T.logW) ** T.f


def test_table_sizes_match_paper():
    """K = 4096 slots of 16 B (FP64) / 12 B (FP32) give 64 KB / 48 KB (Sec. V-A)."""
    P = O.csr_params(64)
    K = 1 << P.logK
    assert K * (4 + 8 + 2 * 2) == 64 * 1024
    assert K * (4 + 4 + 2 * 2) == 48 * 1024


def test_paper_csr_example_spmv():
    """Fig. "CSR example": values 7,5,3,2,4,1, columns 1,3,0,2,1,3, row start
    0,2,4,5,6; with x = (1,2,3,4), y = A x = (34, 9, 8, 4)."""
    rp = np.array([0, 2, 4, 5, 6])
    cols = np.array([1, 3, 0, 2, 1, 3], np.uint32)
    vals = np.array([7, 5, 3, 2, 4, 1], np.float64)
    x = np.array([1, 2, 3, 4], np.float64)
    y, _ = O.spmm_ref(rp, cols, vals, x)
    assert y.tolist() == [34, 9, 8, 4]
    assert O.dense_spmv(rp, cols, vals, 4, x).tolist() == [34, 9, 8, 4]
    # y = A x + y (Sec. III-A) with the previous y
    y2, _ = O.spmm_ref(rp, cols, vals, x, beta=1.0, Y=np.array([1, 1, 1, 1.0]))
    assert y2.tolist() == [35, 10, 9, 5]
    # and its encoding round-trips
    E = O.encode_matrix(rp, cols, vals, 4)
    rp2, c2, v2 = O.decode_matrix(E)
    assert rp2.tolist() == rp.tolist() and c2.tolist() == cols.tolist() and v2.tolist() == vals.tolist()


def test_spmm_ref_matches_dense_brute_force():
    for seed in range(5):
        A = WL.random_csr(seed, 37, 29, 5.0, integer_valued=True, empty_frac=0.2)
        rng = np.random.default_rng(seed)
        x = rng.integers(-5, 6, A["n"]).astype(np.float64)
        y, _ = O.spmm_ref(A["row_ptr"], A["cols"], A["vals"], x)
        yd = O.dense_spmv(A["row_ptr"], A["cols"], A["vals"], A["n"], x)
        assert np.array_equal(y, yd)
        X = rng.integers(-5, 6, (A["n"], 3)).astype(np.float64)
        Y, _ = O.spmm_ref(A["row_ptr"], A["cols"], A["vals"], X)
        for b in range(3):
            assert np.array_equal(Y[:, b], O.dense_spmv(A["row_ptr"], A["cols"], A["vals"], A["n"], X[:, b]))


def _transpose(A):
    m, n = A["m"], A["n"]
    rows = np.repeat(np.arange(m), np.diff(A["row_ptr"]))
    order = np.lexsort((rows, A["cols"]))
    ct = rows[order].astype(np.uint32)
    vt = A["vals"][order]
    rpt = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(A["cols"], minlength=n), out=rpt[1:])
    return rpt, ct, vt


def test_spmm_t_and_vals_grad_brute_force():
    for seed in range(4):
        A = WL.random_csr(seed + 10, 23, 31, 4.0, integer_valued=True)
        rng = np.random.default_rng(seed)
        G = rng.integers(-4, 5, (A["m"], 3)).astype(np.float64)
        X = rng.integers(-4, 5, (A["n"], 3)).astype(np.float64)
        XG, _ = O.spmm_t_ref(A["row_ptr"], A["cols"], A["vals"], A["n"], G)
        rpt, ct, vt = _transpose(A)
        for b in range(3):
            assert np.array_equal(XG[:, b], O.dense_spmv(rpt, ct, vt, A["m"], G[:, b]))
        vg, _ = O.vals_grad_ref(A["row_ptr"], A["cols"], G, X)
        rows = np.repeat(np.arange(A["m"]), np.diff(A["row_ptr"]))
        brute = np.array([sum(G[i, b] * X[j, b] for b in range(3)) for i, j in zip(rows, A["cols"])])
        assert np.array_equal(vg, brute)
        # Euler: L = sum(G * (A X)) is linear in a, so sum_q a_q dL/da_q = L
        Y, _ = O.spmm_ref(A["row_ptr"], A["cols"], A["vals"], X)
        assert float(np.sum(vg * A["vals"])) == float(np.sum(G * Y))


def test_compensated_sum_is_exact_on_cancellation():
    rp = np.array([0, 3])
    cols = np.array([0, 1, 2], np.uint32)
    vals = np.array([1e16, 1.0, -1e16])
    y, ab = O.spmm_ref(rp, cols, vals, np.ones(3))
    assert y[0] == 1.0
    assert ab[0] == 2e16 + 1.0


def _unit_costs(E, dom_tables):
    """CE and L of every unit from the decoded symbols and the table
    multiplicities: CE = sum over slots (pads included) of log2(K/m), L = sum
    over the last segment's slots of log2(m)."""
    K = 4096
    n_u, deltas, vkeys = O.decode_units(E)
    mD, mV = dom_tables
    padD = E.tabD.kept_key[0] if E.tabD.nkept else None
    padV = E.tabV.kept_key[0] if E.tabV.nkept else None
    out = []
    t = 0
    for u in range(E.nunits):
        n = int(n_u[u])
        if n == 0:
            out.append((0.0, 0.0, 0))
            continue
        nseg = (n + 3) // 4
        mults = []
        for i in range(4 * nseg):
            if i < n:
                dk, vk = int(deltas[t + i]), int(vkeys[t + i])
                mults.append(mD.get(dk, mD.get("ESC")))
                mults.append(mV.get(vk, mV.get("ESC")))
            else:
                mults.append(mD[int(padD)] if padD is not None else mD["ESC"])
                mults.append(mV[int(padV)] if padV is not None else mV["ESC"])
        ce = sum(math.log2(K / mm) for mm in mults)
        last = sum(math.log2(mm) for mm in mults[-8:])
        out.append((ce, last, nseg))
        t += n
    return out


@pytest.mark.parametrize("case", ["pr1", "stencil", "powerlaw", "escapes"])
def test_size_bounds_per_unit(case):
    """CE + L <= 32 S <= CE + L + 32 + (#extractions), with S the stored words
    of a unit other than n and raw words, and #extractions = 3 nseg - S
    (every segment consumes 3 words: stored or extracted)."""
    if case == "pr1":
        A = WL.pr1(seed=0, n=512)
    elif case == "stencil":
        A = WL.stencil27(grid=8)
    elif case == "powerlaw":
        A = WL.power_law(rows=2048, seed=5)
    else:
        A = WL.random_csr(3, 300, 5000, 9.0)  # continuous values: nearly all escaped
    E = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], A["n"])
    costs = _unit_costs(E, (E.tabD.multiplicities(), E.tabV.multiplicities()))
    for u, (ce, last, nseg) in enumerate(costs):
        S = int(E.unit_words[u]) - 1 - int(E.unit_raw[u])
        if nseg == 0:
            assert S == 0
            continue
        ext = 3 * nseg - S
        assert 0 <= ext <= 2 * (nseg - 1)
        assert ce + last <= 32 * S + 1e-9
        assert 32 * S <= ce + last + 32 + ext + 1e-9
    # exact word-count identity of the interleaved stream
    assert E.nwords == int(E.unit_words.sum())
    # global invariant: >= 8 bits per nonzero, so at most 12x (FP64) below CSR
    assert 32 * (E.nwords - E.nunits) >= 8 * E.nnz


def test_closed_form_sixteen_uniform_symbols():
    """16 equally frequent symbols per domain: every m = 256 = M, every group of
    4 digits has radix 2^32 = W, every check extracts, so a unit of n entries
    stores exactly 4 + (ceil(n/4) - 1) words (n, 3 initial, 1 per later segment)."""
    m, L = 64, 32
    deltas = 1 + (np.arange(m * L) % 16)
    cols = np.cumsum(deltas.reshape(m, L), axis=1).reshape(-1).astype(np.uint32)
    consts = np.linspace(-1, 1, 16)
    vals = consts[np.arange(m * L) % 16]
    rp = np.arange(0, m * L + 1, L)
    E = O.encode_matrix(rp, cols, vals, int(cols.max()) + 1)
    assert set(E.tabD.multiplicities().values()) == {256} and len(E.tabD.multiplicities()) == 16
    assert set(E.tabV.multiplicities().values()) == {256} and len(E.tabV.multiplicities()) == 16
    assert (E.unit_words == 4 + (L // 4 - 1)).all()
    assert E.unit_loads.sum() == 0 and E.unit_raw.sum() == 0
    assert E.nwords == m * (4 + L // 4 - 1)
    # compression vs CSR-FP64 (12 bytes/nnz + row starts) tends to 12x as L grows
    csr = 12 * m * L + 4 * (m + 1)
    assert csr / (4 * E.nwords) < 12


def test_cost_at_least_shannon_bound():
    for A in (WL.pr1(seed=1, n=1024), WL.power_law(rows=4096, seed=9)):
        E = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], A["n"])
        for dom, t in ((0, E.tabD), (1, E.tabV)):
            keys, counts = E.hist[dom]
            H = O.entropy(counts)
            assert t.cost_bits >= counts.sum() * H - 1e-6
            # m <= M = 256 of K = 4096: at least 4 bits per symbol
            assert t.cost_bits >= 4 * counts.sum() - 1e-6


@pytest.mark.parametrize("n", [2, 5, 40])
def test_first_delta_conventions_on_tridiagonal(n):
    """Delta histograms of the n x n tridiagonal matrix, worked by hand from the
    definitions.  Absolute first deltas (Sec. IV-A): row 0 starts at column 0,
    row i >= 1 at column i - 1, every other delta is 1.  Row-relative first
    deltas: 0 for row 0 and (i - 1) - i = -1 = 2^32 - 1 for every later row."""
    rows, cols = [], []
    for i in range(n):
        for j in (i - 1, i, i + 1):
            if 0 <= j < n:
                rows.append(i)
                cols.append(j)
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rp[1:])
    cols = np.array(cols, np.uint32)
    vals = np.ones(len(cols))
    ones = 2 * (n - 1)  # 3 per interior row and 2 per end row, minus one first delta per row
    expect_abs = {1: ones}
    for i in range(n):
        f = 0 if i == 0 else i - 1
        expect_abs[f] = expect_abs.get(f, 0) + 1
    expect_rel = {1: ones, 0: 1, 2 ** 32 - 1: n - 1}
    for fd, expect in ((0, expect_abs), (1, expect_rel)):
        E = O.encode_matrix(rp, cols, vals, n, first_delta=fd)
        keys, counts = E.hist[0]
        assert dict(zip(keys.tolist(), counts.tolist())) == expect
        rp2, c2, v2 = O.decode_matrix(E)
        assert np.array_equal(c2, cols) and np.array_equal(rp2, rp)


def test_row_relative_first_delta_removes_stencil_escapes():
    """On the periodic 27-point stencil every interior row's first column is
    row - g^2 - g - 1, so row-relative first deltas take a handful of values and
    no first delta is escaped; absolute first deltas are all distinct, and once
    the rows outnumber the table's K = 4096 slots most of them are escaped (one
    raw word each).  g = 24: 13,824 rows."""
    A = WL.stencil27(grid=24)
    E0 = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], A["n"])
    E1 = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], A["n"], first_delta=1)
    assert E1.unit_raw.sum() == 0
    assert E0.unit_raw.sum() > A["m"] // 2
    assert E1.nwords < E0.nwords
    assert len(E1.hist[0][0]) <= 40


def _codebook_case(seed, m=37, n=29, T=5, density=0.3, k=3):
    """Small integer-valued weight-shared matrix: every product and sum below
    is an exact FP64 integer."""
    rng = np.random.default_rng(seed)
    codebook = rng.choice(np.arange(-9, 10), size=T, replace=False).astype(np.float64)
    mask = rng.random((m, n)) < density
    assign = rng.integers(0, T, (m, n))
    rp = np.zeros(m + 1, np.int64)
    np.cumsum(mask.sum(1), out=rp[1:])
    rows, cols = np.nonzero(mask)
    vals = codebook[assign[rows, cols]]
    G = rng.integers(-4, 5, (m, k)).astype(np.float64)
    X = rng.integers(-4, 5, (n, k)).astype(np.float64)
    return codebook, mask, assign, rp, cols.astype(np.uint32), vals, G, X


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_codebook_grad_finite_difference_dense(seed):
    """L(c) = sum(G .* (A(c) X)) is linear in the codebook c, so
    L(c + e_r) - L(c) is exactly d L / d c_r; computed here on the dense
    matrix with integer arithmetic."""
    codebook, mask, assign, rp, cols, vals, G, X = _codebook_case(seed)
    grad, _ = O.codebook_grad_ref(rp, cols, vals, codebook, G, X)

    def L(cb):
        A = np.where(mask, cb[assign], 0).astype(np.int64)
        return int((G.astype(np.int64) * (A @ X.astype(np.int64))).sum())

    base = L(codebook.astype(np.int64))
    for r in range(len(codebook)):
        e = np.zeros(len(codebook), np.int64)
        e[r] = 1
        assert grad[r] == L(codebook.astype(np.int64) + e) - base
    assert grad[-1] == 0  # every value is in the codebook


def test_codebook_grad_euler_identity_and_escape_bin():
    """sum_r c_r dL/dc_r = L for L linear in c (Euler); entries whose value is
    not in the codebook land in the last entry, which then equals the sum of
    their per-entry gradients."""
    codebook, mask, assign, rp, cols, vals, G, X = _codebook_case(7, k=4)
    grad, _ = O.codebook_grad_ref(rp, cols, vals, codebook, G, X)
    Y, _ = O.spmm_ref(rp, cols, vals, X)
    assert float((codebook * grad[:-1]).sum()) == float((G * Y).sum())
    vals2 = vals.copy()
    vals2[::4] = 100.0  # not in the codebook
    grad2, _ = O.codebook_grad_ref(rp, cols, vals2, codebook, G, X)
    vg, _ = O.vals_grad_ref(rp, cols, G, X)
    assert grad2[-1] == vg[::4].sum()
    assert grad2[:-1].sum() + grad2[-1] == vg.sum()


@pytest.mark.parametrize("chain", [2, 5, 64])
def test_chained_units_closed_form_sixteen_uniform_symbols(chain):
    """Chains of units (one dtANS sequence per lane over `chain` slices) in the
    closed-form case above: every check extracts, so a lane's chain of units
    with S segments in total stores its n words, 3 initial words and one word
    per segment but the chain's final one -- the 3-word tail of every other
    unit is gone.  Word count, by hand: m rows of L entries, 32 rows a slice."""
    m, L = 32 * 7, 32
    deltas = 1 + (np.arange(m * L) % 16)
    cols = np.cumsum(deltas.reshape(m, L), axis=1).reshape(-1).astype(np.uint32)
    consts = np.linspace(-1, 1, 16)
    vals = consts[np.arange(m * L) % 16]
    rp = np.arange(0, m * L + 1, L)
    E = O.encode_matrix(rp, cols, vals, int(cols.max()) + 1, chain=chain)
    nslices = m // 32
    expect = 0
    for c0 in range(0, nslices, chain):
        nk = min(chain, nslices - c0)  # units per lane in this chain
        S = nk * (L // 4)
        expect += 32 * (nk + 3 + S - 1)
    assert E.nwords == expect
    assert E.unit_loads.sum() == 0 and E.unit_raw.sum() == 0
    assert E.nwords == int(E.unit_words.sum())
    rp2, c2, v2 = O.decode_matrix(E)
    assert np.array_equal(c2, cols) and np.array_equal(v2, vals)


@pytest.mark.parametrize("case", ["pr1", "powerlaw_split", "escapes", "empty_rows"])
@pytest.mark.parametrize("chain", [3, 8])
def test_chained_units_word_identity_and_tail_saving(case, chain):
    """Chained units: the interleaved stream has exactly the words the decoder
    reads (sum of per-unit counts), every unit but a lane's chain-final one
    reads its segments' words like a middle segment, and the stream is never
    longer than the one-sequence-per-unit stream of the same matrix."""
    kw = {}
    if case == "pr1":
        A = WL.pr1(seed=0, n=1024)
    elif case == "powerlaw_split":
        A = WL.power_law(rows=3000, seed=5, max_len=300)
        kw = dict(unit_max_nnz=8, row_order=1)
    elif case == "escapes":
        A = WL.random_csr(3, 700, 5000, 9.0)
    else:
        A = WL.random_csr(9, 3333, 50, 2.0, empty_frac=0.5)
    E1 = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], A["n"], **kw)
    E = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], A["n"], chain=chain, **kw)
    assert E.nwords == int(E.unit_words.sum())
    assert E.nwords <= E1.nwords
    assert np.array_equal(E.unit_raw, E1.unit_raw)  # escapes do not depend on the chaining


SPLITMIX = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_reference_outputs.txt")


def test_splitmix64_matches_published_reference_outputs():
    """The slot permutation's generator reproduces SplitMix64's reference
    outputs (tests/golden/splitmix64_reference_outputs.txt)."""
    seen = 0
    for line in open(SPLITMIX):
        if line.startswith("#") or not line.strip():
            continue
        seed, vals = line.split(":")
        want = [int(v) for v in vals.split()]
        got = O.splitmix64(int(seed), len(want))
        assert [int(v) for v in got] == want
        seen += 1
    assert seen == 2


@pytest.mark.parametrize("seeds", [(1, 0), (0, 99), (12345, 678)])
def test_slot_permutation_moves_only_used_slots(seeds):
    """The permutation maps the canonical used slots (kept symbols, then the
    escape symbol) one to one onto themselves and leaves the unused tail in
    place; it depends only on the seed, and a seed of 0 keeps the canonical
    layout."""
    A = WL.random_csr(31, 700, 900, 12.0, nvals=5)  # 5 value symbols: 1280 of 4096 value slots used
    E1 = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], A["n"], perm_seeds=seeds)
    E2 = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], A["n"], perm_seeds=seeds)
    for t, perm, perm2, seed in ((E1.tabD, E1.permD, E2.permD, seeds[0]), (E1.tabV, E1.permV, E2.permV, seeds[1])):
        if seed == 0:
            assert perm is None
            continue
        K = len(perm)
        u = int(np.max(np.nonzero(t.slot_kind != 0)[0])) + 1
        assert np.all(t.slot_kind[:u] != 0) and np.all(t.slot_kind[u:] == 0)  # used slots are a prefix
        assert sorted(perm[:u].tolist()) == list(range(u))
        assert np.array_equal(perm[u:], np.arange(u, K))
        assert np.array_equal(perm, perm2)
        assert not np.array_equal(perm[:u], np.arange(u))
    if seeds[1]:
        assert int(np.count_nonzero(E1.tabV.slot_kind)) == 5 * 256


# ---------------------------------------------------------------------------
# Hand-worked multi-lane slices (tests/golden/*.txt, derivations in the files)
# ---------------------------------------------------------------------------

def _num(t: str) -> int:
    return int(t, 16) if t.lower().startswith("0x") else int(t)


def _hand_slice(name: str):
    """Parses a hand-worked slice file: parameters, the matrix and the
    expected arrays."""
    g = {}
    rows = []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        line = line.rstrip("\n")
        if not line.strip() or line.startswith("#"):
            continue
        k, _, v = line.partition(":")
        if k.startswith("row"):
            rows.append([(int(e.split(":")[0]), float(e.split(":")[1])) for e in v.split()])
        else:
            g[k] = v.strip()
    if g["params"] == "csr":
        P = O.csr_params(64, 32)
    else:
        kv = dict(e.split("=") for e in g["params"].split())
        P = O.Params()
        P.logK, P.logW, P.M, P.l, P.o, P.f, P.spi = (int(kv[k]) for k in ("logK", "logW", "M", "l", "o", "f", "spi"))
        P.raw_words[0], P.raw_words[1] = (int(t) for t in kv["raw_words"].split(","))
        P.raw_bits[0], P.raw_bits[1] = (int(t) for t in kv["raw_bits"].split(","))
        P.slice = int(kv["slice"])
    row_ptr = np.zeros(len(rows) + 1, np.int64)
    row_ptr[1:] = np.cumsum([len(r) for r in rows])
    cols = np.array([c for r in rows for c, _ in r], np.uint32)
    vals = np.array([v for r in rows for _, v in r], np.float64)
    arr = {k: np.array([_num(t) for t in v.split()], np.int64) for k, v in g.items()
           if k not in ("params", "delta_slots", "value_slots")}
    return P, dict(row_ptr=row_ptr, cols=cols, vals=vals, n=int(g["n"]), m=len(rows)), arr, g


def test_hand_worked_slice_with_escapes_and_early_end():
    """Three lanes of 5, 1 and 4 entries and an empty fourth unit, escaped
    deltas and escaped FP64 values in two lanes (tests/golden/
    interleave_escapes_small.txt): the oracle's stream equals the hand-worked
    one word for word, in-stream and with the separate escape stream, and its
    decoder reads the hand-worked words back to the matrix.  Pins the lane
    and program-point order of the interleave (P_n, P_w, then per segment
    E, C1, C2, U) and the escape raw-word order (slot order, low word of a
    value first) of Sec. II, IV-B and IV-F."""
    P, A, g, raw = _hand_slice("interleave_escapes_small.txt")
    E = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], A["n"], params=P)
    assert E.words.astype(np.int64).tolist() == g["stream"].tolist()
    assert E.slice_off.tolist() == g["slice_off"].tolist()
    # tables as derived: kept deltas 0..6 and values 1.0..7.0 in slots 0..6, escape in slot 7, all bases 1
    kd = [int(t) for t in raw["delta_slots"].split()]
    kv = O.value_keys(np.array([float(t) for t in raw["value_slots"].split()]))
    assert E.tabD.slot_key[:7].tolist() == kd and E.tabV.slot_key[:7].tolist() == kv.tolist()
    for t in (E.tabD, E.tabV):
        assert t.slot_kind.tolist() == [1] * 7 + [2] and t.slot_base.tolist() == [1] * 8
    Es = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], A["n"], params=P, escape_stream=1)
    assert Es.words.astype(np.int64).tolist() == g["stream_sep"].tolist()
    assert Es.slice_off.tolist() == g["slice_off_sep"].tolist()
    assert Es.esc_words.astype(np.int64).tolist() == g["esc_words"].tolist()
    assert Es.esc_off.tolist() == g["esc_off"].tolist()
    # decoding the hand-worked words (not the oracle's own) gives the matrix back
    rp, c, v = O.decode_matrix(E, g["stream"].astype(np.uint32), g["slice_off"])
    assert np.array_equal(rp, A["row_ptr"]) and np.array_equal(c, A["cols"])
    assert np.array_equal(O.value_keys(v), O.value_keys(A["vals"]))
    rp, c, v = O.decode_matrix(Es, g["stream_sep"].astype(np.uint32), g["slice_off_sep"],
                               esc_words=g["esc_words"].astype(np.uint32), esc_off=g["esc_off"])
    assert np.array_equal(c, A["cols"]) and np.array_equal(O.value_keys(v), O.value_keys(A["vals"]))


def test_hand_worked_slot_permutation_placement():
    """The slot permutation of a four-slot value table from SplitMix64's
    published outputs for seed 1234567, worked by hand
    (tests/golden/slot_permutation_small.txt): the oracle's permutation and
    the stream it encodes through it equal the hand-worked ones, and the
    hand-worked stream decodes back to the matrix."""
    P, A, g, raw = _hand_slice("slot_permutation_small.txt")
    seeds = tuple(int(t) for t in raw["perm_seeds"].split())
    E = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], A["n"], params=P, perm_seeds=seeds)
    assert E.permD is None
    assert E.permV.tolist() == g["value_perm"].tolist()
    assert E.words.astype(np.int64).tolist() == g["stream"].tolist()
    assert E.slice_off.tolist() == g["slice_off"].tolist()
    rp, c, v = O.decode_matrix(E, g["stream"].astype(np.uint32), g["slice_off"])
    assert np.array_equal(c, A["cols"]) and np.array_equal(v, A["vals"])


def test_hand_worked_csr_dtans_slice():
    """Three lanes in the real CSR-dtANS parameters (K = 2^12, W = 2^32),
    16 equally frequent symbols per domain so that every check group has
    radix exactly W (tests/golden/csr_dtans_slice_radix_w.txt): the stream
    equals the hand-worked words (12-bit slot packing, byte digits, lane
    order, pads, the lane that ends in its first segment)."""
    P, A, g, _ = _hand_slice("csr_dtans_slice_radix_w.txt")
    E = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], A["n"])
    assert E.words.astype(np.int64).tolist() == g["stream"].tolist()
    assert E.slice_off.tolist() == g["slice_off"].tolist()
    assert E.tabD.slot_base.tolist() == [256] * 4096 and E.tabV.slot_base.tolist() == [256] * 4096
    rp, c, v = O.decode_matrix(E, g["stream"].astype(np.uint32), g["slice_off"])
    assert np.array_equal(c, A["cols"]) and np.array_equal(v, A["vals"])


@pytest.mark.parametrize("kind", ["mixed_exponents", "cancellation", "integer_rows"])
def test_reference_product_within_dot2_bound_of_exact_sum(kind):
    """The oracle's y (compensated dot products, Dot2 of Ogita, Rump and Oishi,
    "Accurate sum and dot product", 2005) against the exact rational sum of
    each row: |y - s| <= u |s| + gamma_n^2 sum |a x| with u = 2^-53 and
    gamma_n = n u / (1 - n u), the published bound of that algorithm.  The
    inputs are the adversarial ones the GPU parity tests use: x whose
    exponents spread over 2^+-600, rows whose terms cancel to a tiny result,
    and small-integer values (the integer-coefficient form's tables)."""
    from fractions import Fraction
    rng = np.random.default_rng({"mixed_exponents": 1, "cancellation": 2, "integer_rows": 3}[kind])
    m, n = 300, 400
    lens = rng.integers(1, 40, m)
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    cols = np.concatenate([np.sort(rng.choice(n, L, replace=False)) for L in lens]).astype(np.uint32)
    if kind == "integer_rows":
        vals = rng.integers(-9, 10, len(cols)).astype(np.float64)
    else:
        vals = rng.uniform(-1, 1, len(cols)) * np.exp2(rng.integers(-30, 30, len(cols)))
    x = rng.uniform(1, 2, n) * rng.choice([-1.0, 1.0], n)
    if kind == "mixed_exponents":
        x *= np.exp2(rng.integers(-600, 600, n))
    elif kind == "cancellation":
        # the last term of each row cancels the rounded sum of the others
        for i in range(m):
            a, b = rp[i], rp[i + 1]
            if b - a >= 2:
                s = float(np.dot(vals[a:b - 1], x[cols[a:b - 1]]))
                x[cols[b - 1]] = -s / vals[b - 1]
    y, ab = O.spmm_ref(rp, cols, vals, x)
    u = 2.0 ** -53
    checked = 0
    for i in range(m):
        a, b = rp[i], rp[i + 1]
        exact = sum((Fraction(float(vals[q])) * Fraction(float(x[cols[q]])) for q in range(a, b)), Fraction(0))
        g = (b - a) * u / (1 - (b - a) * u)
        bound = u * abs(float(exact)) + g * g * ab[i]
        assert abs(Fraction(float(y[i])) - exact) <= Fraction(bound) * (1 + 2 ** -40), (i, float(exact), y[i])
        checked += 1
    assert checked == m
