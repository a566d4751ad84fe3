"""Host side of the library (no GPU): the C++ encoder is bit-exact with the
oracle, the shared library exports every declared symbol, and the handle's
error paths and file format behave as documented in include/dtans.h."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_2603_01915_gb300 as D
import workloads as WL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "dtans.h")).read()
    declared = set(re.findall(r"^\s*(?:dtans_status|void|const char \*)\s*\*?\s*(dtans_\w+)\s*\(", hdr, re.M))
    assert declared, "no declarations parsed"
    L = D.lib()
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert declared == set(D.EXPORTS)


def _cases():
    yield "pr1", WL.pr1(seed=0, n=700), {}
    yield "stencil", WL.stencil27(grid=6), {}
    yield "powerlaw", WL.power_law(rows=3000, seed=2), {}
    yield "escapes", WL.random_csr(2, 500, 100000, 12.0), {}
    yield "f32", WL.random_csr(8, 400, 700, 9.0, nvals=40, dtype=np.float32), {}
    yield "split", WL.power_law(rows=1200, seed=3, max_len=200), dict(unit_max_nnz=8, row_order=1)
    yield "split_natural", WL.power_law(rows=1200, seed=4, max_len=200), dict(unit_max_nnz=16, row_order=0)
    yield "perm", WL.pr1(seed=6, n=500), dict(perm_seeds=(99, 1234567))
    yield "empty_rows", WL.random_csr(9, 333, 50, 2.0, empty_frac=0.5), {}
    yield "sorted_unsplit", WL.power_law(rows=1200, seed=6, max_len=200), dict(unit_max_nnz=0, row_order=1)
    yield "chain8", WL.pr1(seed=7, n=900), dict(chain=8)
    yield "chain3_split_rel", WL.power_law(rows=1500, seed=8, max_len=200), dict(unit_max_nnz=8, row_order=1,
                                                                                 first_delta=1, chain=3)
    yield "chain64_empty", WL.random_csr(9, 3333, 50, 2.0, empty_frac=0.5), dict(chain=64)
    yield "esc_stream", WL.random_csr(2, 500, 100000, 12.0), dict(escape_stream=1)
    yield "esc_stream_chain", WL.power_law(rows=1500, seed=9, max_len=200), dict(escape_stream=1, chain=4)
    yield "stencil_rel", WL.stencil27(grid=6), dict(first_delta=1)
    yield "split_rel", WL.power_law(rows=1200, seed=5, max_len=200), dict(unit_max_nnz=8, row_order=1, first_delta=1)
    yield "window", WL.power_law(rows=2500, seed=10, max_len=200), dict(unit_max_nnz=16, row_order=1,
                                                                         order_window=300)
    yield "window_unsplit_chain", WL.power_law(rows=2000, seed=11, max_len=200), dict(row_order=1, order_window=77,
                                                                                       chain=2)
    yield "unsorted_dups", WL.unsorted_duplicates(WL.pr1(seed=12, n=800), seed=1), {}
    yield "unsorted_dups_f32_split_rel", WL.unsorted_duplicates(WL.power_law(rows=1500, seed=13, max_len=200), seed=2,
                                                                dup_frac=0.3), dict(unit_max_nnz=8, row_order=1,
                                                                                    first_delta=1)
    yield "unsorted_dups_stencil_chain", WL.unsorted_duplicates(WL.stencil27(grid=7), seed=3), dict(chain=4)


@pytest.mark.parametrize("name,A,kw", list(_cases()), ids=[c[0] for c in _cases()])
def test_encoder_bit_exact_with_oracle(name, A, kw):
    okw = dict(unit_max_nnz=kw.get("unit_max_nnz", 0), row_order=kw.get("row_order", 0),
               perm_seeds=kw.get("perm_seeds", (0, 0)), first_delta=kw.get("first_delta", 0),
               chain=kw.get("chain", 1), escape_stream=kw.get("escape_stream", 0),
               order_window=kw.get("order_window", 0))
    E = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], A["n"], **okw)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), **okw)
    v = M.view()
    inf = M.info
    assert inf.nwords == E.nwords and inf.nunits == E.nunits and inf.nslices == E.nslices
    assert inf.order_window == okw["order_window"]
    assert np.array_equal(v["words"], E.words)
    assert np.array_equal(v["slice_off"].astype(np.int64), E.slice_off)
    assert np.array_equal(v["unit_row"].astype(np.int64), E.unit_row)
    assert np.array_equal(v["unit_len"].astype(np.int64), E.unit_len)
    if kw.get("escape_stream"):
        assert np.array_equal(v["esc_words"], E.esc_words) and np.array_equal(v["esc_off"].astype(np.int64), E.esc_off)
        assert inf.nesc == len(E.esc_words) and inf.bytes_esc == 4 * inf.nesc + 8 * (inf.nslices + 1)
    else:
        assert v["esc_words"] is None and inf.nesc == 0
    for name_, t in (("delta", E.tabD), ("value", E.tabV)):
        assert np.array_equal(v[f"{name_}_kind"], t.slot_kind)
        assert np.array_equal(v[f"{name_}_key"], t.slot_key)
        assert np.array_equal(v[f"{name_}_digit"].astype(np.uint32), t.slot_digit)
        assert np.array_equal(v[f"{name_}_base"].astype(np.uint32), t.slot_base)
    assert inf.cost_bits_delta == E.tabD.cost_bits and inf.cost_bits_value == E.tabV.cost_bits
    if E.permD is not None:
        assert np.array_equal(v["delta_perm"], E.permD) and np.array_equal(v["value_perm"], E.permV)
    M.close()


def test_encoder_independent_of_thread_count():
    A = WL.power_law(rows=5000, seed=12)
    w = [D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), num_threads=t).view()["words"]
         for t in (1, 3, 8)]
    assert np.array_equal(w[0], w[1]) and np.array_equal(w[0], w[2])


def test_oracle_decodes_library_stream():
    A = WL.power_law(rows=2000, seed=13)
    E = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], A["n"])
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]))
    v = M.view()
    rp, c, vals = O.decode_matrix(E, v["words"], v["slice_off"].astype(np.int64))
    cs, vs = O.sort_rows(A["row_ptr"], A["cols"], A["vals"])
    assert np.array_equal(c, cs) and np.array_equal(vals.view(np.uint32), vs.view(np.uint32))


def test_info_sizes():
    A = WL.pr1(seed=1, n=1000)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]))
    inf = M.info
    assert inf.bytes_tables == 4096 * 8 + 4096 * 16
    assert inf.bytes_words == 4 * inf.nwords
    assert inf.bytes_slice_off == 8 * (inf.nslices + 1)
    assert inf.bytes_unit_meta == 0
    assert inf.bytes_compressed == inf.bytes_words + inf.bytes_slice_off + inf.bytes_tables
    M32 = D.Matrix(A["row_ptr"], A["cols"], A["vals"].astype(np.float32), (A["m"], A["n"]))
    assert M32.info.bytes_tables == 4096 * 8 + 4096 * 8


def test_encode_rejects_bad_input():
    rp = np.array([0, 2, 1], np.int64)
    with pytest.raises(D.DtansError) as e:
        D.Matrix(rp, np.array([0, 1], np.uint32), np.ones(2), (2, 4))
    assert e.value.status == -1
    with pytest.raises(D.DtansError):
        D.Matrix(np.array([0, 2]), np.array([0, 9], np.uint32), np.ones(2), (1, 4))  # column >= n
    with pytest.raises(D.DtansError):
        D.Matrix(np.array([1, 2]), np.array([0], np.uint32), np.ones(1), (1, 4))  # row_ptr[0] != 0
    with pytest.raises(TypeError):
        D.Matrix(np.array([0, 1]), np.array([0], np.uint32), np.ones(1, np.int32), (1, 4))
    with pytest.raises(D.DtansError) as e:
        D.Matrix(np.array([0, 1]), np.array([0], np.uint32), np.ones(1), (1, 4), row_order=1, order_window=-1)
    assert e.value.status == -1


def test_calls_before_upload_fail_with_state_error():
    A = WL.pr1(seed=2, n=64)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]))
    st = D.lib().dtans_spmv(M.h, C.c_void_p(0), C.c_void_p(0), 0.0, C.c_void_p(0))
    assert st == -7
    assert b"not uploaded" in D.lib().dtans_last_error()
    assert D.lib().dtans_spmv(C.c_void_p(0), C.c_void_p(0), C.c_void_p(0), 0.0, C.c_void_p(0)) == -1


def test_save_load_round_trip(tmp_path):
    A = WL.power_law(rows=1500, seed=14, max_len=100)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), unit_max_nnz=8, row_order=1,
                 perm_seeds=(5, 6), first_delta=1, chain=4, escape_stream=1, order_window=500)
    p = str(tmp_path / "m.dtans")
    M.save(p)
    M2 = D.Matrix.load(p)
    a, b = M.view(), M2.view()
    for k in a:
        if a[k] is None:
            assert b[k] is None
        else:
            assert np.array_equal(a[k], b[k]), k
    i1, i2 = M.info, M2.info
    assert (i1.m, i1.n, i1.nnz, i1.nwords, i1.dtype) == (i2.m, i2.n, i2.nnz, i2.nwords, i2.dtype)
    assert i1.first_delta == i2.first_delta == 1 and i1.chain_slices == i2.chain_slices == 4
    assert i1.escape_stream == i2.escape_stream == 1 and i1.nesc == i2.nesc
    assert i1.order_window == i2.order_window == 500
    # a matrix whose escape stream is not empty
    B = WL.random_csr(2, 500, 100000, 12.0)
    M = D.Matrix(B["row_ptr"], B["cols"], B["vals"], (B["m"], B["n"]), escape_stream=1, chain=3)
    M.save(p)
    M2 = D.Matrix.load(p)
    a, b = M.view(), M2.view()
    assert M.info.nesc > 0 and np.array_equal(a["esc_words"], b["esc_words"])
    assert np.array_equal(a["esc_off"], b["esc_off"]) and np.array_equal(a["words"], b["words"])


def test_load_accepts_version_1_and_2_files(tmp_path):
    """Files of the earlier format versions load: version 2 (no order_window
    field) and version 1 (no first_delta, chain_slices, escape_stream, nesc
    fields either) -- built from a version-3 file by dropping the 32-byte
    version-3 header and then the 32-byte version-2 header."""
    A = WL.pr1(seed=3, n=300)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), row_order=1)
    p = tmp_path / "v3.dtans"
    M.save(str(p))
    raw = p.read_bytes()
    assert raw[:8] == b"DTANSv3\0"
    hdr = 8 + 8 * 13  # magic + version-1 header (13 int64 fields)
    assert int.from_bytes(raw[hdr:hdr + 8], "little") == 0  # first_delta
    assert int.from_bytes(raw[hdr + 8:hdr + 16], "little") == 1  # chain_slices
    assert int.from_bytes(raw[hdr + 16:hdr + 24], "little") == 0  # escape_stream
    assert int.from_bytes(raw[hdr + 32:hdr + 40], "little") == 0  # order_window
    v2 = tmp_path / "v2.dtans"
    v2.write_bytes(b"DTANSv2\0" + raw[8:hdr + 32] + raw[hdr + 64:])
    v1 = tmp_path / "v1.dtans"
    v1.write_bytes(b"DTANSv1\0" + raw[8:hdr] + raw[hdr + 64:])
    for f in (v1, v2):
        M1 = D.Matrix.load(str(f))
        assert M1.info.first_delta == 0 and M1.info.order_window == 0 and M1.info.row_order == 1
        assert np.array_equal(M1.view()["words"], M.view()["words"])
        assert np.array_equal(M1.view()["unit_row"], M.view()["unit_row"])


def test_load_rejects_corrupt_files(tmp_path):
    A = WL.pr1(seed=3, n=200)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]))
    p = str(tmp_path / "m.dtans")
    M.save(p)
    raw = open(p, "rb").read()
    bad = tmp_path / "bad.dtans"
    bad.write_bytes(b"XXXXXXXX" + raw[8:])
    with pytest.raises(D.DtansError) as e:
        D.Matrix.load(str(bad))
    assert e.value.status == -4
    bad.write_bytes(raw[: len(raw) // 2])
    with pytest.raises(D.DtansError):
        D.Matrix.load(str(bad))
    hdr = 8 + 8 * 13 + 32  # the version-3 header's order_window
    bad.write_bytes(raw[:hdr] + (-1).to_bytes(8, "little", signed=True) + raw[hdr + 8:])
    with pytest.raises(D.DtansError) as e:
        D.Matrix.load(str(bad))
    assert e.value.status == -4
    with pytest.raises(D.DtansError) as e:
        D.Matrix.load(str(tmp_path / "missing.dtans"))
    assert e.value.status == -6


def test_codebook_get_and_set_on_host(tmp_path):
    """dtans_codebook returns the kept value symbols in the table's rank order
    (the oracle's kept keys); dtans_set_codebook replaces them in every slot of
    their symbol without touching the stream, and a saved file keeps them."""
    A = WL.pruned_linear(dim=300, batch=2)
    E = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], A["n"])
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]))
    cb = M.codebook()
    assert cb.dtype == np.float32 and len(cb) == M.info.kept_value == E.tabV.nkept
    assert np.array_equal(O.value_keys(cb), E.tabV.kept_key[: E.tabV.nkept])
    words0 = M.view()["words"].copy()
    new = (np.arange(len(cb)) * 0.25 - 1.0).astype(np.float32)
    M.set_codebook(new)
    assert np.array_equal(M.codebook(), new)
    v = M.view()
    assert np.array_equal(v["words"], words0)
    kept = v["value_kind"] == 1
    assert set(O.value_keys(new).tolist()) == set(v["value_key"][kept].tolist())
    p = str(tmp_path / "cb.dtans")
    M.save(p)
    assert np.array_equal(D.Matrix.load(p).codebook(), new)
    with pytest.raises(ValueError):
        M.set_codebook(new[:-1])


def _random_option_cases(count=40, seed=2024):
    rng = np.random.default_rng(seed)
    for i in range(count):
        m = int(rng.integers(1, 900))
        n = int(rng.integers(1, 3000))
        dt = np.float64 if rng.random() < 0.5 else np.float32
        A = WL.random_csr(int(rng.integers(1 << 30)), m, n, float(rng.uniform(0.5, 40.0)),
                          nvals=int(rng.integers(2, 300)) if rng.random() < 0.7 else None, dtype=dt,
                          empty_frac=float(rng.choice([0.0, 0.3])))
        order = int(rng.integers(0, 2))
        kw = dict(unit_max_nnz=int(rng.choice([0, 1, 4, 7, 32])), row_order=order,
                  order_window=int(rng.choice([0, 1, 33, 500])) if order else 0,
                  first_delta=int(rng.integers(0, 2)), chain=int(rng.choice([1, 1, 2, 5, 64])),
                  escape_stream=int(rng.integers(0, 2)),
                  perm_seeds=(int(rng.integers(0, 2)) * 77, int(rng.integers(0, 2)) * 991))
        yield i, A, kw


@pytest.mark.parametrize("i,A,kw", list(_random_option_cases()), ids=[f"r{c[0]}" for c in _random_option_cases()])
def test_encoder_bit_exact_random_options(i, A, kw):
    """Random shapes, densities, value sets and combinations of every encoder
    option: the library's stream, slice offsets, unit layout and escape arrays
    equal the oracle's word for word."""
    E = O.encode_matrix(A["row_ptr"], A["cols"], A["vals"], A["n"], **kw)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), **kw)
    v, inf = M.view(), M.info
    assert inf.nwords == E.nwords and inf.nunits == E.nunits
    assert np.array_equal(v["words"], E.words)
    assert np.array_equal(v["slice_off"].astype(np.int64), E.slice_off)
    assert np.array_equal(v["unit_row"].astype(np.int64), E.unit_row)
    assert np.array_equal(v["unit_len"].astype(np.int64), E.unit_len)
    if kw["escape_stream"]:
        assert np.array_equal(v["esc_words"], E.esc_words)
    # and the oracle decodes it back to the sorted input
    rp, c, val = O.decode_matrix(E)
    cs, vs = O.sort_rows(A["row_ptr"], A["cols"], A["vals"])
    assert np.array_equal(rp, A["row_ptr"]) and np.array_equal(c, cs)
    assert np.array_equal(O.value_keys(val), O.value_keys(vs))
    M.close()


_FUZZ = r'''
import os, random, sys, tempfile
import paper_2603_01915_gb300 as D, workloads as WL
A = WL.power_law(rows=1500, seed=14, max_len=100)
M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), unit_max_nnz=8, row_order=1,
             perm_seeds=(5, 6), first_delta=1, chain=4, escape_stream=1, order_window=500)
d = tempfile.mkdtemp()
p = os.path.join(d, "m.dtans")
M.save(p)
raw = open(p, "rb").read()
rng = random.Random(int(sys.argv[1]))
loaded = rejected = 0
for it in range(300):
    b = bytearray(raw)
    kind = rng.random()
    if kind < 0.8:
        span = 2048 if kind < 0.5 else len(b)
        for _ in range(rng.randint(1, 4)):
            b[rng.randrange(min(len(b), span))] = rng.randrange(256)
    else:
        b = b[: rng.randrange(len(b))]
    q = os.path.join(d, "f.dtans")
    open(q, "wb").write(bytes(b))
    try:
        M2 = D.Matrix.load(q)
        M2.info, M2.view()
        M2.close()
        loaded += 1
    except D.DtansError as e:
        assert e.status in (-4, -6), e.status
        rejected += 1
print(loaded, rejected)
'''


@pytest.mark.parametrize("seed", [7, 8])
def test_load_survives_corrupted_files(seed):
    """dtans_load on 300 randomly corrupted or truncated copies of a file that
    uses every option: each either loads into a handle whose info and view
    can be read, or fails with DTANS_ERR_CORRUPT / DTANS_ERR_IO -- never a
    crash (run in a child process so a crash fails the test)."""
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "-c", _FUZZ, str(seed)], capture_output=True, text=True, timeout=300,
                       cwd=ROOT, env=dict(os.environ, PYTHONPATH=ROOT))
    assert r.returncode == 0, r.stderr[-2000:]
    loaded, rejected = map(int, r.stdout.split())
    assert loaded + rejected == 300 and rejected > 0


def test_every_entry_point_rejects_null_arguments():
    """Each C entry point given a null handle (or null output) returns
    DTANS_ERR_ARG without touching the GPU; the destroy calls accept null."""
    L = D.lib()
    null = None
    calls = {
        "dtans_upload": (null, null),
        "dtans_spmv": (null, null, null, 0.0, null),
        "dtans_spmv_noalloc": (null, null, null, 0.0, null),
        "dtans_spmv_host": (null, null, null, 0.0, null),
        "dtans_spmm": (null, 2, null, null, 0.0, null),
        "dtans_spmv_T": (null, 2, null, null, 0.0, null),
        "dtans_vals_grad": (null, 2, null, null, null, null),
        "dtans_decode_csr": (null, null, null, null),
        "dtans_codebook": (null, null),
        "dtans_set_codebook": (null, null, null),
        "dtans_codebook_grad": (null, 2, null, null, null, null),
        "dtans_info": (null, null),
        "dtans_view": (null, null),
        "dtans_check": (null, null),
        "dtans_save": (null, b"/nonexistent/x"),
        "dtans_load": (null, null),
        "dtans_set_launch": (null, 1, 32),
        "dtans_set_warps": (null, 24),
        "dtans_set_tile_policy": (null, 0),
        "dtans_set_accumulate": (null, 0),
        "dtans_set_scatter": (null, 0),
        "dtans_tune_warps": (null, 1, null, null, null),
        "dtans_batch_create": (null, 0, null),
        "dtans_batch_bind": (null, null, null),
        "dtans_batch_spmv": (null, 0.0, null),
        "dtans_encode": (2, 2, null, null, null, 2, null, null),
        "dtans_tune": (2, 2, null, null, null, 2, null, null, null, null),
    }
    for name, args in calls.items():
        assert getattr(L, name)(*args) == -1, name
        assert L.dtans_last_error(), name
    L.dtans_destroy(None)
    L.dtans_batch_destroy(None)
    assert set(calls) | {"dtans_destroy", "dtans_batch_destroy", "dtans_last_error"} == set(D.EXPORTS)


def test_library_stream_equals_hand_worked_csr_slice():
    """The library encoder reproduces the hand-worked CSR-dtANS slice of
    tests/golden/csr_dtans_slice_radix_w.txt (three lanes, radix-W groups)
    word for word: a pin that does not go through the oracle."""
    rows, g = [], {}
    for line in open(os.path.join(ROOT, "tests", "golden", "csr_dtans_slice_radix_w.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        k, _, v = line.partition(":")
        if k.startswith("row"):
            rows.append([(int(e.split(":")[0]), float(e.split(":")[1])) for e in v.split()])
        else:
            g[k] = v.split()
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    cols = np.array([c for r in rows for c, _ in r], np.uint32)
    vals = np.array([v for r in rows for _, v in r], np.float64)
    M = D.Matrix(rp, cols, vals, (len(rows), int(g["n"][0])))
    v = M.view()
    want = [int(t, 16) if t.startswith("0x") else int(t) for t in g["stream"]]
    assert v["words"].tolist() == want
    assert v["slice_off"].tolist() == [int(t) for t in g["slice_off"]]
    M.close()
