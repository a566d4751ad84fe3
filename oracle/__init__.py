"""CPU oracle for CSR-dtANS (test infrastructure only).

Plain, slow, obviously correct reference of "Fast Entropy Decoding for Sparse
MVM on GPUs" (arXiv 2603.01915): coding tables (Sec. III-D, IV-C), the dtANS
encoder (Sec. IV-E) and decoder (Algorithm 3 with the check placement of the
Sec. IV-D worked example), warp interleaving (Sec. II, IV-B), and compensated
FP64 products y = A x + beta y (Sec. III-A), A^T g and the value gradient.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline and
reference legs may import this package.  The product package never does, and
the two share no code.  The arithmetic lives in ``dtans_oracle.c`` (plain C,
compiled here with gcc on first use); this module only marshals arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dtans_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (-O2, no FP contraction) and returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Params(C.Structure):
    _fields_ = [("logK", C.c_int32), ("logW", C.c_int32), ("M", C.c_int32), ("l", C.c_int32),
                ("o", C.c_int32), ("f", C.c_int32), ("spi", C.c_int32),
                ("raw_words", C.c_int32 * 2), ("raw_bits", C.c_int32 * 2), ("slice", C.c_int32)]


class _Table(C.Structure):
    _fields_ = [("nkept", C.c_int64), ("has_esc", C.c_int32), ("pad_esc", C.c_int32),
                ("pad_key", C.c_uint64), ("esc_first", C.c_uint32), ("esc_mult", C.c_uint32),
                ("cost_bits", C.c_double),
                ("kept_key", C.c_void_p), ("kept_first", C.c_void_p), ("kept_mult", C.c_void_p),
                ("slot_key", C.c_void_p), ("slot_digit", C.c_void_p), ("slot_base", C.c_void_p),
                ("slot_kind", C.c_void_p)]


def _p(a: np.ndarray):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
            L.or_entropy.restype = dbl
            L.or_entropy.argtypes = [i64, vp]
            L.or_cross_entropy.restype = dbl
            L.or_cross_entropy.argtypes = [i64, vp, vp]
            L.or_build_table.restype = C.c_int
            L.or_build_table.argtypes = [C.POINTER(Params), i32, i64, vp, vp, C.POINTER(_Table)]
            L.or_encode_string.restype = i64
            L.or_encode_string.argtypes = [C.POINTER(Params), C.POINTER(_Table), i64, vp, vp, i64, vp]
            L.or_decode_string.restype = i64
            L.or_decode_string.argtypes = [C.POINTER(Params), C.POINTER(_Table), vp, i64, vp, vp]
            L.or_splitmix64_seq.restype = None
            L.or_splitmix64_seq.argtypes = [C.c_uint64, i64, vp]
            L.or_layout.restype = i64
            L.or_layout.argtypes = [i64, vp, i64, i32, i64, vp, vp, vp]
            L.or_sort_rows.restype = None
            L.or_sort_rows.argtypes = [i64, vp, vp, vp, vp, vp]
            L.or_encode_matrix.restype = vp
            L.or_encode_matrix.argtypes = [C.POINTER(Params), i64, i64, vp, vp, vp, i64, i32, i64, i32, i32, i32,
                                           C.POINTER(_Table), C.POINTER(_Table), C.c_uint64, C.c_uint64,
                                           vp, vp, C.POINTER(C.c_int32)]
            L.or_matrix_get.restype = i64
            L.or_matrix_get.argtypes = [vp, i32]
            L.or_matrix_copy.restype = None
            L.or_matrix_copy.argtypes = [vp] + [vp] * 9
            L.or_matrix_copy_esc.restype = None
            L.or_matrix_copy_esc.argtypes = [vp, vp, vp]
            L.or_matrix_hist.restype = None
            L.or_matrix_hist.argtypes = [vp, i32, vp, vp]
            L.or_matrix_free.restype = None
            L.or_matrix_free.argtypes = [vp]
            L.or_decode_slices.restype = i32
            L.or_decode_slices.argtypes = [C.POINTER(Params), C.POINTER(_Table), C.POINTER(_Table), vp, vp,
                                           vp, vp, i64, i64, i64, i32, vp, vp, vp, vp, i64]
            L.or_spmm_ref.restype = None
            L.or_spmm_ref.argtypes = [i64, vp, vp, vp, i64, vp, dbl, vp, vp, vp]
            L.or_spmm_t_ref.restype = None
            L.or_spmm_t_ref.argtypes = [i64, i64, vp, vp, vp, i64, vp, dbl, vp, vp, vp]
            L.or_vals_grad_ref.restype = None
            L.or_vals_grad_ref.argtypes = [i64, vp, vp, i64, vp, vp, vp, vp]
            L.or_dense_spmv.restype = None
            L.or_dense_spmv.argtypes = [i64, i64, vp, vp, vp, vp, vp]
            _lib = L
    return _lib


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------

def csr_params(value_bits: int = 64, slice_width: int = 32) -> Params:
    """CSR-dtANS: K = 2^12, W = 2^32, M = 2^8, l = 8, o = 3, f = 2 (Sec. IV-D),
    symbols alternate (delta, value); escaped deltas cost one 32-bit word and
    escaped values one (FP32) or two (FP64) words."""
    P = Params()
    P.logK, P.logW, P.M, P.l, P.o, P.f, P.spi = 12, 32, 256, 8, 3, 2, 2
    P.raw_words[0], P.raw_words[1] = 1, (2 if value_bits == 64 else 1)
    P.raw_bits[0], P.raw_bits[1] = 32, value_bits
    P.slice = slice_width
    return P


def toy_params() -> Params:
    """The worked dtANS example of Sec. IV-D: K = 8, W = 4 (2-bit words), M = 4,
    l = 2 slots from o = 3 words, f = 2 checks, one symbol per item."""
    P = Params()
    P.logK, P.logW, P.M, P.l, P.o, P.f, P.spi = 3, 2, 4, 2, 3, 2, 1
    P.raw_words[0], P.raw_words[1] = 0, 0
    P.raw_bits[0], P.raw_bits[1] = 64, 64
    P.slice = 1
    return P


# ---------------------------------------------------------------------------
# tables
# ---------------------------------------------------------------------------

class Table:
    """One domain's coding table; numpy views of the slot arrays."""

    def __init__(self, K: int):
        self.K = K
        self.kept_key = np.zeros(K, np.uint64)
        self.kept_first = np.zeros(K, np.uint32)
        self.kept_mult = np.zeros(K, np.uint32)
        self.slot_key = np.zeros(K, np.uint64)
        self.slot_digit = np.zeros(K, np.uint32)
        self.slot_base = np.zeros(K, np.uint32)
        self.slot_kind = np.zeros(K, np.uint8)
        self.c = _Table()
        self._bind()

    def _bind(self):
        c = self.c
        c.kept_key, c.kept_first, c.kept_mult = (self.kept_key.ctypes.data, self.kept_first.ctypes.data,
                                                 self.kept_mult.ctypes.data)
        c.slot_key, c.slot_digit, c.slot_base, c.slot_kind = (self.slot_key.ctypes.data,
                                                              self.slot_digit.ctypes.data,
                                                              self.slot_base.ctypes.data,
                                                              self.slot_kind.ctypes.data)

    @property
    def nkept(self):
        return int(self.c.nkept)

    @property
    def has_esc(self):
        return bool(self.c.has_esc)

    @property
    def cost_bits(self):
        return float(self.c.cost_bits)

    @property
    def esc_mult(self):
        return int(self.c.esc_mult)

    @property
    def pad_esc(self):
        return bool(self.c.pad_esc)

    def multiplicities(self):
        """{key: m} for kept symbols, plus 'ESC' when present."""
        d = {int(self.kept_key[i]): int(self.kept_mult[i]) for i in range(self.nkept)}
        if self.has_esc:
            d["ESC"] = self.esc_mult
        return d

    @staticmethod
    def explicit(P: Params, layout):
        """A table given slot by slot: layout = [(key, multiplicity), ...] in slot
        order (used for the paper's worked example, whose table is printed)."""
        K = 1 << P.logK
        t = Table(K)
        slot = 0
        for i, (key, m) in enumerate(layout):
            t.kept_key[i], t.kept_first[i], t.kept_mult[i] = key, slot, m
            for dg in range(m):
                t.slot_key[slot], t.slot_digit[slot], t.slot_base[slot], t.slot_kind[slot] = key, dg, m, 1
                slot += 1
        t.c.nkept = len(layout)
        t.c.has_esc, t.c.pad_esc = 0, 0
        t.c.pad_key = layout[0][0]
        return t


def build_table(P: Params, dom: int, keys, counts) -> Table:
    keys = np.ascontiguousarray(keys, np.uint64)
    counts = np.ascontiguousarray(counts, np.uint64)
    t = Table(1 << P.logK)
    rc = lib().or_build_table(C.byref(P), dom, len(keys), _p(keys), _p(counts), C.byref(t.c))
    if rc != 0:
        raise RuntimeError(f"or_build_table failed: {rc}")
    return t


def entropy(counts) -> float:
    c = np.ascontiguousarray(counts, np.uint64)
    return lib().or_entropy(len(c), _p(c))


def cross_entropy(counts, q) -> float:
    c = np.ascontiguousarray(counts, np.uint64)
    qq = np.ascontiguousarray(q, np.float64)
    return lib().or_cross_entropy(len(c), _p(c), _p(qq))


# ---------------------------------------------------------------------------
# plain strings (worked example)
# ---------------------------------------------------------------------------

def encode_string(P: Params, table: Table, syms):
    syms = np.ascontiguousarray(syms, np.uint64)
    ips = P.l // P.spi
    nseg = (len(syms) + ips - 1) // ips
    cap = P.o + nseg * (P.o + 2 * P.l) + 4
    body = np.zeros(cap, np.uint32)
    flags = np.zeros(max(1, nseg * P.f), np.uint8)
    nb = lib().or_encode_string(C.byref(P), C.byref(table.c), len(syms), _p(syms), _p(body), cap, _p(flags))
    if nb < 0:
        raise RuntimeError(f"or_encode_string failed: {nb}")
    return body[:nb].copy(), flags[: nseg * P.f].reshape(nseg, P.f).copy()


def decode_string(P: Params, table: Table, stream, n: int):
    stream = np.ascontiguousarray(stream, np.uint32)
    out = np.zeros(max(1, n * P.spi), np.uint64)
    n_out = np.zeros(1, np.int64)
    used = lib().or_decode_string(C.byref(P), C.byref(table.c), _p(stream), len(stream), _p(out), _p(n_out))
    if used < 0:
        raise RuntimeError("corrupt stream")
    return out[: int(n_out[0]) * P.spi].copy(), int(used)


# ---------------------------------------------------------------------------
# matrices
# ---------------------------------------------------------------------------

def value_keys(vals: np.ndarray) -> np.ndarray:
    """FP64 / FP32 values as their bit patterns (u64; FP32 zero-extended)."""
    vals = np.ascontiguousarray(vals)
    if vals.dtype == np.float64:
        return vals.view(np.uint64).copy()
    if vals.dtype == np.float32:
        return vals.view(np.uint32).astype(np.uint64)
    raise TypeError(vals.dtype)


def keys_to_values(keys: np.ndarray, dtype) -> np.ndarray:
    if np.dtype(dtype) == np.float64:
        return keys.astype(np.uint64).view(np.float64)
    return keys.astype(np.uint32).view(np.float32)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """First n outputs of the slot permutation's generator (SplitMix64)."""
    out = np.zeros(max(n, 1), np.uint64)
    lib().or_splitmix64_seq(seed, n, _p(out))
    return out[:n]


def layout(row_ptr, unit_max_nnz: int = 0, row_order: int = 0, order_window: int = 0):
    rp = np.ascontiguousarray(row_ptr, np.int64)
    m = len(rp) - 1
    nu = lib().or_layout(m, _p(rp), unit_max_nnz, row_order, order_window, None, None, None)
    ur, us, ul = (np.zeros(max(nu, 1), np.int64) for _ in range(3))
    lib().or_layout(m, _p(rp), unit_max_nnz, row_order, order_window, _p(ur), _p(us), _p(ul))
    return ur[:nu], us[:nu], ul[:nu]


def sort_rows(row_ptr, cols, vals):
    """Each row's entries by ascending column (stable for duplicates)."""
    rp = np.ascontiguousarray(row_ptr, np.int64)
    c = np.ascontiguousarray(cols, np.uint32)
    k = value_keys(vals)
    cs = np.zeros(max(len(c), 1), np.uint32)
    ks = np.zeros(max(len(c), 1), np.uint64)
    lib().or_sort_rows(len(rp) - 1, _p(rp), _p(c), _p(k), _p(cs), _p(ks))
    return cs[: len(c)], keys_to_values(ks[: len(c)], vals.dtype)


class Encoded:
    """Oracle-side CSR-dtANS encoding of one matrix."""


def encode_matrix(row_ptr, cols, vals, n: int, unit_max_nnz: int = 0, row_order: int = 0,
                  slice_width: int = 32, perm_seeds=(0, 0), first_delta: int = 0, chain: int = 1,
                  escape_stream: int = 0, order_window: int = 0, params: Params | None = None) -> Encoded:
    """first_delta 0: a unit's first delta is its absolute column (Sec. IV-A);
    1: the column minus the unit's row, modulo 2^32 (an option, not the
    paper's format).  chain > 1: each lane's units of `chain` consecutive
    slices form one dtANS sequence (an option: the paper's format is one
    sequence per unit).  escape_stream = 1: the escape points' raw words go
    to a separate array (E.esc_words, E.esc_off per slice), the alternative
    the paper describes in Sec. IV-F.  order_window > 0 with row_order = 1
    orders rows by unit length only within consecutive blocks of that many
    rows (an option; 0 orders all rows together).  params (default: the
    CSR-dtANS parameters of csr_params) runs the same encoder with other
    (K, W, M, l, o, f); it must alternate (delta, value) symbols (spi = 2),
    and its raw word counts must match the value type."""
    vals = np.ascontiguousarray(vals)
    vbits = 64 if vals.dtype == np.float64 else 32
    P = csr_params(vbits, slice_width) if params is None else params
    rp = np.ascontiguousarray(row_ptr, np.int64)
    c = np.ascontiguousarray(cols, np.uint32)
    k = value_keys(vals)
    K = 1 << P.logK
    tD, tV = Table(K), Table(K)
    permD = np.zeros(K, np.uint32)
    permV = np.zeros(K, np.uint32)
    err = C.c_int32(0)
    h = lib().or_encode_matrix(C.byref(P), len(rp) - 1, n, _p(rp), _p(c), _p(k), unit_max_nnz, row_order,
                               int(order_window), int(first_delta), int(chain), int(escape_stream), C.byref(tD.c), C.byref(tV.c), perm_seeds[0], perm_seeds[1], _p(permD),
                               _p(permV), C.byref(err))
    if not h:
        raise RuntimeError(f"or_encode_matrix failed: {err.value}")
    L = lib()
    try:
        g = [L.or_matrix_get(h, i) for i in range(9)]
        m_, n_, nnz, nu, ns, nw, SD, SV, ne = g
        E = Encoded()
        E.P, E.dtype, E.m, E.n, E.nnz, E.nunits, E.nslices, E.nwords = P, vals.dtype, m_, n_, nnz, nu, ns, nw
        E.words = np.zeros(max(nw, 1), np.uint32)
        E.slice_off = np.zeros(ns + 1, np.int64)
        arrs = [np.zeros(max(nu, 1), np.int64) for _ in range(7)]
        L.or_matrix_copy(h, _p(E.words), _p(E.slice_off), *[_p(a) for a in arrs])
        E.words = E.words[:nw]
        E.esc_words = np.zeros(max(ne, 1), np.uint32)
        E.esc_off = np.zeros(ns + 1, np.int64)
        L.or_matrix_copy_esc(h, _p(E.esc_words), _p(E.esc_off))
        E.esc_words = E.esc_words[:ne]
        (E.unit_row, E.unit_start, E.unit_len, E.unit_words, E.unit_loads, E.unit_extr,
         E.unit_raw) = [a[:nu] for a in arrs]
        E.hist = []
        for dom, S in ((0, SD), (1, SV)):
            hk = np.zeros(max(S, 1), np.uint64)
            hc = np.zeros(max(S, 1), np.uint64)
            L.or_matrix_hist(h, dom, _p(hk), _p(hc))
            E.hist.append((hk[:S], hc[:S]))
    finally:
        L.or_matrix_free(h)
    E.tabD, E.tabV = tD, tV
    E.permD = permD if perm_seeds[0] else None
    E.permV = permV if perm_seeds[1] else None
    E.unit_max_nnz, E.row_order, E.first_delta, E.chain = unit_max_nnz, row_order, int(first_delta), int(chain)
    E.order_window = int(order_window)
    E.escape_stream = int(escape_stream)
    return E


def _inverse(p):
    if p is None:
        return None
    inv = np.zeros_like(p)
    inv[p] = np.arange(len(p), dtype=p.dtype)
    return inv


def decode_units(E: Encoded, words=None, slice_off=None, s0: int = 0, s1: int | None = None, esc_words=None,
                 esc_off=None):
    """Decodes slices [s0, s1) from (words, slice_off) -- and, for a separate
    escape stream, (esc_words, esc_off) -- with E's tables.
    Returns (n per unit, deltas, value keys) in unit order."""
    words = E.words if words is None else np.ascontiguousarray(words, np.uint32)
    slice_off = E.slice_off if slice_off is None else np.ascontiguousarray(slice_off, np.int64)
    esc = getattr(E, "escape_stream", 0)
    esc_words = (E.esc_words if esc_words is None else np.ascontiguousarray(esc_words, np.uint32)) if esc else None
    esc_off = (E.esc_off if esc_off is None else np.ascontiguousarray(esc_off, np.int64)) if esc else None
    s1 = E.nslices if s1 is None else s1
    u0, u1 = s0 * E.P.slice, min(s1 * E.P.slice, E.nunits)
    cap = int(E.unit_len[u0:u1].sum()) if u1 > u0 else 0
    out_n = np.zeros(max(u1 - u0, 1), np.int64)
    out_sym = np.zeros(max(2 * cap, 2), np.uint64)
    pD, pV = _inverse(E.permD), _inverse(E.permV)
    rc = lib().or_decode_slices(C.byref(E.P), C.byref(E.tabD.c), C.byref(E.tabV.c), _p(pD), _p(pV),
                                _p(words), _p(slice_off), E.nunits, s0, s1, int(getattr(E, "chain", 1)),
                                _p(esc_words) if esc else None, _p(esc_off) if esc else None, _p(out_n),
                                _p(out_sym), cap)
    if rc != 0:
        raise RuntimeError(f"or_decode_slices failed: {rc}")
    syms = out_sym[: 2 * cap]
    return out_n[: u1 - u0], syms[0::2].copy(), syms[1::2].copy()


def decode_matrix(E: Encoded, words=None, slice_off=None, esc_words=None, esc_off=None):
    """Full decode back to CSR (rows sorted by column): (row_ptr, cols, vals).
    A unit's columns are the running sums of its deltas (the first delta is
    absolute, Sec. IV-A), taken modulo 2^32 as the deltas are 32-bit words;
    with first_delta = 1 the running sum starts at the unit's row."""
    n_u, deltas, vkeys = decode_units(E, words, slice_off, esc_words=esc_words, esc_off=esc_off)
    m = E.m
    row_len = np.zeros(m, np.int64)
    np.add.at(row_len, E.unit_row, n_u)
    row_ptr = np.zeros(m + 1, np.int64)
    np.cumsum(row_len, out=row_ptr[1:])
    total = int(n_u.sum())
    run = np.cumsum(deltas.astype(np.uint64))
    ustart = np.zeros(len(n_u), np.int64)
    np.cumsum(n_u[:-1], out=ustart[1:])
    if total:
        before = np.where(ustart > 0, run[np.maximum(ustart - 1, 0)], np.uint64(0))
    else:
        before = np.zeros(len(n_u), np.uint64)
    start = np.repeat(E.unit_row.astype(np.uint64), n_u) if getattr(E, "first_delta", 0) else np.uint64(0)
    cols_u = ((run - np.repeat(before, n_u) + start) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    dest = np.repeat(row_ptr[E.unit_row] + E.unit_start - ustart, n_u) + np.arange(total)
    cols = np.zeros(total, np.uint32)
    vk = np.zeros(total, np.uint64)
    cols[dest] = cols_u
    vk[dest] = vkeys
    return row_ptr, cols, keys_to_values(vk, E.dtype)


# ---------------------------------------------------------------------------
# products
# ---------------------------------------------------------------------------

def spmm_ref(row_ptr, cols, vals, X, beta: float = 0.0, Y=None):
    """Y = A X + beta Y with Dot2 compensated sums; returns (Y, sum |a x|)."""
    rp = np.ascontiguousarray(row_ptr, np.int64)
    c = np.ascontiguousarray(cols, np.uint32)
    v = np.ascontiguousarray(vals, np.float64)
    X = np.asarray(X, np.float64)
    vec = X.ndim == 1
    X2 = np.ascontiguousarray(X.reshape(X.shape[0], -1))
    m, k = len(rp) - 1, X2.shape[1]
    Yin = np.ascontiguousarray(np.asarray(Y, np.float64).reshape(m, k)) if (Y is not None and beta != 0) else None
    out = np.zeros((m, k), np.float64)
    ab = np.zeros((m, k), np.float64)
    lib().or_spmm_ref(m, _p(rp), _p(c), _p(v), k, _p(X2), float(beta), _p(Yin), _p(out), _p(ab))
    return (out[:, 0], ab[:, 0]) if vec else (out, ab)


def spmm_t_ref(row_ptr, cols, vals, n: int, G, beta: float = 0.0, XG=None):
    """XG = A^T G + beta XG with compensated sums; returns (XG, sum |a g|)."""
    rp = np.ascontiguousarray(row_ptr, np.int64)
    c = np.ascontiguousarray(cols, np.uint32)
    v = np.ascontiguousarray(vals, np.float64)
    G = np.asarray(G, np.float64)
    vec = G.ndim == 1
    G2 = np.ascontiguousarray(G.reshape(G.shape[0], -1))
    m, k = len(rp) - 1, G2.shape[1]
    Xin = np.ascontiguousarray(np.asarray(XG, np.float64).reshape(n, k)) if (XG is not None and beta != 0) else None
    out = np.zeros((n, k), np.float64)
    ab = np.zeros((n, k), np.float64)
    lib().or_spmm_t_ref(m, n, _p(rp), _p(c), _p(v), k, _p(G2), float(beta), _p(Xin), _p(out), _p(ab))
    return (out[:, 0], ab[:, 0]) if vec else (out, ab)


def vals_grad_ref(row_ptr, cols, G, X):
    """vals_grad[q] = sum_b G[i, b] X[j, b] per stored entry q = (i, j)."""
    rp = np.ascontiguousarray(row_ptr, np.int64)
    c = np.ascontiguousarray(cols, np.uint32)
    G2 = np.ascontiguousarray(np.asarray(G, np.float64).reshape(len(rp) - 1, -1))
    k = G2.shape[1]
    X2 = np.ascontiguousarray(np.asarray(X, np.float64).reshape(-1, k))
    out = np.zeros(max(len(c), 1), np.float64)
    ab = np.zeros(max(len(c), 1), np.float64)
    lib().or_vals_grad_ref(len(rp) - 1, _p(rp), _p(c), k, _p(G2), _p(X2), _p(out), _p(ab))
    return out[: len(c)], ab[: len(c)]


def codebook_grad_ref(row_ptr, cols, vals, codebook, G, X):
    """Gradient of L = sum(G .* (A X)) with respect to the codebook values of
    a weight-shared matrix: entry r is the sum, over the stored entries
    q = (i, j) whose value has the bit pattern of codebook[r], of
    d L / d a_q = sum_b G[i, b] X[j, b]; a last entry collects the stored
    entries that match no codebook value (escaped values).  cols and vals in
    the same (sorted-CSR) order.  Per-entry products come from vals_grad_ref
    (compensated), the per-value sums from math.fsum (correctly rounded).
    Returns (grad[T + 1], sum of |G X| per entry of grad)."""
    import math
    p, ab = vals_grad_ref(row_ptr, cols, G, X)
    keys = value_keys(np.asarray(vals))
    ck = value_keys(np.asarray(codebook))
    T = len(ck)
    bins = np.full(len(keys), T, np.int64)
    for r in range(T):
        bins[keys == ck[r]] = r
    grad = np.array([math.fsum(p[bins == r]) for r in range(T + 1)])
    absum = np.array([math.fsum(ab[bins == r]) for r in range(T + 1)])
    return grad, absum


def dense_spmv(row_ptr, cols, vals, n: int, x):
    rp = np.ascontiguousarray(row_ptr, np.int64)
    c = np.ascontiguousarray(cols, np.uint32)
    v = np.ascontiguousarray(vals, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    y = np.zeros(max(len(rp) - 1, 1), np.float64)
    lib().or_dense_spmv(len(rp) - 1, n, _p(rp), _p(c), _p(v), _p(x), _p(y))
    return y[: len(rp) - 1]
