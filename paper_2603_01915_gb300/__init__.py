"""CSR-dtANS on GB300: Python binding of the C-ABI library ``libdtans.so``.

The binding only marshals arguments: every step of the encoder runs in the
library's C++ host code and every step of the products runs in its CUDA
kernels (sm_103a).  The entry points keep the C names (``dtans_encode``,
``dtans_spmv``, ...); ``Matrix`` wraps a handle and ``CompressedLinear`` is the
torch.autograd.Function around the compressed operator.  There is no CPU
fallback: if the library is missing or was built for another architecture,
loading fails with an error.
"""
from __future__ import annotations

import ctypes as C
import functools
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_CSRC = os.path.join(_HERE, "csrc")
_INC = os.path.join(_ROOT, "include")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "libdtans.so")

ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
              "--expt-relaxed-constexpr", "-I", _INC, "-I", _CSRC]

DTANS_F32, DTANS_F64 = 1, 2
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_ALLOC", -3: "ERR_CUDA", -4: "ERR_CORRUPT", -5: "ERR_UNSUPPORTED",
          -6: "ERR_IO", -7: "ERR_STATE"}


def _sources():
    return sorted(os.path.join(_CSRC, f) for f in os.listdir(_CSRC) if f.endswith((".cu", ".cpp")))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles the library for sm_103a (one translation unit per nvcc job, in parallel)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = _sources()
    deps = srcs + [os.path.join(_CSRC, f) for f in os.listdir(_CSRC) if f.endswith((".h", ".cuh"))] + \
        [os.path.join(_INC, "dtans.h")]
    if not force and os.path.exists(LIB_PATH):
        t = os.path.getmtime(LIB_PATH)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB_PATH
    nvcc = os.environ.get("NVCC", "nvcc")

    def compile_one(src):
        obj = os.path.join(_BUILD, os.path.basename(src) + ".o")
        cmd = [nvcc] + ARCH_FLAGS + NVCC_FLAGS + ["-c", src, "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose:
        for _, err in results:
            if err:
                print(err)
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH_FLAGS + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


BASELINE_LIB_PATH = os.path.join(_BUILD, "libdtans_cusparse.so")


def build_baseline(force: bool = False) -> str:
    """Compiles the measurement helpers used by bench.py (not part of the
    library): the cuSPARSE baselines and the ceiling microbenchmarks."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, "csrc_baseline", f) for f in ("cusparse_baseline.cpp", "ceilings.cu")]
    if not force and os.path.exists(BASELINE_LIB_PATH) and \
            os.path.getmtime(BASELINE_LIB_PATH) >= max(os.path.getmtime(s) for s in srcs):
        return BASELINE_LIB_PATH
    tmp = BASELINE_LIB_PATH + f".tmp{os.getpid()}"
    cmd = [os.environ.get("NVCC", "nvcc")] + ARCH_FLAGS + ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                                                           "-o", tmp] + srcs + ["-lcusparse"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for the cuSPARSE baseline:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, BASELINE_LIB_PATH)
    return BASELINE_LIB_PATH


# ---------------------------------------------------------------------------
# ctypes declarations (mirror include/dtans.h)
# ---------------------------------------------------------------------------

class EncodeOpts(C.Structure):
    _fields_ = [("unit_max_nnz", C.c_int32), ("row_order", C.c_int32), ("perm_seed_delta", C.c_uint64),
                ("perm_seed_value", C.c_uint64), ("num_threads", C.c_int32), ("first_delta", C.c_int32),
                ("chain_slices", C.c_int32), ("escape_stream", C.c_int32), ("order_window", C.c_int32),
                ("reserved", C.c_int32 * 3)]


class Info(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("nnz", C.c_int64), ("nunits", C.c_int64),
                ("nslices", C.c_int64), ("nwords", C.c_int64), ("bytes_words", C.c_int64),
                ("bytes_slice_off", C.c_int64), ("bytes_tables", C.c_int64), ("bytes_unit_meta", C.c_int64),
                ("bytes_compressed", C.c_int64), ("kept_delta", C.c_int64), ("kept_value", C.c_int64),
                ("esc_delta", C.c_int32), ("esc_value", C.c_int32), ("dtype", C.c_int32), ("uploaded", C.c_int32),
                ("cost_bits_delta", C.c_double), ("cost_bits_value", C.c_double), ("unit_max_nnz", C.c_int32),
                ("row_order", C.c_int32), ("grid", C.c_int32), ("block", C.c_int32), ("first_delta", C.c_int32),
                ("warps", C.c_int32), ("chain_slices", C.c_int32), ("escape_stream", C.c_int32),
                ("nesc", C.c_int64), ("bytes_esc", C.c_int64), ("tile_policy", C.c_int32),
                ("order_window", C.c_int32), ("int_coefficients", C.c_int32), ("int_exp", C.c_int32),
                ("accumulate", C.c_int32), ("scatter", C.c_int32), ("int_products", C.c_int32)]


class View(C.Structure):
    _fields_ = [("words", C.c_void_p), ("slice_off", C.c_void_p), ("unit_row", C.c_void_p),
                ("unit_len", C.c_void_p), ("unit_pos", C.c_void_p), ("slot_key", C.c_void_p * 2),
                ("slot_digit", C.c_void_p * 2), ("slot_base", C.c_void_p * 2), ("slot_kind", C.c_void_p * 2),
                ("perm", C.c_void_p * 2), ("esc_words", C.c_void_p), ("esc_off", C.c_void_p)]


EXPORTS = ["dtans_encode", "dtans_upload", "dtans_spmv", "dtans_spmm", "dtans_spmv_T", "dtans_vals_grad",
           "dtans_decode_csr", "dtans_info", "dtans_view", "dtans_check", "dtans_save", "dtans_load",
           "dtans_set_launch", "dtans_destroy", "dtans_last_error", "dtans_batch_create", "dtans_batch_bind",
           "dtans_batch_spmv", "dtans_batch_destroy", "dtans_tune", "dtans_spmv_noalloc", "dtans_codebook",
           "dtans_set_codebook", "dtans_codebook_grad", "dtans_set_warps", "dtans_tune_warps",
           "dtans_set_tile_policy", "dtans_spmv_host", "dtans_set_accumulate",
           "dtans_set_scatter"]

TUNE_MAX = 64


class TuneOpts(C.Structure):
    _fields_ = [("k", C.c_int32), ("reps", C.c_int32), ("num_threads", C.c_int32), ("n_candidates", C.c_int32),
                ("unit_max_nnz", C.c_int32 * TUNE_MAX), ("row_order", C.c_int32 * TUNE_MAX),
                ("first_delta", C.c_int32 * TUNE_MAX), ("first_delta_default", C.c_int32),
                ("order_window", C.c_int32 * TUNE_MAX)]


class TuneReport(C.Structure):
    _fields_ = [("n", C.c_int32), ("best", C.c_int32), ("unit_max_nnz", C.c_int32 * TUNE_MAX),
                ("row_order", C.c_int32 * TUNE_MAX), ("first_delta", C.c_int32 * TUNE_MAX),
                ("warps", C.c_int32 * TUNE_MAX), ("tile_policy", C.c_int32 * TUNE_MAX),
                ("ms", C.c_double * TUNE_MAX), ("order_window", C.c_int32 * TUNE_MAX)]

_lib = None


def lib(path: str | None = None):
    """Loads libdtans.so (building it first if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or build()
    L = C.CDLL(p)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    st = C.c_int
    sig = {
        "dtans_encode": (st, [i64, i64, vp, vp, vp, i32, C.POINTER(EncodeOpts), C.POINTER(vp)]),
        "dtans_upload": (st, [vp, vp]),
        "dtans_spmv": (st, [vp, vp, vp, dbl, vp]),
        "dtans_spmv_noalloc": (st, [vp, vp, vp, dbl, vp]),
        "dtans_spmv_host": (st, [vp, vp, vp, dbl, vp]),
        "dtans_spmm": (st, [vp, i32, vp, vp, dbl, vp]),
        "dtans_spmv_T": (st, [vp, i32, vp, vp, dbl, vp]),
        "dtans_vals_grad": (st, [vp, i32, vp, vp, vp, vp]),
        "dtans_decode_csr": (st, [vp, vp, vp, vp]),
        "dtans_codebook": (st, [vp, vp]),
        "dtans_set_codebook": (st, [vp, vp, vp]),
        "dtans_codebook_grad": (st, [vp, i32, vp, vp, vp, vp]),
        "dtans_info": (st, [vp, C.POINTER(Info)]),
        "dtans_view": (st, [vp, C.POINTER(View)]),
        "dtans_check": (st, [vp, vp]),
        "dtans_save": (st, [vp, C.c_char_p]),
        "dtans_load": (st, [C.c_char_p, C.POINTER(vp)]),
        "dtans_set_launch": (st, [vp, i32, i32]),
        "dtans_set_warps": (st, [vp, i32]),
        "dtans_set_tile_policy": (st, [vp, i32]),
        "dtans_set_accumulate": (st, [vp, i32]),
        "dtans_set_scatter": (st, [vp, i32]),
        "dtans_tune_warps": (st, [vp, i32, C.POINTER(i32), C.POINTER(dbl), vp]),
        "dtans_destroy": (None, [vp]),
        "dtans_last_error": (C.c_char_p, []),
        "dtans_batch_create": (st, [vp, i32, C.POINTER(vp)]),
        "dtans_batch_bind": (st, [vp, vp, vp]),
        "dtans_batch_spmv": (st, [vp, dbl, vp]),
        "dtans_batch_destroy": (None, [vp]),
        "dtans_tune": (st, [i64, i64, vp, vp, vp, i32, C.POINTER(TuneOpts), C.POINTER(vp), C.POINTER(TuneReport),
                            vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    _lib = L
    return L


class DtansError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(status: int):
    if status != 0:
        raise DtansError(status, lib().dtans_last_error().decode(errors="replace"))


def _ptr(t) -> C.c_void_p:
    """Device or host address of a torch tensor or numpy array (no copies)."""
    if t is None:
        return C.c_void_p(0)
    if isinstance(t, np.ndarray):
        return C.c_void_p(t.ctypes.data)
    return C.c_void_p(t.data_ptr())


def _stream(stream=None) -> C.c_void_p:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------
# C entry points with the same names
# ---------------------------------------------------------------------------

def dtans_encode(row_ptr, col_idx, vals, m: int, n: int, unit_max_nnz: int = 0, row_order: int = 0,
                 perm_seeds=(0, 0), num_threads: int = 0, first_delta: int = 0, chain: int = 1,
                 escape_stream: int = 0, order_window: int = 0) -> C.c_void_p:
    rp = np.ascontiguousarray(row_ptr, np.int64)
    ci = np.ascontiguousarray(col_idx, np.uint32)
    v = np.ascontiguousarray(vals)
    if v.dtype == np.float64:
        dt = DTANS_F64
    elif v.dtype == np.float32:
        dt = DTANS_F32
    else:
        raise TypeError(f"values must be float32 or float64, not {v.dtype}")
    o = EncodeOpts(unit_max_nnz, row_order, perm_seeds[0], perm_seeds[1], num_threads, first_delta, chain,
                   escape_stream, order_window)
    h = C.c_void_p()
    _check(lib().dtans_encode(m, n, _ptr(rp), _ptr(ci), _ptr(v), dt, C.byref(o), C.byref(h)))
    return h


def dtans_upload(h, stream=None):
    _check(lib().dtans_upload(h, _stream(stream)))


def dtans_spmv(h, x, y, beta: float = 0.0, stream=None):
    _check(lib().dtans_spmv(h, _ptr(x), _ptr(y), float(beta), _stream(stream)))


def dtans_spmm(h, k: int, X, Y, beta: float = 0.0, stream=None):
    _check(lib().dtans_spmm(h, k, _ptr(X), _ptr(Y), float(beta), _stream(stream)))


def dtans_spmv_T(h, k: int, G, XG, beta: float = 0.0, stream=None):
    _check(lib().dtans_spmv_T(h, k, _ptr(G), _ptr(XG), float(beta), _stream(stream)))


def dtans_vals_grad(h, k: int, G, X, out, stream=None):
    _check(lib().dtans_vals_grad(h, k, _ptr(G), _ptr(X), _ptr(out), _stream(stream)))


def dtans_decode_csr(h, cols_out, vals_out, stream=None):
    _check(lib().dtans_decode_csr(h, _ptr(cols_out), _ptr(vals_out), _stream(stream)))


def dtans_codebook(h, values):
    _check(lib().dtans_codebook(h, _ptr(values)))


def dtans_set_codebook(h, values, stream=None):
    _check(lib().dtans_set_codebook(h, _ptr(values), _stream(stream) if _has_torch_cuda() else C.c_void_p(0)))


def dtans_codebook_grad(h, k: int, G, X, out, stream=None):
    _check(lib().dtans_codebook_grad(h, k, _ptr(G), _ptr(X), _ptr(out), _stream(stream)))


def _has_torch_cuda() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except ImportError:
        return False


def _host_ptr(a):
    """Address of a contiguous host buffer (numpy array or CPU tensor)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host buffer must be contiguous")
        return C.c_void_p(a.ctypes.data)
    if a.is_cuda or not a.is_contiguous():
        raise ValueError("host buffer must be a contiguous CPU tensor")
    return C.c_void_p(a.data_ptr())


def dtans_spmv_host(h, x_ptr, y_ptr, beta: float = 0.0, stream=None):
    _check(lib().dtans_spmv_host(h, x_ptr, y_ptr, float(beta), _stream(stream)))


def dtans_info(h) -> Info:
    inf = Info()
    _check(lib().dtans_info(h, C.byref(inf)))
    return inf


def dtans_check(h, stream=None):
    _check(lib().dtans_check(h, _stream(stream)))


def dtans_save(h, path: str):
    _check(lib().dtans_save(h, path.encode()))


def dtans_load(path: str) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib().dtans_load(path.encode(), C.byref(h)))
    return h


def dtans_set_launch(h, grid: int, block: int):
    _check(lib().dtans_set_launch(h, grid, block))


def dtans_set_accumulate(h, mode: int):
    _check(lib().dtans_set_accumulate(h, mode))


def dtans_set_warps(h, warps: int):
    _check(lib().dtans_set_warps(h, warps))


def dtans_tune_warps(h, reps: int = 5, stream=None):
    """Times the single-vector product per warp count, keeps the fastest on
    the handle; returns (warps, {warps: median ms})."""
    best = C.c_int32(0)
    ms = (C.c_double * 4)()
    _check(lib().dtans_tune_warps(h, reps, C.byref(best), ms, _stream(stream)))
    return best.value, dict(zip((20, 24, 28, 32), list(ms)))


def dtans_destroy(h):
    lib().dtans_destroy(h)


def dtans_view(h) -> dict:
    """Copies of the handle's host-side stream and canonical tables (numpy)."""
    inf = dtans_info(h)
    v = View()
    _check(lib().dtans_view(h, C.byref(v)))

    def arr(p, ctype, count, dtype):
        if count == 0 or not p:
            return np.zeros(0, dtype)
        return np.ctypeslib.as_array(C.cast(p, C.POINTER(ctype)), shape=(count,)).astype(dtype, copy=True)

    K = 4096
    out = dict(words=arr(v.words, C.c_uint32, inf.nwords, np.uint32),
               slice_off=arr(v.slice_off, C.c_uint64, inf.nslices + 1, np.uint64),
               unit_row=arr(v.unit_row, C.c_uint32, inf.nunits, np.uint32),
               unit_len=arr(v.unit_len, C.c_uint32, inf.nunits, np.uint32),
               unit_pos=arr(v.unit_pos, C.c_uint64, inf.nunits, np.uint64),
               esc_words=arr(v.esc_words, C.c_uint32, inf.nesc, np.uint32) if v.esc_off else None,
               esc_off=arr(v.esc_off, C.c_uint64, inf.nslices + 1, np.uint64) if v.esc_off else None)
    for d, name in ((0, "delta"), (1, "value")):
        out[f"{name}_key"] = arr(v.slot_key[d], C.c_uint64, K, np.uint64)
        out[f"{name}_digit"] = arr(v.slot_digit[d], C.c_uint16, K, np.uint16)
        out[f"{name}_base"] = arr(v.slot_base[d], C.c_uint16, K, np.uint16)
        out[f"{name}_kind"] = arr(v.slot_kind[d], C.c_uint8, K, np.uint8)
        out[f"{name}_perm"] = arr(v.perm[d], C.c_uint32, K, np.uint32) if v.perm[d] else None
    return out


# ---------------------------------------------------------------------------
# Matrix: an encoded matrix on the device
# ---------------------------------------------------------------------------

class Matrix:
    """A CSR-dtANS matrix: host encode at construction, device upload on demand.

    Encoder options (fields of dtans_encode_opts; all zero is the paper's
    canonical format): unit_max_nnz splits rows longer than it into units;
    row_order = 1 orders rows by their longest unit, within blocks of
    order_window rows when that is > 0; first_delta = 1 stores a unit's first
    delta relative to its row; chain > 1 chains each lane's units over that
    many slices; escape_stream = 1 moves escaped raw words to their own
    array; perm_seeds permute the used table slots.
    """

    def __init__(self, row_ptr, col_idx, vals, shape, unit_max_nnz: int = 0, row_order: int = 0,
                 perm_seeds=(0, 0), num_threads: int = 0, handle=None, first_delta: int = 0, chain: int = 1,
                 escape_stream: int = 0, order_window: int = 0):
        self.shape = tuple(int(s) for s in shape)
        if handle is not None:
            self.h = handle
        else:
            self.h = dtans_encode(row_ptr, col_idx, vals, self.shape[0], self.shape[1], unit_max_nnz, row_order,
                                  perm_seeds, num_threads, first_delta, chain, escape_stream, order_window)
        inf = dtans_info(self.h)
        self.dtype_code = inf.dtype
        self.nnz = int(inf.nnz)

    @classmethod
    def load(cls, path: str) -> "Matrix":
        h = dtans_load(path)
        inf = dtans_info(h)
        return cls(None, None, None, (inf.m, inf.n), handle=h)

    def save(self, path: str):
        dtans_save(self.h, path)

    @property
    def torch_dtype(self):
        import torch
        return torch.float64 if self.dtype_code == DTANS_F64 else torch.float32

    @property
    def info(self) -> Info:
        return dtans_info(self.h)

    def view(self) -> dict:
        return dtans_view(self.h)

    def cuda(self, stream=None) -> "Matrix":
        dtans_upload(self.h, stream)
        return self

    def _out(self, shape, like):
        import torch
        return torch.empty(shape, dtype=self.torch_dtype, device=like.device)

    def spmv(self, x, y=None, beta: float = 0.0, stream=None):
        if y is None:
            y = self._out((self.shape[0],), x)
        dtans_spmv(self.h, x, y, beta, stream)
        return y

    def spmv_host(self, x, y, beta: float = 0.0, stream=None, sync: bool = True):
        """y = A x + beta y with x and y in host memory (numpy arrays or CPU
        tensors of the matrix's type, contiguous; pinned memory lets
        consecutive calls overlap their copies with the products):
        dtans_spmv_host, which copies x in, multiplies and copies y out on the
        handle's own streams.  With sync=False the call returns once the work
        is enqueued and ``stream`` (default: the current stream) must be
        synchronized before y is read."""
        dtans_spmv_host(self.h, _host_ptr(x), _host_ptr(y), beta, stream)
        if sync:
            import torch
            (stream or torch.cuda.current_stream()).synchronize()
        return y

    def spmm(self, X, Y=None, beta: float = 0.0, stream=None):
        k = X.shape[1]
        if Y is None:
            Y = self._out((self.shape[0], k), X)
        dtans_spmm(self.h, k, X, Y, beta, stream)
        return Y

    def spmv_T(self, G, XG=None, beta: float = 0.0, stream=None):
        k = 1 if G.dim() == 1 else G.shape[1]
        if XG is None:
            XG = self._out((self.shape[1],) if G.dim() == 1 else (self.shape[1], k), G)
        dtans_spmv_T(self.h, k, G, XG, beta, stream)
        return XG

    def vals_grad(self, G, X, out=None, stream=None):
        k = 1 if G.dim() == 1 else G.shape[1]
        if out is None:
            out = self._out((self.nnz,), G)
        dtans_vals_grad(self.h, k, G, X, out, stream)
        return out

    @property
    def _np_dtype(self):
        return np.float64 if self.dtype_code == DTANS_F64 else np.float32

    def codebook(self) -> np.ndarray:
        """The kept value symbols c_0 .. c_{T-1} in the table's rank order."""
        out = np.zeros(int(self.info.kept_value), self._np_dtype)
        dtans_codebook(self.h, out)
        return out

    def set_codebook(self, values, stream=None):
        """Replaces the codebook (T values, rank order); no re-encoding."""
        v = np.ascontiguousarray(np.asarray(values, self._np_dtype))
        if v.shape != (int(self.info.kept_value),):
            raise ValueError(f"codebook must have {int(self.info.kept_value)} values")
        dtans_set_codebook(self.h, v, stream)

    def codebook_grad(self, G, X, out=None, stream=None):
        """d sum(G .* (A X)) / d c_r for r < T, and the escaped entries' sum at T."""
        k = 1 if G.dim() == 1 else G.shape[1]
        if out is None:
            out = self._out((int(self.info.kept_value) + 1,), G)
        dtans_codebook_grad(self.h, k, G, X, out, stream)
        return out

    def decode_csr(self, device="cuda", stream=None):
        import torch
        cols = torch.empty(self.nnz, dtype=torch.int32, device=device)
        vals = torch.empty(self.nnz, dtype=self.torch_dtype, device=device)
        dtans_decode_csr(self.h, cols, vals, stream)
        return cols, vals

    def check(self, stream=None):
        dtans_check(self.h, stream)

    # A^T as a second CSR-dtANS stream: the alternative to the atomic scatter
    # of dtans_spmv_T for x_grad = A^T g, attached when it measures faster.
    transpose = None

    def attach_transpose(self, MT: "Matrix"):
        if MT is not None and tuple(MT.shape) != (self.shape[1], self.shape[0]):
            raise ValueError("transpose has the wrong shape")
        self.transpose = MT

    def xgrad(self, G, XG=None, stream=None):
        """A^T G through the attached transposed stream if any, else dtans_spmv_T."""
        if self.transpose is None:
            return self.spmv_T(G, XG, stream=stream)
        if G.dim() == 1:
            return self.transpose.spmv(G, XG, stream=stream)
        return self.transpose.spmm(G, XG, stream=stream)

    def set_launch(self, grid: int, block: int):
        dtans_set_launch(self.h, grid, block)

    def set_warps(self, warps: int):
        dtans_set_warps(self.h, warps)

    def set_accumulate(self, mode: int):
        """0: FP64 fused multiply-adds (default); 1: exact integer-coefficient
        products where the value table allows them (dtans_set_accumulate)."""
        dtans_set_accumulate(self.h, mode)

    def set_scatter(self, mode: int):
        """x_grad scatter of spmv_T: 0 one atomic per entry (default), 1
        warp-aggregated atomics (dtans_set_scatter)."""
        _check(lib().dtans_set_scatter(self.h, mode))

    def set_tile_policy(self, policy: int):
        _check(lib().dtans_set_tile_policy(self.h, policy))

    def tune_warps(self, reps: int = 5, stream=None):
        return dtans_tune_warps(self.h, reps, stream)

    def close(self):
        if getattr(self, "h", None):
            dtans_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dtans_tune(row_ptr, col_idx, vals, m: int, n: int, k: int = 1, reps: int = 5, candidates=None,
               num_threads: int = 0, stream=None, first_delta: int = 0):
    """Encodes one handle per candidate layout, times each on the device and
    returns (fastest uploaded handle, report as a list of dicts, best index).
    candidates: (U, row_order[, first_delta[, order_window]]) tuples; the
    default list uses first_delta (0, 1, or 2 = both)."""
    rp = np.ascontiguousarray(row_ptr, np.int64)
    ci = np.ascontiguousarray(col_idx, np.uint32)
    v = np.ascontiguousarray(vals)
    dt = DTANS_F64 if v.dtype == np.float64 else DTANS_F32
    o = TuneOpts()
    o.k, o.reps, o.num_threads, o.first_delta_default = k, reps, num_threads, first_delta
    if candidates:
        o.n_candidates = len(candidates)
        for i, c in enumerate(candidates):
            o.unit_max_nnz[i], o.row_order[i] = c[0], c[1]
            o.first_delta[i] = c[2] if len(c) > 2 else 0
            o.order_window[i] = c[3] if len(c) > 3 else 0
    rep = TuneReport()
    h = C.c_void_p()
    _check(lib().dtans_tune(m, n, _ptr(rp), _ptr(ci), _ptr(v), dt, C.byref(o), C.byref(h), C.byref(rep),
                            _stream(stream)))
    rows = [dict(unit_max_nnz=rep.unit_max_nnz[i], row_order=rep.row_order[i], first_delta=rep.first_delta[i],
                 order_window=rep.order_window[i], warps=rep.warps[i], tile_policy=rep.tile_policy[i],
                 ms=rep.ms[i]) for i in range(rep.n)]
    return h, rows, rep.best


def tune(row_ptr, col_idx, vals, shape, k: int = 1, reps: int = 5, candidates=None, stream=None,
         first_delta: int = 0):
    """Autotuned Matrix (already on the device) and the timing report."""
    h, rows, best = dtans_tune(row_ptr, col_idx, vals, shape[0], shape[1], k, reps, candidates, stream=stream,
                               first_delta=first_delta)
    return Matrix(None, None, None, shape, handle=h), rows, best


def transpose_csr(row_ptr, col_idx, vals, shape):
    """Host CSR of A^T (rows sorted by column), for a transposed stream."""
    rp = np.asarray(row_ptr, np.int64)
    ci = np.asarray(col_idx, np.int64)
    m, n = int(shape[0]), int(shape[1])
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(rp))
    order = np.lexsort((rows, ci))
    rpt = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(ci, minlength=n), out=rpt[1:])
    return rpt, rows[order].astype(np.uint32), np.asarray(vals)[order]


def choose_xgrad(A: "Matrix", AT: "Matrix", k: int, reps: int = 5):
    """Times x_grad = A^T G with k columns three ways: one atomic per entry
    over A's stream, warp-aggregated atomics over A's stream
    (dtans_set_scatter), and a multiply over A^T's stream.  Keeps the fastest
    on A (the scatter mode, and AT attached when the transposed stream wins).
    Returns (choice, {way: median ms})."""
    import torch
    dev = torch.device("cuda")
    G = torch.zeros((A.shape[0], k) if k > 1 else (A.shape[0],), dtype=A.torch_dtype, device=dev).uniform_(-1, 1)
    XG = torch.empty((A.shape[1], k) if k > 1 else (A.shape[1],), dtype=A.torch_dtype, device=dev)
    times = {}

    def scatter(mode):
        def fn():
            A.set_scatter(mode)
            A.spmv_T(G, XG)
        return fn

    ways = {"atomics": scatter(0), "aggregated": scatter(1),
            "transposed": (lambda: AT.spmm(G, XG)) if k > 1 else (lambda: AT.spmv(G, XG))}
    for way, fn in ways.items():
        for _ in range(2):
            fn()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        times[way] = sorted(ts)[len(ts) // 2]
    choice = min(times, key=times.get)
    A.set_scatter(1 if choice == "aggregated" else 0)
    A.attach_transpose(AT if choice == "transposed" else None)
    return choice, times


class Batch:
    """Many uploaded matrices multiplied in one persistent kernel launch."""

    def __init__(self, mats):
        self.mats = list(mats)
        arr = (C.c_void_p * len(self.mats))(*[m.h for m in self.mats])
        self.b = C.c_void_p()
        _check(lib().dtans_batch_create(arr, len(self.mats), C.byref(self.b)))

    def bind(self, xs, ys):
        xa = (C.c_void_p * len(xs))(*[t.data_ptr() for t in xs])
        ya = (C.c_void_p * len(ys))(*[t.data_ptr() for t in ys])
        _check(lib().dtans_batch_bind(self.b, xa, ya))
        self._keep = (xs, ys)

    def spmv(self, beta: float = 0.0, stream=None):
        _check(lib().dtans_batch_spmv(self.b, float(beta), _stream(stream)))

    def close(self):
        if getattr(self, "b", None):
            lib().dtans_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_encoded_values(A: Matrix, vals):
    """Raises ValueError unless ``vals`` equals A's encoded values (sorted-CSR
    order) bit for bit.  A tensor already checked at its current version is
    not decoded again."""
    import torch

    key = (vals.data_ptr(), vals._version, tuple(vals.shape), vals.dtype)
    if getattr(A, "_vals_checked", None) == key:
        return
    if vals.numel() != A.nnz:
        raise ValueError(f"vals has {vals.numel()} entries, the matrix stores {A.nnz}")
    _, enc = A.decode_csr()
    v = vals.detach().reshape(-1).to(device=enc.device, dtype=enc.dtype)
    ib = torch.int64 if enc.dtype == torch.float64 else torch.int32
    if not torch.equal(v.view(ib), enc.view(ib)):
        raise ValueError("vals differs from the values encoded in the matrix (the forward would not use it); "
                         "re-encode the matrix or train a codebook with CodebookLinear")
    A._vals_checked = key


@functools.lru_cache(maxsize=None)
def _autograd():
    import torch

    class CompressedLinear(torch.autograd.Function):
        """Y = A X for a CSR-dtANS matrix A (forward: dtans_spmm).

        ``vals`` is an nnz-long tensor that stands for A's stored values in
        sorted-CSR order; the forward multiplies with the values encoded in the
        stream, so it first checks that ``vals`` still equals them bit for bit
        (decoded on the device once per tensor version) and raises
        ValueError when they differ, e.g. after an optimizer step on ``vals``
        (re-encode the matrix, or train a codebook with CodebookLinear).
        Backward returns
        X_grad = A^T G (dtans_spmv_T) and vals_grad_q = <G[i, :], X[j, :]>
        (dtans_vals_grad) for each stored entry q = (i, j).  X_grad goes
        through A's attached transposed stream when one is attached
        (choose_xgrad picks by measurement), else the atomic scatter."""

        @staticmethod
        def forward(ctx, A: Matrix, vals, X):
            _check_encoded_values(A, vals)
            ctx.A = A
            ctx.save_for_backward(X)
            vec = X.dim() == 1
            X2 = X.reshape(X.shape[0], -1).contiguous()
            Y = A.spmm(X2)
            return Y.reshape(-1) if vec else Y

        @staticmethod
        def backward(ctx, G):
            (X,) = ctx.saved_tensors
            A = ctx.A
            vec = X.dim() == 1
            G2 = G.reshape(G.shape[0], -1).contiguous()
            X2 = X.reshape(X.shape[0], -1).contiguous()
            gx = gv = None
            if ctx.needs_input_grad[2]:
                gx = A.xgrad(G2 if not vec else G2.reshape(-1))
                gx = gx.reshape(X.shape)
            if ctx.needs_input_grad[1]:
                gv = A.vals_grad(G2 if not vec else G2.reshape(-1), X2 if not vec else X2.reshape(-1))
            return None, gv, gx

    class CodebookLinear(torch.autograd.Function):
        """Y = A X for a CSR-dtANS matrix A whose stored values are a trainable
        codebook (weight sharing): ``codebook`` holds the T kept value symbols
        in the table's rank order (Matrix.codebook()).  Forward installs the
        codebook (dtans_set_codebook, also on an attached transposed stream)
        and multiplies (dtans_spmm); backward returns X_grad = A^T G and
        codebook_grad_r = sum over entries with value c_r of <G[i, :], X[j, :]>
        (dtans_codebook_grad)."""

        @staticmethod
        def forward(ctx, A: Matrix, codebook, X):
            cb = codebook.detach().to("cpu").numpy()
            A.set_codebook(cb)
            if A.transpose is not None:
                A.transpose.set_codebook(cb)
            ctx.A = A
            ctx.save_for_backward(X)
            vec = X.dim() == 1
            X2 = X.reshape(X.shape[0], -1).contiguous()
            Y = A.spmm(X2)
            return Y.reshape(-1) if vec else Y

        @staticmethod
        def backward(ctx, G):
            (X,) = ctx.saved_tensors
            A = ctx.A
            vec = X.dim() == 1
            G2 = G.reshape(G.shape[0], -1).contiguous()
            X2 = X.reshape(X.shape[0], -1).contiguous()
            gx = gc = None
            if ctx.needs_input_grad[2]:
                gx = A.xgrad(G2 if not vec else G2.reshape(-1)).reshape(X.shape)
            if ctx.needs_input_grad[1]:
                gc = A.codebook_grad(G2 if not vec else G2.reshape(-1), X2 if not vec else X2.reshape(-1))[:-1]
            return None, gc, gx

    return CompressedLinear, CodebookLinear


def __getattr__(name):
    if name == "CompressedLinear":
        return _autograd()[0]
    if name == "CodebookLinear":
        return _autograd()[1]
    raise AttributeError(name)
