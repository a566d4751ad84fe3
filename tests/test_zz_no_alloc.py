"""The no-allocation SpMV entry point (dtans_spmv_noalloc) against dtans_spmv.

dtans_spmv_noalloc serves callers that must not allocate device memory when
they multiply: it keeps its per-warp slice ranges in a fixed device array
compiled into the library instead of a buffer allocated on first use.  These
tests call both entry points through the C ABI on the same inputs and require
the same result within the row bound used by the other parity tests
(8 * len * u * sum |a x|), on two calls in a row (the second call reuses the
array the first one filled).  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2603_01915_gb300 as D  # noqa: E402

U = {np.dtype(np.float64): 2.0 ** -53, np.dtype(np.float32): 2.0 ** -24}


def _call(name, M, x, y, beta):
    L = D.lib()
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(L, name)(M.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), float(beta), st)
    assert rc == 0, L.dtans_last_error()


def _compare(A, M, x, y_in, beta):
    dt = A["vals"].dtype
    tdt = torch.float64 if dt == np.float64 else torch.float32
    xd = torch.from_numpy(x.astype(dt)).cuda()
    y_ref = torch.from_numpy(y_in.astype(dt)).cuda()
    y_new = y_ref.clone()
    _call("dtans_spmv", M, xd, y_ref, beta)
    _call("dtans_spmv_noalloc", M, xd, y_new, beta)
    torch.cuda.synchronize()
    M.check()
    _, ab = O.spmm_ref(A["row_ptr"], A["cols"], A["vals"].astype(np.float64), x.astype(np.float64), beta=beta,
                       Y=y_in.astype(np.float64))
    lens = np.diff(A["row_ptr"]) + (1 if beta else 0)
    tol = 8.0 * lens * U[np.dtype(dt)] * ab
    diff = np.abs(y_new.cpu().numpy().astype(np.float64) - y_ref.cpu().numpy().astype(np.float64))
    assert y_new.dtype == tdt
    assert (diff <= tol).all(), f"{int((diff > tol).sum())} rows differ beyond the row bound"


@pytest.mark.parametrize("case", ["stencil_fp64", "powerlaw_split_fp32", "pr1_chained"])
def test_noalloc_matches_spmv_on_two_calls(case):
    rng = np.random.default_rng(11)
    if case == "stencil_fp64":
        A = WL.stencil27(grid=24)
        M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"])).cuda()
        betas = (0.0, 1.0)
    elif case == "powerlaw_split_fp32":
        A = WL.power_law(rows=30000, seed=12, max_len=800)
        M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), unit_max_nnz=16, row_order=1).cuda()
        betas = (0.5, 0.0)
    else:
        A = WL.pr1(seed=13, n=8192)
        M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), chain=8).cuda()
        betas = (0.0, 1.0)
    for beta in betas:  # two calls in a row, with fresh x and y each time
        x = rng.uniform(-1, 1, A["n"])
        y_in = rng.uniform(-1, 1, A["m"])
        _compare(A, M, x, y_in, beta)


def test_noalloc_after_another_matrix_and_launch_shape():
    """A second matrix and a smaller launch shape overwrite the shared ranges;
    the result must follow the new call, not the previous one."""
    rng = np.random.default_rng(12)
    A1 = WL.pr1(seed=3, n=4096)
    M1 = D.Matrix(A1["row_ptr"], A1["cols"], A1["vals"], (A1["m"], A1["n"])).cuda()
    A2 = WL.random_csr(13, 5000, 3000, 7.0, nvals=20)
    M2 = D.Matrix(A2["row_ptr"], A2["cols"], A2["vals"], (A2["m"], A2["n"])).cuda()
    M2.set_launch(7, 0)
    M2.set_warps(20)
    _compare(A1, M1, rng.uniform(-1, 1, A1["n"]), rng.uniform(-1, 1, A1["m"]), 0.0)
    _compare(A2, M2, rng.uniform(-1, 1, A2["n"]), rng.uniform(-1, 1, A2["m"]), 0.0)
    _compare(A1, M1, rng.uniform(-1, 1, A1["n"]), rng.uniform(-1, 1, A1["m"]), 0.0)


def test_noalloc_rejects_launch_shapes_beyond_its_array():
    A = WL.pr1(seed=4, n=512)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"])).cuda()
    M.set_launch(257, 0)
    M.set_warps(32)  # 257 CTAs x 32 warps > 8192 warps
    x = torch.zeros(A["n"], dtype=torch.float64, device="cuda")
    y = torch.zeros(A["m"], dtype=torch.float64, device="cuda")
    L = D.lib()
    rc = L.dtans_spmv_noalloc(M.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), 0.0,
                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1 and b"no-alloc scratch" in L.dtans_last_error()
