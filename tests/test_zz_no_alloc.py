"""The no-allocation SpMV entry point (dtans_spmv_noalloc).

dtans_spmv_noalloc serves callers that must not allocate device memory when
they multiply (a real-time loop, an allocator-free runtime, a pool that has
handed out all its memory): it keeps its per-warp slice ranges in a fixed
device array compiled into the library instead of a buffer allocated on
first use.  These tests call it through the C ABI and require
- its y within the row bound of the other parity tests
  (8 * len * u * sum |a x|) of the oracle's y;
- the same y as dtans_spmv: bit for bit when both run the same kernel on
  the same slice ranges (no row split over several units, FP64 fused
  multiply-adds), within the row bound otherwise (split rows add their parts
  atomically, in any order; dtans_spmv's integer-coefficient kernel rounds
  each row once);
- two calls in a row (the second reuses the array the first one filled), for
  beta = 0, 1 and 0.5;
- no change of the device's free memory across calls.
This file is collected last on purpose.
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
    y_lib = torch.from_numpy(y_in.astype(dt)).cuda()
    y_new = y_lib.clone()
    _call("dtans_spmv", M, xd, y_lib, beta)
    _call("dtans_spmv_noalloc", M, xd, y_new, beta)
    torch.cuda.synchronize()
    M.check()
    assert y_new.dtype == tdt
    y_or, ab = O.spmm_ref(A["row_ptr"], A["cols"], A["vals"].astype(np.float64), x.astype(dt).astype(np.float64),
                          beta=beta, Y=y_in.astype(dt).astype(np.float64))
    lens = np.diff(A["row_ptr"]) + (1 if beta else 0)
    tol = 8.0 * lens * U[np.dtype(dt)] * ab
    yn = y_new.cpu().numpy().astype(np.float64)
    diff = np.abs(yn - y_or)
    assert (diff <= tol).all(), f"{int((diff > tol).sum())} rows differ from the oracle beyond the row bound"
    yl = y_lib.cpu().numpy().astype(np.float64)
    if M.info.nunits > M.shape[0] or M.info.int_products:
        # split rows add their parts atomically in any order, and dtans_spmv's
        # integer-coefficient kernel rounds once per row where the no-alloc
        # call runs FP64 fused multiply-adds: equal within the row bound
        assert (np.abs(yn - yl) <= 2 * tol).all(), "no-alloc and dtans_spmv differ beyond the row bound"
    else:
        assert np.array_equal(y_new.cpu().numpy(), y_lib.cpu().numpy()), "no-alloc differs from dtans_spmv"


@pytest.mark.parametrize("case", ["stencil_fp64", "stencil_fp64_int", "powerlaw_split_fp32", "pr1_chained"])
def test_noalloc_matches_spmv_on_two_calls(case):
    rng = np.random.default_rng(11)
    if case in ("stencil_fp64", "stencil_fp64_int"):
        A = WL.stencil27(grid=24)
        M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"])).cuda()
        if case == "stencil_fp64_int":
            M.set_accumulate(1)  # dtans_spmv on the integer-coefficient kernel: within the row bound
        betas = (0.0, 1.0, 0.5)
    elif case == "powerlaw_split_fp32":
        A = WL.power_law(rows=30000, seed=12, max_len=800)
        M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), unit_max_nnz=16, row_order=1).cuda()
        betas = (0.5, 0.0, 1.0)
    else:
        A = WL.pr1(seed=13, n=8192)
        M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), chain=8).cuda()
        betas = (0.0, 1.0, 0.5)
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


def test_noalloc_leaves_free_device_memory_unchanged():
    """After one call of each kind has loaded the kernels it launches, further
    calls change nothing in the device's free memory (cudaMemGetInfo)."""
    rng = np.random.default_rng(14)
    A = WL.power_law(rows=20000, seed=15, max_len=600)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), unit_max_nnz=16, row_order=1).cuda()
    B = WL.pr1(seed=16, n=4096)
    N = D.Matrix(B["row_ptr"], B["cols"], B["vals"], (B["m"], B["n"])).cuda()
    bufs = []
    for Am in (A, B):
        dt = torch.float32 if Am["vals"].dtype == np.float32 else torch.float64
        bufs.append((torch.from_numpy(rng.uniform(-1, 1, Am["n"])).to(dt).cuda(),
                     torch.from_numpy(rng.uniform(-1, 1, Am["m"])).to(dt).cuda()))
    calls = [(M, bufs[0], b) for b in (0.0, 1.0, 0.5)] + [(N, bufs[1], b) for b in (0.0, 1.0, 0.5)]
    for Mx, (x, y), beta in calls:  # warm-up: loads every kernel these calls launch
        _call("dtans_spmv_noalloc", Mx, x, y, beta)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        for Mx, (x, y), beta in calls:
            _call("dtans_spmv_noalloc", Mx, x, y, beta)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    M.check()
    N.check()
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
