"""Parity at the full sizes of the five benchmark workloads, in the launch
configuration bench.py times (persistent kernels, default grid).

Decoded streams equal the input CSR bit for bit; every output row (or column)
satisfies the row bound against the oracle's compensated product.  The oracle
products are plain C loops and finish in seconds even at 84 M entries.
"""
import numpy as np
import pytest

import oracle as O
import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2603_01915_gb300 as D  # noqa: E402

U = {np.dtype(np.float64): 2.0 ** -53, np.dtype(np.float32): 2.0 ** -24}


def _bound_ok(y, yref, ab, lens, dt, extra=0):
    err = np.abs(np.asarray(y, np.float64) - yref)
    lens = np.asarray(lens, np.float64)
    if yref.ndim == 2:
        lens = lens[:, None]
    bound = 8.0 * (lens + extra) * U[np.dtype(dt)] * ab
    bad = int((err > bound).sum())
    assert bad == 0, f"{bad} outputs outside the row bound"


def _decode_ok(A, M):
    cols, vals = M.decode_csr()
    torch.cuda.synchronize()
    M.check()
    cs, vs = O.sort_rows(A["row_ptr"], A["cols"], A["vals"])
    assert np.array_equal(cols.cpu().numpy().view(np.uint32), cs)
    assert np.array_equal(O.value_keys(vals.cpu().numpy()), O.value_keys(vs))


def _spmv_ok(A, M, beta=0.0):
    dt = A["vals"].dtype
    rng = np.random.default_rng(1)
    y0 = rng.uniform(-1, 1, A["m"]).astype(dt)
    y = torch.from_numpy(y0.copy()).cuda()
    M.spmv(torch.from_numpy(A["x"].astype(dt)).cuda(), y, beta=beta)
    torch.cuda.synchronize()
    M.check()
    yref, ab = O.spmm_ref(A["row_ptr"], A["cols"], A["vals"].astype(np.float64), A["x"].astype(np.float64),
                          beta=beta, Y=y0.astype(np.float64))
    _bound_ok(y.cpu().numpy(), yref, ab, np.diff(A["row_ptr"]), dt, 1 if beta else 0)


@pytest.mark.parametrize("first_delta,chain", [(0, 1), (1, 1), (1, 8)])
def test_stencil_128_full(first_delta, chain):
    A = WL.stencil27(128, seed=1)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), first_delta=first_delta,
                 chain=chain).cuda()
    _decode_ok(A, M)
    _spmv_ok(A, M)
    _spmv_ok(A, M, beta=1.0)


@pytest.mark.parametrize("U,window", [(16, 0), (32, 2048)])
def test_power_law_4m_full(U, window):
    A = WL.power_law(seed=2)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), unit_max_nnz=U, row_order=1,
                 order_window=window).cuda()
    _decode_ok(A, M)
    _spmv_ok(A, M)


def test_batched_64_and_multi_rhs_full():
    mats = WL.batched(seed=3)
    Ms = [D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"])).cuda() for A in mats]
    xs = [torch.from_numpy(A["x"]).cuda() for A in mats]
    ys = [torch.empty(A["m"], dtype=torch.float64, device="cuda") for A in mats]
    B = D.Batch(Ms)
    B.bind(xs, ys)
    B.spmv()
    torch.cuda.synchronize()
    for A, y in zip(mats, ys):
        yref, ab = O.spmm_ref(A["row_ptr"], A["cols"], A["vals"], A["x"])
        _bound_ok(y.cpu().numpy(), yref, ab, np.diff(A["row_ptr"]), np.float64)
    A = WL.multi_rhs(seed=3, k=16)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"])).cuda()
    for k in (1, 4, 8, 16):
        X = np.ascontiguousarray(A["X"][:, :k])
        Y = M.spmm(torch.from_numpy(X).cuda())
        torch.cuda.synchronize()
        Yref, ab = O.spmm_ref(A["row_ptr"], A["cols"], A["vals"], X)
        _bound_ok(Y.cpu().numpy(), Yref, ab, np.diff(A["row_ptr"]), np.float64)


def test_pruned_linear_full_forward_backward():
    """Forward, x_grad, value gradient and codebook gradient of the pruned
    layer at full size, with the layout the autotuner picks for k = 32."""
    A = WL.pruned_linear(seed=4)
    M, _, _ = D.tune(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), k=32, reps=2)
    X = torch.from_numpy(A["X"]).cuda()
    G = torch.from_numpy(A["G"]).cuda()
    Y = M.spmm(X)
    XG = M.spmv_T(G)
    VG = M.vals_grad(G, X)
    torch.cuda.synchronize()
    Xd, Gd = A["X"].astype(np.float64), A["G"].astype(np.float64)
    vals = A["vals"].astype(np.float64)
    Yref, ab = O.spmm_ref(A["row_ptr"], A["cols"], vals, Xd)
    _bound_ok(Y.cpu().numpy(), Yref, ab, np.diff(A["row_ptr"]), np.float32)
    XGref, ab = O.spmm_t_ref(A["row_ptr"], A["cols"], vals, A["n"], Gd)
    _bound_ok(XG.cpu().numpy(), XGref, ab, np.bincount(A["cols"], minlength=A["n"]), np.float32)
    VGref, ab = O.vals_grad_ref(A["row_ptr"], A["cols"], Gd, Xd)
    _bound_ok(VG.cpu().numpy(), VGref, ab, np.full(len(VGref), 32), np.float32)
    # codebook gradient (16 symbols): each bin sums count * 32 products
    CG = M.codebook_grad(G, X)
    torch.cuda.synchronize()
    M.check()
    cb = M.codebook()
    CGref, ab = O.codebook_grad_ref(A["row_ptr"], A["cols"], A["vals"], cb, Gd, Xd)
    keys = O.value_keys(A["vals"])
    counts = np.array([(keys == c).sum() for c in O.value_keys(cb)] + [0])
    counts[-1] = len(keys) - counts.sum()
    _bound_ok(CG.cpu().numpy(), CGref, ab, np.maximum(counts * 32, 1), np.float32)


def test_stencil_128_full_integer_products():
    """The integer-coefficient form the bench times beside the FMA form:
    every row within the row bound, and sampled rows bit-equal to the
    correctly rounded exact product (x uniform in [-1, 1] lies within the
    2^40 window, so no entry takes the FMA chain)."""
    from fractions import Fraction
    A = WL.stencil27(128, seed=1)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), first_delta=1).cuda()
    M.set_accumulate(1)
    assert M.info.int_products == 1
    x = A["x"].astype(np.float64)
    y = torch.zeros(A["m"], dtype=torch.float64, device="cuda")
    M.spmv(torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    M.check()
    yh = y.cpu().numpy()
    yref, ab = O.spmm_ref(A["row_ptr"], A["cols"], A["vals"], x)
    _bound_ok(yh, yref, ab, np.diff(A["row_ptr"]), np.float64)
    rp, cols, vals = A["row_ptr"], A["cols"], A["vals"]
    for i in np.random.default_rng(5).choice(A["m"], 400, replace=False):
        s = sum(Fraction(float(vals[q])) * Fraction(float(x[cols[q]])) for q in range(rp[i], rp[i + 1]))
        assert yh[i] == float(s), f"row {i} is not the correctly rounded product"


def test_stencil_128_full_host_vectors():
    """dtans_spmv_host at the bench's size: consecutive calls on pinned host
    vectors (three buffer sets in turn, the fourth call reusing the first),
    each y within the row bound of the oracle."""
    A = WL.stencil27(128, seed=1)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), first_delta=1).cuda()
    xs = [torch.from_numpy(A["x"] * s).pin_memory() for s in (1.0, -0.5, 2.0, 0.25)]
    ys = [torch.empty(A["m"], dtype=torch.float64).pin_memory() for _ in xs]
    for xh, yh in zip(xs, ys):
        M.spmv_host(xh, yh, sync=False)
    torch.cuda.current_stream().synchronize()
    M.check()
    for xh, yh in zip(xs, ys):
        yref, ab = O.spmm_ref(A["row_ptr"], A["cols"], A["vals"], xh.numpy())
        _bound_ok(yh.numpy(), yref, ab, np.diff(A["row_ptr"]), np.float64)


def test_power_law_4m_full_transposed_products():
    """x_grad = A^T g on the power-law layout the bench times, with one
    atomic per entry and with warp-aggregated atomics: every column within
    the column bound of the oracle's A^T g."""
    A = WL.power_law(seed=2)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), unit_max_nnz=32, row_order=1,
                 order_window=2048).cuda()
    g = A["x"][:A["m"]].astype(np.float32)
    gd = torch.from_numpy(g).cuda()
    XGref, ab = O.spmm_t_ref(A["row_ptr"], A["cols"], A["vals"].astype(np.float64), A["n"], g.astype(np.float64))
    lens = np.bincount(A["cols"], minlength=A["n"])
    for mode in (0, 1):
        M.set_scatter(mode)
        XG = M.spmv_T(gd)
        torch.cuda.synchronize()
        M.check()
        _bound_ok(XG.cpu().numpy(), XGref, ab, lens, np.float32)
