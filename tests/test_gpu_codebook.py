"""GPU parity of the codebook entry points (dtans_codebook_grad,
dtans_set_codebook) and of CodebookLinear against the CPU oracle, through the
C ABI.  Bins are sums of many products in an unfixed order, so each bin r is
held to 8 * n_r * u * sum |G X| with n_r its number of terms."""
import numpy as np
import pytest

import oracle as O
import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2603_01915_gb300 as D  # noqa: E402

U = {np.dtype(np.float64): 2.0 ** -53, np.dtype(np.float32): 2.0 ** -24}


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _weight_shared(seed, dim, dtype, escaped_frac=0.0):
    """The pruned-linear construction; with escaped_frac > 0 that share of the
    entries gets unique continuous values (more than the table's 4096 slots),
    so the encoder escapes them."""
    A = WL.pruned_linear(seed=seed, dim=dim, batch=4, dtype=dtype)
    if escaped_frac:
        rng = np.random.default_rng(seed + 100)
        # at least 6000 unique values: more symbols than the table can keep
        pick = rng.random(len(A["vals"])) < max(escaped_frac, 6000 / len(A["vals"]))
        A["vals"] = A["vals"].copy()
        A["vals"][pick] = rng.uniform(0.5, 1.5, int(pick.sum())).astype(dtype)
    return A


def _check_bins(got, ref, ab, counts, k, dt, what):
    bound = 8.0 * np.maximum(counts * k, 1) * U[np.dtype(dt)] * ab
    err = np.abs(got.astype(np.float64) - ref)
    bad = np.nonzero(err > bound)[0]
    assert len(bad) == 0, f"{what}: bins {bad[:5]} err {err[bad][:5]} bound {bound[bad][:5]}"


@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("k", [1, 5, 32])
@pytest.mark.parametrize("layout", [{}, dict(unit_max_nnz=16, row_order=1, first_delta=1, chain=3, escape_stream=1)])
def test_codebook_grad_matches_oracle(dt, k, layout):
    A = _weight_shared(3 + k, 1024 if k < 32 else 512, dt, escaped_frac=0.08)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), **layout).cuda()
    T = int(M.info.kept_value)
    assert M.info.esc_value  # the unique values are escaped
    rng = np.random.default_rng(k)
    G = rng.uniform(-1, 1, (A["m"], k)).astype(dt)
    X = rng.uniform(-1, 1, (A["n"], k)).astype(dt)
    out = M.codebook_grad(_dev(G) if k > 1 else _dev(G[:, 0]), _dev(X) if k > 1 else _dev(X[:, 0]))
    torch.cuda.synchronize()
    M.check()
    assert out.shape == (T + 1,)
    cs, vs = O.sort_rows(A["row_ptr"], A["cols"], A["vals"])
    cb = M.codebook()
    ref, ab = O.codebook_grad_ref(A["row_ptr"], cs, vs, cb, G.astype(np.float64), X.astype(np.float64))
    keys = O.value_keys(vs)
    counts = np.array([(keys == c).sum() for c in O.value_keys(cb)] + [0])
    counts[-1] = len(keys) - counts.sum()
    _check_bins(out.cpu().numpy(), ref, ab, counts, k, dt, "codebook grad")


@pytest.mark.parametrize("k", [32, 40, 64])
@pytest.mark.parametrize("layout", ["plain", "split", "chain", "relative", "offset"])
def test_codebook_grad_fp32_persistent(k, layout):
    """FP32 codebook gradients in passes of 32 columns on the persistent ring
    kernel (each entry's dot product added to its value symbol's bin in
    shared memory, the CTA's bins added to the output at the end; the rest of
    k on the one-slice-per-warp kernel): every bin within its bound for split
    rows, chained units, row-relative first deltas and G and X 16- but not
    32-byte aligned."""
    A = _weight_shared(50 + k, 600, np.float32, escaped_frac=0.08)
    kw = {"plain": {}, "split": dict(unit_max_nnz=8, row_order=1), "chain": dict(chain=3),
          "relative": dict(first_delta=1, row_order=1, order_window=128), "offset": {}}[layout]
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), **kw).cuda()
    T = int(M.info.kept_value)
    rng = np.random.default_rng(k)
    G = rng.uniform(-1, 1, (A["m"], k)).astype(np.float32)
    X = rng.uniform(-1, 1, (A["n"], k)).astype(np.float32)

    def dev(Z):
        if layout != "offset":
            return _dev(Z)
        buf = torch.zeros(Z.size + 4, dtype=torch.float32, device="cuda")  # 16 bytes in
        t = buf[4:].view(Z.shape)
        t.copy_(torch.from_numpy(Z))
        assert t.data_ptr() % 32 == 16
        return t

    out = M.codebook_grad(dev(G), dev(X))
    torch.cuda.synchronize()
    M.check()
    assert out.shape == (T + 1,)
    cs, vs = O.sort_rows(A["row_ptr"], A["cols"], A["vals"])
    cb = M.codebook()
    ref, ab = O.codebook_grad_ref(A["row_ptr"], cs, vs, cb, G.astype(np.float64), X.astype(np.float64))
    keys = O.value_keys(vs)
    counts = np.array([(keys == c).sum() for c in O.value_keys(cb)] + [0])
    counts[-1] = len(keys) - counts.sum()
    _check_bins(out.cpu().numpy(), ref, ab, counts, k, np.float32, "codebook grad")


def test_set_codebook_changes_products_not_stream():
    A = _weight_shared(11, 768, np.float64, escaped_frac=0.05)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"])).cuda()
    cb = M.codebook()
    new = cb * -3.0 + 0.125
    M.set_codebook(new)
    # the matrix the stream now stands for: every kept value replaced
    cs, vs = O.sort_rows(A["row_ptr"], A["cols"], A["vals"])
    keys, ck = O.value_keys(vs), O.value_keys(cb)
    vs2 = vs.copy()
    for r in range(len(cb)):
        vs2[keys == ck[r]] = new[r]
    cols, vals = M.decode_csr()
    torch.cuda.synchronize()
    assert np.array_equal(cols.cpu().numpy().view(np.uint32), cs)
    assert np.array_equal(O.value_keys(vals.cpu().numpy()), O.value_keys(vs2))
    x = A["X"][:, 0].astype(np.float64)
    y = torch.empty(A["m"], dtype=torch.float64, device="cuda")
    M.spmv(_dev(x), y)
    torch.cuda.synchronize()
    yref, ab = O.spmm_ref(A["row_ptr"], cs, vs2, x)
    lens = np.diff(A["row_ptr"]).astype(np.float64)
    assert (np.abs(y.cpu().numpy() - yref) <= 8 * lens * U[np.dtype(np.float64)] * ab).all()


def test_codebook_linear_autograd_and_finite_differences():
    """CodebookLinear on a 256 x 256 FP64 instance of the pruned construction:
    gradients against the oracle, and FP64 central differences of
    L = sum(G .* (A(c) X)) in a random codebook direction (rel. err <= 1e-6),
    each perturbed codebook installed with dtans_set_codebook."""
    A = WL.pruned_linear(dim=256, batch=4, dtype=np.float64, seed=21)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"])).cuda()
    CL = D.CodebookLinear
    cb0 = M.codebook()
    cb = torch.tensor(cb0, device="cuda", requires_grad=True)
    X = torch.tensor(A["X"], device="cuda", requires_grad=True)
    G = torch.tensor(A["G"], device="cuda")
    (CL.apply(M, cb, X) * G).sum().backward()
    cs, vs = O.sort_rows(A["row_ptr"], A["cols"], A["vals"])
    ref, _ = O.codebook_grad_ref(A["row_ptr"], cs, vs, cb0, A["G"], A["X"])
    np.testing.assert_allclose(cb.grad.cpu().numpy(), ref[:-1], rtol=1e-11, atol=1e-11)
    XGref, _ = O.spmm_t_ref(A["row_ptr"], A["cols"], A["vals"], A["n"], A["G"])
    np.testing.assert_allclose(X.grad.cpu().numpy(), XGref, rtol=1e-12, atol=1e-12)

    def loss(c):
        with torch.no_grad():
            return float((CL.apply(M, torch.tensor(c, device="cuda"), X) * G).sum())

    rng = np.random.default_rng(0)
    d = rng.normal(size=cb0.shape)
    h = 1e-3
    fd = (loss(cb0 + h * d) - loss(cb0 - h * d)) / (2 * h)
    an = float((cb.grad.cpu().numpy() * d).sum())
    assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
