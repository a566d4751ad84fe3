"""GPU parity of the integer-coefficient products (dtans_set_accumulate mode 1).

FP64 tables whose kept values are all c * 2^e (one e, |c| < 2^15) take the
integer path: x becomes exact fixed point, each unit's sum of c x is
accumulated exactly and rounded once.  So for a row whose x all lie within
2^40 of the largest |x| (and whose values were not escaped) y must equal the
correctly rounded exact product bit for bit; every row must stay within the
row bound of the other parity tests; entries outside the window, escaped
values, infinities and NaNs take the FMA chain.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2603_01915_gb300 as D  # noqa: E402

U = 2.0 ** -53


def _exact_rows(A, x, beta=0.0, y0=None):
    """Correctly rounded y = A x + beta y0 per row, from exact rational sums."""
    rp, cols, vals = A["row_ptr"], A["cols"], A["vals"]
    out = np.empty(A["m"])
    for i in range(A["m"]):
        s = Fraction(0)
        for q in range(rp[i], rp[i + 1]):
            s += Fraction(float(vals[q])) * Fraction(float(x[cols[q]]))
        if beta:
            s += Fraction(beta) * Fraction(float(y0[i]))
        out[i] = float(s)
    return out


def _run(M, x, y0=None, beta=0.0):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    y = torch.from_numpy(np.ascontiguousarray(y0 if y0 is not None else np.zeros(M.shape[0]))).cuda()
    M.spmv(xd, y, beta=beta)
    torch.cuda.synchronize()
    M.check()
    return y.cpu().numpy()


def _check_bound(A, x, y, beta=0.0, y0=None):
    yref, ab = O.spmm_ref(A["row_ptr"], A["cols"], A["vals"], x, beta=beta, Y=y0)
    lens = np.diff(A["row_ptr"]) + (1 if beta else 0)
    fin = np.isfinite(yref)
    err = np.abs(y[fin] - yref[fin])
    tol = 8.0 * lens[fin] * U * ab[fin]
    assert (err <= tol).all(), f"{int((err > tol).sum())} rows outside the row bound"
    # rows the oracle finds non-finite are non-finite on the GPU too (NaN and infinities propagate)
    assert (~np.isfinite(y[~fin])).all()
    return yref


def test_stencil_takes_integer_path_and_rounds_correctly():
    A = WL.stencil27(grid=12)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), first_delta=1).cuda()
    assert M.info.int_coefficients == 1 and M.info.int_products == 0  # mode 0 (FMA) by default
    M.set_accumulate(1)
    inf = M.info
    assert inf.int_products == 1 and inf.int_exp == 0
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, A["n"])
    y = _run(M, x)
    assert np.array_equal(y, _exact_rows(A, x)), "integer path differs from the correctly rounded product"
    for beta in (1.0, -0.5):
        y0 = rng.uniform(-1, 1, A["m"])
        yb = _run(M, x, y0, beta)
        _check_bound(A, x, yb, beta, y0)
    # the FMA form (mode 0) gives the same products within the row bound
    M.set_accumulate(0)
    assert M.info.int_products == 0
    y1 = _run(M, x)
    _check_bound(A, x, y1)


@pytest.mark.parametrize("kind", ["mixed_exponents", "cancellation", "out_of_window", "special"])
def test_adversarial_x(kind):
    """x with exponents over the whole FP64 range, rows that cancel to (near)
    zero, entries far below the window, and infinities, NaNs, zeros and
    subnormals: every finite row within the row bound of the oracle, the
    non-finite rows non-finite, and rows whose x are all inside the window
    bit-equal to the correctly rounded product."""
    A = WL.random_csr(40, 700, 900, 9.0, integer_valued=True)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"])).cuda()
    M.set_accumulate(1)
    assert M.info.int_products == 1
    rng = np.random.default_rng({"mixed_exponents": 2, "cancellation": 3, "out_of_window": 4, "special": 5}[kind])
    n = A["n"]
    if kind == "mixed_exponents":
        # most x within 2^30 of each other, the rest spread down to 2^-1000
        far = rng.random(n) < 0.3
        ex = np.where(far, rng.integers(-1000, 30, n), rng.integers(0, 30, n))
        x = rng.uniform(1, 2, n) * np.exp2(ex) * rng.choice([-1.0, 1.0], n)
    elif kind == "cancellation":
        x = rng.uniform(-1, 1, n)
        # give each row a partner column so that the two products cancel almost exactly
        rp, cols, vals = A["row_ptr"], A["cols"], A["vals"]
        for i in range(0, A["m"], 3):
            if rp[i + 1] - rp[i] >= 2:
                a, b = rp[i], rp[i] + 1
                if vals[a] != 0 and vals[b] != 0:
                    x[cols[b]] = -x[cols[a]] * vals[a] / vals[b] * (1 + 2.0 ** -50)
    elif kind == "out_of_window":
        x = rng.uniform(-1, 1, n)
        small = rng.random(n) < 0.2
        x[small] *= 2.0 ** -60  # far below the 2^40 window of the largest |x|
        x[rng.random(n) < 0.05] *= 2.0 ** -1070  # subnormal
    else:
        x = rng.uniform(-1, 1, n)
        x[rng.random(n) < 0.1] = 0.0
        x[rng.random(n) < 0.1] = -0.0
        x[rng.random(n) < 0.02] = np.inf
        x[rng.random(n) < 0.02] = -np.inf
        x[rng.random(n) < 0.02] = np.nan
        x[rng.random(n) < 0.05] = 5e-324
    y = _run(M, x)
    _check_bound(A, x, y)
    if kind in ("cancellation", "mixed_exponents"):
        ex = _exact_rows(A, x)
        if kind == "cancellation":  # every x inside the window: the integer path is exact
            assert np.array_equal(y, ex)
        else:  # only rows whose x all lie inside the window are exact
            big = np.max(np.abs(x))
            win = np.abs(x) >= big * 2.0 ** -40
            rows = np.repeat(np.arange(A["m"]), np.diff(A["row_ptr"]))
            ok = np.ones(A["m"], bool)
            np.logical_and.at(ok, rows, win[A["cols"]])
            assert ok.any() and np.array_equal(y[ok], ex[ok])


def test_escaped_integer_values_take_the_fma_chain():
    """More distinct integer values than table slots: the kept ones are
    integer coefficients, the escaped ones are read raw and multiplied in
    FP64; products within the row bound."""
    rng = np.random.default_rng(6)
    A = WL.random_csr(41, 3000, 2500, 12.0)
    A["vals"] = rng.integers(-20000, 20001, len(A["vals"])).astype(np.float64)
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"])).cuda()
    M.set_accumulate(1)
    inf = M.info
    assert inf.esc_value == 1 and inf.int_products == 1
    x = rng.uniform(-1, 1, A["n"])
    y = _run(M, x)
    _check_bound(A, x, y)


@pytest.mark.parametrize("kw", [dict(unit_max_nnz=8, row_order=1), dict(chain=4, first_delta=1),
                                dict(row_order=1, order_window=100)])
def test_integer_path_layouts(kw):
    """Split rows (parts added atomically), chained units and windowed
    orders on the integer path."""
    A = WL.power_law(rows=6000, seed=42, max_len=300)
    A["vals"] = np.rint(A["vals"].astype(np.float64) * 32.0)  # FP64 integers
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"]), **kw).cuda()
    M.set_accumulate(1)
    assert M.info.int_products == 1
    rng = np.random.default_rng(7)
    x = rng.uniform(-1, 1, A["n"])
    for beta in (0.0, 1.0, 0.5):
        y0 = rng.uniform(-1, 1, A["m"])
        y = _run(M, x, y0, beta)
        _check_bound(A, x, y, beta, y0 if beta else None)


def test_non_integer_tables_keep_the_fma_path():
    A = WL.pr1(seed=3, n=2048)  # 16 random constants: not small integer multiples of one power of two
    M = D.Matrix(A["row_ptr"], A["cols"], A["vals"], (A["m"], A["n"])).cuda()
    M.set_accumulate(1)
    assert M.info.int_coefficients == 0 and M.info.int_products == 0
    B = WL.random_csr(43, 500, 500, 6.0, integer_valued=True)
    B["vals"] = B["vals"] * 40001.0  # integers, but c = 40001 v needs more than 15 bits
    MB = D.Matrix(B["row_ptr"], B["cols"], B["vals"], (B["m"], B["n"])).cuda()
    MB.set_accumulate(1)
    inf = MB.info
    assert inf.int_coefficients == 0
    x = np.random.default_rng(8).uniform(-1, 1, B["n"])
    _check_bound(B, x, _run(MB, x))
