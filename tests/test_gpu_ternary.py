"""GPU parity of the ternary function ite(a, b, c) = a > 0 ? b : c (type code
4, 20 on a Modi node): the kernels push the condition's sign bits on a
per-lane condition stack and select between the branches with a binary
form.  Checked against the FP64 oracle on random populations that mix ite
with the SR function set (single output and Modi, several launch shapes),
bit for bit on the selection itself (zero, negative zero, NaN and infinite
conditions), on the nesting limit of pending conditions, and on the adjoint,
which reports ite trees instead of differentiating them."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2501_17168_gb300 import _lib, api, workloads as W
from parity import assert_mse_strict_floor, assert_strict_floor, compare_mse, compare_points

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_17168_gb300 import build
    build.build_all()
    _lib.load()


def _forward(p, X, O=1, config=None):
    t, v, s = api.population_to(p, DEV)
    out, st = api.tgp_eval_forward(t, v, s, torch.from_numpy(X).to(DEV), O, max_len=p.max_len,
                                   config=config)
    api.tgp_check_device_error()
    return out.cpu().numpy(), st.cpu().numpy()


def _check(orc, p, X, O=1, config=None):
    g, gst = _forward(p, X, O, config)
    ref, err, st = orc.evaluate(p.type, p.val, p.size, X, n_outputs=O, with_err=True,
                                max_len=p.max_len)
    np.testing.assert_array_equal(gst, st)
    ok = st == 0
    stats = compare_points(g[ok], ref[ok], err[ok])
    assert stats.failed == 0, (stats, stats.examples)
    assert_strict_floor(g[ok], ref[ok], err[ok], p.type[ok], p.val[ok], p.size[ok], X, O)
    return stats


@pytest.mark.parametrize("cfg", [None, {"points_per_lane": 4},
                                 {"points_per_lane": 8, "trees_per_block": 3, "points_per_tile": 512}])
def test_ite_population_forward_and_mse(orc, cfg):
    p = W.random_population(201, 150, 127, (1, 127), max_depth=8, n_features=4,
                            fset=W.TERNARY_FSET)
    assert (p.type == W.TFUNC).sum() > 200
    X = np.random.default_rng(31).standard_normal((1234, 4)).astype(np.float32)
    _check(orc, p, X, config=cfg)
    y = np.random.default_rng(32).standard_normal((1234, 1)).astype(np.float32)
    t, v, s = api.population_to(p, DEV)
    m, st = api.tgp_fitness_mse(t, v, s, torch.from_numpy(X).to(DEV), torch.from_numpy(y).to(DEV), 1,
                                max_len=p.max_len, config=cfg)
    m = m.cpu().numpy()
    ref, allow, _ = orc.mse(p.type, p.val, p.size, X, y, rel_tol=1e-5)
    r = compare_mse(m, ref, allow)
    assert len(r["failed"]) == 0 and len(r["class_mismatch"]) == 0, r
    assert_mse_strict_floor(m, ref, allow, p.type, p.val, p.size, X, y)


def test_ite_modi_population(orc):
    p = W.random_population(202, 120, 255, (9, 255), max_depth=8, n_features=5, fset=W.TERNARY_FSET,
                            n_outputs=3, modi=True, modi_max=8)
    assert (p.type == W.TFUNC + W.MODI).sum() > 5
    X = np.random.default_rng(33).uniform(-2, 2, (900, 5)).astype(np.float32)
    _check(orc, p, X, O=3)


def test_ite_selection_is_exact():
    """The selection copies the chosen branch bit for bit; a zero, negative
    zero or NaN condition selects the third child."""
    p = W.stack([W.encode(["ite", ("x", 0), ("x", 1), ("x", 2)]),
                 W.encode(["ite", ("x", 0), ("c", 0.25), ("x", 2)]),
                 W.encode(["ite", ("c", -1.0), ("x", 1), ("x", 2)]),
                 W.encode(["ite", "sin", ("x", 0), "mul", ("x", 1), ("x", 2), ("x", 2)])])
    conds = np.array([1.0, -1.0, 0.0, -0.0, np.nan, 1e-45, -1e-45, np.inf, -np.inf, 3e38, -2.5, 7.0],
                     np.float32)
    r = np.random.default_rng(34)
    X = np.stack([np.tile(conds, 50), r.standard_normal(600), r.standard_normal(600)], 1).astype(np.float32)
    g, st = _forward(p, X)
    assert (st == 0).all()
    c, b, e = X[:, 0], X[:, 1], X[:, 2]
    np.testing.assert_array_equal(g[0, 0], np.where(c > 0, b, e))
    np.testing.assert_array_equal(g[1, 0], np.where(c > 0, np.float32(0.25), e))
    np.testing.assert_array_equal(g[2, 0], e)
    s = g[3, 0]
    # sin(x0) > 0 decides; the branch value is the float32 product
    with np.errstate(invalid="ignore"):
        pick = np.sin(c.astype(np.float64)) > 0
    with np.errstate(invalid="ignore"):
        sure = (np.abs(c) < 1e4) & (np.abs(np.sin(c.astype(np.float64))) > 1e-5)
    np.testing.assert_array_equal(s[sure & pick], (b * e)[sure & pick])
    np.testing.assert_array_equal(s[sure & ~pick], e[sure & ~pick])


def _nested(depth):
    """ite nested `depth` deep in the second branch: every condition is
    pending while the innermost branch is evaluated."""
    toks = []
    for _ in range(depth):
        toks += ["ite", ("x", 0)]
    toks += ["add", ("x", 1), ("x", 2)]
    toks += [("x", 2)] * depth
    return W.encode(toks)


def test_ite_nesting_limit(orc):
    """Eight pending conditions fit the condition stack; a ninth is reported
    as TGP_TREE_DEPTH (the oracle has no such limit), and that tree alone."""
    ok, deep = _nested(8), _nested(9)
    P = W.stack([ok, deep])
    X = np.random.default_rng(35).standard_normal((300, 3)).astype(np.float32)
    g, st = _forward(P, X)
    assert st[0] == 0 and st[1] == _lib.TREE_DEPTH
    ref, _ = orc.evaluate(ok.type, ok.val, ok.size, X)
    np.testing.assert_allclose(g[0, 0], ref[0, 0], rtol=1e-6, atol=1e-6)
    assert np.isnan(g[1]).all()


def test_adjoint_reports_ite_trees(orc):
    """The adjoint differentiates no ite: such trees get TGP_TREE_NO_ADJOINT and
    NaN results, every other tree its normal gradient."""
    plain = W.random_population(203, 40, 63, (1, 63), max_depth=6, n_features=3,
                                fset=(W.ADD, W.SUB, W.MUL, W.SIN, W.COS))
    tern = W.stack([W.encode(["ite", ("x", 0), ("c", 1.0), ("x", 1)], 63)])
    P = W.stack([plain, tern], ld=63)
    X = np.random.default_rng(36).uniform(-1, 1, (400, 3)).astype(np.float32)
    y = np.random.default_rng(37).standard_normal((400, 1)).astype(np.float32)
    t, v, s = api.population_to(P, DEV)
    g = torch.ones((P.pop, 1), dtype=torch.float64)
    mse, gv, gx, st = api.tgp_eval_backward(t, v, s, torch.from_numpy(X).to(DEV),
                                            torch.from_numpy(y).to(DEV), g, 1, max_len=63)
    api.tgp_check_device_error()
    st, mse, gv = st.cpu().numpy(), mse.cpu().numpy(), gv.cpu().numpy()
    assert st[-1] == _lib.TREE_NO_ADJOINT and (st[:-1] == 0).all()
    assert np.isnan(mse[-1]).all() and np.isnan(gv[-1]).all()
    rm, rgv, rgx, _ = orc.grad(plain.type, plain.val, plain.size, X, y, 1.0, max_len=63)
    with np.errstate(invalid="ignore"):
        np.testing.assert_allclose(mse[:-1], rm, rtol=1e-4)
        const = plain.type == W.CONST
        np.testing.assert_allclose(gv[:-1][const], rgv[const], rtol=1e-3, atol=1e-3)
    # the forward of the same population evaluates the ite tree
    fo, fst = _forward(P, X)
    assert (fst == 0).all() and np.isfinite(fo[-1]).all()
