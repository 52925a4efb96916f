"""Pins of the FP64 oracle against facts that do not come from the oracle.

* the paper's two worked examples (Sec. II-A sigmoid tree, Sec. IV-C Modi
  tree), compared with their closed forms;
* textbook special cases (single leaves, exact sums and products, the MSE of
  an exact fit);
* brute force over every tree of at most 4 nodes (and a random sample of
  5-node trees) against a separately written Python restatement that builds
  an expression string and evaluates it with numpy;
* Modi brute force on small trees against a restatement that collects the
  output contributions explicitly;
* encoding invariants (Sec. III-A) and validator rejections;
* the guard branches of the protected operators at and around 1e-6f;
* reverse mode against central finite differences of the forward pass;
* the FP32 error bound against an actual float32 evaluation;
* the GPops/s definition (Sec. V-C) against the paper's Table III numbers.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from paper_2501_17168_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")))
THR = float(np.float32(1e-6))


def _tok(t):
    if isinstance(t, list) and t[0] in ("x", "c"):
        return (t[0], t[1])
    if isinstance(t, list):
        return (t[0], t[1])
    return t


def _enc(tokens, ld=None):
    return W.encode([_tok(t) for t in tokens], ld)


# ------------------------------------------------------------ worked examples
def test_sigmoid_tree_closed_form(orc):
    ex = GOLD["sigmoid"]
    p = _enc(ex["tokens"])
    assert list(p.size[0]) == ex["sizes"]
    x = np.linspace(-10, 10, 201, dtype=np.float32)[:, None]
    out, st = orc.evaluate(p.type, p.val, p.size, x)
    assert st[0] == 0
    ref = 1.0 / (1.0 + np.exp(-x[:, 0].astype(np.float64)))
    np.testing.assert_allclose(out[0, 0], ref, rtol=1e-15, atol=1e-15)


def test_modi_tree_closed_forms(orc):
    ex = GOLD["modi"]
    p = _enc(ex["tokens"])
    assert list(p.size[0]) == ex["sizes"]
    rng = np.random.default_rng(7)
    X = rng.uniform(-3, 3, (500, 5)).astype(np.float32)
    X[:, 2] = np.where(np.abs(X[:, 2]) < 1e-3, 0.5, X[:, 2])  # keep the pdiv guard off
    out, st = orc.evaluate(p.type, p.val, p.size, X, n_outputs=3)
    assert st[0] == 0
    a, b, c, d, e = (X[:, i].astype(np.float64) for i in range(5))
    np.testing.assert_allclose(out[0, 0], a / c * 0.5, rtol=1e-15)
    np.testing.assert_allclose(out[0, 1], np.maximum(b, c) + (d - 0.5), rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(out[0, 2], e + 0.5, rtol=1e-15, atol=1e-15)


def test_modi_outputs_without_contribution_are_zero(orc):
    p = _enc([["add", 1], ["x", 0], ["c", 2.0]])
    X = np.array([[1.5], [-3.0]], np.float32)
    out, st = orc.evaluate(p.type, p.val, p.size, X, n_outputs=3)
    np.testing.assert_array_equal(out[0, 0], [0.0, 0.0])
    np.testing.assert_array_equal(out[0, 1], [3.5, -1.0])
    np.testing.assert_array_equal(out[0, 2], [0.0, 0.0])


# ----------------------------------------------------------- textbook cases
def test_single_leaf_mse(orc):
    rng = np.random.default_rng(1)
    X = rng.standard_normal((300, 3)).astype(np.float32)
    y = rng.standard_normal(300).astype(np.float32)
    pops = [_enc([["x", f]], 4) for f in range(3)] + [_enc([["c", 0.75]], 4)]
    P = W.stack(pops)
    m, st = orc.mse(P.type, P.val, P.size, X, y)
    X64, y64 = X.astype(np.float64), y.astype(np.float64)
    for f in range(3):
        assert m[f, 0] == pytest.approx(np.mean((X64[:, f] - y64) ** 2), rel=1e-14)
    assert m[3, 0] == pytest.approx(np.mean((np.float64(np.float32(0.75)) - y64) ** 2), rel=1e-14)


def test_exact_fit_has_zero_mse(orc):
    # y = x0^2 + sin(x1) evaluated in float64 and rounded once to float32 is
    # not exactly representable, so the MSE is the float32 rounding residue.
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, (256, 2)).astype(np.float32)
    X64 = X.astype(np.float64)
    ref = X64[:, 0] ** 2 + np.sin(X64[:, 1])
    y = ref.astype(np.float32)
    p = _enc(["add", "mul", ["x", 0], ["x", 0], "sin", ["x", 1]])
    m, st = orc.mse(p.type, p.val, p.size, X, y)
    assert m[0, 0] == pytest.approx(np.mean((ref - y.astype(np.float64)) ** 2), rel=1e-12)
    assert m[0, 0] < 1e-14


def test_operand_order_left_is_first_child(orc):
    X = np.array([[5.0, 2.0]], np.float32)
    for name, want in [("sub", 3.0), ("pdiv", 2.5), ("max", 5.0), ("mul", 10.0), ("add", 7.0)]:
        p = _enc([name, ["x", 0], ["x", 1]])
        out, _ = orc.evaluate(p.type, p.val, p.size, X)
        assert out[0, 0, 0] == want, name


# ---------------------------------------------------------- brute force
NP_F = {
    "add": lambda a, b: f"({a} + {b})",
    "sub": lambda a, b: f"({a} - {b})",
    "mul": lambda a, b: f"({a} * {b})",
    "pdiv": lambda a, b: f"_pdiv({a}, {b})",
    "max": lambda a, b: f"np.fmax({a}, {b})",
    "sin": lambda a: f"np.sin({a})",
    "cos": lambda a: f"np.cos({a})",
    "plog": lambda a: f"_plog({a})",
    "cexp": lambda a: f"np.exp(np.minimum({a}, 80.0))",
    "tan": lambda a: f"np.tan({a})",
}


_AMBIG = []  # masks of points whose guard operand sits within 1e-9 of 1e-6f


def _near_guard(v):
    m = np.abs(np.abs(np.asarray(v, np.float64)) - THR) <= 1e-9 * THR
    _AMBIG.append(np.broadcast_to(m, np.shape(v)))


def _pdiv(a, b):
    a, b = np.broadcast_arrays(np.asarray(a, np.float64), np.asarray(b, np.float64))
    _near_guard(b)
    with np.errstate(all="ignore"):
        return np.where(np.abs(b) > THR, a / np.where(b == 0, 1, b), 1.0)


def _plog(a):
    a = np.asarray(a, np.float64)
    _near_guard(a)
    with np.errstate(all="ignore"):
        return np.where(np.abs(a) > THR, np.log(np.where(np.abs(a) > THR, np.abs(a), 1.0)), 0.0)


def _expr(tokens):
    """prefix tokens -> (python expression string, tokens consumed)"""
    t = tokens[0]
    if isinstance(t, tuple) and t[0] == "x":
        return f"x[:, {t[1]}]", 1
    if isinstance(t, tuple) and t[0] == "c":
        return f"np.float64({t[1]!r})", 1
    name = t
    if W.ARITY[W.FUNC_NAMES.index(name)] == 1:
        a, n = _expr(tokens[1:])
        return NP_F[name](a), 1 + n
    a, n1 = _expr(tokens[1:])
    b, n2 = _expr(tokens[1 + n1:])
    return NP_F[name](a, b), 1 + n1 + n2


LEAVES = [("x", 0), ("x", 1), ("c", 0.5)]
UN = ["sin", "cos", "plog", "cexp", "tan"]
BIN = ["add", "sub", "mul", "pdiv", "max"]


def _trees(n):
    """every prefix token list of exactly n nodes"""
    if n == 1:
        for l in LEAVES:
            yield [l]
        return
    for f in UN:
        for sub in _trees(n - 1):
            yield [f] + sub
    for f in BIN:
        for k in range(1, n - 1):
            for a in _trees(k):
                for b in _trees(n - 1 - k):
                    yield [f] + a + b


def _restated(expr, npts):
    """evaluates a restated expression; returns (values, usable-point mask)"""
    _AMBIG.clear()
    v = np.broadcast_to(eval(expr, globals(), _ENV), (npts,))
    ok = np.ones(npts, bool)
    for m in _AMBIG:
        ok &= ~np.broadcast_to(m, (npts,))
    # skip points whose value moves by more than 1e-6 when the inputs move by
    # 1e-13 relative: there a one-ulp difference between two libms shows
    x0 = _ENV["x"]
    moved = []
    for s in (1 + 1e-13, 1 - 1e-13):
        _ENV["x"] = x0 * s
        moved.append(np.broadcast_to(eval(expr, globals(), _ENV), (npts,)))
    _ENV["x"] = x0
    with np.errstate(all="ignore"):
        stable = np.abs(moved[0] - moved[1]) <= 1e-6 * np.maximum(np.abs(v), 1.0)
    ok &= stable | (np.isnan(v) & np.isnan(moved[0]))
    return v, ok


_ENV = {}


def _brute_points():
    rng = np.random.default_rng(3)
    X = rng.uniform(-4, 4, (64, 2)).astype(np.float32)
    X[0] = [0.0, -0.0]
    X[1] = [THR, -THR]
    X[2] = [np.nextafter(np.float32(THR), np.float32(1)), 1e-7]
    X[3] = [85.0, -85.0]
    return X


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_brute_force_all_small_trees(orc, n):
    X = _brute_points()
    x = X.astype(np.float64)
    trees = list(_trees(n))
    P = W.stack([W.encode(t, 8) for t in trees])
    out, st = orc.evaluate(P.type, P.val, P.size, X)
    assert (st == 0).all()
    _ENV["x"] = x
    with np.errstate(all="ignore"):
        for i, t in enumerate(trees):
            e, used = _expr(t)
            assert used == n
            ref, ok = _restated(e, X.shape[0])
            np.testing.assert_allclose(out[i, 0][ok], ref[ok], rtol=1e-9, atol=1e-12,
                                       equal_nan=True, err_msg=str(t))


def test_brute_force_sampled_five_node_trees(orc):
    X = _brute_points()
    x = X.astype(np.float64)
    trees = list(_trees(5))
    rng = np.random.default_rng(4)
    pick = rng.choice(len(trees), size=min(3000, len(trees)), replace=False)
    trees = [trees[i] for i in pick]
    P = W.stack([W.encode(t, 8) for t in trees])
    out, st = orc.evaluate(P.type, P.val, P.size, X)
    _ENV["x"] = x
    with np.errstate(all="ignore"):
        for i, t in enumerate(trees):
            ref, ok = _restated(_expr(t)[0], X.shape[0])
            np.testing.assert_allclose(out[i, 0][ok], ref[ok], rtol=1e-9, atol=1e-12,
                                       equal_nan=True, err_msg=str(t))


def _modi_restated(tokens, x):
    """Restatement of Sec. IV-C over explicit contribution lists: returns
    (value seen by the parent, list of (output, value))."""
    contrib = []

    def go(i):
        t = tokens[i]
        if isinstance(t, tuple) and t[0] == "x":
            return x[t[1]], i + 1
        if isinstance(t, tuple) and t[0] == "c":
            return float(t[1]), i + 1
        name, out = (t, None) if isinstance(t, str) else t
        kids = []
        j = i + 1
        for _ in range(W.ARITY[W.FUNC_NAMES.index(name)]):
            v, j = go(j)
            kids.append(v)
        args = ", ".join(repr(float(k)) for k in kids)
        with np.errstate(all="ignore"):
            val = float(eval(NP_F[name](*[f"np.float64({float(k)!r})" for k in kids])))
        if out is None:
            return val, j
        contrib.append((out, val))
        return kids[-1], j

    v, end = go(0)
    assert end == len(tokens)
    return v, contrib


def test_modi_brute_force(orc):
    rng = np.random.default_rng(5)
    X = rng.uniform(-3, 3, (16, 2)).astype(np.float32)
    trees = []
    for n in (2, 3, 4):
        for t in _trees(n):
            fpos = [i for i, tok in enumerate(t) if isinstance(tok, str)]
            for mask in range(1, 2 ** len(fpos)):
                tt = list(t)
                for b, i in enumerate(fpos):
                    if mask >> b & 1:
                        tt[i] = (tt[i], (i + b) % 2)
                trees.append(tt)
    pick = rng.choice(len(trees), size=min(2000, len(trees)), replace=False)
    trees = [trees[i] for i in pick]
    P = W.stack([W.encode(t, 8) for t in trees])
    out, st = orc.evaluate(P.type, P.val, P.size, X, n_outputs=2)
    assert (st == 0).all()
    def outputs(t, xd):
        _, contrib = _modi_restated(t, xd)
        want = np.zeros(2)
        for o, v in contrib:
            want[o] += v
        return want

    n_cmp = 0
    for i, t in enumerate(trees):
        for d in range(X.shape[0]):
            xd = X[d].astype(np.float64)
            want = outputs(t, xd)
            hi, lo = outputs(t, xd * (1 + 1e-13)), outputs(t, xd * (1 - 1e-13))
            with np.errstate(all="ignore"):
                ok = np.abs(hi - lo) <= 1e-6 * np.maximum(np.abs(want), 1.0)
            n_cmp += ok.sum()
            np.testing.assert_allclose(out[i, :, d][ok], want[ok], rtol=1e-9, atol=1e-12,
                                       equal_nan=True, err_msg=str(t))
    assert n_cmp > 0.9 * len(trees) * X.shape[0] * 2


# ---------------------------------------------------------- invariants
def test_generated_trees_satisfy_size_invariants(orc):
    for p in (W.sr_small().pop, W.random_population(11, 500, 255, max_depth=8, n_features=16),
              W.modi(pop=300, D=10).pop):
        st, ln = orc.validate(p.type, p.val, p.size, 32, 8)
        assert (st == 0).all()
        assert (ln == p.size[:, 0]).all()
        for k in range(p.pop):
            L = ln[k]
            s = p.size[k, :L].astype(int)
            ar = [0 if t in (0, 1) else (1 if (int(t) & 3) == 2 else 2) for t in p.type[k, :L]]
            for i in range(L):
                assert i + s[i] <= L
                kids, j = 0, i + 1
                for _ in range(ar[i]):
                    kids += s[j]
                    j += s[j]
                assert s[i] == 1 + kids
            assert np.isnan(p.type[k, L:]).all() and np.isnan(p.size[k, L:]).all()


def test_validator_rejections(orc):
    base = _enc(["add", ["x", 0], "sin", ["c", 1.0]], 6)

    def st_of(mut, F=1, O=1, max_len=6):
        t, v, s = base.type.copy(), base.val.copy(), base.size.copy()
        mut(t, v, s)
        return orc.validate(t, v, s, F, O, max_len)[0][0]

    assert st_of(lambda t, v, s: None) == 0
    assert st_of(lambda t, v, s: s.__setitem__((0, 0), 7)) == orc.ST_LEN
    assert st_of(lambda t, v, s: s.__setitem__((0, 0), np.nan)) == orc.ST_LEN
    assert st_of(lambda t, v, s: None, max_len=3) == orc.ST_LEN
    assert st_of(lambda t, v, s: t.__setitem__((0, 1), 5)) == orc.ST_TYPE
    assert st_of(lambda t, v, s: v.__setitem__((0, 0), 5)) == orc.ST_FUNC      # sin on a binary node
    assert st_of(lambda t, v, s: v.__setitem__((0, 0), 12)) == orc.ST_FUNC     # unknown id
    assert st_of(lambda t, v, s: v.__setitem__((0, 0), 256)) == orc.ST_FUNC    # output index on a plain node
    assert st_of(lambda t, v, s: v.__setitem__((0, 1), 1)) == orc.ST_VAR
    assert st_of(lambda t, v, s: v.__setitem__((0, 1), 0.5)) == orc.ST_VAR
    assert st_of(lambda t, v, s: v.__setitem__((0, 3), np.inf)) == orc.ST_CONST
    assert st_of(lambda t, v, s: s.__setitem__((0, 2), 1)) == orc.ST_SIZE
    assert st_of(lambda t, v, s: (t.__setitem__((0, 0), 19), v.__setitem__((0, 0), 512))) == orc.ST_MODI
    assert st_of(lambda t, v, s: (t.__setitem__((0, 0), 19), v.__setitem__((0, 0), 512)), O=3) == 0
    # a tree whose prefix ends early: [add, x0] with size 2
    t = np.array([[3, 0, np.nan]], np.float32)
    v = np.array([[0, 0, np.nan]], np.float32)
    s = np.array([[2, 1, np.nan]], np.float32)
    assert orc.validate(t, v, s, 1)[0][0] == orc.ST_SIZE


# ---------------------------------------------------------- guards
def test_guard_branches(orc):
    thr = np.float32(1e-6)
    up = np.nextafter(thr, np.float32(1))
    dn = np.nextafter(thr, np.float32(0))
    den = np.float32(1e-40)
    bs = np.array([thr, -thr, up, -up, dn, -dn, 0.0, -0.0, den, -den, 1.0], np.float32)
    X = np.stack([np.full_like(bs, 3.0), bs], 1)
    p = _enc(["pdiv", ["x", 0], ["x", 1]])
    out, _ = orc.evaluate(p.type, p.val, p.size, X)
    for b, o in zip(bs, out[0, 0]):
        if abs(float(b)) > float(thr):
            assert o == 3.0 / float(b)
        else:
            assert o == 1.0
    p = _enc(["plog", ["x", 1]])
    out, _ = orc.evaluate(p.type, p.val, p.size, X)
    for b, o in zip(bs, out[0, 0]):
        if abs(float(b)) > float(thr):
            assert o == math.log(abs(float(b)))
        else:
            assert o == 0.0
    p = _enc(["cexp", ["x", 1]])
    X2 = np.array([[0, 79.5], [0, 80.0], [0, 80.5], [0, 1e30], [0, -200.0]], np.float32)
    out, _ = orc.evaluate(p.type, p.val, p.size, X2)
    assert list(out[0, 0]) == [math.exp(79.5), math.exp(80.0), math.exp(80.0), math.exp(80.0),
                               math.exp(-200.0)]


# ---------------------------------------------------------- reverse mode
def test_reverse_mode_matches_central_differences(orc):
    pop = W.random_population(21, 40, 31, (5, 31), max_depth=10, n_features=3, p_var=0.4)
    rng = np.random.default_rng(6)
    X = rng.uniform(-1.5, 1.5, (12, 3)).astype(np.float32)
    y = rng.standard_normal(12).astype(np.float32)
    g = rng.uniform(0.5, 1.5, (pop.pop, 1))
    m, gv, gx, st = orc.grad(pop.type, pop.val, pop.size, X, y, g)
    m2, _ = orc.mse(pop.type, pop.val, pop.size, X, y)
    np.testing.assert_array_equal(m, m2)
    checked = skipped = 0

    # constants: perturb by a float32-exact step h = 2^-10 * max(|c|, 1), a
    # step of 8 ulp or more is representable exactly in float32
    for k in range(pop.pop):
        L = int(pop.size[k, 0])
        for i in range(L):
            if pop.type[k, i] != W.CONST:
                continue
            c = float(pop.val[k, i])
            h = 2.0 ** -12 * max(1.0, 2.0 ** math.ceil(math.log2(max(abs(c), 1e-30))))
            vals = []
            for s in (+1, -1):
                pv = pop.val[k:k + 1].copy()
                pv[0, i] = np.float32(c + s * h)
                assert float(pv[0, i]) == c + s * h
                mm, _ = orc.mse(pop.type[k:k + 1], pv, pop.size[k:k + 1], X, y)
                vals.append(mm[0, 0])
            fd = g[k, 0] * (vals[0] - vals[1]) / (2 * h)
            ref = gv[k, i]
            if not np.isfinite(ref) or not np.isfinite(fd):
                skipped += 1
                continue
            # the second difference bounds the truncation error of the FD
            if abs(fd - ref) > 1e-4 * max(abs(ref), 1.0):
                skipped += 1          # kink (guard, clamp, max tie) or strong curvature
                continue
            checked += 1
    assert checked >= 30
    assert skipped <= 0.1 * (checked + skipped)
    # non-constant positions carry no gradient
    nonconst = pop.type != W.CONST
    assert (gv[nonconst] == 0).all()


def test_reverse_mode_input_gradient_fd(orc):
    pop = W.random_population(22, 20, 25, (5, 25), max_depth=10, n_features=2)
    rng = np.random.default_rng(8)
    X = rng.uniform(-1, 1, (6, 2)).astype(np.float32)
    y = rng.standard_normal(6).astype(np.float32)
    g = np.ones((pop.pop, 1))
    m, gv, gx, st = orc.grad(pop.type, pop.val, pop.size, X, y, g)
    h = 2.0 ** -14
    good = bad = 0
    base_m, _ = orc.mse(pop.type, pop.val, pop.size, X, y)
    ok_tree = np.isfinite(base_m[:, 0]) & (np.abs(base_m[:, 0]) < 1e8)
    g2 = g * ok_tree[:, None]
    m, gv, gx, st = orc.grad(pop.type, pop.val, pop.size, X, y, g2)
    for d in range(X.shape[0]):
        for f in range(2):
            vals = []
            for s in (+1, -1):
                Xp = X.copy()
                Xp[d, f] = np.float32(float(X[d, f]) + s * h)
                mm, _ = orc.mse(pop.type, pop.val, pop.size, Xp, y)
                vals.append(np.sum(g2[:, 0] * np.where(ok_tree, mm[:, 0], 0.0)))
            fd = (vals[0] - vals[1]) / (2 * h)
            if abs(fd - gx[d, f]) <= 1e-4 * max(abs(gx[d, f]), 1.0):
                good += 1
            else:
                bad += 1
    assert good >= 10 and bad <= 2


def test_modi_reverse_mode_closed_form(orc):
    ex = GOLD["modi"]
    p = _enc(ex["tokens"])
    rng = np.random.default_rng(9)
    X = rng.uniform(0.5, 2.0, (7, 5)).astype(np.float32)
    Y = rng.standard_normal((7, 3)).astype(np.float32)
    g = np.array([[0.7, 1.3, -0.4]])
    m, gv, gx, st = orc.grad(p.type, p.val, p.size, X, Y, g, n_outputs=3)
    a, b, c, d, e = (X[:, i].astype(np.float64) for i in range(5))
    y = Y.astype(np.float64)
    r1 = a / c * 0.5 - y[:, 0]
    r2 = np.maximum(b, c) + (d - 0.5) - y[:, 1]
    r3 = e + 0.5 - y[:, 2]
    D = 7
    s1, s2, s3 = 2 * g[0, 0] * r1 / D, 2 * g[0, 1] * r2 / D, 2 * g[0, 2] * r3 / D
    np.testing.assert_allclose(gx[:, 0], s1 * 0.5 / c, rtol=1e-12)
    np.testing.assert_allclose(gx[:, 1], s2 * (b >= c), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(gx[:, 2], s1 * (-a * 0.5 / c ** 2) + s2 * (c > b), rtol=1e-12)
    np.testing.assert_allclose(gx[:, 3], s2, rtol=1e-12)
    np.testing.assert_allclose(gx[:, 4], s3, rtol=1e-12)
    # the constant 0.5 (position 10) enters o1 (factor a/c), o2 (-1) and o3 (+1)
    want = np.sum(s1 * a / c - s2 + s3)
    assert gv[0, 10] == pytest.approx(want, rel=1e-12)


# ---------------------------------------------------------- error bound
def _f32_eval(tokens, x):
    """float32 evaluation with numpy's float32 kernels (correctly rounded
    basic ops, ~1 ulp transcendental functions)."""
    f = np.float32

    def go(i):
        t = tokens[i]
        if isinstance(t, tuple) and t[0] == "x":
            return x[:, t[1]].astype(f), i + 1
        if isinstance(t, tuple) and t[0] == "c":
            return np.full(x.shape[0], t[1], f), i + 1
        a, j = go(i + 1)
        if W.ARITY[W.FUNC_NAMES.index(t)] == 2:
            b, j = go(j)
        with np.errstate(all="ignore"):
            r = {"add": lambda: a + b, "sub": lambda: a - b, "mul": lambda: a * b,
                 "pdiv": lambda: np.where(np.abs(b) > f(1e-6), a / b, f(1)),
                 "max": lambda: np.fmax(a, b), "sin": lambda: np.sin(a), "cos": lambda: np.cos(a),
                 "plog": lambda: np.where(np.abs(a) > f(1e-6), np.log(np.abs(a)), f(0)),
                 "cexp": lambda: np.exp(np.minimum(a, f(80))), "tan": lambda: np.tan(a)}[t]()
        return r.astype(f), j

    return go(0)[0]


def _decode(pop, k):
    toks = []
    L = int(pop.size[k, 0])
    for i in range(L):
        t, v = int(pop.type[k, i]), float(pop.val[k, i])
        toks.append(("x", int(v)) if t == 0 else ("c", v) if t == 1 else W.FUNC_NAMES[int(v) % 256])
    return toks


def test_error_bound_covers_float32_evaluation(orc):
    pop = W.random_population(31, 300, 63, (1, 63), max_depth=8, n_features=3)
    rng = np.random.default_rng(10)
    X = rng.standard_normal((200, 3)).astype(np.float32)
    out, err, st = orc.evaluate(pop.type, pop.val, pop.size, X, with_err=True)
    n_fin = n_viol = 0
    for k in range(pop.pop):
        v32 = _f32_eval(_decode(pop, k), X).astype(np.float64)
        ok = np.isfinite(err[k, 0]) & np.isfinite(out[k, 0])
        n_fin += ok.sum()
        n_viol += (np.abs(v32[ok] - out[k, 0][ok]) > err[k, 0][ok]).sum()
    assert n_fin > 0.8 * pop.pop * X.shape[0]
    assert n_viol == 0


def test_error_bound_flags_ill_conditioned_points(orc):
    # (x0 + 1) - 1 cancels: the bound must grow as 1/|x0| relative to the value
    p = _enc(["sub", "add", ["x", 0], ["c", 1.0], ["c", 1.0]])
    X = np.array([[1e-3], [1e-6], [2.0]], np.float32)
    out, err, _ = orc.evaluate(p.type, p.val, p.size, X, with_err=True)
    assert err[0, 0, 1] / abs(out[0, 0, 1]) > err[0, 0, 2] / abs(out[0, 0, 2]) * 1e4
    # a guard operand within its error of the threshold makes the bound
    # infinite: 3 * fl(1/3) rounds in FP32 by ~3e-8, and the difference to
    # fl(1 - 1e-6) lands 4e-8 above the 1e-6f threshold
    p = _enc(["pdiv", ["c", 1.0], "sub", "mul", ["x", 0], ["x", 1], ["x", 2]])
    X = np.array([[3.0, 1.0 / 3.0, 1.0 - 1e-6]], np.float32)
    out, err, _ = orc.evaluate(p.type, p.val, p.size, X, with_err=True)
    assert np.isinf(err[0, 0, 0])
    # the same operand computed exactly (Sterbenz subtraction) is not ambiguous
    p = _enc(["pdiv", ["c", 1.0], "sub", ["x", 0], ["c", 1.0]])
    X = np.array([[np.float32(1.0) + np.float32(1e-6)]], np.float32)
    out, err, _ = orc.evaluate(p.type, p.val, p.size, X, with_err=True)
    assert out[0, 0, 0] == 1.0 and err[0, 0, 0] < 1e-30


# ---------------------------------------------------------- GPops/s
def test_gpops_definition_reproduces_table():
    from paper_2501_17168_gb300.metrics import gpops
    g = GOLD["gpops"]
    assert gpops(g["G"], g["P"], g["S"], g["D"], g["T"]) == pytest.approx(g["gpops"], rel=5e-3)


# ---------------------------------------------------------- gradient bound
def test_gradient_bound_covers_float32_reverse_mode(orc):
    """The oracle's per-element bound on the FP32 gradient covers a plain
    float32 restatement of the reverse mode (numpy float32 per point, FP64
    sums, so no FP32 partial sums: acc_terms = 1) on random single-output
    and Modi populations."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from parity import f32_grad
    rng = np.random.default_rng(3)
    cases = []
    p = W.random_population(31, 300, 63, (1, 63), max_depth=8, n_features=3, max_consts=16)
    cases.append((p, rng.standard_normal((200, 3)).astype(np.float32),
                  rng.standard_normal((200, 1)).astype(np.float32), 1))
    q = W.random_population(32, 200, 31, (1, 31), max_depth=6, n_features=2,
                            fset=(W.ADD, W.SUB, W.MUL, W.SIN, W.COS, W.MAX))
    cases.append((q, rng.uniform(-1, 1, (150, 2)).astype(np.float32),
                  rng.standard_normal((150, 1)).astype(np.float32), 1))
    m = W.modi(pop=100, D=150, n_outputs=3)
    cases.append((m.pop, m.X, rng.standard_normal((150, 3)).astype(np.float32), 3))
    n_c = n_x = 0
    for p, X, y, O in cases:
        rm, rgv, rgx, rst, egv, egx = orc.grad(p.type, p.val, p.size, X, y, 1.0, n_outputs=O,
                                               with_err=True, acc_terms=1)
        gv32, gx32 = f32_grad(p.type, p.val, p.size, X, y, 1.0, O)
        const = p.type == W.CONST
        with np.errstate(all="ignore"):
            okc = const & np.isfinite(egv)
            okx = np.isfinite(egx)
            assert not (np.abs(gv32 - rgv) > egv)[okc].any()
            assert not (np.abs(gx32 - rgx) > egx)[okx].any()
        n_c += int(okc.sum())
        n_x += int(okx.sum())
    assert n_c > 2000 and n_x > 1000


def test_gradient_bound_is_tight_on_well_conditioned_trees(orc):
    """For c * x0 and sin(c * x0 + x1) over well-scaled data the bound is a
    small multiple of u times the sum of the magnitudes of the contributions
    (not vacuous), and it grows with the FP32 partial-sum length; the max
    rule's undecided ties count as a unit derivative error, guards left
    undecided by their operand's error make the bound infinite."""
    u = 2.0 ** -24
    rng = np.random.default_rng(4)
    X = rng.uniform(0.5, 2, (400, 2)).astype(np.float32)
    y = np.zeros((400, 1), np.float32)
    for toks in (["mul", ("c", 0.75), ("x", 0)],
                 ["sin", "add", "mul", ("c", 0.75), ("x", 0), ("x", 1)]):
        p = _enc(toks)
        _, gv, gx, st, egv, egx = orc.grad(p.type, p.val, p.size, X, y, 1.0, with_err=True, acc_terms=1)
        c = int(np.flatnonzero(p.type[0] == W.CONST)[0])
        out, _ = orc.evaluate(p.type, p.val, p.size, X)
        # per point |adjoint of c| = |2 o / D * do/dc| <= 2 |o| |x0| / D here
        mag = np.sum(2 * np.abs(out[0, 0]) * X[:, 0].astype(np.float64) / 400)
        assert 0 < egv[0, c] <= 64 * u * mag, (egv[0, c], mag)
        _, _, _, _, egv2, _ = orc.grad(p.type, p.val, p.size, X, y, 1.0, with_err=True, acc_terms=400)
        assert egv2[0, c] >= egv[0, c] + 300 * u * abs(gv[0, c])
    # max(x0, x0 + c) at c = 0 and c tiny: an exact tie is decided, a tie the
    # rounding of x0 + c may break is a unit derivative error
    # (the adjoint reaches x0 through the max, so the input gradient shows it)
    p = _enc(["mul", ("c", 1.0), "max", ("x", 0), "add", ("x", 0), ("c", 1e-9)])
    _, gv, gx, _, egv, egx = orc.grad(p.type, p.val, p.size, X, y, 1.0, with_err=True, acc_terms=1)
    assert np.isfinite(egx[:, 0]).all() and (egx[:, 0] > 0.1 * np.abs(gx[:, 0])).all()
    assert egv[0, 1] <= 64 * u * np.sum(np.abs(gx[:, 0] * X[:, 0]))
    p = _enc(["mul", ("c", 1.0), "max", ("x", 0), ("x", 0)])
    _, gv, gx, _, egv, egx = orc.grad(p.type, p.val, p.size, X, y, 1.0, with_err=True, acc_terms=1)
    assert (egx[:, 0] <= 64 * u * np.abs(gx[:, 0])).all()
    # a protected division whose divisor lies within its error of the guard
    p = _enc(["pdiv", ("c", 1.0), "sub", "mul", ("x", 0), ("x", 1), ("x", 2)])
    Xg = np.array([[3.0, 1.0 / 3.0, 1.0 - 1e-6]], np.float32)
    out, err, _ = orc.evaluate(p.type, p.val, p.size, Xg, with_err=True)
    _, _, _, _, egv, _ = orc.grad(p.type, p.val, p.size, Xg, np.zeros((1, 1), np.float32), 1.0,
                                  with_err=True)
    assert not np.isfinite(err[0, 0, 0]) and np.isinf(egv[0, 1])


# ---------------------------------------------------------- ternary ite
def test_ite_selects_by_the_sign_of_its_condition(orc):
    """ite(a, b, c) = a > 0 ? b : c (the library's ternary function; type
    code 4, the arity the encoding's (type, value) pair names, Sec. III-A):
    exact selection, a zero, negative zero or NaN condition selects c."""
    p = _enc(["ite", ["x", 0], ["x", 1], ["x", 2]])
    assert list(p.type[0]) == [W.TFUNC, W.VAR, W.VAR, W.VAR] and p.size[0, 0] == 4
    conds = np.array([1.0, -1.0, 0.0, -0.0, np.nan, 1e-45, -1e-45, np.inf, -np.inf, 3e38],
                     np.float32)
    rng = np.random.default_rng(21)
    X = np.stack([conds, rng.standard_normal(10), rng.standard_normal(10)], 1).astype(np.float32)
    out, st = orc.evaluate(p.type, p.val, p.size, X)
    assert st[0] == 0
    want = np.where(X[:, 0] > 0, X[:, 1], X[:, 2]).astype(np.float64)
    np.testing.assert_array_equal(out[0, 0], want)


def test_ite_modi_passes_its_third_child(orc):
    # add·M(o0)(ite·M(o1)(x0, x1, x2), x3): output 1 = ite(x0, x1, x2); the
    # ite node hands its parent x2, so output 0 = x2 + x3
    p = _enc([("add", 0), ("ite", 1), ["x", 0], ["x", 1], ["x", 2], ["x", 3]])
    X = np.random.default_rng(22).standard_normal((64, 4)).astype(np.float32)
    out, st = orc.evaluate(p.type, p.val, p.size, X, n_outputs=2)
    x = X.astype(np.float64)
    np.testing.assert_array_equal(out[0, 1], np.where(x[:, 0] > 0, x[:, 1], x[:, 2]))
    np.testing.assert_allclose(out[0, 0], x[:, 2] + x[:, 3], rtol=1e-15)


def test_ite_validator_and_gradient_routing(orc):
    ok = _enc(["ite", ["x", 0], ["c", 1.0], ["x", 1]])
    t, v, s = ok.type.copy(), ok.val.copy(), ok.size.copy()
    st, _ = orc.validate(t, v, s, 2)
    assert st[0] == 0
    bad = t.copy(); bad[0, 0] = W.BFUNC          # ite under the binary type
    assert orc.validate(bad, v, s, 2)[0][0] & orc.ST_FUNC
    bad = t.copy(); bv = v.copy(); bv[0, 0] = W.ADD   # a binary id under the ternary type
    assert orc.validate(bad, bv, s, 2)[0][0] & orc.ST_FUNC
    bs = s.copy(); bs[0, 0] = 3                    # sizes that do not tile three children
    assert orc.validate(t, v, bs, 2)[0][0] & orc.ST_SIZE
    # d MSE / d x1 reaches x1 only where x0 <= 0; the condition gets nothing
    p = _enc(["mul", ["c", 1.5], "ite", ["x", 0], ["x", 1], ["x", 2]])
    X = np.random.default_rng(23).standard_normal((200, 3)).astype(np.float32)
    y = np.zeros((200, 1), np.float32)
    m, gv, gx, st = orc.grad(p.type, p.val, p.size, X, y, 1.0)
    x = X.astype(np.float64)
    sel = np.where(x[:, 0] > 0, x[:, 1], x[:, 2])
    o = 1.5 * sel
    np.testing.assert_allclose(gx[:, 0], 0.0)
    np.testing.assert_allclose(gx[:, 1], np.where(x[:, 0] > 0, 2 * o * 1.5 / 200, 0.0), rtol=1e-12)
    np.testing.assert_allclose(gx[:, 2], np.where(x[:, 0] > 0, 0.0, 2 * o * 1.5 / 200), rtol=1e-12)
    np.testing.assert_allclose(gv[0, 1], np.sum(2 * o * sel / 200), rtol=1e-12)


def test_ite_bound_is_infinite_where_the_sign_is_undecided(orc):
    # sub(x0, x1) = 1e-30 - 1e-30 rounds exactly (0); (x0 * x1) - x2 carries
    # rounding error around 0: the branch is undecided there
    p = _enc(["ite", "sub", "mul", ["x", 0], ["x", 1], ["x", 2], ["c", 1.0], ["c", -1.0]])
    X = np.array([[3.0, 1.0 / 3.0, 1.0], [3.0, 1.0, 1.0], [2.0, 2.0, 1.0]], np.float32)
    out, err, _ = orc.evaluate(p.type, p.val, p.size, X, with_err=True)
    assert np.isinf(err[0, 0, 0])          # 3 * fl(1/3) - 1 is within its rounding of 0
    assert err[0, 0, 2] == 0.0 and out[0, 0, 2] == 1.0


def test_error_bound_covers_float32_evaluation_with_ite(orc):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from parity import f32_eval
    pop = W.random_population(33, 300, 63, (1, 63), max_depth=8, n_features=3, fset=W.TERNARY_FSET)
    m = W.random_population(34, 100, 63, (5, 63), max_depth=8, n_features=3, fset=W.TERNARY_FSET,
                            n_outputs=3, modi=True)
    assert (pop.type == W.TFUNC).sum() > 100 and (m.type == W.TFUNC + W.MODI).sum() > 5
    X = np.random.default_rng(12).standard_normal((200, 3)).astype(np.float32)
    for p, O in ((pop, 1), (m, 3)):
        out, err, st = orc.evaluate(p.type, p.val, p.size, X, n_outputs=O, with_err=True)
        assert (st == 0).all()
        v32 = f32_eval(p.type, p.val, p.size, X, O).astype(np.float64)
        ok = np.isfinite(err) & np.isfinite(out)
        assert ok.mean() > 0.8
        assert not (np.abs(v32[ok] - out[ok]) > err[ok]).any()
