"""Pins of the genetic-operator oracle (``oracle/genetic.py``) against facts
that do not come from it.

* subtree exchange (Sec. III-B) against token surgery: the child's prefix
  token list is spliced with subtree extents found by counting arities, and
  its subtree sizes are recomputed from scratch by the input encoder -- so a
  wrong ancestor set, a wrong dn or a wrong segment boundary fails;
* the ancestor walk against the definition (k lies inside the subtree of i);
* closed forms: the evaluated child of a hand-built crossover equals the
  algebraic expression it must become;
* special cases: exchanging a subtree with itself is the identity; hoisting at
  the root yields the chosen subtree; the size limit is inclusive and a
  rejected child is the old tree;
* tournament selection against a vectorised restatement (numpy lexicographic
  argmin) and against the closed-form probability that the best tree wins;
* classification accuracy against numpy's argmax and a two-output Modi tree
  whose prediction has a closed form.
"""
import numpy as np
import pytest

from paper_2501_17168_gb300 import workloads as W


@pytest.fixture(scope="module")
def gen(orc):
    from oracle import genetic
    return genetic


def _tokens(t, v, s):
    """Prefix token list of one tree (the input encoder's vocabulary)."""
    out = []
    for i in range(int(s[0])):
        ty, va = int(t[i]), float(v[i])
        if ty == 0:
            out.append(("x", int(va)))
        elif ty == 1:
            out.append(("c", va))
        else:
            name = W.FUNC_NAMES[int(va) % 256]
            out.append((name, int(va) // 256) if ty >= 16 else name)
    return out


def _arity(tok):
    if isinstance(tok, tuple) and tok[0] in ("x", "c"):
        return 0
    name = tok if isinstance(tok, str) else tok[0]
    return W.ARITY[W.FUNC_NAMES.index(name)]


def _extent(tokens, k):
    """End of the subtree at k, by counting open child slots."""
    need, i = 1, k
    while need:
        need += _arity(tokens[i]) - 1
        i += 1
    return i


def _row(pop, i):
    n = int(pop.size[i, 0])
    return pop.type[i, :n], pop.val[i, :n], pop.size[i, :n]


def _same(a, b):
    return np.array_equal(np.asarray(a, np.float32), np.asarray(b, np.float32), equal_nan=True)


def test_ancestors_match_definition(gen):
    pop = W.random_population(5, 60, 63, (1, 63), max_depth=8, n_features=2)
    for p in range(pop.pop):
        t, v, s = _row(pop, p)
        toks = _tokens(t, v, s)
        n = len(toks)
        for k in range(n):
            want = [i for i in range(k) if _extent(toks, i) > k]
            assert gen.ancestors(t, s, k) == want


def test_exchange_matches_token_surgery(gen):
    rng = np.random.default_rng(1)
    a = W.random_population(6, 80, 63, (1, 63), max_depth=8, n_features=3)
    b = W.random_population(7, 80, 63, (1, 63), max_depth=8, n_features=3)
    for p in range(a.pop):
        ta, va, sa = _row(a, p)
        tb, vb, sb = _row(b, p)
        k = int(rng.integers(len(ta)))
        j = int(rng.integers(len(tb)))
        m = int(sb[j])
        t, v, z, st = gen.exchange(ta, va, sa, k, tb[j:j + m], vb[j:j + m], sb[j:j + m], 10 ** 6)
        assert st == gen.DONE
        old, don = _tokens(ta, va, sa), _tokens(tb, vb, sb)
        want = old[:k] + don[j:_extent(don, j)] + old[_extent(old, k):]
        ref = W.encode(want)
        assert _same(t, ref.type[0]) and _same(v, ref.val[0]) and _same(z, ref.size[0])


def test_exchange_closed_form(gen, orc):
    # mul(add(x0, 1.5), sin(x1)) with add(...) replaced by cos(x0) -> cos(x0) * sin(x1)
    old = W.encode(["mul", "add", ("x", 0), ("c", 1.5), "sin", ("x", 1)])
    new = W.encode(["cos", ("x", 0)])
    t, v, z, st = gen.exchange(old.type[0], old.val[0], old.size[0], 1, new.type[0], new.val[0],
                               new.size[0], 64)
    assert st == gen.DONE and list(z) == [5, 2, 1, 2, 1]
    X = np.random.default_rng(2).uniform(-2, 2, (50, 2)).astype(np.float32)
    out, _ = orc.evaluate(t, v, z, X)
    x = X.astype(np.float64)
    np.testing.assert_allclose(out[0, 0], np.cos(x[:, 0]) * np.sin(x[:, 1]), rtol=1e-15)


def test_exchange_with_own_subtree_is_identity(gen):
    pop = W.random_population(8, 40, 127, (1, 127), max_depth=10, n_features=2)
    for p in range(pop.pop):
        t, v, s = _row(pop, p)
        for k in range(len(t)):
            m = int(s[k])
            c = gen.exchange(t, v, s, k, t[k:k + m], v[k:k + m], s[k:k + m], len(t))
            assert c[3] == gen.DONE and _same(c[0], t) and _same(c[1], v) and _same(c[2], s)


def test_size_limit_is_inclusive_and_rejection_keeps_old_tree(gen):
    old = W.encode(["add", ("x", 0), ("x", 1)])
    new = W.encode(["mul", ("x", 0), ("c", 2.0)])
    args = (old.type[0], old.val[0], old.size[0], 2, new.type[0], new.val[0], new.size[0])
    t, v, z, st = gen.exchange(*args, 5)          # 3 + 2 = 5 nodes: allowed
    assert st == gen.DONE and list(z) == [5, 1, 3, 1, 1]
    t, v, z, st = gen.exchange(*args, 4)          # one over: the old tree comes back
    assert st == gen.TOO_LARGE and _same(t, old.type[0]) and _same(z, old.size[0])


def test_population_modes_and_statuses(gen, orc):
    rng = np.random.default_rng(3)
    a = W.random_population(9, 50, 63, (1, 63), max_depth=8, n_features=2)
    b = W.random_population(10, 30, 63, (1, 63), max_depth=8, n_features=2)
    n = 200
    oi = rng.integers(0, a.pop, n).astype(np.int32)
    di = rng.integers(0, b.pop, n).astype(np.int32)
    r1 = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    r2 = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    old, don = (a.type, a.val, a.size), (b.type, b.val, b.size)
    # crossover: splice the chosen subtree of the donor at the chosen node
    t, v, z, st = gen.subtree_exchange(old, don, oi, r1, di, r2, gen.RANDOM, 80, 96)
    assert set(st) <= {gen.DONE, gen.TOO_LARGE}
    for i in range(n):
        ta, va, sa = _row(a, oi[i])
        tb, vb, sb = _row(b, di[i])
        k, j = int(r1[i]) % len(ta), int(r2[i]) % len(tb)
        oldt, dont = _tokens(ta, va, sa), _tokens(tb, vb, sb)
        want = oldt[:k] + dont[j:_extent(dont, j)] + oldt[_extent(oldt, k):]
        if len(want) > 80:
            want = oldt
            assert st[i] == gen.TOO_LARGE
        ref = W.encode(want, 96)
        assert _same(t[i], ref.type[0]) and _same(v[i], ref.val[0]) and _same(z[i], ref.size[0])
    good = st == gen.DONE
    vs, _ = orc.validate(t[good], v[good], z[good], 2, 1, 80)
    assert (vs == 0).all()
    # hoist: a subtree inside the chosen subtree replaces it; never grows
    t, v, z, st = gen.subtree_exchange(old, None, oi, r1, None, r2, gen.HOIST, 63, 63)
    assert (st == gen.DONE).all()
    for i in range(n):
        ta, va, sa = _row(a, oi[i])
        k = int(r1[i]) % len(ta)
        j = k + int(r2[i]) % int(sa[k])
        toks = _tokens(ta, va, sa)
        want = toks[:k] + toks[j:_extent(toks, j)] + toks[_extent(toks, k):]
        ref = W.encode(want, 63)
        assert _same(t[i], ref.type[0]) and _same(z[i], ref.size[0])
        assert z[i, 0] <= sa[0]
    # hoist at the root gives the chosen subtree itself
    zero = np.zeros(n, np.uint32)
    t, v, z, st = gen.subtree_exchange(old, None, oi, zero, None, r2, gen.HOIST, 63, 63)
    for i in range(n):
        ta, va, sa = _row(a, oi[i])
        j = int(r2[i]) % int(sa[0])
        m = int(sa[j])
        assert _same(t[i, :m], ta[j:j + m]) and _same(z[i, :m], sa[j:j + m])
        assert np.isnan(t[i, m:]).all()
    # statuses: indices out of range and malformed lengths or sizes
    bad_t = a.type.copy(), a.val.copy(), a.size.copy()
    bad_t[2][1, 0] = np.nan                      # tree 1: no length
    bad_t[2][2, 1] = 1000.0                      # tree 2: size[1] beyond the tree
    oi2 = np.array([-1, a.pop, 1, 2, 0, 0], np.int32)
    k2 = np.array([0, 0, 0, 1, 10 ** 6, 0], np.uint32)
    j2 = np.array([0, 0, 0, 0, 0, 10 ** 6], np.uint32)
    di2 = np.zeros(6, np.int32)
    t, v, z, st = gen.subtree_exchange(bad_t, don, oi2, k2, di2, j2, gen.EXPLICIT, 63, 63)
    assert list(st) == [gen.BAD_INDEX, gen.BAD_INDEX, gen.BAD_TREE, gen.BAD_TREE, gen.BAD_INDEX,
                        gen.BAD_INDEX]
    assert np.isnan(t).all() and np.isnan(z).all()
    # operator probability: children whose word is not below the threshold are copies
    aw = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    thr = int(0.3 * 2 ** 32)
    t, v, z, st = gen.subtree_exchange(old, don, oi, r1, di, r2, gen.RANDOM, 80, 96, apply_word=aw,
                                       apply_below=thr)
    t0, v0, z0, st0 = gen.subtree_exchange(old, don, oi, r1, di, r2, gen.RANDOM, 80, 96)
    on = aw < thr
    assert (st[~on] == gen.SKIPPED).all() and (st[on] == st0[on]).all()
    assert _same(t[on], t0[on]) and _same(z[on], z0[on])
    for i in np.flatnonzero(~on):
        ta, va, sa = _row(a, oi[i])
        L = len(ta)
        assert _same(t[i, :L], ta) and _same(v[i, :L], va) and _same(z[i, :L], sa)
        assert np.isnan(t[i, L:]).all()


def _tournament_vectorised(f, words, minimize):
    P = f.shape[0]
    c = (words.astype(np.int64) % P)
    val = f[c] if minimize else -f[c]
    nan = np.isnan(val)
    val = np.where(nan, 0.0, val)
    m = np.arange(words.shape[1])[None, :].repeat(words.shape[0], 0)
    out = np.empty(words.shape[0], np.int32)
    for i in range(words.shape[0]):
        order = np.lexsort((m[i], val[i], nan[i]))   # NaN last, then value, then draw order
        out[i] = c[i, order[0]]
    return out


def test_tournament_against_vectorised_restatement(gen):
    rng = np.random.default_rng(4)
    for P, t, spread in ((1, 3, 0), (7, 1, 0), (50, 20, 0), (1000, 20, 0), (300, 64, 0),
                         (50, 20, 3), (200, 8, 2)):
        f = rng.standard_normal(P)
        if spread:                                   # ties at the optimum
            f = rng.integers(0, spread, P).astype(np.float64)
        f[rng.random(P) < 0.1] = np.nan
        f[rng.random(P) < 0.1] = np.inf
        f[rng.random(P) < 0.2] = 0.5                 # ties
        w = rng.integers(0, 2 ** 32, (400, t), dtype=np.uint64).astype(np.uint32)
        for mn in (True, False):
            assert (gen.tournament(f, w, mn) == _tournament_vectorised(f, w, mn)).all()


def test_tournament_best_tree_probability(gen):
    # distinct fitness: the best of P trees wins a size-t tournament with
    # probability 1 - (1 - 1/P)^t (contestants drawn with replacement)
    rng = np.random.default_rng(5)
    P, t, n = 100, 20, 200_000
    f = rng.permutation(P).astype(np.float64)
    w = rng.integers(0, 2 ** 32, (n, t), dtype=np.uint64).astype(np.uint32)
    win = _tournament_vectorised(f, w, True)
    p = 1 - (1 - 1 / P) ** t
    got = np.mean(f[win] == 0)
    assert abs(got - p) < 5 * np.sqrt(p * (1 - p) / n)
    sub = w[:2000]
    assert (gen.tournament(f, sub) == win[:2000]).all()


def _predict_loop(o):
    """First index of the largest non-NaN value, scanning once; -1 if none."""
    pred, best = -1, None
    for k, v in enumerate(o):
        if v != v:
            continue
        if pred < 0 or v > best:
            pred, best = k, v
    return pred


def test_accuracy_from_outputs_against_scan(gen):
    rng = np.random.default_rng(6)
    P, C, D = 6, 5, 300
    out = rng.integers(-2, 3, (P, C, D)).astype(np.float32)      # many ties
    out[rng.random((P, C, D)) < 0.15] = np.nan
    out[rng.random((P, C, D)) < 0.05] = -np.inf
    out[0, :, :10] = np.nan                                      # points with no prediction
    out[1, :, :10] = -np.inf                                     # all -inf: class 0
    out[2, 0, :10], out[2, 1:, :10] = np.nan, -np.inf            # NaN then -inf: class 1
    lab = rng.integers(0, C, D).astype(np.int32)
    acc, cnt = gen.accuracy_from_outputs(out, lab)
    pred = np.array([[_predict_loop(out[p, :, d]) for d in range(D)] for p in range(P)])
    assert (pred[1, :10] == 0).all() and (pred[2, :10] == 1).all() and (pred[0, :10] == -1).all()
    assert (gen.predict(out) == pred).all()
    want = ((pred >= 0) & (pred == lab[None, :])).sum(1)
    assert (cnt == want).all()
    np.testing.assert_array_equal(acc, want / D)


def test_accuracy_of_two_output_modi_tree(gen, orc):
    # add_M0(sub_M1(x1, 0), x0): output 1 is x1, output 0 is 0 + x0
    tree = W.encode([("add", 0), ("sub", 1), ("x", 1), ("c", 0.0), ("x", 0)])
    rng = np.random.default_rng(7)
    X = rng.standard_normal((500, 2)).astype(np.float32)
    X[:20, 1] = X[:20, 0]                                        # exact ties -> class 0
    lab = rng.integers(0, 2, 500).astype(np.int32)
    acc, cnt, amb, st = gen.accuracy(tree.type, tree.val, tree.size, X, lab, 2)
    pred = (X[:, 1] > X[:, 0]).astype(np.int32)
    assert st[0] == 0 and cnt[0] == np.sum(pred == lab)
    assert acc[0] == np.sum(pred == lab) / 500
    assert amb[0] >= 20                                          # ties are ambiguous in FP32
