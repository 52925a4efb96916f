"""Property tests (hypothesis) of the oracle and the host logic, on CPU.

Random prefix trees drawn by a recursive strategy (any shape, any mix of
functions, variables and constants), random padding widths and random point
counts:

* encoding invariants of Sec. III-A: size[i] = 1 + sizes of its children,
  len = size[0], validation passes, padding is never read (the result does
  not change with the padding width or its contents);
* the MSE is the mean of the squared residuals of the evaluated outputs
  (Sec. III-C), and its point-sharded combination equals the whole;
* subtree exchange (Sec. III-B): the child is valid, has the length
  len_old - size_old[k] + size_donor[j], and evaluates exactly like the old
  tree with the subtree at k replaced (the child built by token surgery);
* tournament selection: the winner is a contestant, its fitness is the best
  among them (a number beats NaN) and no earlier contestant ties it;
* accuracy is unchanged when the points (with their labels) are permuted.
"""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import HealthCheck, given, settings, strategies as st  # noqa: E402

from paper_2501_17168_gb300 import shard, workloads as W  # noqa: E402

SETTINGS = settings(max_examples=60, deadline=None,
                    suppress_health_check=[HealthCheck.too_slow, HealthCheck.data_too_large])
FUNCS = list(W.FUNC_NAMES)


def _leaf(F):
    return st.one_of(st.tuples(st.just("x"), st.integers(0, F - 1)),
                     st.tuples(st.just("c"), st.floats(-3, 3, width=32)))


def _tree(F, max_leaves=12):
    """Nested trees: a leaf, or (function, [children])."""
    return st.recursive(
        _leaf(F),
        lambda kids: st.one_of(
            st.tuples(st.sampled_from([f for f in FUNCS if W.ARITY[FUNCS.index(f)] == 1]),
                      st.lists(kids, min_size=1, max_size=1)),
            st.tuples(st.sampled_from([f for f in FUNCS if W.ARITY[FUNCS.index(f)] == 2]),
                      st.lists(kids, min_size=2, max_size=2))),
        max_leaves=max_leaves)


def _tokens(t):
    """Prefix tokens of a nested tree."""
    out = []

    def go(n):
        if isinstance(n, tuple) and n[0] in ("x", "c") and not isinstance(n[1], list):
            out.append(n)
            return
        f, kids = n
        out.append(f)
        for c in kids:
            go(c)
    go(t)
    return out


def _arity(tok):
    if isinstance(tok, tuple) and tok[0] in ("x", "c"):
        return 0
    return W.ARITY[FUNCS.index(tok if isinstance(tok, str) else tok[0])]


def _extent(tokens, k):
    need, i = 1, k
    while need:
        need += _arity(tokens[i]) - 1
        i += 1
    return i


@SETTINGS
@given(t=_tree(3), pad=st.integers(0, 9), fill=st.sampled_from([np.nan, 0.0, 7.0]))
def test_encoding_invariants_and_padding_is_never_read(orc, t, pad, fill):
    toks = _tokens(t)
    p = W.encode(toks)
    n = len(toks)
    s = p.size[0]
    assert s[0] == n
    for i in range(n):
        kids, j = [], i + 1
        for _ in range(_arity(toks[i])):
            kids.append(int(s[j]))
            j += int(s[j])
        assert s[i] == 1 + sum(kids)
    st_, ln = orc.validate(p.type, p.val, p.size, 3)
    assert st_[0] == 0 and ln[0] == n
    wide = W.encode(toks, n + pad)
    for a in (wide.type, wide.val, wide.size):
        a[0, n:] = fill
    X = np.random.default_rng(0).uniform(-2, 2, (17, 3)).astype(np.float32)
    o1, _ = orc.evaluate(p.type, p.val, p.size, X)
    o2, _ = orc.evaluate(wide.type, wide.val, wide.size, X)
    assert np.array_equal(o1, o2, equal_nan=True)


@SETTINGS
@given(t=_tree(2), D=st.integers(1, 40), cut=st.integers(0, 40))
def test_mse_is_mean_squared_residual_and_shards_combine(orc, t, D, cut):
    p = W.encode(_tokens(t))
    r = np.random.default_rng(D)
    X = r.uniform(-2, 2, (D, 2)).astype(np.float32)
    y = r.standard_normal((D, 1)).astype(np.float32)
    m, _ = orc.mse(p.type, p.val, p.size, X, y)
    out, _ = orc.evaluate(p.type, p.val, p.size, X)
    with np.errstate(all="ignore"):
        ref = np.mean((out[0, 0] - y[:, 0].astype(np.float64)) ** 2)
        c = min(cut, D)
        parts = [(orc.mse(p.type, p.val, p.size, X[a:b], y[a:b])[0][0, 0], b - a)
                 for a, b in ((0, c), (c, D)) if b > a]
        comb = sum(v * n for v, n in parts) / D
    if np.isfinite(ref):
        assert abs(m[0, 0] - ref) <= 1e-12 * max(abs(ref), 1e-300)
        assert abs(comb - ref) <= 1e-12 * max(abs(ref), 1e-300)
    else:
        assert not np.isfinite(m[0, 0])


@SETTINGS
@given(a=_tree(2, 16), b=_tree(2, 16), data=st.data())
def test_exchange_child_is_the_spliced_tree(orc, a, b, data):
    from oracle import genetic
    ta, tb = _tokens(a), _tokens(b)
    k = data.draw(st.integers(0, len(ta) - 1))
    j = data.draw(st.integers(0, len(tb) - 1))
    A, B = W.encode(ta), W.encode(tb)
    m = int(B.size[0, j])
    t, v, z, status = genetic.exchange(A.type[0], A.val[0], A.size[0], k, B.type[0, j:j + m],
                                       B.val[0, j:j + m], B.size[0, j:j + m], 10 ** 6)
    assert status == genetic.DONE
    assert len(t) == len(ta) - int(A.size[0, k]) + m
    want = W.encode(ta[:k] + tb[j:_extent(tb, j)] + ta[_extent(ta, k):])
    assert np.array_equal(z, want.size[0]) and np.array_equal(t, want.type[0])
    st_, _ = orc.validate(t[None], v[None], z[None], 2)
    assert st_[0] == 0
    X = np.random.default_rng(1).uniform(-2, 2, (9, 2)).astype(np.float32)
    o1, _ = orc.evaluate(t[None], v[None], z[None], X)
    o2, _ = orc.evaluate(want.type, want.val, want.size, X)
    assert np.array_equal(o1, o2, equal_nan=True)


@SETTINGS
@given(f=st.lists(st.one_of(st.floats(allow_nan=True, allow_infinity=True),
                            st.integers(-3, 3).map(float)), min_size=1, max_size=30),
       words=st.lists(st.lists(st.integers(0, 2 ** 32 - 1), min_size=1, max_size=12),
                      min_size=1, max_size=12),
       minimize=st.booleans())
def test_tournament_winner_is_the_first_best_contestant(f, words, minimize):
    from oracle import genetic
    t = min(len(w) for w in words)
    w = np.array([row[:t] for row in words], dtype=np.uint32)
    fit = np.array(f, dtype=np.float64)
    win = genetic.tournament(fit, w, minimize)
    for i in range(w.shape[0]):
        c = [int(x) % len(fit) for x in w[i]]
        assert win[i] in c
        vals = [fit[x] for x in c]
        num = [x for x in vals if not np.isnan(x)]
        if not num:
            assert win[i] == c[0]
            continue
        best = min(num) if minimize else max(num)
        assert fit[win[i]] == best
        first = next(m for m, x in enumerate(vals) if x == best)
        assert win[i] == c[first]


@SETTINGS
@given(P=st.integers(1, 4), C=st.integers(1, 5), D=st.integers(1, 50), seed=st.integers(0, 99))
def test_accuracy_is_invariant_to_point_order(P, C, D, seed):
    from oracle import genetic
    r = np.random.default_rng(seed)
    out = r.integers(-2, 3, (P, C, D)).astype(np.float32)
    out[r.random((P, C, D)) < 0.2] = np.nan
    lab = r.integers(0, C, D).astype(np.int32)
    perm = r.permutation(D)
    a1, c1 = genetic.accuracy_from_outputs(out, lab)
    a2, c2 = genetic.accuracy_from_outputs(out[:, :, perm], lab[perm])
    assert (c1 == c2).all() and np.array_equal(a1, a2)


@SETTINGS
@given(n=st.integers(0, 10 ** 6), world=st.integers(1, 64))
def test_population_ranges_partition(n, world):
    rs = [shard.population_range(n, r, world) for r in range(world)]
    assert rs[0][0] == 0 and rs[-1][1] == n
    assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
    assert max(b - a for a, b in rs) - min(b - a for a, b in rs) <= 1
