"""Seeded synthetic inputs for population fitness evaluation.

Input construction only -- nothing here evaluates a tree.  It builds
populations in the three-array encoding of Sec. III-A (types, values and
subtree sizes as float32 ``[P, Lmax]`` arrays padded with NaN), feature
matrices, target noise and ground-truth trees.  Targets ``y = GT(X) + noise``
are formed by the caller with whichever evaluator it owns (the FP64 oracle in
the tests, the library itself in the benchmark), so that no arithmetic of the
method lives in this module.

Encoding (our reading; Sec. III-A leaves the codes open):
  type  0 variable, 1 constant, 2 unary function, 3 binary function,
        4 ternary function; +16 marks a Modi node (Sec. IV-C).
  value variable -> feature index, constant -> the constant,
        function -> func_id + 256 * output_index (output index on Modi only).
  func  0 add, 1 sub, 2 mul, 3 protected div, 4 max, 5 sin, 6 cos,
        7 protected log, 8 clamped exp, 9 tan, 10 ite (a > 0 ? b : c).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

VAR, CONST, UFUNC, BFUNC, TFUNC, MODI = 0, 1, 2, 3, 4, 16
ADD, SUB, MUL, PDIV, MAX, SIN, COS, PLOG, CEXP, TAN, ITE = range(11)
FUNC_NAMES = ("add", "sub", "mul", "pdiv", "max", "sin", "cos", "plog", "cexp", "tan", "ite")
ARITY = (2, 2, 2, 2, 2, 1, 1, 1, 1, 1, 3)

#: function set of the plain-SR workloads
SR_FSET = (ADD, SUB, MUL, PDIV, SIN, COS, PLOG, CEXP, MAX)
#: function set of the paper's experiments (Table "Configuration of GP")
PAPER_FSET = (ADD, SUB, MUL, PDIV, SIN, COS, TAN)
#: function set with the ternary if-then-else (classification-style rules)
TERNARY_FSET = SR_FSET + (ITE,)
#: ground-truth trees use a tame subset so that targets stay finite
GT_FSET = (ADD, SUB, MUL, SIN, COS, MAX)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "treegen.c")
_SO = os.path.join(_HERE, "_build", "libtgp_treegen.so")
_lock = threading.Lock()
_lib = None


def build_treegen(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_treegen()
            lib = ctypes.CDLL(_SO)
            fp = ctypes.POINTER(ctypes.c_float)
            I, L, D = ctypes.c_int, ctypes.c_long, ctypes.c_double
            lib.tg_population.argtypes = [L, L, I, I, I, ctypes.POINTER(ctypes.c_int), I, I, D, D,
                                          D, I, I, I, I, ctypes.c_uint64, fp, fp, fp, I]
            lib.tg_population.restype = I
            _lib = lib
    return _lib


@dataclass
class Population:
    """Three NaN-padded float32 arrays ``[P, ld]`` (Sec. III-A)."""
    type: np.ndarray
    val: np.ndarray
    size: np.ndarray
    max_len: int

    @property
    def pop(self) -> int:
        return self.type.shape[0]

    @property
    def ld(self) -> int:
        return self.type.shape[1]

    def lengths(self) -> np.ndarray:
        return self.size[:, 0].astype(np.int64)

    def take(self, idx) -> "Population":
        return Population(self.type[idx], self.val[idx], self.size[idx], self.max_len)

    def nodes(self) -> int:
        return int(self.lengths().sum())


def random_population(seed: int, pop: int, max_len: int, len_range=None, max_depth: int = 20,
                      fset=SR_FSET, n_features: int = 1, const_range=(-2.0, 2.0),
                      p_var: float = 0.5, max_consts: int = -1, n_outputs: int = 1,
                      modi: bool = False, modi_max: int = 16, ld: int | None = None,
                      threads: int | None = None) -> Population:
    """Random prefix trees; lengths uniform on ``len_range`` (default [1, max_len])."""
    lo, hi = len_range if len_range is not None else (1, max_len)
    ld = max_len if ld is None else ld
    fs = (ctypes.c_int * len(fset))(*fset)
    t = np.empty((pop, ld), np.float32)
    v = np.empty((pop, ld), np.float32)
    s = np.empty((pop, ld), np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    rc = _load().tg_population(pop, ld, lo, hi, max_depth, fs, len(fset), n_features,
                               const_range[0], const_range[1], p_var, max_consts, n_outputs,
                               int(modi), modi_max, ctypes.c_uint64(seed & (2**64 - 1)),
                               t.ctypes.data_as(fp), v.ctypes.data_as(fp), s.ctypes.data_as(fp),
                               threads or (os.cpu_count() or 1))
    if rc != 0:
        raise ValueError(f"tree generator rejected its arguments (code {rc})")
    return Population(t, v, s, max_len)


def encode(tokens, ld: int | None = None) -> Population:
    """Builds one tree from prefix tokens.

    A token is ``("x", f)`` for a variable, ``("c", value)`` for a constant, a
    function name such as ``"add"``, or ``("add", out)`` for a Modi node that
    feeds output ``out``.  Subtree sizes come from the arities.
    """
    n = len(tokens)
    ld = n if ld is None else ld
    t = np.full(ld, np.nan, np.float32)
    v = np.full(ld, np.nan, np.float32)
    s = np.full(ld, np.nan, np.float32)
    ar = []
    for i, tok in enumerate(tokens):
        if isinstance(tok, tuple) and tok[0] == "x":
            t[i], v[i] = VAR, tok[1]
            ar.append(0)
        elif isinstance(tok, tuple) and tok[0] == "c":
            t[i], v[i] = CONST, tok[1]
            ar.append(0)
        else:
            name, out = (tok, None) if isinstance(tok, str) else tok
            f = FUNC_NAMES.index(name)
            t[i] = (UFUNC, BFUNC, TFUNC)[ARITY[f] - 1] | (MODI if out is not None else 0)
            v[i] = f + 256 * (out or 0)
            ar.append(ARITY[f])

    # subtree sizes from the arities, right to left with a stack of sizes
    stk = []
    for i in range(n - 1, -1, -1):
        if len(stk) < ar[i]:
            raise ValueError("tokens do not form exactly one prefix tree")
        kids = [stk.pop() for _ in range(ar[i])]
        s[i] = 1 + sum(kids)
        stk.append(int(s[i]))
    if len(stk) != 1:
        raise ValueError("tokens do not form exactly one prefix tree")
    return Population(t[None], v[None], s[None], ld)


def stack(pops, ld: int | None = None) -> Population:
    """Concatenates populations along P, padding to a common ``ld`` with NaN."""
    ld = max(p.ld for p in pops) if ld is None else ld

    def pad(a):
        out = np.full((a.shape[0], ld), np.nan, np.float32)
        out[:, :a.shape[1]] = a
        return out

    return Population(np.concatenate([pad(p.type) for p in pops]),
                      np.concatenate([pad(p.val) for p in pops]),
                      np.concatenate([pad(p.size) for p in pops]),
                      max(p.max_len for p in pops))


# --------------------------------------------------------------- workloads
@dataclass
class Problem:
    """One SR problem: a population, features, target noise and GT trees."""
    name: str
    pop: Population
    X: np.ndarray                  # [D, F] float32
    noise: np.ndarray              # [D, O] float32
    gt: Population                 # [O] ground-truth trees (one per output)
    n_outputs: int = 1
    meta: dict = field(default_factory=dict)

    @property
    def D(self) -> int:
        return self.X.shape[0]

    @property
    def F(self) -> int:
        return self.X.shape[1]


def _rng(seed: int, *key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, *key])))


def _seed64(seed: int, *key: int) -> int:
    return int(np.random.SeedSequence([seed, *key]).generate_state(1, np.uint64)[0])


def _gt_trees(seed: int, key: int, n_out: int, F: int, length: int = 31) -> Population:
    return random_population(_seed64(seed, key, 99), n_out, length, (length, length),
                             max_depth=10, fset=GT_FSET, n_features=F)


def sr_small(seed: int = 0) -> Problem:
    """64 trees, length <= 63 and depth <= 5, 2 features U(-1,1), 256 points,
    y = x0^2 + sin(x1) (the exact tree ``add(mul(x0,x0), sin(x1))``)."""
    pop = random_population(_seed64(seed, 1), 64, 63, (1, 63), max_depth=5, fset=SR_FSET,
                            n_features=2)
    X = _rng(seed, 1, 1).uniform(-1, 1, (256, 2)).astype(np.float32)
    gt = encode(["add", "mul", ("x", 0), ("x", 0), "sin", ("x", 1)])
    return Problem("sr_small", pop, X, np.zeros((256, 1), np.float32), gt)


def sr_scale(seed: int = 0, pop: int = 5000, D: int = 100_000) -> Problem:
    """5,000 trees, length <= 255, depth <= 8, 16 features N(0,1), 100,000
    points, y = GT tree of length 31 + N(0, 0.01^2)."""
    p = random_population(_seed64(seed, 2), pop, 255, (1, 255), max_depth=8, fset=SR_FSET,
                          n_features=16)
    r = _rng(seed, 2, 1)
    X = r.standard_normal((D, 16), dtype=np.float32)
    noise = (0.01 * r.standard_normal((D, 1))).astype(np.float32)
    return Problem("sr_scale", p, X, noise, _gt_trees(seed, 2, 1, 16))


def diff(seed: int = 0, pop: int = 10_000, D: int = 200_000) -> Problem:
    """10,000 trees, length <= 127, <= 16 constants, 4 features U(-3,3),
    200,000 points, y = GT tree + N(0, 0.01^2)."""
    p = random_population(_seed64(seed, 4), pop, 127, (1, 127), max_depth=10, fset=SR_FSET,
                          n_features=4, max_consts=16)
    r = _rng(seed, 4, 1)
    X = r.uniform(-3, 3, (D, 4)).astype(np.float32)
    noise = (0.01 * r.standard_normal((D, 1))).astype(np.float32)
    return Problem("diff", p, X, noise, _gt_trees(seed, 4, 1, 4))


def modi(seed: int = 0, pop: int = 20_000, D: int = 1_000_000, n_outputs: int = 8) -> Problem:
    """20,000 Modi trees, length <= 255, 8 outputs, 32 features N(0,1),
    1,000,000 points, targets from 8 GT trees + N(0, 0.01^2)."""
    p = random_population(_seed64(seed, 5), pop, 255, (1, 255), max_depth=10, fset=SR_FSET,
                          n_features=32, n_outputs=n_outputs, modi=True, modi_max=16)
    r = _rng(seed, 5, 1)
    X = r.standard_normal((D, 32), dtype=np.float32)
    noise = (0.01 * r.standard_normal((D, n_outputs))).astype(np.float32)
    return Problem("modi", p, X, noise, _gt_trees(seed, 5, n_outputs, 32), n_outputs)


def batched_uneven(seed: int = 0, n_problems: int = 8, pop_range=(1000, 20000),
                   d_range=(1000, 1_000_000), f_range=(4, 32), len_range=(7, 511),
                   scale: float = 1.0) -> list[Problem]:
    """8 independent SR problems: P ~ U{1k..20k}, D log-uniform on [1e3, 1e6],
    F ~ U{4..32}, lengths U[7, 511]; ``scale`` shrinks P and D for tests."""
    r = _rng(seed, 3)
    probs = []
    for i in range(n_problems):
        P = int(r.integers(pop_range[0], pop_range[1] + 1))
        D = int(round(math.exp(r.uniform(math.log(d_range[0]), math.log(d_range[1])))))
        F = int(r.integers(f_range[0], f_range[1] + 1))
        P = max(1, int(P * scale))
        D = max(1, int(D * scale))
        p = random_population(_seed64(seed, 3, i), P, len_range[1], len_range, max_depth=10,
                              fset=SR_FSET, n_features=F)
        rr = _rng(seed, 3, i, 1)
        X = rr.standard_normal((D, F), dtype=np.float32)
        noise = (0.01 * rr.standard_normal((D, 1))).astype(np.float32)
        probs.append(Problem(f"batched_{i}", p, X, noise, _gt_trees(seed, 300 + i, 1, F)))
    return probs


# ------------------------------------------------ paper-shape sweep inputs
#: (points, features) of the paper's SR data sets (table "Details of Symbolic
#: Regression Datasets"; Auto MPG as counted in the GPops/s summary table)
SR_DATASET_SHAPES = {"daily_demand": (60, 12), "auto_mpg": (392, 7),
                     "california_housing": (20_640, 8), "feynman_i_9_18": (100_000, 9)}
#: population sizes of the GPops/s summary table
SWEEP_POPS = (100, 500, 1000, 5000, 10_000, 50_000, 100_000, 500_000, 1_000_000)


def sweep_population(seed: int = 0, pop: int = 1_000_000) -> Population:
    """Trees for the paper-shape sweep: lengths U[300, 511] in rows of 512
    (mean ~405, the scale of the paper's S-bar), the paper's function set,
    feature indices below 7 so that every data set shape can use them."""
    return random_population(_seed64(seed, 11), pop, 512, (300, 511), max_depth=20,
                             fset=PAPER_FSET, n_features=7)


def sweep_data(seed: int, name: str) -> tuple[np.ndarray, np.ndarray]:
    """X ~ N(0, 1) and targets ~ N(0, 1) of a data set's shape."""
    D, F = SR_DATASET_SHAPES[name]
    r = _rng(seed, 11, sorted(SR_DATASET_SHAPES).index(name))
    return (r.standard_normal((D, F), dtype=np.float32),
            r.standard_normal((D, 1), dtype=np.float32))


# ------------------------------------------------- threshold study inputs
#: population sizes and data-set sizes of the threshold study (Sec. V-B: the
#: Pagie polynomial at populations 100, 1,000, 5,000 and 10,000 over a sweep
#: of data-set sizes across the hybrid / data-parallel switch)
E1_POPS = (100, 1000, 5000, 10_000)
E1_POINTS = (64, 256, 1024, 4096, 10_496, 16_384, 65_536, 262_144)


def e1_population(seed: int = 0, pop: int = 10_000) -> Population:
    """Random SR trees for the threshold study: the paper's function set,
    lengths U[1, 255] in rows of 256, two features (x, y)."""
    return random_population(_seed64(seed, 12), pop, 256, (1, 255), max_depth=12,
                             fset=PAPER_FSET, n_features=2)


def e1_data(seed: int, D: int) -> tuple[np.ndarray, np.ndarray]:
    """Pagie polynomial data (Sec. V-B): (x, y) ~ U(-5, 5) and the target
    f = 1/(1 + x^-4) + 1/(1 + y^-4) = x^4/(1 + x^4) + y^4/(1 + y^4), formed
    in FP64 and rounded (a data-generating function, not a tree)."""
    r = _rng(seed, 12, D)
    X = r.uniform(-5, 5, (D, 2)).astype(np.float32)
    x4 = X.astype(np.float64) ** 4
    y = (x4[:, 0] / (1 + x4[:, 0]) + x4[:, 1] / (1 + x4[:, 1])).astype(np.float32)[:, None]
    return X, y


# ------------------------------------------------- genetic-operator inputs
def random_words(seed: int, shape, *key: int) -> np.ndarray:
    """Uniform 32-bit words (the random numbers the operators consume)."""
    return _rng(seed, 7, *key).integers(0, 2 ** 32, shape, dtype=np.uint64).astype(np.uint32)


@dataclass
class GeneticInputs:
    """A population, a pool of new subtrees and the random words of one round
    of crossover / mutation / selection over ``n`` children."""
    pop: Population
    pool: Population
    n: int
    old_index: np.ndarray    # int32 [n]
    donor_index: np.ndarray  # int32 [n]
    pool_index: np.ndarray   # int32 [n]
    node: np.ndarray         # uint32 [n]
    donor_node: np.ndarray   # uint32 [n]
    apply: np.ndarray        # uint32 [n]


def genetic(seed: int = 0, pop: int = 100_000, max_size: int = 512, len_range=(1, 511),
            n: int | None = None, pool: int = 4096, pool_len=(1, 31), n_features: int = 16,
            fset=PAPER_FSET) -> GeneticInputs:
    """Trees of the paper's SR setting (maximum tree size 512, function set
    {+,-,*,/,sin,cos,tan}) with lengths uniform on ``len_range``, a pool of
    small random trees for subtree mutation, uniform parent rows and words."""
    n = pop if n is None else n
    p = random_population(_seed64(seed, 8), pop, max_size, len_range, max_depth=20, fset=fset,
                          n_features=n_features)
    q = random_population(_seed64(seed, 9), pool, pool_len[1], pool_len, max_depth=8, fset=fset,
                          n_features=n_features, ld=pool_len[1])
    r = _rng(seed, 8, 1)
    rows = lambda m: r.integers(0, m, n).astype(np.int32)
    return GeneticInputs(p, q, n, rows(pop), rows(pop), rows(pool), random_words(seed, n, 1),
                         random_words(seed, n, 2), random_words(seed, n, 3))


#: (features, classes, points) of the paper's classification data sets
#: (table "Details of Classification Datasets")
CLASSIFICATION_SHAPES = {"wine": (13, 3, 178), "kidney": (24, 3, 400), "breast": (30, 2, 569),
                         "yeast": (8, 10, 1484)}


@dataclass
class ClassProblem:
    name: str
    pop: Population
    X: np.ndarray       # [D, F] float32
    labels: np.ndarray  # [D] int32
    n_classes: int


def classification(seed: int = 0, shape: str = "yeast", pop: int = 5000, max_len: int = 255,
                   D: int | None = None) -> ClassProblem:
    """Modi trees with one output per class (Sec. IV-C) on a synthetic data
    set of the named shape: X ~ N(0, 1), labels uniform over the classes."""
    F, C, D0 = CLASSIFICATION_SHAPES[shape]
    D = D0 if D is None else D
    key = sorted(CLASSIFICATION_SHAPES).index(shape)
    p = random_population(_seed64(seed, 10, key), pop, max_len, (1, max_len), max_depth=10,
                          fset=SR_FSET, n_features=F, n_outputs=C, modi=True, modi_max=16)
    r = _rng(seed, 10, key)
    X = r.standard_normal((D, F), dtype=np.float32)
    labels = r.integers(0, C, D).astype(np.int32)
    return ClassProblem(shape, p, X, labels, C)


WORKLOADS = {
    "sr_small": sr_small,
    "sr_scale": sr_scale,
    "batched_uneven": batched_uneven,
    "diff": diff,
    "modi": modi,
}
