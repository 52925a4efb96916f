"""Each FP32 function body of the kernels, alone, against the FP64 oracle and
its per-function error allowance.

One-node trees f(x0) and f(x0, x1) over sweeps of exact float32 arguments
run through the real forward kernels (the leaf-fused forms that every tree
uses); per point the GPU value must lie within the oracle's first-order FP32
bound, which for exact operands is the function's own allowance (Sec. II-A
functions with the guards and clamp of the library's reading):
  sin/cos/tan  |x| up to 1e5, including the float32 neighbours of multiples
               of pi/2 (the argument reduction's hardest inputs);
  plog         |x| from below the 1e-6 guard up to 3e38, and the guard's
               float32 neighbours;
  cexp         [-100, 80.5] and the clamp's neighbours;
  pdiv         |b| across the whole normal float32 range, including values
               above 2^126 whose reciprocal is subnormal (flushed to zero,
               which the allowance states), with small and huge numerators,
               and the guard's neighbours;
  add/sub/mul/max  operands of every magnitude.
This pins the allowances the parity tests use to widen the 1e-5 bar: an
allowance too small for the kernel's actual error fails here, as does a
function body that loses accuracy in some range.  The derivative bodies of
the adjoint are swept the same way against the oracle's reverse mode.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2501_17168_gb300 import _lib, api, workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
F32 = np.float32


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_17168_gb300 import build
    build.build_all()
    _lib.load()


def _tree(f):
    """[f, x0] or [f, x0, x1] in the three-array encoding."""
    if W.ARITY[f] == 1:
        t, v, s = [W.UFUNC, W.VAR], [f, 0], [2, 1]
    else:
        t, v, s = [W.BFUNC, W.VAR, W.VAR], [f, 0, 1], [3, 1, 1]
    a = lambda x: np.array([x], np.float32)
    return a(t), a(v), a(s)


def _neighbours(x, k=3):
    x = np.asarray(x, F32)
    out = [x]
    up, dn = x.copy(), x.copy()
    for _ in range(k):
        up = np.nextafter(up, F32(np.inf))
        dn = np.nextafter(dn, F32(-np.inf))
        out += [up, dn]
    return np.concatenate(out)


def _logspace(lo, hi, n, signs=True):
    m = np.logspace(lo, hi, n)
    m = m[np.isfinite(m.astype(F32)) & (m.astype(F32) > 0)]
    v = m.astype(F32)
    return np.concatenate([v, -v]) if signs else v


def _check(orc, f, x0, x1=None):
    x0 = np.asarray(x0, F32)
    X = np.stack([x0, x0 if x1 is None else np.asarray(x1, F32)], 1)
    X = np.ascontiguousarray(X)
    t, v, s = _tree(f)
    td, vd, sd = (torch.from_numpy(a).to(DEV) for a in (t, v, s))
    out, st = api.tgp_eval_forward(td, vd, sd, torch.from_numpy(X).to(DEV), 1, max_len=t.shape[1])
    api.tgp_check_device_error()
    assert int(st[0]) == 0
    g = out.cpu().numpy()[0, 0].astype(np.float64)
    ref, err, ost = orc.evaluate(t, v, s, X, with_err=True)
    ref, err = ref[0, 0], err[0, 0]
    with np.errstate(all="ignore"):
        d = np.abs(g - ref)
        usable = np.isfinite(err) & np.isfinite(ref)
        bad = usable & ~(d <= err)
    n_skip = int((~usable).sum())
    if bad.any():
        i = np.flatnonzero(bad)[:8]
        raise AssertionError(
            f"{W.FUNC_NAMES[f]}: {int(bad.sum())} of {int(usable.sum())} points beyond the allowance; "
            f"x0={X[i, 0].tolist()} x1={X[i, 1].tolist()} gpu={g[i].tolist()} ref={ref[i].tolist()} "
            f"err={err[i].tolist()}")
    # the sweep must actually exercise the function (few skipped points)
    assert n_skip <= 0.05 * len(g), (W.FUNC_NAMES[f], n_skip)
    return g, ref, err


def _trig_args():
    k = np.arange(-20000, 20001)
    halfpi = (k * (np.pi / 2)).astype(F32)
    return np.concatenate([_logspace(-8, 5, 4000), _neighbours(halfpi[::7], 2),
                           np.linspace(-10, 10, 2001).astype(F32),
                           _neighbours(np.array([1e5, -1e5, 65536.0, 12345.678], F32), 3)])


@pytest.mark.parametrize("f", [W.SIN, W.COS])
def test_sin_cos_within_allowance(orc, f):
    _check(orc, f, _trig_args())


def test_tan_within_allowance(orc):
    x = _trig_args()
    _check(orc, W.TAN, x)


def test_plog_within_allowance_and_guard(orc):
    guard = F32(1e-6)
    x = np.concatenate([_logspace(-12, 38.5, 6000), _neighbours(np.array([guard, -guard]), 4),
                        np.array([0.0, 1.0, -1.0, 3.4e38, -3.4e38, 1e-45, -1e-45], F32),
                        np.linspace(0.5, 2.0, 3001).astype(F32)])
    g, ref, _ = _check(orc, W.PLOG, x)
    # guard branch: exactly 0 where |x| <= 1e-6f
    at = np.abs(x) <= guard
    assert (g[at] == 0.0).all() and (ref[at] == 0.0).all()


def test_cexp_within_allowance_and_clamp(orc):
    x = np.concatenate([np.linspace(-100, 80.5, 8001).astype(F32),
                        _neighbours(np.array([80.0, 0.0, -87.0, 88.7], F32), 4),
                        _logspace(-10, 1.9, 1000)])
    g, ref, _ = _check(orc, W.CEXP, x)
    over = x > 80.0
    assert (g[over] == g[np.argmin(np.abs(x - 80.0))]).all()


def test_pdiv_within_allowance_and_guard(orc):
    guard = F32(1e-6)
    b = np.concatenate([_logspace(np.log10(1.2e-38), 38.5, 1500), _neighbours(np.array([guard, -guard]), 4),
                        _neighbours(np.array([2.0 ** 126, -2.0 ** 126, 2.0 ** 127, 3.0e38], F32), 3),
                        np.array([0.0, -0.0, 1e-45, 1.0, -1.0], F32)])
    nums = np.array([1.0, -3.5, 7.0e3, 1.0e20, 2.0 ** 100, -3.0e38, 1.0e-20, 0.0], F32)
    a = np.repeat(nums, len(b))
    bb = np.tile(b, len(nums))
    g, ref, _ = _check(orc, W.PDIV, a, bb)
    at = np.abs(bb) <= guard
    assert (g[at] == 1.0).all() and (ref[at] == 1.0).all()


@pytest.mark.parametrize("f", [W.ADD, W.SUB, W.MUL, W.MAX])
def test_arithmetic_within_allowance(orc, f):
    r = np.random.default_rng(f)
    n = 20000
    # magnitudes whose products and sums stay inside the float32 range
    mag = lambda: (10.0 ** r.uniform(-18, 18, n)) * r.choice([-1.0, 1.0], n)
    a, b = mag().astype(F32), mag().astype(F32)
    # close magnitudes (cancellation) and exact ties
    a[:2000] = b[:2000] * F32(1.0000001)
    a[2000:2100] = b[2000:2100]
    _check(orc, f, a, b)


@pytest.mark.parametrize("f", [W.SIN, W.COS, W.PLOG, W.CEXP, W.PDIV, W.MUL, W.MAX, W.SUB])
def test_adjoint_derivative_bodies(orc, f):
    """d MSE / d x of the one-node tree f(x0[, x1]) with y = 0 is
    2 f(x) f'(x) / D per point: the adjoint's function and derivative bodies
    against the oracle's reverse mode (1e-3 relative to max(|ref|, 1), the
    gradient bar), on arguments away from guards, the clamp and max ties."""
    r = np.random.default_rng(100 + f)
    D = 4096
    if f in (W.SIN, W.COS):
        x0 = r.uniform(-30, 30, D)
    elif f == W.PLOG:
        x0 = 10.0 ** r.uniform(-4, 4, D) * r.choice([-1, 1], D)
    elif f == W.CEXP:
        x0 = r.uniform(-20, 6, D)
    else:
        x0 = r.uniform(-3, 3, D)
    x1 = r.uniform(0.1, 3, D) * r.choice([-1, 1], D)
    X = np.ascontiguousarray(np.stack([x0, x1], 1).astype(F32))
    t, v, s = _tree(f)
    y = np.zeros((D, 1), F32)
    td, vd, sd = (torch.from_numpy(a).to(DEV) for a in (t, v, s))
    Xd = torch.from_numpy(X).to(DEV)
    g = torch.ones((1, 1), dtype=torch.float64, device=DEV)
    m, gv, gx, st = api.tgp_eval_backward(td, vd, sd, Xd, torch.from_numpy(y).to(DEV), g, 1,
                                          max_len=t.shape[1])
    api.tgp_check_device_error()
    mo, gvo, gxo, sto = orc.grad(t, v, s, X, y, 1.0)
    gx = gx.cpu().numpy()
    tol = 1e-3 * np.maximum(np.abs(gxo), 1.0 / D)
    bad = ~(np.abs(gx - gxo) <= tol)
    assert not bad.any(), (W.FUNC_NAMES[f], int(bad.sum()), X[bad][:4], gx[bad][:4], gxo[bad][:4])
    assert abs(float(m.cpu()[0, 0]) - mo[0, 0]) <= 1e-4 * abs(mo[0, 0]) + 1e-12
