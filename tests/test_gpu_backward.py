"""GPU parity of the reverse-mode adjoint (tgp_eval_backward) against the
oracle's FP64 reverse mode and against central finite differences, plus the
autograd.Function wrapper and a short Adam run on the constants.

The oracle also bounds, per gradient element, how far an FP32 evaluation of
the same gradient may land (its forward bounds carried through the seeds and
local derivatives, one rounding per product and sum, FP32 partial sums before
FP64).  Every element is checked: within the bar |gpu - ref| <= 1e-3 *
max(|ref|, 1) (strict), or within 2x that bound where the bound says no FP32
evaluation can meet the bar (widened, counted).  Only trees whose gradient
bound is infinite somewhere (a guard, clamp or max tie the FP32 path may
decide the other way, or an adjoint that may leave the FP32 range) get a
zero upstream gradient and are counted; each test asserts the fraction of
trees checked.  The GPU's strict count is held against a plain float32
restatement of the reverse mode on the same elements.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2501_17168_gb300 import _lib, api, autograd as ag, workloads as W
from parity import GradStats, compare_grads, compare_mse, f32_grad

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL_GRAD = 1e-3
from parity import ACC_TERMS  # FP32 terms per constant before FP64 in the adjoint kernel


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_17168_gb300 import build
    build.build_all()
    _lib.load()


def gradient_checkable(orc, p, X, y, O=1):
    """Trees whose oracle gradient bound is finite for every constant (one
    oracle pass with g = 1 on every tree: constant bounds are per tree)."""
    _, _, _, st, egv, _ = orc.grad(p.type, p.val, p.size, X, y, 1.0, n_outputs=O, max_len=p.max_len,
                                   with_err=True, acc_terms=ACC_TERMS)
    const = p.type == W.CONST
    with np.errstate(invalid="ignore"):
        fin = np.where(const, np.isfinite(egv), True).all(1)
    return (st == 0) & fin


def gpu_backward(p, X, y, g, O=1, want_mse=True):
    t, v, s = api.population_to(p, DEV)
    mse, gv, gx, st = api.tgp_eval_backward(t, v, s, torch.from_numpy(X).to(DEV),
                                            torch.from_numpy(np.ascontiguousarray(y, np.float32)).to(DEV),
                                            torch.from_numpy(np.ascontiguousarray(g, np.float64)), O,
                                            max_len=p.max_len, want_mse=want_mse)
    api.tgp_check_device_error()
    cpu = lambda x: None if x is None else x.cpu().numpy()
    return cpu(mse), cpu(gv), cpu(gx), cpu(st)


def check_grads(orc, p, X, y, O, rng, min_frac=0.5):
    ok = gradient_checkable(orc, p, X, y, O)
    assert ok.mean() >= min_frac, (int(ok.sum()), p.pop)
    g = rng.uniform(0.5, 1.5, (p.pop, O)) * ok[:, None]
    mse, gv, gx, st = gpu_backward(p, X, y, g, O)
    rm, rgv, rgx, rst, egv, egx = orc.grad(p.type, p.val, p.size, X, y, g, n_outputs=O,
                                           max_len=p.max_len, with_err=True, acc_terms=ACC_TERMS)
    np.testing.assert_array_equal(st, rst)
    gv32, gx32 = f32_grad(p.type, p.val, p.size, X, y, g, O)
    # constant gradients of the included trees (zero elsewhere by contract)
    const = (p.type == W.CONST)
    sel = ok[:, None] & const
    sc = compare_grads(gv[sel], rgv[sel], egv[sel], f32=gv32[sel])
    assert sc.skipped == 0, sc
    assert (gv[(st == 0)[:, None] & ~const] == 0).all()
    # input gradients (sum over the included trees)
    sx = compare_grads(gx, rgx, egx, f32=gx32)
    assert sx.skipped <= 0.05 * gx.size, sx
    # fused MSE (the forward's rule: 1e-4, or what the per-point bounds allow)
    ref, allow, _ = orc.mse(p.type, p.val, p.size, X, y, n_outputs=O, rel_tol=1e-5, max_len=p.max_len)
    r = compare_mse(mse, ref, allow)
    assert len(r["failed"]) == 0 and len(r["class_mismatch"]) == 0, r
    print(f"trees checked {int(ok.sum())}/{p.pop}; constants {sc}; inputs {sx}")
    return int(ok.sum()), int(sel.sum())


def test_backward_matches_oracle_sr(orc):
    # differentiation workload shape, scaled down: <= 16 constants, 4 features U(-3,3)
    rng = np.random.default_rng(11)
    p = W.random_population(71, 400, 127, (1, 127), max_depth=10, n_features=4, max_consts=16)
    X = rng.uniform(-3, 3, (1111, 4)).astype(np.float32)     # ragged last tile
    y = rng.standard_normal((1111, 1)).astype(np.float32)
    check_grads(orc, p, X, y, 1, rng)


def test_backward_matches_oracle_tame(orc):
    # functions whose derivatives stay well conditioned: nearly every tree counts
    rng = np.random.default_rng(12)
    p = W.random_population(72, 300, 63, (1, 63), max_depth=10, n_features=3,
                            fset=(W.ADD, W.SUB, W.MUL, W.SIN, W.COS, W.MAX))
    X = rng.uniform(-1, 1, (600, 3)).astype(np.float32)
    y = rng.standard_normal((600, 1)).astype(np.float32)
    n_ok, n_const = check_grads(orc, p, X, y, 1, rng, min_frac=0.9)
    assert n_const > 500


def test_backward_modi(orc):
    rng = np.random.default_rng(13)
    prob = W.modi(pop=200, D=700, n_outputs=4)
    p = prob.pop
    X = prob.X
    y = rng.standard_normal((700, 4)).astype(np.float32)
    check_grads(orc, p, X, y, 4, rng)


def test_backward_single_output_mixed_modi(orc):
    rng = np.random.default_rng(14)
    plain = W.random_population(81, 60, 31, n_features=2)
    modi = W.random_population(82, 60, 31, (5, 31), n_features=2, n_outputs=1, modi=True, modi_max=4)
    P = W.stack([plain, modi])
    X = rng.uniform(-1, 1, (300, 2)).astype(np.float32)
    y = rng.standard_normal((300, 1)).astype(np.float32)
    check_grads(orc, P, X, y, 1, rng, min_frac=0.7)


def test_gpu_gradient_against_central_differences(orc):
    # independent of the oracle's reverse mode: central differences of the
    # oracle's FP64 MSE in constants that are exact in float32
    rng = np.random.default_rng(15)
    p = W.random_population(91, 40, 31, (5, 31), max_depth=10, n_features=2,
                            fset=(W.ADD, W.SUB, W.MUL, W.SIN, W.COS, W.CEXP), p_var=0.4)
    X = rng.uniform(-1, 1, (256, 2)).astype(np.float32)
    y = rng.standard_normal((256, 1)).astype(np.float32)
    g = np.ones((p.pop, 1))
    mse, gv, gx, st = gpu_backward(p, X, y, g)
    checked = 0
    for k in range(p.pop):
        for i in range(int(p.size[k, 0])):
            if p.type[k, i] != W.CONST:
                continue
            c = float(p.val[k, i])
            h = 2.0 ** -12
            vals = []
            for sgn in (1, -1):
                pv = p.val[k:k + 1].copy()
                pv[0, i] = np.float32(c + sgn * h)
                m, _ = orc.mse(p.type[k:k + 1], pv, p.size[k:k + 1], X, y)
                vals.append(m[0, 0])
            fd = (vals[0] - vals[1]) / (2 * h)
            if np.isfinite(fd) and np.isfinite(gv[k, i]):
                assert abs(gv[k, i] - fd) <= 2e-3 * max(abs(fd), 1.0), (k, i, gv[k, i], fd)
                checked += 1
    assert checked >= 20


def test_autograd_function_matches_direct_call():
    rng = np.random.default_rng(16)
    p = W.random_population(93, 50, 31, n_features=3, fset=(W.ADD, W.MUL, W.SIN, W.COS))
    t, v, s = api.population_to(p, DEV)
    X = torch.from_numpy(rng.uniform(-1, 1, (500, 3)).astype(np.float32)).to(DEV)
    y = torch.from_numpy(rng.standard_normal((500, 1)).astype(np.float32)).to(DEV)
    w = torch.from_numpy(rng.uniform(0.5, 2, (50, 1))).to(DEV)
    val = v.clone().requires_grad_(True)
    Xg = X.clone().requires_grad_(True)
    mse = ag.fitness(val, Xg, t, s, y, 1, max_len=p.max_len)
    (w * mse).sum().backward()
    _, gv, gx, _ = api.tgp_eval_backward(t, v, s, X, y, w, 1, max_len=p.max_len, want_mse=False)
    assert torch.equal(torch.nan_to_num(val.grad), torch.nan_to_num(gv))
    assert torch.allclose(Xg.grad, gx, rtol=1e-5, atol=1e-6)


def test_grad_X_accumulates_and_zero_g_skips():
    rng = np.random.default_rng(17)
    p = W.random_population(94, 30, 31, n_features=2, fset=(W.ADD, W.MUL, W.SIN))
    t, v, s = api.population_to(p, DEV)
    X = torch.from_numpy(rng.uniform(-1, 1, (300, 2)).astype(np.float32)).to(DEV)
    y = torch.zeros((300, 1), device=DEV)
    g = torch.ones((30, 1), dtype=torch.float64)
    _, _, gx1, _ = api.tgp_eval_backward(t, v, s, X, y, g, 1, max_len=p.max_len)
    _, _, gx2, _ = api.tgp_eval_backward(t, v, s, X, y, g, 1, max_len=p.max_len, grad_X=gx1.clone())
    assert torch.allclose(gx2, 2 * gx1, rtol=1e-5, atol=1e-6)
    z = torch.zeros((30, 1), dtype=torch.float64)
    mse, gv, gx, _ = api.tgp_eval_backward(t, v, s, X, y, z, 1, max_len=p.max_len, want_mse=False)
    assert mse is None and (gv == 0).all() and (gx == 0).all()


def test_adam_on_constants_reduces_the_loss():
    # differentiation workload pattern: constants gathered into [P, 16] and
    # optimised with Adam through the autograd.Function
    rng = np.random.default_rng(18)
    p = W.random_population(95, 200, 63, (5, 63), max_depth=10, n_features=4, max_consts=16,
                            fset=(W.ADD, W.SUB, W.MUL, W.SIN, W.COS, W.MAX))
    t, v, s = api.population_to(p, DEV)
    Xn = rng.uniform(-3, 3, (2000, 4)).astype(np.float32)
    X = torch.from_numpy(Xn).to(DEV)
    y = torch.from_numpy((np.sin(Xn[:, 0]) * Xn[:, 1] + 0.5 * Xn[:, 2])[:, None].astype(np.float32)).to(DEV)
    const = (t == W.CONST)
    idx = torch.zeros((p.pop, 16), dtype=torch.long, device=DEV)
    mask = torch.zeros((p.pop, 16), dtype=torch.bool, device=DEV)
    for k in range(p.pop):
        pos = torch.nonzero(const[k]).flatten()
        idx[k, :len(pos)] = pos
        mask[k, :len(pos)] = True
    consts = torch.gather(v, 1, idx).clone().requires_grad_(True)
    opt = torch.optim.Adam([consts], lr=1e-2)
    first = None
    for step in range(20):
        val = v.scatter(1, idx, torch.where(mask, consts, torch.gather(v, 1, idx)))
        mse = ag.fitness(val, X, t, s, y, 1, max_len=p.max_len)
        loss = torch.nan_to_num(mse, nan=0.0, posinf=0.0).clamp(max=1e6).sum()
        if first is None:
            first = mse.detach().clone()
        opt.zero_grad()
        loss.backward()
        consts.grad = torch.nan_to_num(consts.grad) * mask
        opt.step()
    last = mse.detach()
    fin = torch.isfinite(first) & torch.isfinite(last) & mask.any(1, keepdim=True)
    improved = (last[fin] < first[fin]).float().mean().item()
    assert improved > 0.8, improved


def test_zero_upstream_tree_that_overflows_leaves_grad_X_finite(orc):
    # the fused MSE needs the forward of every tree, but a tree with zero
    # upstream gradient must contribute nothing to the X gradient even where
    # its value overflows (0 * inf would be NaN)
    over = W.encode(["cexp", "cexp", "mul", ("c", 3.0), ("x", 0)])      # exp(exp(3 x0)) -> inf
    tame = W.encode(["add", "mul", ("x", 0), ("c", 0.5), "sin", ("x", 1)])
    p = W.stack([over, tame])
    X = np.random.default_rng(19).uniform(-3, 3, (777, 2)).astype(np.float32)
    y = np.zeros((777, 1), np.float32)
    g = np.array([[0.0], [1.0]])
    mse, gv, gx, st = gpu_backward(p, X, y, g)
    assert np.isinf(mse[0, 0]) or mse[0, 0] > 1e30
    rm, rgv, rgx, rst = orc.grad(p.type, p.val, p.size, X, y, g, max_len=p.max_len)
    assert np.isfinite(gx).all()
    np.testing.assert_allclose(gx, rgx, rtol=1e-3, atol=1e-3)
    np.testing.assert_allclose(gv[1], rgv[1], rtol=1e-3, atol=1e-3)
    assert (gv[0] == 0).all()


def test_backward_feature_limit_is_reported():
    # the adjoint holds a tile of X and of its gradient in shared memory: 256
    # features do not fit, and the call says so instead of launching
    p = W.random_population(96, 10, 63, n_features=256)
    t, v, s = api.population_to(p, DEV)
    X = torch.zeros((300, 256), device=DEV)
    y = torch.zeros((300, 1), device=DEV)
    g = torch.ones((10, 1), dtype=torch.float64)
    with pytest.raises(_lib.TGPError) as e:
        api.tgp_eval_backward(t, v, s, X, y, g, 1, max_len=p.max_len)
    assert e.value.code == _lib.TGP_ERR_UNSUPPORTED


def test_backward_sixteen_outputs(orc):
    rng = np.random.default_rng(20)
    p = W.random_population(97, 40, 63, (5, 63), max_depth=8, n_features=2, n_outputs=16,
                            modi=True, modi_max=20, fset=(W.ADD, W.SUB, W.MUL, W.SIN, W.COS, W.MAX))
    X = rng.uniform(-1, 1, (400, 2)).astype(np.float32)
    y = rng.standard_normal((400, 16)).astype(np.float32)
    check_grads(orc, p, X, y, 16, rng)
