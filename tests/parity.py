"""Comparison helpers for the CUDA path against the FP64 oracle.

Per output point the bar is |gpu - ref| <= 1e-5 * max(|ref|, 1).  Where the
oracle's first-order FP32 error bound e shows that no FP32 evaluation can meet
it (2e above the tolerance), the point must still satisfy |gpu - ref| <= 2e,
and it is counted; points whose bound is infinite (a guard decided within
rounding error, or an intermediate that may leave the FP32 range) are
skipped and counted.  MSE: |gpu - ref| <= 1e-4 |ref| + the deviation that the
per-point allowances can produce (oracle's mse_allow), skipped where that is
infinite; divergence classes (non-finite or > 1e30) must agree.
"""
import numpy as np

TOL_POINT = 1e-5
TOL_MSE = 1e-4
DIVERGENT = 1e30


class PointStats:
    def __init__(self):
        self.n = self.strict = self.widened = self.skipped = self.failed = 0
        self.worst = 0.0
        self.examples = []

    def frac_strict(self):
        return self.strict / max(self.n, 1)

    def __repr__(self):
        return (f"points={self.n} strict={self.strict} ({self.frac_strict():.4f}) "
                f"widened={self.widened} skipped={self.skipped} failed={self.failed}")


def compare_points(gpu, ref, err, stats=None, where=""):
    stats = stats or PointStats()
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.asarray(err, np.float64)
    with np.errstate(all="ignore"):
        tol = TOL_POINT * np.maximum(np.abs(ref), 1.0)
        d = np.abs(gpu - ref)
        usable = np.isfinite(err) & np.isfinite(ref)
        strict = usable & (d <= tol)
        widened = usable & ~strict & (d <= 2 * err)
        failed = usable & ~strict & ~widened
    stats.n += int(usable.sum())
    stats.strict += int(strict.sum())
    stats.widened += int(widened.sum())
    stats.skipped += int((~usable).sum())
    stats.failed += int(failed.sum())
    if failed.any():
        idx = np.argwhere(failed)[:5]
        for i in idx:
            i = tuple(i)
            stats.examples.append((where, i, float(gpu[i]), float(ref[i]), float(err[i])))
    return stats


def compare_mse(gpu, ref, allow):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    with np.errstate(all="ignore"):
        div_ref = ~np.isfinite(ref) | (ref > DIVERGENT)
        div_gpu = ~np.isfinite(gpu) | (gpu > DIVERGENT)
        usable = np.isfinite(allow)
        both_ok = usable & ~div_ref
        d = np.abs(gpu - ref)
        ok = d <= TOL_MSE * np.abs(ref) + allow
        strict = d <= TOL_MSE * np.abs(ref)
    res = {
        "n": int(both_ok.sum()),
        "strict": int((both_ok & strict).sum()),
        "failed": np.argwhere(both_ok & (~ok | div_gpu)).ravel(),
        "class_mismatch": np.argwhere(usable & (div_ref != div_gpu)).ravel(),
        "skipped": int((~usable).sum()),
    }
    return res
