"""Plain reference of the population-parallel genetic operators.

TEST INFRASTRUCTURE ONLY.  Like the rest of ``oracle/``, this module is the
independent reference the CUDA library is checked against; only the tests,
the smoke check and the CPU-baseline leg of the benchmark import it.  It
shares no code with the CUDA path.  The operators work on one tree (one
selection) at a time with numpy slices, in the order the paper states the
steps; the accuracy is plain numpy over the whole output array.

What it computes:

* ``exchange`` -- the subtree exchange of Sec. III-B ("Tensorized
  Operations"): the child's three arrays are the old tree's prefix before the
  replaced subtree, the new subtree, and the old tree's suffix after it; the
  subtree sizes of the ancestors of the replaced root grow by
  ``dn = size_new[root] - size_old[k]``; a child longer than the maximum tree
  size is rejected and the old tree is returned unchanged.  Ancestors are
  found by walking down from the root through the child that contains ``k``
  (first child at ``i+1``, second at ``i+1+size[i+1]``), i.e. from the tree
  structure, not from an interval test on the size array.
* node choice -- how the operators of Sec. III-B choose their nodes from
  random words the caller draws: one-point crossover and subtree mutation take
  ``k = r mod len(T_old)`` and ``j = r' mod len(T_donor)``; hoist mutation
  takes ``k = r mod len(T)`` and a node ``j = k + (r' mod size[k])`` inside the
  subtree of ``k`` of the same tree, whose subtree then replaces it.
* ``tournament`` -- tournament selection (Algorithm 1 "Select parents";
  tournament size in the table "Configuration of Genetic Programming"):
  contestant ``m`` of selection ``i`` is tree ``r[i, m] mod P``; the winner has
  the best fitness, ties going to the earliest contestant, NaN losing to every
  number.
* ``predict`` / ``accuracy_from_outputs`` / ``accuracy`` -- classification fitness
  (Sec. V-D classification tasks, measured by accuracy): the predicted class
  of a point is the first index of the largest non-NaN output; accuracy is
  the fraction of points whose prediction equals the label.

Readings (the paper names the operators but leaves these open): random node
choice by ``mod`` of a 32-bit word; the status codes below; an all-NaN
output vector predicts no class.
"""
from __future__ import annotations

import numpy as np

from . import evaluate as _evaluate

# restated encoding (Sec. III-A): arity of each node type
_ARITY = {0: 0, 1: 0, 2: 1, 3: 2, 4: 3, 18: 1, 19: 2, 20: 3}

# per-child status of an exchange (the library's reading, restated)
DONE, TOO_LARGE, SKIPPED, BAD_INDEX, BAD_TREE = 1, 0, 2, -1, -2
# node choice modes
EXPLICIT, RANDOM, HOIST = 0, 1, 2


def _count(x, hi):
    """x as an int if it is an integer in [1, hi], else None."""
    x = float(x)
    if not np.isfinite(x) or x != np.floor(x) or x < 1 or x > hi:
        return None
    return int(x)


def ancestors(type_row, size_row, k):
    """Proper ancestors of node k, from the root down, by walking the
    structure: at each node descend into the child whose subtree holds k.
    Defined for well-formed trees (those that pass validation)."""
    out = []
    i = 0
    while i < k:
        out.append(i)
        ar = _ARITY[int(type_row[i])]
        c1 = i + 1
        if ar == 2 and k >= c1 + int(size_row[c1]):
            i = c1 + int(size_row[c1])
        else:
            i = c1
    return out


def exchange(old_t, old_v, old_s, k, new_t, new_v, new_s, max_size):
    """Sec. III-B subtree exchange of one tree.

    ``old_*`` are the old tree's arrays (at least len(T_old) long), ``k`` the
    root of the replaced subtree, ``new_*`` the new subtree's arrays (exactly
    its nodes).  Returns (type, value, size, status) with arrays of the
    child's length.
    """
    n_old = int(old_s[0])
    s, e = k, k + int(old_s[k])
    dn = int(new_s[0]) - int(old_s[k])
    if n_old + dn > max_size:
        return (np.array(old_t[:n_old]), np.array(old_v[:n_old]), np.array(old_s[:n_old]),
                TOO_LARGE)
    upd = np.array(old_s[:s], dtype=np.float32)
    for a in ancestors(old_t, old_s, k):
        upd[a] = upd[a] + dn
    t = np.concatenate([old_t[:s], new_t, old_t[e:n_old]]).astype(np.float32)
    v = np.concatenate([old_v[:s], new_v, old_v[e:n_old]]).astype(np.float32)
    z = np.concatenate([upd, new_s, old_s[e:n_old]]).astype(np.float32)
    return t, v, z, DONE


def subtree_exchange(old, donor, old_index, node, donor_index, donor_node, mode, max_size,
                     out_ld, old_max_len=None, donor_max_len=None, apply_word=None,
                     apply_below=0):
    """Exchange over a list of children.

    ``old`` and ``donor`` are (type, value, size) float32 arrays [P, ld];
    ``node`` / ``donor_node`` hold node positions (EXPLICIT) or 32-bit random
    words (RANDOM, HOIST), read as unsigned; ``donor_node`` None means 0.
    In HOIST mode ``donor`` and ``donor_index`` are ignored: the donor is the
    old tree itself.  Returns
    out arrays [n, out_ld] (NaN padded) and the int32 status per child.
    Children with an index out of range or a malformed length / subtree size
    get an all-NaN row.  With ``apply_word`` given, child i takes part only
    when ``apply_word[i] < apply_below`` (the operator's probability as a
    threshold on a 32-bit word); the others are copies of their old tree
    (SKIPPED).  Steps per child, in order:
      0. old index in range, else BAD_INDEX; its length an integer in
         [1, max_len], else BAD_TREE; not applied -> SKIPPED (a copy);
      1. donor index in range, else BAD_INDEX;
      2. donor length an integer in [1, max_len], else BAD_TREE;
      3. k: the position, or r mod len(T_old); out of range -> BAD_INDEX;
      4. size_old[k] an integer in [1, len(T_old) - k], else BAD_TREE;
      5. j: the position, r' mod len(T_donor), or k + r' mod size_old[k]
         (hoist); out of range -> BAD_INDEX;
      6. size_donor[j] an integer in [1, len(T_donor) - j], else BAD_TREE;
      7. the exchange (TOO_LARGE keeps the old tree).
    """
    ot, ov, os_ = old
    n = len(old_index)
    out = [np.full((n, out_ld), np.nan, np.float32) for _ in range(3)]
    status = np.zeros(n, np.int32)
    oml = ot.shape[1] if old_max_len is None else old_max_len
    for i in range(n):
        a = int(old_index[i])
        if not 0 <= a < ot.shape[0]:
            status[i] = BAD_INDEX
            continue
        n_old = _count(os_[a, 0], oml)
        if n_old is None:
            status[i] = BAD_TREE
            continue
        if apply_word is not None and (int(apply_word[i]) & 0xFFFFFFFF) >= apply_below:
            for arr, src in zip(out, (ot, ov, os_)):
                arr[i, :n_old] = src[a, :n_old]
            status[i] = SKIPPED
            continue
        if mode == HOIST:
            dt, dv, ds, b, dml = ot, ov, os_, a, oml
        else:
            dt, dv, ds = donor
            b = int(donor_index[i])
            dml = dt.shape[1] if donor_max_len is None else donor_max_len
        if not 0 <= b < dt.shape[0]:
            status[i] = BAD_INDEX
            continue
        n_don = _count(ds[b, 0], dml)
        if n_don is None:
            status[i] = BAD_TREE
            continue
        r = int(node[i]) & 0xFFFFFFFF
        r2 = 0 if donor_node is None else int(donor_node[i]) & 0xFFFFFFFF
        k = r if mode == EXPLICIT else r % n_old
        if k >= n_old:
            status[i] = BAD_INDEX
            continue
        sub_old = _count(os_[a, k], n_old - k)
        if sub_old is None:
            status[i] = BAD_TREE
            continue
        j = r2 if mode == EXPLICIT else (r2 % n_don if mode == RANDOM else k + r2 % sub_old)
        if j >= n_don:
            status[i] = BAD_INDEX
            continue
        m = _count(ds[b, j], n_don - j)
        if m is None:
            status[i] = BAD_TREE
            continue
        t, v, z, st = exchange(ot[a], ov[a], os_[a], k, dt[b, j:j + m], dv[b, j:j + m],
                               ds[b, j:j + m], max_size)
        out[0][i, :len(t)], out[1][i, :len(v)], out[2][i, :len(z)] = t, v, z
        status[i] = st
    return out[0], out[1], out[2], status


def tournament(fitness, words, minimize=True):
    """Winner index per selection; ``words`` is [n, t] uint32."""
    f = np.asarray(fitness, np.float64)
    P = f.shape[0]
    n, t = words.shape
    win = np.empty(n, np.int32)
    for i in range(n):
        best = None
        for m in range(t):
            c = int(words[i, m]) % P
            v = f[c]
            if best is None:
                best = c
                continue
            b = f[best]
            if np.isnan(v):
                continue
            if np.isnan(b) or (v < b if minimize else v > b):
                best = c
        win[i] = best
    return win


def predict(out):
    """Predicted class [P, D] of outputs [P, C, D]: the first index whose
    output equals the largest non-NaN output of the point; -1 when all of
    the point's outputs are NaN."""
    out = np.asarray(out)
    allnan = np.isnan(out).all(axis=1)
    with np.errstate(invalid="ignore"):
        best = np.max(np.where(np.isnan(out), -np.inf, out), axis=1)
    first = np.argmax(out == best[:, None, :], axis=1)
    return np.where(allnan, -1, first)


def accuracy_from_outputs(out, labels):
    """Accuracy [P] (float64) and correct counts [P] of outputs [P, C, D]."""
    pred = predict(out)
    lab = np.asarray(labels)[None, :]
    cnt = ((pred >= 0) & (pred == lab)).sum(axis=1).astype(np.int64)
    D = pred.shape[1]
    acc = cnt / np.float64(D) if D else np.full(pred.shape[0], np.nan)
    return acc, cnt


def accuracy(type_, val, size, X, labels, n_classes, max_len=None):
    """Accuracy from the FP64 forward outputs, plus per tree the number of
    points whose prediction an FP32 evaluation could change: the predicted
    output lies within the summed error bounds of another output, a bound or
    an output is not finite, or there is no prediction."""
    out, err, st = _evaluate(type_, val, size, X, n_classes, with_err=True, max_len=max_len)
    acc, cnt = accuracy_from_outputs(out, labels)
    pred = predict(out)
    pk = np.maximum(pred, 0)[:, None, :]
    o_p = np.take_along_axis(out, pk, axis=1)
    e_p = np.take_along_axis(err, pk, axis=1)
    with np.errstate(invalid="ignore"):
        close = (o_p - out <= e_p + err)
    close &= np.arange(n_classes)[None, :, None] != pk
    bad = (pred < 0) | ~np.isfinite(err).all(axis=1) | ~np.isfinite(out).all(axis=1)
    amb = (close.any(axis=1) | bad).sum(axis=1).astype(np.int64)
    acc[st != 0] = np.nan
    return acc, cnt, amb, st
