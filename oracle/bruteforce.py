"""Brute-force EFM enumeration over every reaction support (tiny networks).

TEST INFRASTRUCTURE ONLY.  Written straight from Def. 2 and Def. 3 on the
split (irreversible) network: a set T of columns with no forward/reverse pair
is the support of an elementary flux mode iff S_int[:, T] has a one-dimensional
null space whose generator is nonzero on every column of T with a single sign.
Candidate supports are screened with numpy's SVD rank in batches, and every
support kept is then confirmed exactly with sympy (rational null space).
"""
from __future__ import annotations

from itertools import combinations

import numpy as np


def split(net):
    """Dense S_int over split columns, twin list and full split S."""
    S = net.dense()
    cols = []
    for j in range(net.n_rxn):
        cols.append((j, 1))
        if net.reversible[j]:
            cols.append((j, -1))
    full = np.stack([S[:, j] * d for (j, d) in cols], axis=1) if cols else np.zeros((net.n_met, 0), np.int64)
    internal = np.flatnonzero(net.external == 0)
    twin = [-1] * len(cols)
    for k in range(len(cols) - 1):
        if cols[k][0] == cols[k + 1][0]:
            twin[k], twin[k + 1] = k + 1, k
    return full[internal, :], twin, full


def exact_kernel(A):
    """Rational null space basis of an integer matrix (sympy)."""
    import sympy

    return sympy.Matrix(A.tolist()).nullspace()


def is_efm_support(S_int, cols):
    """Exact Def. 3 test for the support `cols` (columns of S_int)."""
    A = S_int[:, list(cols)]
    if A.shape[0] == 0:
        return len(cols) == 1
    ker = exact_kernel(A)
    if len(ker) != 1:
        return False
    v = [ker[0][i] for i in range(len(cols))]
    return all(x > 0 for x in v) or all(x < 0 for x in v)


def efm_supports(net, max_size=None):
    """Every EFM support of the split network (as sorted column tuples)."""
    S_int, twin, _ = split(net)
    M, N = S_int.shape
    top = N if max_size is None else min(N, max_size)
    top = min(top, (np.linalg.matrix_rank(S_int) if M else 0) + 1)
    pairs = [(a, twin[a]) for a in range(N) if twin[a] > a]
    found = []
    for k in range(1, top + 1):
        idx = np.fromiter((x for c in combinations(range(N), k) for x in c), dtype=np.int64).reshape(-1, k)
        if idx.size == 0:
            continue
        keep = np.ones(len(idx), dtype=bool)
        for a, b in pairs:
            keep &= ~((idx == a).any(axis=1) & (idx == b).any(axis=1))
        idx = idx[keep]
        for start in range(0, len(idx), 65536):
            chunk = idx[start:start + 65536]
            if M == 0:
                sel = chunk if k == 1 else chunk[:0]
            else:
                mats = S_int[:, chunk].transpose(1, 0, 2).astype(np.float64)  # [b, M, k]
                ranks = np.linalg.matrix_rank(mats)
                sel_mask = (k - ranks) == 1
                if not sel_mask.any():
                    continue
                sub = mats[sel_mask]
                # null vector = last right singular vector; screen the sign
                # pattern in floating point, then confirm exactly below
                _, _, vt = np.linalg.svd(sub)
                v = vt[:, -1, :]
                one_sign = (np.all(v > 1e-9, axis=1) | np.all(v < -1e-9, axis=1))
                sel = chunk[sel_mask][one_sign]
            for c in sel:
                c = tuple(int(x) for x in c)
                if is_efm_support(S_int, c):
                    found.append(c)
    return found


def seeds_of(net, target):
    """Columns producing the target (all columns for target -1)."""
    _, _, full = split(net)
    if target < 0:
        return set(range(full.shape[1]))
    return {k for k in range(full.shape[1]) if full[target, k] > 0}
