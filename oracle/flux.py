"""Exact flux vectors of results (TEST INFRASTRUCTURE ONLY).

A result's support U has nullity(S_int[:, U]) = 1, so the balanced flux
modes on U form one ray (Def. 3): the kernel of S_int[:, U].  Its
representative here is the primitive integer vector (entries with gcd 1),
oriented positive; on a result every entry is then strictly positive.
Computed exactly with sympy's rational null space.
"""
from __future__ import annotations

from math import gcd

import numpy as np


def flux_vector(S_int, cols):
    """Primitive positive kernel vector of S_int[:, cols] (ascending column
    order), or None when the kernel is not one ray positive on every column."""
    import sympy

    A = sympy.Matrix(np.asarray(S_int)[:, list(cols)].tolist())
    ns = A.nullspace()
    if len(ns) != 1:
        return None
    v = ns[0]
    den = 1
    for x in v:
        den = den * x.q // gcd(den, x.q)
    ints = [int(x * den) for x in v]
    g = 0
    for x in ints:
        g = gcd(g, abs(x))
    ints = [x // g for x in ints]
    if ints[0] < 0:
        ints = [-x for x in ints]
    if any(x <= 0 for x in ints):
        return None
    return ints


def flux_vectors(net, supports):
    """Flux vectors of uint64[n, W] supports: list of int lists (None where
    the support is not a single positive ray)."""
    from . import bruteforce, supports_to_lists

    S_int, _, _ = bruteforce.split(net)
    return [flux_vector(S_int, cols) for cols in supports_to_lists(supports)]
