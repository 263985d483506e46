"""Flux-dependent reactions (Def. 11), the output of the DEPTHy pre-pass
(Alg. 2).  TEST INFRASTRUCTURE ONLY.

Reading: for an internal metabolite i, an output column o of i (it
consumes i) and an input column c of i (it produces i) are flux-dependent
with respect to i when some walk in the metabolite graph leaves i through o
and comes back to i for the first time through c, using at most L columns.
A step of a walk goes from metabolite m through a column k that consumes m
to an internal metabolite that k produces.  Both flows of Def. 11 are the
same cycle read in opposite directions: in a forward flow o is the primary
output and c the secondary input; in a backward flow c is the primary input
and o the secondary output.

Output: dep_out[i][k] = 1 when column k is the leaving column of such a
walk, dep_in[i][k] = 1 when k is its returning column (boolean M x N).
Computed by plain depth-first enumeration of the walks.
"""
from __future__ import annotations

import numpy as np


def edges_of(S_int):
    """Steps from each internal metabolite, in the order (column, product row)."""
    M, N = S_int.shape
    out = []
    for m in range(M):
        e = []
        for k in range(N):
            if S_int[m, k] < 0:
                for m2 in range(M):
                    if S_int[m2, k] > 0:
                        e.append((k, m2))
        out.append(e)
    return out


def dependent_reactions(net, L):
    from . import bruteforce

    S_int, _, _ = bruteforce.split(net)
    M, N = S_int.shape
    E = edges_of(S_int)
    dep_out = np.zeros((M, N), dtype=bool)
    dep_in = np.zeros((M, N), dtype=bool)
    for i in range(M):
        stack = [(i, -1, 0)]  # (metabolite, leaving column, columns used)
        while stack:
            m, first, used = stack.pop()
            for k, m2 in E[m]:
                f = k if first < 0 else first
                if m2 == i:
                    dep_out[i, f] = True
                    dep_in[i, k] = True
                elif used + 1 < L:
                    stack.append((m2, f, used + 1))
    return dep_out, dep_in


def r_max(net):
    """Largest number of steps out of one internal metabolite."""
    from . import bruteforce

    S_int, _, _ = bruteforce.split(net)
    return max((len(e) for e in edges_of(S_int)), default=0)
