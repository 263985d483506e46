"""Seeded synthetic metabolic networks.

This module only draws random networks; it holds none of the pathway
method's arithmetic.  Both the CPU oracle and the CUDA path read the arrays
it returns, so a test hands the very same network to both sides.

A network is a stoichiometric matrix S (metabolites x reactions, Sec. 2.1)
stored as CSR by metabolite (row_ptr, col_idx, coef), a reversibility flag
per reaction and an external flag per metabolite.  Shapes follow the two
networks the paper studies (Sec. 4.2): a 12 x 18 core model and a genome-scale
model of 1668 metabolites x 2382 reactions whose cofactors are set external.
Neither model is shipped with the paper, so seeded stand-ins of the same
shape are drawn here:

* degree: metabolites get Chung-Lu weights w_m ~ (m + m0)^(-1/(gamma-1))
  (power law, gamma = 2.2) unless `uniform` is set;
* size:   each reaction touches `size_range` metabolites (uniform);
* coef:   drawn from `coef_probs` ({value: probability});
* roles:  externals are split into product targets, hub cofactors and
  uptake substrates; every internal metabolite gets at least one producer
  and one consumer (a consistent network, Lemma 2), every target at least
  one producer, every reaction at least one substrate and one product.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

CORE_COEFS = {1: 0.90, 2: 0.08, 3: 0.01, 4: 0.01}
TINY_COEFS = {1: 0.5, 2: 0.5}


@dataclass
class Network:
    n_met: int
    n_rxn: int
    row_ptr: np.ndarray  # int32 [n_met + 1]
    col_idx: np.ndarray  # int32 [nnz], reaction index, ascending within a row
    coef: np.ndarray  # int32 [nnz], nonzero net stoichiometric coefficient
    reversible: np.ndarray  # uint8 [n_rxn]
    external: np.ndarray  # uint8 [n_met]
    targets: list = field(default_factory=list)  # metabolite indices
    name: str = ""
    seed: int = 0

    def dense(self) -> np.ndarray:
        """Dense S (int64, metabolites x reactions)."""
        S = np.zeros((self.n_met, self.n_rxn), dtype=np.int64)
        for m in range(self.n_met):
            for p in range(self.row_ptr[m], self.row_ptr[m + 1]):
                S[m, self.col_idx[p]] = self.coef[p]
        return S

    @staticmethod
    def from_dense(S, reversible, external, targets=(), name="", seed=0) -> "Network":
        S = np.asarray(S, dtype=np.int64)
        n_met, n_rxn = S.shape
        row_ptr = [0]
        cols, vals = [], []
        for m in range(n_met):
            nz = np.nonzero(S[m])[0]
            cols.extend(int(j) for j in nz)
            vals.extend(int(S[m, j]) for j in nz)
            row_ptr.append(len(cols))
        return Network(
            n_met=n_met,
            n_rxn=n_rxn,
            row_ptr=np.asarray(row_ptr, dtype=np.int32),
            col_idx=np.asarray(cols, dtype=np.int32),
            coef=np.asarray(vals, dtype=np.int32),
            reversible=np.asarray(reversible, dtype=np.uint8).reshape(n_rxn),
            external=np.asarray(external, dtype=np.uint8).reshape(n_met),
            targets=list(int(t) for t in targets),
            name=name,
            seed=seed,
        )

    def split_columns(self) -> int:
        return int(self.n_rxn + int(self.reversible.sum()))


def _draw_coef(rng, probs, size):
    vals = np.array(sorted(probs), dtype=np.int64)
    p = np.array([probs[v] for v in vals], dtype=np.float64)
    p /= p.sum()
    return rng.choice(vals, size=size, p=p)


def _powerlaw_weights(rng, n, gamma, m0=1.0):
    if n == 0:
        return np.zeros(0)
    w = (np.arange(n, dtype=np.float64) + m0) ** (-1.0 / (gamma - 1.0))
    rng.shuffle(w)
    return w / w.sum()


def generate(
    *,
    n_int: int,
    n_targets: int,
    n_hubs: int,
    n_substrates: int,
    n_rxn: int,
    n_rev: int,
    size_range=(2, 6),
    coef_probs=None,
    gamma: float | None = 2.2,
    hub_degree=(30, 60),
    seed: int = 0,
    name: str = "",
    shuffle_ids: bool = True,
) -> Network:
    """Draw one seeded network with the roles described in the module doc."""
    rng = np.random.Generator(np.random.PCG64(seed))
    coef_probs = coef_probs or CORE_COEFS
    n_ext = n_targets + n_hubs + n_substrates
    n_met = n_int + n_ext
    internal = np.arange(n_int)
    targets = np.arange(n_int, n_int + n_targets)
    hubs = np.arange(n_int + n_targets, n_int + n_targets + n_hubs)
    subs = np.arange(n_int + n_targets + n_hubs, n_met)
    if gamma is None:
        w = np.full(n_int, 1.0 / max(n_int, 1))
    else:
        w = _powerlaw_weights(rng, n_int, gamma)

    # reaction -> {metabolite: coefficient}
    rxns: list[dict] = []

    def pick_internal(k, exclude=()):
        k = min(k, n_int - len(exclude))
        if k <= 0:
            return []
        ww = w.copy()
        for e in exclude:
            ww[e] = 0.0
        ww /= ww.sum()
        return list(rng.choice(internal, size=k, replace=False, p=ww))

    n_up = max(1, int(round(0.03 * n_rxn))) if n_substrates else 0
    n_exp = n_targets
    n_body = n_rxn - n_up - n_exp
    if n_body < 1:
        raise ValueError("too few reactions for the requested roles")
    # uptake: substrate -> 1-2 internal products
    for r in range(n_up):
        s = int(subs[r % n_substrates])
        prods = pick_internal(int(rng.integers(1, 3)))
        cs = _draw_coef(rng, coef_probs, len(prods) + 1)
        d = {s: -int(cs[0])}
        for m, c in zip(prods, cs[1:]):
            d[int(m)] = int(c)
        rxns.append(d)
    # export: 1-2 internal substrates -> target
    for t in targets:
        srcs = pick_internal(int(rng.integers(1, 3)))
        cs = _draw_coef(rng, coef_probs, len(srcs) + 1)
        d = {int(t): int(cs[0])}
        for m, c in zip(srcs, cs[1:]):
            d[int(m)] = -int(c)
        rxns.append(d)
    # body reactions among internal metabolites
    lo, hi = size_range
    for r in range(n_body):
        sz = int(rng.integers(lo, hi + 1))
        mets = pick_internal(sz)
        if len(mets) < 2:
            raise ValueError("network too small for reaction size")
        n_sub = int(rng.integers(1, len(mets)))
        cs = _draw_coef(rng, coef_probs, len(mets))
        d = {}
        for i, (m, c) in enumerate(zip(mets, cs)):
            d[int(m)] = -int(c) if i < n_sub else int(c)
        rxns.append(d)
    body0 = n_up + n_exp
    # hub cofactors: fixed degree, attached to random body reactions
    for h in hubs:
        deg = int(rng.integers(hub_degree[0], hub_degree[1] + 1))
        deg = max(1, min(deg, n_body))
        for r in rng.choice(n_body, size=deg, replace=False):
            side = 1 if rng.random() < 0.5 else -1
            rxns[body0 + int(r)][int(h)] = side
    # repair: every internal metabolite needs a producer and a consumer
    for m in internal:
        m = int(m)
        has_p = any(d.get(m, 0) > 0 for d in rxns)
        has_c = any(d.get(m, 0) < 0 for d in rxns)
        for need, sign in ((not has_p, 1), (not has_c, -1)):
            if not need:
                continue
            order = rng.permutation(n_body)
            for r in order:
                d = rxns[body0 + int(r)]
                if m not in d:
                    d[m] = sign
                    break
    # reversibility
    rev = np.zeros(n_rxn, dtype=np.uint8)
    if n_rev:
        rev[rng.choice(n_rxn, size=n_rev, replace=False)] = 1
    # reaction order shuffled, metabolite ids shuffled
    rperm = rng.permutation(n_rxn) if shuffle_ids else np.arange(n_rxn)
    mperm = rng.permutation(n_met) if shuffle_ids else np.arange(n_met)
    S = np.zeros((n_met, n_rxn), dtype=np.int64)
    for r, d in enumerate(rxns):
        for m, c in d.items():
            S[mperm[m], rperm[r]] = c
    revp = np.zeros(n_rxn, dtype=np.uint8)
    revp[rperm] = rev
    ext = np.zeros(n_met, dtype=np.uint8)
    ext[mperm[n_int:]] = 1
    tg = [int(mperm[t]) for t in targets]
    return Network.from_dense(S, revp, ext, tg, name=name, seed=seed)


# ---------------------------------------------------------------------------
# Workloads.  Sizes follow the two networks of Sec. 4.2 and the batched and
# genome-scale settings the library is built for.
# ---------------------------------------------------------------------------

def tiny(seed: int = 0) -> Network:
    """12 metabolites (8 internal, 4 external), 16 reactions (4 reversible),
    2-4 metabolites per reaction chosen uniformly, coefficients from {1, 2}.
    Targets: the 4 externals (ALL = -1 is added by callers that want it)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_met, n_int, n_rxn = 12, 8, 16
    while True:
        S = np.zeros((n_met, n_rxn), dtype=np.int64)
        for r in range(n_rxn):
            sz = int(rng.integers(2, 5))
            mets = rng.choice(n_met, size=sz, replace=False)
            n_sub = int(rng.integers(1, sz))
            cs = rng.integers(1, 3, size=sz)
            for i, m in enumerate(mets):
                S[m, r] = -cs[i] if i < n_sub else cs[i]
        ext = np.zeros(n_met, dtype=np.uint8)
        ext[rng.choice(n_met, size=n_met - n_int, replace=False)] = 1
        # consistency: every internal metabolite produced and consumed
        ok = all(((S[m] > 0).any() and (S[m] < 0).any()) for m in range(n_met) if not ext[m])
        if ok:
            break
    rev = np.zeros(n_rxn, dtype=np.uint8)
    rev[rng.choice(n_rxn, size=4, replace=False)] = 1
    tg = [int(m) for m in range(n_met) if ext[m]]
    return Network.from_dense(S, rev, ext, tg, name=f"tiny-{seed}", seed=seed)


def core(seed: int = 1_000_000) -> Network:
    """Core-metabolism shape: 72 metabolites (58 internal; 14 external =
    8 targets + 5 hub cofactors + 1 substrate), 95 reactions, 19 reversible,
    2-6 metabolites per reaction, coefficients 1 (90%), 2 (8%), 3-4 (2%),
    power-law degree, hubs of degree 30-60."""
    return generate(n_int=58, n_targets=8, n_hubs=5, n_substrates=1, n_rxn=95, n_rev=19,
                    size_range=(2, 6), coef_probs=CORE_COEFS, gamma=2.2, hub_degree=(30, 60),
                    seed=seed, name=f"core-{seed}")


def batched_member(index: int, base_seed: int = 2_000_000) -> Network:
    """One network of the uneven batch: 10-120 metabolites (80% internal),
    15-200 reactions, 20% reversible, core coefficient/degree laws; hub count
    max(1, round(5 M / 72)), hub degree scaled by R / 95 and capped at R / 2.
    One target: a producible external."""
    seed = base_seed + index
    rng = np.random.Generator(np.random.PCG64(seed))
    while True:
        M = int(rng.integers(10, 121))
        R = int(rng.integers(15, 201))
        n_int = int(round(0.8 * M))
        n_ext = M - n_int
        hubs = max(1, int(round(5 * M / 72)))
        hubs = min(hubs, max(0, n_ext - 2))
        n_sub = 1
        n_tg = n_ext - hubs - n_sub
        if n_tg >= 1 and R - n_tg - max(1, round(0.03 * R)) >= 2 and n_int >= 6:
            break
    scale = R / 95.0
    hlo = max(1, min(int(round(30 * scale)), R // 2))
    hhi = max(hlo, min(int(round(60 * scale)), R // 2))
    net = generate(n_int=n_int, n_targets=n_tg, n_hubs=hubs, n_substrates=n_sub, n_rxn=R,
                   n_rev=int(round(0.2 * R)), size_range=(2, 6), coef_probs=CORE_COEFS,
                   gamma=2.2, hub_degree=(hlo, hhi), seed=seed, name=f"batch-{index}")
    pick = int(rng.integers(0, len(net.targets)))
    net.targets = [net.targets[pick]]
    return net


def genome(seed: int = 3_000_000, n_targets: int = 256) -> Network:
    """Genome-scale shape: 1000 metabolites (850 internal, 150 external),
    2500 reactions, 625 reversible, power law gamma 2.2, 20 hubs of degree
    200-600.  Targets: every non-hub external with a producer, then seeded
    internal metabolites until `n_targets`."""
    n_sub = 10
    net = generate(n_int=850, n_targets=150 - 20 - n_sub, n_hubs=20, n_substrates=n_sub,
                   n_rxn=2500, n_rev=625, size_range=(2, 6), coef_probs=CORE_COEFS,
                   gamma=2.2, hub_degree=(200, 600), seed=seed, name=f"genome-{seed}")
    rng = np.random.Generator(np.random.PCG64(seed + 17))
    tg = list(net.targets)
    internal = [m for m in range(net.n_met) if not net.external[m]]
    extra = rng.permutation(internal)
    for m in extra:
        if len(tg) >= n_targets:
            break
        tg.append(int(m))
    net.targets = tg[:n_targets]
    return net


def type1(seed: int, n_int: int = 7, n_ext: int = 3, n_rxn: int = 14, n_rev: int = 3) -> Network:
    """Network whose reactions each have at most one internal substrate and
    at most one internal product, all coefficients 1 (pathways of Type I,
    Lemma 2).  External metabolites may sit on either side."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_met = n_int + n_ext
    S = np.zeros((n_met, n_rxn), dtype=np.int64)
    for r in range(n_rxn):
        while True:
            s = int(rng.integers(-1, n_int)) if rng.random() < 0.85 else -1
            p = int(rng.integers(-1, n_int)) if rng.random() < 0.85 else -1
            if s != p or s == -1:
                break
        es = int(rng.integers(n_int, n_met))
        ep = int(rng.integers(n_int, n_met))
        if s >= 0:
            S[s, r] = -1
        elif es != ep:
            S[es, r] = -1
        if p >= 0:
            S[p, r] = 1
        elif ep != es or s >= 0:
            S[ep, r] = 1
        if not S[:, r].any():
            S[n_int, r] = 1
    ext = np.zeros(n_met, dtype=np.uint8)
    ext[n_int:] = 1
    rev = np.zeros(n_rxn, dtype=np.uint8)
    if n_rev:
        rev[rng.choice(n_rxn, size=n_rev, replace=False)] = 1
    return Network.from_dense(S, rev, ext, list(range(n_int, n_met)), name=f"type1-{seed}", seed=seed)


# largest |coefficient| the C-ABI loader accepts (EFM_MAX_COEF)
MAX_COEF = 524287


def maximal(seed: int = 4_000_000) -> Network:
    """A network at the library's size limits: exactly 1024 internal
    metabolites and 4096 split columns (support width 64 words), with
    coefficients up to MAX_COEF.

    Two parts that share no metabolite:

    * a chain that reaches the length limit: target T is made by r_0 from
      m_0, r_i (i = 1..62) makes m_{i-1} from m_i, and r_63 makes m_62 from
      the uptake X, so {r_0..r_63} is one 64-column pathway.  Coefficients
      are 1 except a few (MAX_COEF, 2, 3) that scale the flux along the
      chain.  Side branches: an uptake X' makes m_10, m_20, m_30, m_40 and
      m_50 (shorter pathways); r_30 is reversible (twin rule); a reaction
      q turns m_44 into m_46, closing the cycle q, r_46, r_45 (secondary
      steps and a non-elementary balanced support).
    * a random filler of 961 internal and 8 external metabolites (uniform
      degree, 2-6 metabolites per reaction, coefficients mostly 1-3 with 3%
      drawn up to MAX_COEF, 800 of 3225 reactions reversible), whose first
      external is a second target.

    Targets: T, then the filler target."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_chain, n_fill_int, n_fill_ext = 63, 961, 8
    n_int = n_chain + n_fill_int
    T, X, Xalt = n_int, n_int + 1, n_int + 2
    fext0 = n_int + 3
    n_met = fext0 + n_fill_ext
    cols = []
    rev = []

    def add(entries, reversible=False):
        c = np.zeros(n_met, dtype=np.int64)
        for m, v in entries:
            c[m] += v
        cols.append(c)
        rev.append(1 if reversible else 0)

    a = {5: MAX_COEF, 12: 2, 33: 3}  # consumption coefficients of r_i on m_i
    b = {20: MAX_COEF, 27: 3, 51: 2}  # production coefficients of r_i on m_{i-1}
    add([(0, -1), (T, 1)])
    for i in range(1, n_chain):
        add([(i, -a.get(i, 1)), (i - 1, b.get(i, 1))], reversible=(i == 30))
    add([(X, -1), (n_chain - 1, 1)])
    for i in (10, 20, 30, 40, 50):
        add([(Xalt, -1), (i, 1)])
    add([(44, -1), (46, 1)])
    n_fixed_cols = len(cols) + sum(rev)
    n_fill_rev = 800
    n_fill = 4096 - n_fixed_cols - n_fill_rev
    fill_mets = np.concatenate([np.arange(n_chain, n_int), np.arange(fext0, n_met)])
    big = 0
    for r in range(n_fill):
        sz = int(rng.integers(2, 7))
        mets = rng.choice(fill_mets, size=sz, replace=False)
        n_sub = int(rng.integers(1, sz))
        ent = []
        for j, m in enumerate(mets):
            v = int(rng.integers(1, 4))
            if rng.random() < 0.03:
                v = MAX_COEF if big < 2 else int(rng.integers(4, MAX_COEF + 1))
                big += 1
            ent.append((int(m), -v if j < n_sub else v))
        if r < 6 and fext0 not in mets:
            ent.append((fext0, 1))  # producers of the filler target
        add(ent)
    S = np.stack(cols, axis=1)
    reversible = np.asarray(rev, dtype=np.uint8)
    fill_rev = rng.choice(np.arange(len(cols) - n_fill, len(cols)), size=n_fill_rev, replace=False)
    reversible[fill_rev] = 1
    ext = np.zeros(n_met, dtype=np.uint8)
    ext[n_int:] = 1
    return Network.from_dense(S, reversible, ext, [T, fext0], name=f"maximal-{seed}", seed=seed)
