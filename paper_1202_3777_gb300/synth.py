"""Seeded synthetic junction trees and evidence cases.

This module only *builds inputs*: tree shapes, variable cardinalities,
potential tables and evidence.  It holds none of the message-passing
arithmetic (no marginalisation, ratio or scattering), so both the FP64 oracle
and the CUDA path can consume its output without sharing any of the method.

Conventions (shared by every consumer):

* A junction tree is a rooted tree of cliques; clique 0 is the root and
  ``parent[0] == -1`` (the "designated root" of Sec. 2.1).
* ``cliques[c]`` lists the variables of clique ``c`` in *table order*: the
  first-listed variable is the most significant digit of the flat index and
  the last-listed varies fastest (the layout Fig. 2 fixes: for {A,B,D}, B=0
  selects entries {0,1,4,5}).
* The separator of edge (c, parent(c)) is the intersection of the two variable
  sets (Sec. 2.1).  Generators only ever copy separator variables from the
  parent, so the running-intersection property holds by construction.
* ``pot`` is the concatenation of all clique tables (``pot_off`` gives the
  start of each), non-negative, float64 or float32.

The workloads stand in for the paper's Bayesian-network junction trees
(Sec. 4.1, Table 1), which are not available; sizes follow the clique and
separator ranges of Table 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np


@dataclass
class Tree:
    """A junction tree with potential tables, in plain numpy arrays."""

    card: np.ndarray                 # int32 [n_vars], card[v] >= 2
    cliques: List[np.ndarray]        # int32 var lists, table order
    parent: np.ndarray               # int32 [n_cliques], parent[0] == -1
    pot: np.ndarray                  # float64 or float32, concatenated tables
    name: str = "tree"
    fresh: List[np.ndarray] = field(default_factory=list)  # vars introduced by each clique
    meta: dict = field(default_factory=dict)                # generator side facts (e.g. CPTs)

    @property
    def n_vars(self) -> int:
        return int(self.card.shape[0])

    @property
    def n_cliques(self) -> int:
        return len(self.cliques)

    def table_sizes(self) -> np.ndarray:
        return np.array([int(np.prod(self.card[c].astype(np.int64))) for c in self.cliques],
                        dtype=np.int64)

    @property
    def pot_off(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.table_sizes())]).astype(np.int64)

    def table(self, c: int) -> np.ndarray:
        off = self.pot_off
        return self.pot[off[c]:off[c + 1]]

    def clique_csr(self):
        """(clique_off int64 [n+1], clique_vars int32 [sum k]) CSR form."""
        ks = np.array([len(c) for c in self.cliques], dtype=np.int64)
        off = np.concatenate([[0], np.cumsum(ks)]).astype(np.int64)
        flat = (np.concatenate(self.cliques).astype(np.int32)
                if self.cliques else np.zeros(0, np.int32))
        return off, flat

    def as_dtype(self, dtype) -> "Tree":
        """Same tree with potentials stored in ``dtype`` (rounded once)."""
        return Tree(self.card.copy(), [c.copy() for c in self.cliques], self.parent.copy(),
                    self.pot.astype(dtype), self.name, [f.copy() for f in self.fresh],
                    dict(self.meta))

    def with_pot(self, pot: np.ndarray, name: Optional[str] = None) -> "Tree":
        return Tree(self.card.copy(), [c.copy() for c in self.cliques], self.parent.copy(),
                    np.ascontiguousarray(pot), name or self.name, [f.copy() for f in self.fresh],
                    dict(self.meta))

    def entries(self) -> int:
        return int(self.table_sizes().sum())

    def work_per_case(self) -> int:
        """Clique entries touched by one full propagation: the numerator of
        Eq. 4 summed over the 2(n-1) messages, sum over edges of
        2 * (|phi_child| + |phi_parent|)."""
        sz = self.table_sizes()
        w = 0
        for c in range(1, self.n_cliques):
            w += 2 * (int(sz[c]) + int(sz[self.parent[c]]))
        return w

    def depth(self) -> np.ndarray:
        d = np.zeros(self.n_cliques, dtype=np.int32)
        for c in range(1, self.n_cliques):
            d[c] = d[self.parent[c]] + 1   # parents always precede children here
        return d


def _uniform_pot(rng: np.random.Generator, n: int) -> np.ndarray:
    """i.i.d. Uniform(0.01, 1] values in FP64."""
    r = rng.random(n)                # [0, 1)
    np.subtract(1.0, r, out=r)       # (0, 1]
    r *= 0.99
    r += 0.01
    return r


def _build(rng: np.random.Generator,
           n_cliques: int,
           root_size: Callable[[], int],
           child_shape: Callable[[int], tuple],
           fresh_card: Callable[[], int],
           choose_parent: Callable[[List[int]], int],
           shuffle: bool = True):
    """Random attachment tree: each new clique attaches to a parent chosen by
    ``choose_parent`` and copies a random subset of the parent's variables
    (its separator) plus fresh variables."""
    cards: List[int] = []
    cliques: List[List[int]] = []
    fresh: List[List[int]] = []
    parent = [-1]
    depth = [0]

    def new_var():
        cards.append(fresh_card())
        return len(cards) - 1

    k0 = root_size()
    root = [new_var() for _ in range(k0)]
    cliques.append(root)
    fresh.append(list(root))
    for c in range(1, n_cliques):
        p = choose_parent(depth)
        pk = len(cliques[p])
        s, n_new = child_shape(pk)
        sep = list(rng.choice(np.array(cliques[p]), size=s, replace=False)) if s > 0 else []
        new = [new_var() for _ in range(n_new)]
        cliques.append([int(v) for v in sep] + new)
        fresh.append(new)
        parent.append(p)
        depth.append(depth[p] + 1)
    if shuffle:
        cliques = [list(rng.permutation(np.array(cl))) for cl in cliques]
    return (np.array(cards, dtype=np.int32),
            [np.array(cl, dtype=np.int32) for cl in cliques],
            np.array(parent, dtype=np.int32),
            [np.array(f, dtype=np.int32) for f in fresh])


def _uniform_parent(rng):
    return lambda depth: int(rng.integers(0, len(depth)))


def _finish(rng, card, cliques, parent, fresh, name, pot=None) -> Tree:
    t = Tree(card, cliques, parent, np.zeros(0), name, fresh)
    if pot is None:
        pot = _uniform_pot(rng, t.entries())
    t.pot = np.ascontiguousarray(pot)
    return t


# --------------------------------------------------------------------------
# The five workloads (plus small variants used for brute-force checks).
# --------------------------------------------------------------------------

def small_tree(seed: int = 1001) -> Tree:
    """32 cliques x 5 variables of cardinality 3 (243 entries); each child
    shares 2 variables with a uniformly chosen existing clique and adds 3
    fresh ones.  Potentials Uniform(0.01, 1] in FP64."""
    rng = np.random.default_rng(seed)
    card, cl, par, fr = _build(rng, 32, lambda: 5, lambda pk: (2, 3), lambda: 3,
                               _uniform_parent(rng))
    return _finish(rng, card, cl, par, fr, "small-32x243")


def small_brute_tree(seed: int = 1011) -> Tree:
    """4 cliques of 5 ternary variables with separator sizes (2, 3, 3): 12
    variables (3^12 joint states), small enough to enumerate the joint."""
    rng = np.random.default_rng(seed)
    shapes = iter([(2, 3), (3, 2), (3, 2)])
    card, cl, par, fr = _build(rng, 4, lambda: 5, lambda pk: next(shapes), lambda: 3,
                               _uniform_parent(rng))
    return _finish(rng, card, cl, par, fr, "small-brute-4x243")


def large_clique_tree(seed: int = 1002, n_cliques: int = 64, n_vars_per: int = 10,
                      card: int = 4, max_depth: int = 8) -> Tree:
    """64 cliques x 10 variables of cardinality 4 (2^20 entries); separators
    of 4-6 variables from the parent; parents at depth ``max_depth`` are
    rejected, so the tree is at most ``max_depth`` deep."""
    rng = np.random.default_rng(seed)

    def choose(depth):
        while True:
            p = int(rng.integers(0, len(depth)))
            if depth[p] < max_depth:
                return p

    def shape(pk):
        s = int(rng.integers(4, 7))
        return s, n_vars_per - s

    cd, cl, par, fr = _build(rng, n_cliques, lambda: n_vars_per, shape, lambda: card, choose)
    return _finish(rng, cd, cl, par, fr, f"large-clique-{n_cliques}x{card}^{n_vars_per}")


def high_card_tree(seed: int = 1003, n_cliques: int = 48, card: int = 32,
                   alpha: float = 0.5) -> Tree:
    """48 cliques x 4 variables of cardinality 32 (2^20 entries), separators
    of 2 variables (1024 entries, 1024-way fan-in).  The potentials are the
    conditional tables of a Bayesian network multiplied into their clique
    (the Initialization step of Algorithm 4): the root holds
    P(v1)P(v2|v1)P(v3|v1,v2)P(v4|v1,v2,v3) and each child with separator
    (a, b) and fresh (f1, f2) holds P(f1|a,b)P(f2|a,b,f1).  Every CPT column
    is Dirichlet(alpha * 1) in FP64, so the joint is normalised (Z = 1)."""
    rng = np.random.default_rng(seed)
    card_arr, cl, par, fr = _build(rng, n_cliques, lambda: 4, lambda pk: (2, 2),
                                   lambda: card, _uniform_parent(rng), shuffle=False)
    K = card

    def cpt(n_parents):
        # one Dirichlet column per parent configuration; last axis = child
        cols = rng.dirichlet(np.full(K, alpha), size=K ** n_parents)
        return cols.reshape((K,) * n_parents + (K,))

    tables = []
    root_prior = None
    for c in range(n_cliques):
        if c == 0:
            root_prior = cpt(0)
            t = (root_prior[:, None, None, None] * cpt(1)[:, :, None, None]
                 * cpt(2)[:, :, :, None] * cpt(3))
        else:
            t = cpt(2)[:, :, :, None] * cpt(3)
        tables.append(t)
    # shuffle each clique's listed order (and transpose its table to match)
    out_cl, flat = [], []
    for c in range(n_cliques):
        perm = rng.permutation(4)
        out_cl.append(cl[c][perm])
        flat.append(np.transpose(tables[c], perm).reshape(-1))
    t = _finish(rng, card_arr, out_cl, par, fr, f"high-card-{n_cliques}x{card}^4",
                pot=np.concatenate(flat))
    t.meta["root_prior_var"] = int(cl[0][0])      # v1, the root's first CPT variable
    t.meta["root_prior"] = root_prior             # P(v1)
    return t


def batched_tree(seed: int = 1004, n_cliques: int = 256) -> Tree:
    """256 cliques of 6-9 variables, fresh cardinalities 2-4 (64 to 262,144
    entries), separators of 2-5 variables (bounded by the parent's size and
    k-1).  Potentials Uniform(0.01, 1]."""
    rng = np.random.default_rng(seed)

    def shape(pk):
        k = int(rng.integers(6, 10))
        s = min(int(rng.integers(2, 6)), pk, k - 1)
        return s, k - s

    card, cl, par, fr = _build(rng, n_cliques, lambda: int(rng.integers(6, 10)), shape,
                               lambda: int(rng.integers(2, 5)), _uniform_parent(rng))
    return _finish(rng, card, cl, par, fr, f"batched-{n_cliques}")


def binary_serving_tree(seed: int = 1005, n_cliques: int = 1024) -> Tree:
    """1024 cliques of 3-6 binary variables; separators of 1..min(3, k-1)
    variables."""
    rng = np.random.default_rng(seed)

    def shape(pk):
        k = int(rng.integers(3, 7))
        s = min(int(rng.integers(1, 4)), pk, k - 1)
        return s, k - s

    card, cl, par, fr = _build(rng, n_cliques, lambda: int(rng.integers(3, 7)), shape,
                               lambda: 2, _uniform_parent(rng))
    return _finish(rng, card, cl, par, fr, f"binary-{n_cliques}")


def random_small_tree(seed: int, n_cliques: int = 5, max_states: float = 1 << 14,
                      card_range=(2, 5), k_range=(2, 4), allow_empty_sep: bool = False,
                      card_choices=None) -> Tree:
    """A random small tree (random cardinalities, separator sizes including
    empty ones if allowed) whose joint has at most ``max_states`` states.
    ``card_choices`` (a sequence) draws each cardinality from it instead of
    from ``card_range``."""
    for attempt in range(1000):
        rng = np.random.default_rng(seed * 7919 + attempt)

        def shape(pk):
            k = int(rng.integers(k_range[0], k_range[1] + 1))
            lo = 0 if allow_empty_sep else 1
            hi = min(pk, k - 1)        # keep at least one fresh variable
            s = int(rng.integers(lo, hi + 1)) if hi >= lo else max(hi, 0)
            return s, k - s

        card, cl, par, fr = _build(rng, n_cliques,
                                   lambda: int(rng.integers(k_range[0], k_range[1] + 1)),
                                   shape,
                                   (lambda: int(rng.integers(card_range[0], card_range[1] + 1)))
                                   if card_choices is None else (lambda: int(rng.choice(card_choices))),
                                   _uniform_parent(rng))
        states = int(np.prod(card.astype(np.int64)))
        if states <= max_states:
            return _finish(rng, card, cl, par, fr, f"random-small-{seed}")
    raise RuntimeError("could not draw a small tree")


def separator_sweep_tree(sep_vars: int, seed: int = 1006, n_cliques: int = 32, k: int = 6,
                         card: int = 4) -> Tree:
    """Trees that differ only in separator size, for the analogue of Fig. 6
    (speedup against average separator table size): ``n_cliques`` cliques
    of ``k`` variables of cardinality ``card``; every child shares exactly
    ``sep_vars`` variables with a uniformly chosen earlier clique, so every
    separator table has card**sep_vars entries and every clique card**k.
    Potentials Uniform(0.01, 1] in FP64."""
    if not 1 <= sep_vars < k:
        raise ValueError("need 1 <= sep_vars < k")
    rng = np.random.default_rng(seed + 97 * sep_vars)
    c_, cl, par, fr = _build(rng, n_cliques, lambda: k, lambda pk: (sep_vars, k - sep_vars),
                             lambda: card, _uniform_parent(rng))
    return _finish(rng, c_, cl, par, fr, f"sep-sweep-{n_cliques}x{card}^{k}-sep{card}^{sep_vars}")


# --------------------------------------------------------------------------
# Alternative potentials with known closed forms (inputs only).
# --------------------------------------------------------------------------

def all_ones(tree: Tree) -> Tree:
    return tree.with_pot(np.ones(tree.entries(), dtype=np.float64), tree.name + "-ones")


def product_form(tree: Tree, seed: int):
    """Potentials phi_C(x) = prod over the variables C introduces of f_v(x_v),
    each variable getting its factor in exactly one clique.  Returns the new
    tree and the factors f (list of arrays, one per variable)."""
    rng = np.random.default_rng(seed)
    f = [0.01 + 0.99 * (1.0 - rng.random(int(k))) for k in tree.card]
    tables = []
    for c, vars_c in enumerate(tree.cliques):
        fresh = set(int(v) for v in tree.fresh[c])
        t = np.ones([int(tree.card[v]) for v in vars_c])
        for ax, v in enumerate(vars_c):
            if int(v) in fresh:
                shape = [1] * len(vars_c)
                shape[ax] = int(tree.card[v])
                t = t * f[int(v)].reshape(shape)
        tables.append(t.reshape(-1))
    return tree.with_pot(np.concatenate(tables), tree.name + "-product"), f


def bn_for_tree(tree: Tree, seed: int, max_parents: int = 3, alpha: float = 1.0):
    """A Bayesian network whose every family fits in a clique of ``tree``.

    Each variable v gets one CPT P(v | pa(v)), with pa(v) up to
    ``max_parents`` variables drawn from the clique that introduces v among
    those created before v (so the network is acyclic and its family lies in
    that clique).  Every CPT column is Dirichlet(alpha * 1) in FP64.  Each
    family is listed in a random order (the table transposed to match), so
    the first-listed variable is the table's most significant digit, as in
    a clique table.  Returns (families: list of int32 arrays, tables: list
    of flat float64 arrays), one per variable, in variable order."""
    rng = np.random.default_rng(seed)
    fam_of, tab_of = {}, {}
    for c, vars_c in enumerate(tree.cliques):
        for v in sorted(int(x) for x in tree.fresh[c]):
            earlier = [int(u) for u in vars_c if int(u) < v]
            k = int(rng.integers(0, min(max_parents, len(earlier)) + 1))
            pa = [int(u) for u in rng.choice(np.array(earlier, dtype=np.int64), size=k, replace=False)] if k else []
            kv = int(tree.card[v])
            n_cols = int(np.prod([int(tree.card[u]) for u in pa], dtype=np.int64))
            cols = rng.dirichlet(np.full(kv, alpha), size=n_cols)          # last axis: v
            t = cols.reshape([int(tree.card[u]) for u in pa] + [kv])
            perm = rng.permutation(k + 1)
            fam = (pa + [v])
            fam_of[v] = np.array([fam[i] for i in perm], dtype=np.int32)
            tab_of[v] = np.ascontiguousarray(np.transpose(t, perm)).reshape(-1)
    order = sorted(fam_of)
    return [fam_of[v] for v in order], [tab_of[v] for v in order]


# --------------------------------------------------------------------------
# Evidence.
# --------------------------------------------------------------------------

def random_evidence(tree: Tree, n_obs: int, seed: int):
    """``n_obs`` distinct variables, each fixed to a uniform state.  Returns
    (vars int32, states int32)."""
    rng = np.random.default_rng(seed)
    n_obs = min(n_obs, tree.n_vars)
    vars_ = np.sort(rng.choice(tree.n_vars, size=n_obs, replace=False)).astype(np.int32)
    states = np.array([int(rng.integers(0, int(tree.card[v]))) for v in vars_], dtype=np.int32)
    return vars_, states


def evidence_matrix(tree: Tree, n_cases: int, frac, base_seed: int) -> np.ndarray:
    """Dense evidence for a batch: int16 [n_cases, n_vars], -1 = unobserved.
    Case ``i`` uses seed ``base_seed + i``; ``frac`` is a fraction of the
    variables, or a (lo, hi) range drawn per case."""
    out = np.full((n_cases, tree.n_vars), -1, dtype=np.int16)
    for i in range(n_cases):
        rng = np.random.default_rng(base_seed + i)
        f = frac if np.isscalar(frac) else float(rng.uniform(frac[0], frac[1]))
        n_obs = int(round(f * tree.n_vars))
        vars_ = rng.choice(tree.n_vars, size=n_obs, replace=False)
        out[i, vars_] = (rng.random(n_obs) * tree.card[vars_]).astype(np.int16)
    return out


def case_from_row(row: np.ndarray):
    vars_ = np.nonzero(row >= 0)[0].astype(np.int32)
    return vars_, row[vars_].astype(np.int32)


# Named workloads: (tree builder, storage dtype, evidence recipe)
WORKLOADS = {
    "small": dict(build=small_tree, dtype=np.float64, n_obs=4),
    "large_clique": dict(build=large_clique_tree, dtype=np.float32, frac=0.05),
    "high_card": dict(build=high_card_tree, dtype=np.float32, n_obs=3),
    "batched": dict(build=batched_tree, dtype=np.float32, frac=0.10, n_cases=4096),
    "binary_serving": dict(build=binary_serving_tree, dtype=np.float32, frac=(0.01, 0.20)),
}


def workload_evidence(name: str, tree: Tree, seed: int):
    """The single evidence case of a named workload."""
    w = WORKLOADS[name]
    if "n_obs" in w:
        return random_evidence(tree, w["n_obs"], seed)
    frac = w["frac"]
    if not np.isscalar(frac):
        frac = float(np.random.default_rng(seed).uniform(frac[0], frac[1]))
    return random_evidence(tree, int(round(frac * tree.n_vars)), seed)
