"""Hugin belief propagation in junction trees, FP64, plain numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): slow, obviously
correct, and sharing no code with the CUDA path.

What it follows, step by step:

* Sec. 3, Eq. 2 (marginalisation): the new separator table is the clique
  table summed over the clique's variables that are not in the separator.
* Sec. 3, Eq. 3 and the sentence after it (scattering): the receiving clique
  is multiplied by new/old separator, with a zero denominator giving zero.
* Eq. 1: a message is Eq. 2 followed by Eq. 3; the separator then holds the
  new table (Algorithm 1 never writes it back, which would make the
  distribute pass divide by a stale separator -- the oracle stores it, the
  standard Hugin update; a brute-force pin fails without it).
* Algorithm 2 (Collect_Evidence): recursive, every child sends to its parent
  after its own subtree has been collected.
* Algorithm 3 (Distribute_Evidence): every parent sends to each child, then
  recurses into it.
* Algorithm 4 (Belief_Propagation): collect then distribute from the root
  (clique 0).  Initialization (multiplying CPTs into cliques) is done by the
  input generator; separators start at 1.
* Sec. 3.1: the index mapping between a clique table and a separator table,
  by decoding each flat index into its state string (first-listed variable
  most significant) and matching the separator variables' states.

Readings where the paper is silent:

* separator tables start at all ones;
* evidence is entered by zeroing, in every clique holding an observed
  variable, the entries whose state disagrees;
* each collect message is divided by its sum (and so is the sending clique,
  which keeps the Hugin invariant joint = prod(cliques) / prod(separators)
  up to the tracked factor); the logs of these sums plus the log of the root
  sum give log Z(e); after the distribute pass every clique holds
  P(x_C | e) and sums to one;
* a separator table is laid out over its variables in ascending variable-id
  order, first most significant;
* children are visited in ascending clique index;
* the marginal of a variable is read from the smallest clique that holds it
  (ties: lowest index).

Pinned by ``tests/test_oracle_pins.py``: Fig. 2 mapping sets, brute-force
joint enumeration, closed forms (all-ones and product-form potentials, the
normalised Bayesian network), calibration invariants, chain rule, root
invariance, and planted-mistake checks.
"""
from __future__ import annotations

import sys
from dataclasses import dataclass
from typing import Dict, List, Sequence

import numpy as np


class NotAJunctionTree(ValueError):
    """The input violates a structural requirement (Sec. 2.1)."""


class ZeroEvidence(ArithmeticError):
    """P(e) = 0: some collect message (or the root) sums to zero."""


# --------------------------------------------------------------------------
# Sec. 3.1 -- index <-> state string, and the index mapping by scanning.
# --------------------------------------------------------------------------

def state_string(index: int, cards: Sequence[int]) -> List[int]:
    """Decode a flat table index into the states of the table's variables,
    first-listed variable most significant (Sec. 3.1, the layout of Fig. 2)."""
    states = [0] * len(cards)
    for pos in range(len(cards) - 1, -1, -1):
        states[pos] = index % cards[pos]
        index //= cards[pos]
    return states


def flat_index(states: Sequence[int], cards: Sequence[int]) -> int:
    """Inverse of :func:`state_string`."""
    idx = 0
    for s, k in zip(states, cards):
        idx = idx * k + s
    return idx


def mapping_tables(clique_vars: Sequence[int], card: Sequence[int],
                   sep_vars: Sequence[int]) -> List[List[int]]:
    """For every separator entry r, the clique entries mapped to it
    (Sec. 3.1 / 3.2): decode r into a state string Y^r over the separator
    variables, scan all clique entries, and keep those whose separator
    variables take the states of Y^r.  Pure Python; small tables only."""
    ccards = [int(card[v]) for v in clique_vars]
    scards = [int(card[v]) for v in sep_vars]
    pos_in_clique = [list(clique_vars).index(v) for v in sep_vars]
    n_clique = int(np.prod(ccards)) if ccards else 1
    n_sep = int(np.prod(scards)) if scards else 1
    out = []
    for r in range(n_sep):
        y = state_string(r, scards)
        hits = []
        for j in range(n_clique):
            x = state_string(j, ccards)
            if all(x[p] == y[i] for i, p in enumerate(pos_in_clique)):
                hits.append(j)
        out.append(hits)
    return out


# --------------------------------------------------------------------------
# Eq. 2 and Eq. 3 on numpy tables.
# --------------------------------------------------------------------------

def separator(vars_i: Sequence[int], vars_j: Sequence[int]) -> List[int]:
    """S_ij = X_i intersect X_j (Sec. 2.1), in ascending variable id."""
    return sorted(set(int(v) for v in vars_i) & set(int(v) for v in vars_j))


def _shaped(table: np.ndarray, vars_: Sequence[int], card) -> np.ndarray:
    return table.reshape([int(card[v]) for v in vars_]) if len(vars_) else table.reshape(())


def marginalize(table: np.ndarray, vars_: Sequence[int], card,
                sep: Sequence[int]) -> np.ndarray:
    """Eq. 2: sum the clique table over X \\ S; result laid out over ``sep``
    (in the order given), first most significant, flattened."""
    t = _shaped(table, vars_, card)
    vars_ = [int(v) for v in vars_]
    drop = tuple(ax for ax, v in enumerate(vars_) if v not in sep)
    m = t.sum(axis=drop) if drop else t
    kept = [v for v in vars_ if v in sep]
    if kept:
        m = np.transpose(m, [kept.index(v) for v in sep])
    return np.ascontiguousarray(m).reshape(-1)


def scatter(table: np.ndarray, vars_: Sequence[int], card, sep: Sequence[int],
            factor: np.ndarray) -> np.ndarray:
    """Eq. 3's product: multiply every clique entry by the separator-table
    entry with the same states of the separator variables."""
    vars_ = [int(v) for v in vars_]
    if not sep:
        return table * factor.reshape(())
    f = factor.reshape([int(card[v]) for v in sep])
    order = sorted(range(len(sep)), key=lambda i: vars_.index(sep[i]))
    f = np.transpose(f, order)       # now in the clique's order of those vars
    shape = [int(card[v]) if v in sep else 1 for v in vars_]
    return (_shaped(table, vars_, card) * f.reshape(shape)).reshape(-1)


def sepset_ratio(new: np.ndarray, old: np.ndarray) -> np.ndarray:
    """new / old with the rule that a zero denominator gives zero (Sec. 3,
    after Eq. 3)."""
    out = np.zeros_like(new)
    nz = old != 0
    out[nz] = new[nz] / old[nz]
    return out


# --------------------------------------------------------------------------
# Validation.
# --------------------------------------------------------------------------

def validate(card, cliques, parent, pot_sizes=None) -> None:
    """Structural checks: a tree rooted at clique 0 with n-1 edges, every
    variable id valid and held by some clique, no duplicate variable inside a
    clique, card >= 2, and
    the running-intersection property (the cliques holding a variable form a
    connected subtree, i.e. (#holders - 1) tree edges have it on both ends)."""
    n = len(cliques)
    if n < 1:
        raise NotAJunctionTree("no cliques")
    card = np.asarray(card)
    if np.any(card < 2):
        raise NotAJunctionTree("cardinality < 2")
    if int(parent[0]) != -1:
        raise NotAJunctionTree("clique 0 must be the root")
    for c in range(1, n):
        p = int(parent[c])
        if not (0 <= p < n) or p == c:
            raise NotAJunctionTree(f"bad parent of clique {c}")
    for c in range(n):               # every clique reaches the root
        seen, x = 0, c
        while x != 0:
            x = int(parent[x])
            seen += 1
            if seen > n:
                raise NotAJunctionTree("cycle in parent links")
    holders: Dict[int, int] = {}
    for c, vs in enumerate(cliques):
        vs = [int(v) for v in vs]
        if len(set(vs)) != len(vs):
            raise NotAJunctionTree(f"duplicate variable in clique {c}")
        for v in vs:
            if not (0 <= v < len(card)):
                raise NotAJunctionTree(f"bad variable id {v}")
            holders[v] = holders.get(v, 0) + 1
    shared: Dict[int, int] = {}
    for c in range(1, n):
        for v in separator(cliques[c], cliques[int(parent[c])]):
            shared[v] = shared.get(v, 0) + 1
    if len(holders) != len(card):
        raise NotAJunctionTree("every variable must appear in some clique")
    for v, h in holders.items():
        if shared.get(v, 0) != h - 1:
            raise NotAJunctionTree(f"running intersection fails for variable {v}")


# --------------------------------------------------------------------------
# Algorithms 2-4.
# --------------------------------------------------------------------------

@dataclass
class Result:
    log_z: float                     # log Z(e)
    marginals: List[np.ndarray]      # P(X = x | e) per variable
    cliques: List[np.ndarray]        # calibrated tables, each = P(x_C | e)
    sepsets: Dict[int, np.ndarray]   # edge (child c) -> final separator table


def enter_evidence(tables: List[np.ndarray], cliques, card,
                   evidence: Dict[int, int]) -> None:
    """Zero, in every clique holding an observed variable, the entries whose
    state of that variable disagrees with the evidence."""
    for c, vs in enumerate(cliques):
        vs = [int(v) for v in vs]
        for v, s in evidence.items():
            if v in vs:
                ax = vs.index(v)
                t = _shaped(tables[c], vs, card)
                idx = [slice(None)] * len(vs)
                keep = np.zeros(int(card[v]), dtype=bool)
                keep[s] = True
                idx[ax] = ~keep
                t[tuple(idx)] = 0.0


def _children(parent) -> List[List[int]]:
    ch = [[] for _ in range(len(parent))]
    for c in range(1, len(parent)):
        ch[int(parent[c])].append(c)
    return ch                        # ascending clique index


def propagate(card, cliques, parent, pot: Sequence[np.ndarray],
              evidence: Dict[int, int] | None = None) -> Result:
    """Belief_Propagation (Algorithm 4) with per-message scaling; returns
    log Z(e), the marginals and the calibrated cliques."""
    card = np.asarray(card, dtype=np.int64)
    cliques = [[int(v) for v in vs] for vs in cliques]
    validate(card, cliques, parent)
    evidence = {int(v): int(s) for v, s in (evidence or {}).items()}
    for v, s in evidence.items():
        if not (0 <= v < len(card)) or not (0 <= s < card[v]):
            raise ValueError("bad evidence")
    phi = [np.array(t, dtype=np.float64).copy() for t in pot]
    for c, t in enumerate(phi):
        if t.size != int(np.prod([card[v] for v in cliques[c]])):
            raise NotAJunctionTree(f"table size of clique {c}")
        if not np.all(np.isfinite(t)) or np.any(t < 0):
            raise ValueError("potentials must be finite and >= 0")
    children = _children(parent)
    sep_vars = {c: separator(cliques[c], cliques[int(parent[c])]) for c in range(1, len(cliques))}
    sep_tab = {c: np.ones(int(np.prod([card[v] for v in sep_vars[c]])))
               for c in sep_vars}                                    # separators start at 1
    enter_evidence(phi, cliques, card, evidence)
    log_scale = [0.0]

    def message(src: int, dst: int, edge: int, normalise: bool) -> None:
        """Eq. 1: marginalise src onto the separator (Eq. 2), scatter the
        new/old ratio into dst (Eq. 3), store the new separator table."""
        s = sep_vars[edge]
        new = marginalize(phi[src], cliques[src], card, s)
        if normalise:
            sigma = float(new.sum())
            if sigma == 0.0:
                raise ZeroEvidence(f"message from clique {src} sums to zero")
            new = new / sigma
            phi[src] = phi[src] / sigma
            log_scale[0] += np.log(sigma)
        ratio = sepset_ratio(new, sep_tab[edge])
        phi[dst] = scatter(phi[dst], cliques[dst], card, s, ratio)
        sep_tab[edge] = new

    def collect(ci: int) -> int:                 # Algorithm 2
        for child in children[ci]:
            message(collect(child), ci, child, normalise=True)
        return ci

    def distribute(ci: int) -> None:             # Algorithm 3
        for child in children[ci]:
            message(ci, child, child, normalise=False)
            distribute(child)

    old_limit = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old_limit, 4 * len(cliques) + 100))
    try:
        collect(0)
        root_sum = float(phi[0].sum())
        if root_sum == 0.0:
            raise ZeroEvidence("root sums to zero")
        phi[0] = phi[0] / root_sum
        log_z = log_scale[0] + np.log(root_sum)
        distribute(0)
    finally:
        sys.setrecursionlimit(old_limit)

    sizes = [t.size for t in phi]
    home: Dict[int, int] = {}
    for c, vs in enumerate(cliques):             # smallest holder, ties -> lowest index
        for v in vs:
            if v not in home or (sizes[c], c) < (sizes[home[v]], home[v]):
                home[v] = c
    marginals = []
    for v in range(len(card)):
        home_c = home[v]
        m = marginalize(phi[home_c], cliques[home_c], card, [v])
        marginals.append(m / m.sum())
    return Result(float(log_z), marginals, phi, sep_tab)


def propagate_tree(tree, evidence=None) -> Result:
    """Convenience wrapper over a ``synth.Tree``-like object (fields card,
    cliques, parent, and ``table(c)``)."""
    off = tree.pot_off
    return propagate(tree.card, tree.cliques, tree.parent,
                     [np.asarray(tree.pot[off[c]:off[c + 1]], dtype=np.float64)
                      for c in range(tree.n_cliques)],
                     evidence)


def evidence_dict(vars_, states) -> Dict[int, int]:
    return {int(v): int(s) for v, s in zip(vars_, states)}
