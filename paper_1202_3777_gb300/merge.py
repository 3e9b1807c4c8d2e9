"""Junction trees with small separators merged away (the remedy the paper
proposes in Sec. 5 for trees of many small cliques and separators: merge
small separators into large ones and propagate over the modified tree).

Merging a clique into its neighbour across their separator replaces the two
cliques by one over the union of their variables; the product of the two
tables, with the separator at its initial value one, is the merged table, so
the tree represents the same joint distribution and every posterior and
P(e) are unchanged.  Merging adjacent cliques keeps the running-intersection
property (a variable shared with any third clique already lies on the path
through both), and leaves every other separator as it was.

This module only does the structural part (which cliques merge, the merged
variable lists, the parent of each merged clique).  The merged tables are
built on the device: the tree is loaded without tables and each original
clique table enters its merged clique as a factor through
``jt_init_from_cpts`` (the product kernel of Algorithm 4's initialisation).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence

import numpy as np


@dataclass
class MergedTree:
    cliques: List[np.ndarray]   # merged variable lists (table order)
    parent: np.ndarray          # int32, parent[0] = -1
    home: np.ndarray            # int32, the merged clique holding each original clique


def _entries(vars_, card) -> int:
    return int(np.prod([int(card[v]) for v in vars_], dtype=np.int64))


def merge_small_separators(card, cliques: Sequence[Sequence[int]], parent: Sequence[int],
                           min_separator_entries: int, max_clique_entries: int,
                           max_clique_vars: int = 32) -> MergedTree:
    """Merge every clique whose separator with its parent has fewer than
    ``min_separator_entries`` entries into the merged clique that holds its
    parent, while the merged table stays within ``max_clique_entries``
    entries and ``max_clique_vars`` variables.

    Cliques are visited in breadth-first order from the root (clique 0), so a
    chain of small separators folds into its topmost clique until the caps
    stop it.  A merged clique lists its topmost clique's variables first,
    then each absorbed clique's new variables in the order of absorption.
    Merged cliques keep the order of their topmost cliques, so the root stays
    clique 0, nothing is renumbered when nothing merges, and parents precede
    children whenever they did in the input."""
    card = [int(k) for k in card]
    n = len(cliques)
    vars_ = [[int(v) for v in c] for c in cliques]
    parent = [int(p) for p in parent]
    if n == 0 or parent[0] != -1:
        raise ValueError("clique 0 must be the root")
    children = [[] for _ in range(n)]
    for c in range(1, n):
        children[parent[c]].append(c)
    order, q = [], [0]
    while q:                                   # breadth-first from the root
        c = q.pop(0)
        order.append(c)
        q.extend(children[c])
    if len(order) != n:
        raise ValueError("not a tree rooted at clique 0")

    group = list(range(n))                     # clique -> topmost clique of its merged group
    gvars = {c: list(vars_[c]) for c in range(n)}
    for c in order[1:]:
        g = group[parent[c]]
        sep = set(vars_[c]) & set(vars_[parent[c]])
        if _entries(sep, card) >= min_separator_entries:
            continue
        new = [v for v in vars_[c] if v not in set(gvars[g])]
        union = gvars[g] + new
        if len(union) > max_clique_vars or _entries(union, card) > max_clique_entries:
            continue
        gvars[g] = union
        group[c] = g
        del gvars[c]

    # merged tree: a group's parent is the group of its topmost clique's parent
    heads = [c for c in range(n) if group[c] == c]
    index = {h: i for i, h in enumerate(heads)}
    m_parent = np.array([-1 if h == 0 else index[group[parent[h]]] for h in heads], dtype=np.int32)
    m_cliques = [np.array(gvars[h], dtype=np.int32) for h in heads]
    home = np.array([index[group[c]] for c in range(n)], dtype=np.int32)
    return MergedTree(m_cliques, m_parent, home)


def load_merged(card, cliques, parent, potentials, min_separator_entries: int, max_clique_entries: int,
                compute=None, max_cases: int = 1, flags: int = 0, stream=None):
    """Load the merged tree of :func:`merge_small_separators` and build its
    tables on the device from the original clique tables.  Returns
    (tree handle, MergedTree).  Evidence, marginals and log Z are per
    variable and need no translation; clique read-out refers to the merged
    cliques."""
    from . import jt
    m = merge_small_separators(card, cliques, parent, min_separator_entries, max_clique_entries)
    h = jt.jt_load_tree(card, m.cliques, m.parent, None, compute=jt.JT_F32 if compute is None else compute,
                        max_cases=max_cases, flags=flags, stream=stream)
    sizes = [_entries(c, card) for c in cliques]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pot = np.asarray(potentials, dtype=np.float64)
    tables = [pot[off[c]:off[c + 1]] for c in range(len(cliques))]
    jt.jt_init_from_cpts(h, [np.asarray(c, dtype=np.int32) for c in cliques], tables, home=m.home, stream=stream)
    return h, m
