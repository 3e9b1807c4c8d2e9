"""Clique potentials from the conditional probability tables of a Bayesian
network, FP64, plain numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): slow, obviously
correct, and sharing no code with the CUDA path.

What it follows: the Initialization step of Algorithm 4 (Sec. 3.3), which
the paper names without spelling out.  The standard Hugin reading, taken
here: every clique and separator table starts at one, and the CPT
P(v | pa(v)) of every variable is multiplied into exactly one clique that
contains its family {v} + pa(v).  The product of the clique tables is then
the network's joint distribution prod_v P(v | pa(v)) (Sec. 2.1: the junction
tree represents the joint).

Readings where the paper is silent:

* a CPT is a table over its family, laid out like a clique table: the
  first-listed variable is the most significant digit;
* a CPT goes to the clique with the fewest entries that contains its family
  (ties: the lowest clique index), unless the caller names the clique;
* the CPTs of one clique are multiplied in ascending CPT order, starting
  from one.

Pinned by ``tests/test_oracle_pins.py``: a three-node chain whose tables,
ancestral marginals and posterior are written out by hand, a deterministic
network (exact zeros), Z = 1 for any normalised network, the home-clique
rule, brute force over the network's own factorisation, and planted
mistakes (a transposed, a dropped and a doubled CPT).
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np


def home_clique(family: Sequence[int], card, cliques) -> int:
    """The clique that receives a CPT over ``family``: among the cliques
    holding every family variable, the one with the fewest table entries,
    ties to the lowest index.  ValueError if no clique holds the family."""
    best, best_n = -1, None
    fam = set(int(v) for v in family)
    for c, vs in enumerate(cliques):
        if fam <= set(int(v) for v in vs):
            n = int(np.prod([int(card[v]) for v in vs], dtype=np.int64))
            if best_n is None or n < best_n:
                best, best_n = c, n
    if best < 0:
        raise ValueError(f"no clique contains the family {sorted(fam)}")
    return best


def cpt_potentials(card, cliques, families: Sequence[Sequence[int]],
                   values: Sequence[np.ndarray],
                   home: Optional[Sequence[int]] = None) -> List[np.ndarray]:
    """Clique tables (listed order, FP64) holding the product of the CPTs
    assigned to each clique, one where a clique receives none.

    ``families[i]`` lists the variables of CPT i in its table order;
    ``values[i]`` is that table, flattened.  ``home[i]`` names the receiving
    clique, or the rule of :func:`home_clique` picks it."""
    card = [int(k) for k in card]
    if len(families) != len(values):
        raise ValueError("one table per family")
    assign = []
    for i, fam in enumerate(families):
        fam = [int(v) for v in fam]
        if not fam or len(set(fam)) != len(fam):
            raise ValueError(f"family {i} is empty or repeats a variable")
        tab = np.asarray(values[i], dtype=np.float64).ravel()
        if tab.size != int(np.prod([card[v] for v in fam], dtype=np.int64)):
            raise ValueError(f"table {i} has the wrong size")
        if not np.all(np.isfinite(tab)) or np.any(tab < 0):
            raise ValueError(f"table {i} must be finite and >= 0")
        c = home_clique(fam, card, cliques) if home is None else int(home[i])
        if not set(fam) <= set(int(v) for v in cliques[c]):
            raise ValueError(f"clique {c} does not hold the family of table {i}")
        assign.append(c)

    out = []
    for c, vs in enumerate(cliques):
        vs = [int(v) for v in vs]
        ccard = [card[v] for v in vs]
        n = int(np.prod(ccard, dtype=np.int64))
        table = np.ones(n, dtype=np.float64)
        # the state of every clique variable at every entry of the table
        states = np.unravel_index(np.arange(n), ccard)
        for i, fam in enumerate(families):
            if assign[i] != c:
                continue
            fam = [int(v) for v in fam]
            # the CPT entry each clique entry selects: the family variables'
            # states, read off the clique's state string
            idx = np.ravel_multi_index([states[vs.index(v)] for v in fam], [card[v] for v in fam])
            table = table * np.asarray(values[i], dtype=np.float64).ravel()[idx]
        out.append(table)
    return out
