"""Brute-force enumeration of the joint distribution (tiny trees only).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

This is the definition that belief propagation reaches exactly (Sec. 2.1:
"from these potential tables we can marginalize and compute P(X|e)"): with
separators starting at one, the junction tree represents the product of its
clique tables, so

    Z(e)          = sum_x  prod_C phi_C(x_C) * prod_{v in E} [x_v = e_v]
    P(X = x | e)  = (1 / Z(e)) * sum_{x' : x'_X = x} (same summand).

The joint is built by broadcasting every clique table onto one array with an
axis per variable (ascending variable id); a library sum does the
marginalisation.  Pinned by closed forms in ``tests/test_oracle_pins.py``
(all-ones potentials give Z = prod of unobserved cardinalities; product-form
potentials give Z and the marginals in closed form).
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np


def joint(card, cliques, pot: Sequence[np.ndarray]) -> np.ndarray:
    """prod_C phi_C(x_C) as an array with one axis per variable."""
    card = [int(k) for k in card]
    n = len(card)
    j = np.ones(card, dtype=np.float64)
    for c, vs in enumerate(cliques):
        vs = [int(v) for v in vs]
        t = np.asarray(pot[c], dtype=np.float64).reshape([card[v] for v in vs])
        order = sorted(range(len(vs)), key=lambda a: vs[a])      # axes by var id
        t = np.transpose(t, order)
        shape = [1] * n
        for v in sorted(vs):
            shape[v] = card[v]
        j = j * t.reshape(shape)
    return j


def brute_force(card, cliques, pot, evidence: Dict[int, int] | None = None
                ) -> Tuple[float, List[np.ndarray]]:
    """(log Z(e), marginals) by enumeration."""
    j = joint(card, cliques, pot)
    for v, s in (evidence or {}).items():
        idx = [slice(None)] * j.ndim
        keep = np.zeros(int(card[v]), dtype=bool)
        keep[int(s)] = True
        idx[int(v)] = ~keep
        j[tuple(idx)] = 0.0
    z = float(j.sum())
    margs = []
    for v in range(j.ndim):
        axes = tuple(a for a in range(j.ndim) if a != v)
        m = j.sum(axis=axes)
        margs.append(m / z if z > 0 else m)
    return (float(np.log(z)) if z > 0 else float("-inf")), margs


def brute_force_tree(tree, evidence=None):
    off = tree.pot_off
    return brute_force(tree.card, tree.cliques,
                       [tree.pot[off[c]:off[c + 1]] for c in range(tree.n_cliques)], evidence)
