"""Merging small separators (the remedy of Sec. 5): the merged tree is a
junction tree over the same variables, every original clique lies in its
merged clique, the caps hold, and -- checked with the FP64 oracle -- the
merged tree with the original tables multiplied into it represents the same
joint: every marginal and log Z are unchanged.  CPU only."""
import numpy as np
import pytest

from oracle import cpt, hugin
from paper_1202_3777_gb300 import synth
from paper_1202_3777_gb300.merge import merge_small_separators


def _tables(tree):
    off = tree.pot_off
    return [np.asarray(tree.pot[off[c]:off[c + 1]], dtype=np.float64) for c in range(tree.n_cliques)]


def _entries(vs, card):
    return int(np.prod([int(card[v]) for v in vs], dtype=np.int64))


def _check_structure(tree, m, min_sep, cap):
    cl = [c.tolist() for c in m.cliques]
    hugin.validate(tree.card, cl, m.parent)
    assert all(m.parent[i] < i for i in range(1, len(cl)))
    assert sorted(set(v for c in cl for v in c)) == list(range(tree.n_vars))
    for c in range(tree.n_cliques):
        assert set(tree.cliques[c].tolist()) <= set(cl[m.home[c]])
    for i, c in enumerate(cl):
        # a merged clique is within the cap unless it is a single original clique
        if sum(1 for h in m.home if h == i) > 1:
            assert _entries(c, tree.card) <= cap
    # every surviving separator is large, or merging across it would break a
    # cap (both merged cliques only grew after the merge was declined)
    for i in range(1, len(cl)):
        sep = set(cl[i]) & set(cl[m.parent[i]])
        if _entries(sep, tree.card) < min_sep:
            union = set(cl[i]) | set(cl[m.parent[i]])
            assert _entries(union, tree.card) > cap or len(union) > 32


def _same_distribution(tree, m, ev):
    pot = cpt.cpt_potentials(tree.card, m.cliques, tree.cliques, _tables(tree), home=m.home)
    r0 = hugin.propagate_tree(tree, ev)
    r1 = hugin.propagate(tree.card, m.cliques, m.parent, pot, ev)
    assert abs(r1.log_z - r0.log_z) <= 1e-12 * max(1.0, abs(r0.log_z))
    assert max(float(np.max(np.abs(a - b))) for a, b in zip(r1.marginals, r0.marginals)) < 1e-12


@pytest.mark.parametrize("builder,min_sep,cap", [
    (lambda: synth.small_tree(), 10, 3 ** 8),                    # separators of 9 entries
    (lambda: synth.binary_serving_tree(n_cliques=200), 8, 1 << 10),
    (lambda: synth.random_small_tree(3, n_cliques=8, max_states=1 << 40), 6, 1 << 9),
    (lambda: synth.separator_sweep_tree(1, k=4), 5, 4 ** 7),
])
def test_merged_tree_represents_the_same_joint(builder, min_sep, cap):
    tree = builder()
    m = merge_small_separators(tree.card, tree.cliques, tree.parent, min_sep, cap)
    assert len(m.cliques) < tree.n_cliques
    _check_structure(tree, m, min_sep, cap)
    for k, seed in ((0, 1), (3, 2)):
        _same_distribution(tree, m, hugin.evidence_dict(*synth.random_evidence(tree, k, seed)))


def test_no_merge_below_threshold_or_cap():
    tree = synth.small_tree()
    for m in (merge_small_separators(tree.card, tree.cliques, tree.parent, 1, 1 << 30),
              merge_small_separators(tree.card, tree.cliques, tree.parent, 1 << 30, 1)):
        assert len(m.cliques) == tree.n_cliques
        assert np.array_equal(m.home, np.arange(tree.n_cliques))
        assert all(np.array_equal(a, b) for a, b in zip(m.cliques, tree.cliques))


def test_everything_folds_into_the_root_without_caps():
    tree = synth.random_small_tree(5, n_cliques=6)
    m = merge_small_separators(tree.card, tree.cliques, tree.parent, 1 << 30, 1 << 30)
    assert len(m.cliques) == 1 and m.parent.tolist() == [-1] and np.all(m.home == 0)
    assert sorted(m.cliques[0].tolist()) == list(range(tree.n_vars))
    _same_distribution(tree, m, {})


def test_rejects_a_tree_not_rooted_at_zero():
    with pytest.raises(ValueError):
        merge_small_separators([2, 2], [[0, 1], [1]], [0, -1], 4, 16)
