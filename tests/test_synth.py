"""The seeded generators are deterministic and produce the stated shapes."""
import numpy as np

from oracle import hugin
from paper_1202_3777_gb300 import synth


def test_deterministic_by_seed():
    a, b = synth.batched_tree(), synth.batched_tree()
    assert np.array_equal(a.pot, b.pot) and np.array_equal(a.parent, b.parent)
    assert all(np.array_equal(x, y) for x, y in zip(a.cliques, b.cliques))
    c = synth.batched_tree(seed=7)
    assert not np.array_equal(a.parent, c.parent)
    e1 = synth.evidence_matrix(a, 8, 0.1, 55)
    e2 = synth.evidence_matrix(a, 8, 0.1, 55)
    assert np.array_equal(e1, e2)
    # case i depends only on base_seed + i
    assert np.array_equal(synth.evidence_matrix(a, 3, 0.1, 56)[0], e1[1])


def test_shapes_of_the_workloads():
    t = synth.small_tree()
    assert t.n_cliques == 32 and all(len(c) == 5 for c in t.cliques)
    assert set(t.card.tolist()) == {3} and t.n_vars == 5 + 31 * 3
    for c in range(1, 32):
        assert len(hugin.separator(t.cliques[c], t.cliques[t.parent[c]])) == 2
    t = synth.batched_tree()
    sizes = t.table_sizes()
    assert t.n_cliques == 256 and sizes.min() >= 64 and sizes.max() <= 4 ** 9
    for c in range(1, t.n_cliques):
        s = len(hugin.separator(t.cliques[c], t.cliques[t.parent[c]]))
        assert 1 <= s <= 5 and s <= len(t.cliques[c]) - 1
    t = synth.binary_serving_tree()
    assert t.n_cliques == 1024 and set(t.card.tolist()) == {2}
    assert all(3 <= len(c) <= 6 for c in t.cliques)
    ev = synth.evidence_matrix(t, 16, (0.01, 0.2), 3)
    frac = (ev >= 0).mean(axis=1)
    assert frac.min() >= 0.005 and frac.max() <= 0.205


def test_large_clique_structure_small_variant():
    t = synth.large_clique_tree(n_cliques=16, n_vars_per=6, card=4, max_depth=3)
    assert t.depth().max() <= 3
    for c in range(1, t.n_cliques):
        s = len(hugin.separator(t.cliques[c], t.cliques[t.parent[c]]))
        assert 4 <= s <= 6
    hugin.validate(t.card, t.cliques, t.parent)


def test_bn_for_tree_is_a_network_over_the_tree():
    """One CPT per variable, its family inside one clique, its parents created
    before it (acyclic), every column a distribution; same seed, same net."""
    t = synth.small_tree()
    fams, vals = synth.bn_for_tree(t, 3)
    assert len(fams) == t.n_vars
    sets = [set(int(v) for v in c) for c in t.cliques]
    for v, (fam, tab) in enumerate(zip(fams, vals)):
        assert v in set(fam.tolist()) and max(fam.tolist()) == v
        assert any(set(fam.tolist()) <= s for s in sets)
        shape = [int(t.card[u]) for u in fam]
        ax = fam.tolist().index(v)
        sums = tab.reshape(shape).sum(axis=ax)
        assert np.allclose(sums, 1.0, atol=1e-12) and np.all(tab >= 0)
    f2, v2 = synth.bn_for_tree(t, 3)
    assert all(np.array_equal(a, b) for a, b in zip(vals, v2))


def test_separator_sweep_trees_differ_only_in_separator_size():
    for s in (1, 3, 5):
        t = synth.separator_sweep_tree(s)
        assert t.n_cliques == 32 and all(len(c) == 6 for c in t.cliques)
        assert np.all(t.table_sizes() == 4 ** 6)
        for c in range(1, t.n_cliques):
            sep = set(t.cliques[c].tolist()) & set(t.cliques[int(t.parent[c])].tolist())
            assert len(sep) == s
        hugin.validate(t.card, [c.tolist() for c in t.cliques], t.parent)
