"""Clique tables built on the GPU from a Bayesian network's CPTs (the
Initialization step of Algorithm 4) against the FP64 oracle, through the C
ABI: every resident table, then log Z and the marginals of propagations on
the initialised tree; explicit home cliques, re-initialisation, a tree
loaded without tables, rejected inputs, and evidence retraction without a
reload."""
import numpy as np
import pytest

from oracle import cpt, hugin
from paper_1202_3777_gb300 import synth
from parity_util import TOL, logz_ok, marg_errors, split_marginals

pytestmark = pytest.mark.gpu

# FP32: every CPT value is rounded once and every product of the (at most a
# few dozen) factors rounds once per factor, each within 2^-24 relative.
TABLE_TOL = {"f32": 1e-5, "f64": 1e-13}
TABLE_FLOOR = {"f32": 1e-30, "f64": 1e-290}


@pytest.fixture(scope="module")
def jt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1202_3777_gb300 import build
    build.build()
    from paper_1202_3777_gb300 import jt as mod
    return mod


def _load_empty(jt, tree, prec, max_cases=1):
    comp = jt.JT_F32 if prec == "f32" else jt.JT_F64
    return jt.jt_load_tree(tree.card, tree.cliques, tree.parent, None, compute=comp, max_cases=max_cases)


def _table_err(got, ref, prec):
    got, ref = np.asarray(got, float), np.asarray(ref, float)
    assert got.shape == ref.shape and np.all(np.isfinite(got))
    big = ref >= TABLE_FLOOR[prec]
    assert np.all(np.abs(got[~big] - ref[~big]) <= TABLE_FLOOR[prec])
    return float(np.max(np.abs(got[big] - ref[big]) / ref[big])) if big.any() else 0.0


def _check_tables(jt, h, tree, ref, prec):
    sizes = tree.table_sizes()
    worst = max(_table_err(jt.jt_get_potential(h, c, int(sizes[c])), ref[c], prec) for c in range(tree.n_cliques))
    assert worst <= TABLE_TOL[prec], worst


def _check_propagation(jt, h, tree, pot, prec, cases):
    for i, (v, s) in enumerate(cases):
        jt.jt_set_evidence(h, i, v, s)
    jt.jt_propagate(h, 0, len(cases))
    lz = jt.jt_get_log_evidence(h, 0, len(cases))
    m = jt.jt_get_marginals(h, 0, len(cases))
    for i, (v, s) in enumerate(cases):
        r = hugin.propagate(tree.card, tree.cliques, tree.parent, pot, hugin.evidence_dict(v, s))
        assert logz_ok(lz[i], r.log_z, prec), (i, lz[i], r.log_z)
        assert marg_errors(split_marginals(m[i], tree.card), r.marginals, prec) <= TOL[prec]


TREES = {
    "small-32x243": lambda: synth.small_tree(),                          # card 3: division path, ragged chunks
    "random-mixed": lambda: synth.random_small_tree(4, n_cliques=7),     # mixed cardinalities
    "large-clique-4x4^10": lambda: synth.large_clique_tree(n_cliques=4),  # card 4: shift path, 128 chunks a clique
    "high-card-6x32^4": lambda: synth.high_card_tree(n_cliques=6),       # card 32, 2^20 entries a clique
}


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("name", list(TREES))
def test_tables_and_propagation_match_the_oracle(jt, name, prec):
    tree = TREES[name]()
    fams, vals = synth.bn_for_tree(tree, 11, max_parents=3)
    ref = cpt.cpt_potentials(tree.card, tree.cliques, fams, vals)
    h = _load_empty(jt, tree, prec, max_cases=3)
    ms = jt.jt_init_from_cpts(h, fams, vals)
    assert ms > 0.0
    _check_tables(jt, h, tree, ref, prec)
    cases = [(np.zeros(0, np.int32), np.zeros(0, np.int32))] + \
        [synth.random_evidence(tree, k, 40 + k) for k in (2, 5)]
    _check_propagation(jt, h, tree, ref, prec, cases)
    # a normalised network: P(no evidence) = 1
    assert abs(jt.jt_get_log_evidence(h, 0, 1)[0]) <= TOL[prec]


def _last_holder(fam, tree):
    return max(c for c, vs in enumerate(tree.cliques) if set(int(v) for v in fam) <= set(int(v) for v in vs))


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_explicit_home_cliques(jt, prec):
    """Homing every CPT in the last clique that holds its family changes the
    tables but not the joint: the tables follow the oracle with the same
    homes, the posteriors equal those of the default homes."""
    tree = synth.random_small_tree(9, n_cliques=6)
    fams, vals = synth.bn_for_tree(tree, 2)
    home = [_last_holder(f, tree) for f in fams]
    ref = cpt.cpt_potentials(tree.card, tree.cliques, fams, vals, home=home)
    h = _load_empty(jt, tree, prec, max_cases=2)
    jt.jt_init_from_cpts(h, fams, vals, home=home)
    _check_tables(jt, h, tree, ref, prec)
    cases = [synth.random_evidence(tree, k, 3 + k) for k in (0, 3)]
    _check_propagation(jt, h, tree, cpt.cpt_potentials(tree.card, tree.cliques, fams, vals), prec, cases)


def test_reinitialisation_invalidates_results(jt):
    tree = synth.small_tree()
    f1, v1 = synth.bn_for_tree(tree, 1)
    f2, v2 = synth.bn_for_tree(tree, 2)
    h = _load_empty(jt, tree, "f64")
    jt.jt_init_from_cpts(h, f1, v1)
    v, s = synth.random_evidence(tree, 3, 5)
    jt.jt_set_evidence(h, 0, v, s)
    jt.jt_propagate(h, 0, 1)
    jt.jt_log_evidence(h, 0)
    jt.jt_init_from_cpts(h, f2, v2)
    with pytest.raises(jt.JtError) as e:
        jt.jt_log_evidence(h, 0)
    assert e.value.status == jt.JT_ERR_STATE
    ref = cpt.cpt_potentials(tree.card, tree.cliques, f2, v2)
    _check_tables(jt, h, tree, ref, "f64")
    _check_propagation(jt, h, tree, ref, "f64", [(v, s)])


def test_tree_loaded_without_tables_starts_at_one(jt):
    """No tables at load: every clique is one, so Z is the product of the
    cardinalities and every marginal is uniform; no CPT at all gives the
    same tables again."""
    tree = synth.random_small_tree(2, n_cliques=5)
    h = _load_empty(jt, tree, "f64")
    sizes = tree.table_sizes()
    for c in range(tree.n_cliques):
        assert np.all(jt.jt_get_potential(h, c, int(sizes[c])) == 1.0)
    jt.jt_propagate(h, 0, 1)
    assert jt.jt_log_evidence(h, 0) == pytest.approx(float(np.sum(np.log(tree.card.astype(float)))), rel=1e-12)
    for v in range(tree.n_vars):
        k = int(tree.card[v])
        assert np.allclose(jt.jt_get_marginal(h, 0, v, k), 1.0 / k, rtol=1e-12, atol=0)
    f, t = synth.bn_for_tree(tree, 1)
    jt.jt_init_from_cpts(h, f, t)
    jt.jt_init_from_cpts(h, [], [])
    for c in range(tree.n_cliques):
        assert np.all(jt.jt_get_potential(h, c, int(sizes[c])) == 1.0)


def test_rejected_cpts_leave_the_tables_unchanged(jt):
    tree = synth.small_tree()
    fams, vals = synth.bn_for_tree(tree, 4)
    h = _load_empty(jt, tree, "f32")
    jt.jt_init_from_cpts(h, fams, vals)
    sizes = tree.table_sizes()
    before = [jt.jt_get_potential(h, c, int(sizes[c])) for c in range(tree.n_cliques)]
    # two variables that share no clique
    sets = [set(int(v) for v in c) for c in tree.cliques]
    a, b = next((a, b) for a in range(tree.n_vars) for b in range(a + 1, tree.n_vars)
                if not any({a, b} <= s for s in sets))
    k = int(tree.card[a]) * int(tree.card[b])
    bad = [
        (fams + [np.array([a, b], np.int32)], vals + [np.ones(k)], None),             # no clique holds it
        (fams + [np.array([a, a], np.int32)], vals + [np.ones(int(tree.card[a]) ** 2)], None),  # repeated variable
        (fams + [np.array([tree.n_vars], np.int32)], vals + [np.ones(2)], None),      # variable out of range
        (fams, [vals[0] * -1.0] + vals[1:], None),                                    # negative values
        (fams, [np.full_like(vals[0], np.nan)] + vals[1:], None),                     # non-finite values
        (fams, vals, [tree.n_cliques] * len(fams)),                                   # home out of range
        (fams, vals, [next(c for c, s in enumerate(sets) if int(fams[-1][0]) not in s)] * len(fams)),  # home lacks it
    ]
    for f, v, home in bad:
        with pytest.raises(jt.JtError) as e:
            jt.jt_init_from_cpts(h, f, v, home=home)
        assert e.value.status == jt.JT_ERR_INVALID_ARG
    after = [jt.jt_get_potential(h, c, int(sizes[c])) for c in range(tree.n_cliques)]
    assert all(np.array_equal(x, y) for x, y in zip(before, after))


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_evidence_retraction_without_reload(jt, prec):
    """Evidence is a per-case mask over resident tables: clearing it and
    propagating again gives the no-evidence result, with the tables as
    loaded."""
    tree = synth.small_tree()
    fams, vals = synth.bn_for_tree(tree, 6)
    ref = cpt.cpt_potentials(tree.card, tree.cliques, fams, vals)
    h = _load_empty(jt, tree, prec, max_cases=2)
    jt.jt_init_from_cpts(h, fams, vals)
    sizes = tree.table_sizes()
    tables = [jt.jt_get_potential(h, c, int(sizes[c])) for c in range(tree.n_cliques)]
    jt.jt_propagate(h, 1, 1)                        # case 1: never any evidence
    clean_lz = jt.jt_get_log_evidence(h, 1, 1)[0]
    clean_m = jt.jt_get_marginals(h, 1, 1)[0]
    v, s = synth.random_evidence(tree, 6, 8)
    jt.jt_set_evidence(h, 0, v, s)
    jt.jt_propagate(h, 0, 1)
    r = hugin.propagate(tree.card, tree.cliques, tree.parent, ref, hugin.evidence_dict(v, s))
    assert logz_ok(jt.jt_log_evidence(h, 0), r.log_z, prec)
    jt.jt_set_evidence(h, 0, [], [])                # retract
    jt.jt_propagate(h, 0, 1)
    # block partial sums meet in L2 in any order: equal up to rounding
    assert logz_ok(jt.jt_get_log_evidence(h, 0, 1)[0], clean_lz, prec)
    assert marg_errors(split_marginals(jt.jt_get_marginals(h, 0, 1)[0], tree.card),
                       split_marginals(clean_m, tree.card), prec) <= TOL[prec]
    assert all(np.array_equal(jt.jt_get_potential(h, c, int(sizes[c])), tables[c]) for c in range(tree.n_cliques))


def test_full_size_large_clique_tree(jt):
    """The benchmark's tree (64 cliques of 4^10 entries, FP32): the tables of
    a network built on the device, every entry, and P(no evidence) = 1."""
    tree = synth.large_clique_tree()
    fams, vals = synth.bn_for_tree(tree, 21)
    ref = cpt.cpt_potentials(tree.card, tree.cliques, fams, vals)
    h = _load_empty(jt, tree, "f32")
    jt.jt_init_from_cpts(h, fams, vals)
    _check_tables(jt, h, tree, ref, "f32")
    jt.jt_propagate(h, 0, 1)
    # log Z adds the logs of 64 FP32 stage totals, each within ~1e-6 relative
    assert abs(jt.jt_log_evidence(h, 0)) <= 1e-4
