"""Pins for the FP64 oracle, against facts fixed outside the oracle itself:
the Fig. 2 mapping sets, brute-force enumeration of the joint, closed forms,
invariants of a calibrated junction tree, and planted mistakes that each pin
must catch.  CPU only."""
import math
import os

import numpy as np
import pytest

from oracle import brute, hugin
from paper_1202_3777_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel_err(a, b, floor=1e-300):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


def max_marg_err(m1, m2):
    """Largest absolute difference; NaN anywhere makes the result NaN."""
    return float(np.max([np.max(np.abs(a - b)) for a, b in zip(m1, m2)]))


# --------------------------------------------------------------------- Fig. 2

def _fig2_rows():
    rows = []
    for line in open(os.path.join(GOLDEN, "fig2_mapping.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        cl, sep, sets = [p.strip() for p in line.split("|")]
        rows.append((cl.split(), sep.split(),
                     [[int(x) for x in s.split()] for s in sets.split(";")]))
    return rows


def test_fig2_mapping_sets():
    names = {"A": 0, "B": 1, "C": 2, "D": 3}
    card = [2, 2, 2, 2]
    rows = _fig2_rows()
    assert len(rows) == 2
    for cl, sep, sets in rows:
        got = hugin.mapping_tables([names[v] for v in cl], card, [names[v] for v in sep])
        assert got == sets


def test_state_string_roundtrip_and_order():
    cards = [3, 2, 4]
    for r in range(24):
        s = hugin.state_string(r, cards)
        assert hugin.flat_index(s, cards) == r
    # first-listed most significant: index 1 changes only the last variable
    assert hugin.state_string(1, cards) == [0, 0, 1]
    assert hugin.state_string(4, cards) == [0, 1, 0]


@pytest.mark.parametrize("seed", range(6))
def test_marginalize_and_scatter_agree_with_mapping_sets(seed):
    """Eq. 2 (numpy sum over axes) and Eq. 3's product equal the per-entry
    sums / products over the Sec. 3.1 mapping sets."""
    rng = np.random.default_rng(seed)
    k = int(rng.integers(2, 5))
    card = [int(c) for c in rng.integers(2, 4, size=6)]
    vars_ = list(rng.permutation(6)[:k])
    ns = int(rng.integers(0, k + 1))
    sep = sorted(int(v) for v in rng.permutation(vars_)[:ns])
    n = int(np.prod([card[v] for v in vars_]))
    table = rng.random(n)
    mu = hugin.mapping_tables(vars_, card, sep)
    m = hugin.marginalize(table, vars_, card, sep)
    assert np.allclose(m, [table[idx].sum() for idx in mu], rtol=1e-14)
    factor = rng.random(len(mu))
    out = hugin.scatter(table, vars_, card, sep, factor)
    expect = table.copy()
    for j, idx in enumerate(mu):
        expect[idx] *= factor[j]
    assert np.allclose(out, expect, rtol=1e-14)
    # every clique entry maps to exactly one separator entry
    assert sorted(i for idx in mu for i in idx) == list(range(n))


def test_sepset_ratio_zero_rule():
    new = np.array([0.0, 2.0, 3.0, 0.0])
    old = np.array([0.0, 4.0, 0.0, 5.0])
    assert np.array_equal(hugin.sepset_ratio(new, old), [0.0, 0.5, 0.0, 0.0])


# ----------------------------------------------------------- brute force joint

def test_brute_force_twelve_variable_tree():
    t = synth.small_brute_tree()
    assert t.n_vars == 12 and [len(c) for c in t.cliques] == [5, 5, 5, 5]
    for seed in range(3):
        ev = hugin.evidence_dict(*synth.random_evidence(t, seed + 1, seed))
        r = hugin.propagate_tree(t, ev)
        lz, m = brute.brute_force_tree(t, ev)
        assert abs(r.log_z - lz) <= 1e-12 * max(1.0, abs(lz))
        for a, b in zip(r.marginals, m):
            assert rel_err(a, b, 1e-290) < 1e-12


@pytest.mark.parametrize("seed", range(20))
def test_brute_force_random_trees(seed):
    t = synth.random_small_tree(seed, n_cliques=int(3 + seed % 5), allow_empty_sep=True)
    ev = hugin.evidence_dict(*synth.random_evidence(t, seed % 4, seed))
    r = hugin.propagate_tree(t, ev)
    lz, m = brute.brute_force_tree(t, ev)
    assert abs(r.log_z - lz) <= 1e-12 * max(1.0, abs(lz))
    assert max_marg_err(r.marginals, m) < 1e-12


def _zero_separator_state(t, c=1):
    """Zero clique ``c``'s entries where one of its separator variables is in
    state 0, so the separator table gets zero entries while P(e) > 0."""
    pot = t.pot.copy()
    off = t.pot_off
    s = hugin.separator(t.cliques[c], t.cliques[int(t.parent[c])])
    ax = list(t.cliques[c]).index(s[0])
    tab = pot[off[c]:off[c + 1]].reshape([int(t.card[v]) for v in t.cliques[c]])
    idx = [slice(None)] * tab.ndim
    idx[ax] = 0
    tab[tuple(idx)] = 0.0
    return t.with_pot(pot)


def test_zero_separator_entries_follow_zero_rule():
    """Zeros in a clique make separator entries zero while P(e) > 0: the
    0/0 := 0 rule must give the brute-force answer (and no NaN)."""
    t0 = _zero_separator_state(synth.small_brute_tree())
    r = hugin.propagate_tree(t0, {})
    lz, m = brute.brute_force_tree(t0, {})
    assert all(np.all(np.isfinite(x)) for x in r.marginals)
    assert abs(r.log_z - lz) <= 1e-12 * max(1, abs(lz))
    assert max_marg_err(r.marginals, m) < 1e-12


def test_zero_evidence_raises():
    t = synth.small_brute_tree()
    pot = t.pot.copy()
    off = t.pot_off
    v = int(t.cliques[2][0])
    pot[off[2]:off[3]].reshape([3] * 5)[1] = 0.0      # x_v = 1 impossible in clique 2
    with pytest.raises(hugin.ZeroEvidence):
        hugin.propagate_tree(t.with_pot(pot), {v: 1})
    lz, _ = brute.brute_force_tree(t.with_pot(pot), {v: 1})
    assert lz == float("-inf")


# --------------------------------------------------------------- closed forms

@pytest.mark.parametrize("builder", [synth.small_tree, synth.batched_tree,
                                     synth.binary_serving_tree])
def test_all_ones_closed_form(builder):
    t = synth.all_ones(builder())
    vars_, states = synth.random_evidence(t, 7, 3)
    ev = hugin.evidence_dict(vars_, states)
    r = hugin.propagate_tree(t, ev)
    expect = sum(math.log(int(t.card[v])) for v in range(t.n_vars) if v not in ev)
    assert abs(r.log_z - expect) <= 1e-12 * max(1, abs(expect))
    for v in range(t.n_vars):
        k = int(t.card[v])
        want = np.full(k, 1.0 / k)
        if v in ev:
            want = np.zeros(k)
            want[ev[v]] = 1.0
        assert np.allclose(r.marginals[v], want, rtol=0, atol=1e-14)


def _product_form_check(t, seed, n_obs, tol):
    tp, f = synth.product_form(t, seed)
    ev = hugin.evidence_dict(*synth.random_evidence(tp, n_obs, seed))
    r = hugin.propagate_tree(tp, ev)
    expect = 0.0
    for v in range(tp.n_vars):
        expect += math.log(f[v][ev[v]]) if v in ev else math.log(f[v].sum())
    assert abs(r.log_z - expect) <= tol * max(1, abs(expect))
    for v in range(tp.n_vars):
        want = f[v] / f[v].sum()
        if v in ev:
            want = np.zeros_like(want)
            want[ev[v]] = 1.0
        assert rel_err(r.marginals[v], want, 1e-300) < tol or np.allclose(
            r.marginals[v], want, rtol=tol, atol=0)


@pytest.mark.parametrize("builder", [synth.small_tree, synth.batched_tree,
                                     synth.binary_serving_tree])
def test_product_form_closed_form(builder):
    _product_form_check(builder(), 11, 9, 1e-12)


@pytest.mark.slow
@pytest.mark.parametrize("builder", [synth.large_clique_tree, synth.high_card_tree])
def test_product_form_closed_form_full_size(builder):
    """2^20-entry cliques, where enumeration is impossible."""
    _product_form_check(builder(), 5, 12, 1e-11)


def test_normalised_bayesian_network():
    """The high-cardinality workload multiplies a BN's CPTs into its cliques:
    Z(empty) = 1 exactly and the root variable's marginal is its prior."""
    t = synth.high_card_tree(n_cliques=6)
    r = hugin.propagate_tree(t, {})
    assert abs(r.log_z) < 1e-12
    v = t.meta["root_prior_var"]
    assert rel_err(r.marginals[v], t.meta["root_prior"], 1e-300) < 1e-11


# ------------------------------------------------------------------ invariants

def test_calibration_invariants():
    t = synth.small_tree()
    ev = hugin.evidence_dict(*synth.random_evidence(t, 4, 9))
    r = hugin.propagate_tree(t, ev)
    for c, tab in enumerate(r.cliques):
        assert abs(tab.sum() - 1.0) < 1e-13                 # every clique = P(x_C | e)
    for c in range(1, t.n_cliques):
        p = int(t.parent[c])
        s = hugin.separator(t.cliques[c], t.cliques[p])
        mc = hugin.marginalize(r.cliques[c], t.cliques[c], t.card, s)
        mp = hugin.marginalize(r.cliques[p], t.cliques[p], t.card, s)
        assert np.allclose(mc, mp, rtol=1e-12, atol=1e-300)  # calibration
        assert np.allclose(mc, r.sepsets[c], rtol=1e-12, atol=1e-300)
    for v in range(t.n_vars):                                # same marginal everywhere
        for c, vs in enumerate(t.cliques):
            if v in vs:
                m = hugin.marginalize(r.cliques[c], vs, t.card, [v])
                assert np.allclose(m, r.marginals[v], rtol=1e-12, atol=1e-300)
        assert abs(r.marginals[v].sum() - 1) < 1e-13
    for v, s in ev.items():
        assert r.marginals[v][s] == pytest.approx(1.0, abs=1e-15)


def test_chain_rule_across_two_queries():
    t = synth.small_tree()
    ev = hugin.evidence_dict(*synth.random_evidence(t, 3, 2))
    r = hugin.propagate_tree(t, ev)
    for v in [0, 17, 55]:
        if v in ev:
            continue
        for x in range(int(t.card[v])):
            ev2 = dict(ev)
            ev2[v] = x
            r2 = hugin.propagate_tree(t, ev2)
            assert math.exp(r2.log_z - r.log_z) == pytest.approx(r.marginals[v][x], rel=1e-12)


def _reroot(t, new_root):
    """Relabel cliques so that ``new_root`` becomes clique 0 (BFS order)."""
    n = t.n_cliques
    adj = [[] for _ in range(n)]
    for c in range(1, n):
        adj[c].append(int(t.parent[c]))
        adj[int(t.parent[c])].append(c)
    order, par_old, seen = [new_root], {new_root: -1}, {new_root}
    i = 0
    while i < len(order):
        x = order[i]
        i += 1
        for y in sorted(adj[x]):
            if y not in seen:
                seen.add(y)
                par_old[y] = x
                order.append(y)
    new_id = {old: k for k, old in enumerate(order)}
    parent = np.array([-1 if par_old[o] < 0 else new_id[par_old[o]] for o in order], np.int32)
    off = t.pot_off
    pot = np.concatenate([t.pot[off[o]:off[o + 1]] for o in order])
    return synth.Tree(t.card.copy(), [t.cliques[o].copy() for o in order], parent, pot,
                      t.name + "-rerooted", [t.fresh[o] for o in order])


def test_root_invariance():
    t = synth.small_tree()
    ev = hugin.evidence_dict(*synth.random_evidence(t, 4, 4))
    r0 = hugin.propagate_tree(t, ev)
    for root in [5, 17, 31]:
        r1 = hugin.propagate_tree(_reroot(t, root), ev)
        assert abs(r1.log_z - r0.log_z) < 1e-12 * max(1, abs(r0.log_z))
        assert max_marg_err(r1.marginals, r0.marginals) < 1e-12


# ------------------------------------------------------------------ validation

def test_validation_rejects_malformed_trees():
    card = [2, 2, 2]
    with pytest.raises(hugin.NotAJunctionTree):          # running intersection broken
        hugin.validate(card, [[0, 1], [1, 2], [0, 2]], [-1, 0, 1])
    with pytest.raises(hugin.NotAJunctionTree):          # cycle
        hugin.validate(card, [[0, 1], [1, 2], [2]], [-1, 2, 1])
    with pytest.raises(hugin.NotAJunctionTree):          # duplicate variable
        hugin.validate(card, [[0, 0], [1, 2]], [-1, 0])
    with pytest.raises(hugin.NotAJunctionTree):          # cardinality < 2
        hugin.validate([1, 2, 2], [[0, 1], [1, 2]], [-1, 0])
    with pytest.raises(hugin.NotAJunctionTree):          # root not clique 0
        hugin.validate(card, [[0, 1], [1, 2]], [1, -1])
    with pytest.raises(hugin.NotAJunctionTree):          # variable in no clique
        hugin.validate([2, 2, 2, 2], [[0, 1], [1, 2]], [-1, 0])
    hugin.validate(card, [[0, 1], [1, 2], [2]], [-1, 0, 1])


# ----------------------------------------------------------- planted mistakes
# Each plant breaks the oracle in one plausible way; a pin above must fail.

def _brute_agrees(t, ev):
    try:
        r = hugin.propagate_tree(t, ev)
    except Exception:
        return False
    lz, m = brute.brute_force_tree(t, ev)
    if not np.isfinite(r.log_z) or abs(r.log_z - lz) > 1e-9 * max(1, abs(lz)):
        return False
    return max_marg_err(r.marginals, m) < 1e-9


def _case():
    t = synth.small_brute_tree()
    return t, hugin.evidence_dict(*synth.random_evidence(t, 2, 1))


def test_plant_separator_not_stored(monkeypatch):
    """Algorithm 1 read literally never writes the new separator back."""
    t, ev = _case()
    assert _brute_agrees(t, ev)
    orig = hugin.sepset_ratio
    store = {}

    def stale_ratio(new, old):
        key = new.shape
        out = orig(new, store.get(key, np.ones_like(new)))
        return out
    monkeypatch.setattr(hugin, "sepset_ratio", stale_ratio)
    assert not _brute_agrees(t, ev)


def test_plant_separator_axes_transposed(monkeypatch):
    t, ev = _case()
    orig = hugin.marginalize

    def transposed(table, vars_, card, sep):
        return orig(table, vars_, card, list(reversed(sep)))
    monkeypatch.setattr(hugin, "marginalize", transposed)
    assert not _brute_agrees(t, ev)


class _NoLogNumpy:
    """numpy as seen from inside the oracle, with the log-scale term dropped."""

    def __getattr__(self, name):
        return getattr(np, name)

    @staticmethod
    def log(x):
        return 0.0 * x


def test_plant_dropped_log_scale(monkeypatch):
    t, ev = _case()
    monkeypatch.setattr(hugin, "np", _NoLogNumpy())
    assert not _brute_agrees(t, ev)


def test_plant_zero_rule_missing(monkeypatch):
    t0 = _zero_separator_state(synth.small_brute_tree())
    assert _brute_agrees(t0, {})
    monkeypatch.setattr(hugin, "sepset_ratio", lambda new, old: new / old)
    with np.errstate(all="ignore"):
        assert not _brute_agrees(t0, {})


def test_plant_last_child_skipped(monkeypatch):
    t, ev = _case()
    orig = hugin._children
    monkeypatch.setattr(hugin, "_children", lambda parent: [c[:-1] for c in orig(parent)])
    assert not _brute_agrees(t, ev)


def test_plant_scatter_wrong_operand(monkeypatch):
    """Scatter by the old separator instead of the ratio (a dropped term)."""
    t, ev = _case()
    monkeypatch.setattr(hugin, "sepset_ratio", lambda new, old: np.where(old != 0, old, 0.0))
    assert not _brute_agrees(t, ev)


# ------------------------------------------ initialisation from CPTs (Alg. 4)

from oracle import cpt  # noqa: E402

# A -> B -> C, binary: P(A), P(B | A), P(C | B); a junction tree {A,B} - {B,C}
# with the cliques listed out of variable order, so the state-string mapping
# between a clique and a CPT is exercised.
_PA = [0.3, 0.7]
_PB_A = [[0.9, 0.1], [0.2, 0.8]]       # row a, column b
_PC_B = [[0.6, 0.4], [0.25, 0.75]]     # row b, column c


def _chain():
    card = [2, 2, 2]
    cliques = [[1, 0], [2, 1]]
    fams = [[0], [0, 1], [1, 2]]
    vals = [np.array(_PA), np.array(_PB_A).ravel(), np.array(_PC_B).ravel()]
    return card, cliques, [-1, 0], fams, vals


def test_cpt_chain_tables_and_closed_forms():
    card, cliques, parent, fams, vals = _chain()
    pot = cpt.cpt_potentials(card, cliques, fams, vals)
    # clique 0 lists (B, A): entry (b, a) = P(a) P(b | a); clique 1 lists
    # (C, B): entry (c, b) = P(c | b).  P(A) and P(B|A) both go to clique 0,
    # the only one holding A.
    for b in range(2):
        for a in range(2):
            assert pot[0][2 * b + a] == pytest.approx(_PA[a] * _PB_A[a][b], abs=0, rel=1e-15)
    for c in range(2):
        for b in range(2):
            assert pot[1][2 * c + b] == _PC_B[b][c]
    # ancestral marginals and a posterior, by hand
    pb0 = 0.3 * 0.9 + 0.7 * 0.2                       # 0.41
    pc0 = pb0 * 0.6 + (1 - pb0) * 0.25
    r = hugin.propagate(card, cliques, parent, pot, {})
    assert abs(r.log_z) < 1e-15
    assert r.marginals[1][0] == pytest.approx(pb0, rel=1e-14)
    assert r.marginals[2][0] == pytest.approx(pc0, rel=1e-14)
    # P(A=0 | C=0) = sum_b P(a=0) P(b|a=0) P(c=0|b) / P(c=0)
    num = 0.3 * (0.9 * 0.6 + 0.1 * 0.25)
    r = hugin.propagate(card, cliques, parent, pot, {2: 0})
    assert r.log_z == pytest.approx(math.log(pc0), rel=1e-14)
    assert r.marginals[0][0] == pytest.approx(num / pc0, rel=1e-14)


def test_cpt_planted_mistakes_fail_the_closed_forms():
    card, cliques, parent, fams, vals = _chain()
    pb0 = 0.41
    # a transposed operand: P(B|A)'s table read as if listed (B, A)
    bad = cpt.cpt_potentials(card, cliques, [[0], [1, 0], [1, 2]], vals)
    assert abs(hugin.propagate(card, cliques, parent, bad, {}).marginals[1][0] - pb0) > 0.05
    # a dropped CPT: Z is no longer one
    bad = cpt.cpt_potentials(card, cliques, fams[:2], vals[:2])
    assert abs(hugin.propagate(card, cliques, parent, bad, {}).log_z) > 0.5
    # a CPT multiplied in twice
    bad = cpt.cpt_potentials(card, cliques, fams + [fams[1]], vals + [vals[1]])
    assert abs(hugin.propagate(card, cliques, parent, bad, {}).log_z) > 0.1


@pytest.mark.parametrize("seed", range(8))
def test_cpt_network_matches_its_own_factorisation(seed):
    """The cliques built from a network's CPTs represent the network: every
    posterior and P(e) equal brute force over prod_v P(v | pa(v)), enumerated
    from the CPTs themselves (not from the clique tables)."""
    t = synth.random_small_tree(seed, n_cliques=int(3 + seed % 4))
    fams, vals = synth.bn_for_tree(t, seed, max_parents=3)
    pot = cpt.cpt_potentials(t.card, t.cliques, fams, vals)
    for n_obs in (0, 2):
        ev = hugin.evidence_dict(*synth.random_evidence(t, n_obs, seed + 7))
        r = hugin.propagate(t.card, t.cliques, t.parent, pot, ev)
        lz, m = brute.brute_force(t.card, fams, vals, ev)
        assert abs(r.log_z - lz) <= 1e-12 * max(1.0, abs(lz))
        assert max_marg_err(r.marginals, m) < 1e-12
        if n_obs == 0:
            assert abs(r.log_z) < 1e-12       # a normalised network: Z = 1


def test_cpt_home_rule_and_empty_cliques():
    card = [2, 3, 2, 2]
    #            0: 12 entries   1: 8 entries   2: 6 entries  3: 6 entries
    cliques = [[0, 1, 2], [0, 2, 3], [1, 2], [2, 1]]
    # {1, 2} fits 0, 2 and 3: cliques 2 and 3 are the smallest; tie -> 2
    assert cpt.home_clique([2, 1], card, cliques) == 2
    # {0, 2} fits 0 (12 entries) and 1 (8 entries) -> 1
    assert cpt.home_clique([0, 2], card, cliques) == 1
    assert cpt.home_clique([3], card, cliques) == 1
    with pytest.raises(ValueError):
        cpt.home_clique([1, 3], card, cliques)
    pot = cpt.cpt_potentials(card, cliques, [[2, 1]], [np.arange(6.0)])
    assert [p.size for p in pot] == [12, 8, 6, 6]
    assert np.all(pot[0] == 1) and np.all(pot[1] == 1) and np.all(pot[3] == 1)
    # clique 2 lists (1, 2), the CPT (2, 1): entry (x1, x2) = table[x2 * 3 + x1]
    assert [pot[2][2 * x1 + x2] for x1 in range(3) for x2 in range(2)] == \
        [float(x2 * 3 + x1) for x1 in range(3) for x2 in range(2)]
    # an explicit home overrides the rule
    pot = cpt.cpt_potentials(card, cliques, [[2, 1]], [np.arange(6.0)], home=[0])
    assert np.all(pot[2] == 1) and sorted(pot[0]) == sorted(np.repeat(np.arange(6.0), 2))


def test_cpt_rejects_bad_tables():
    card, cliques, parent, fams, vals = _chain()
    with pytest.raises(ValueError):
        cpt.cpt_potentials(card, cliques, [[0, 2]], [np.ones(4)])        # no clique holds {A, C}
    with pytest.raises(ValueError):
        cpt.cpt_potentials(card, cliques, [[0, 0]], [np.ones(4)])        # repeated variable
    with pytest.raises(ValueError):
        cpt.cpt_potentials(card, cliques, [[0]], [np.array([0.5, -0.1])])
    with pytest.raises(ValueError):
        cpt.cpt_potentials(card, cliques, [[0]], [np.ones(3)])           # wrong size
    with pytest.raises(ValueError):
        cpt.cpt_potentials(card, cliques, [[0]], [np.ones(2)], home=[1])  # clique 1 lacks A


def test_cpt_deterministic_network():
    """Deterministic CPTs put exact zeros in the clique tables, so separator
    entries are zero and the 0/0 rule decides: B copies A, C = A xor B' where
    B' is a noisy copy of B.  Posteriors by hand and by brute force over the
    factorisation; contradicting evidence gives P(e) = 0."""
    card = [2, 2, 2, 2]                       # A, B, B', C
    cliques = [[0, 1, 2], [0, 2, 3]]          # {A,B,B'} - {A,B',C}
    parent = [-1, 0]
    fams = [[0], [0, 1], [1, 2], [0, 2, 3]]
    pa = np.array([0.3, 0.7])
    copy = np.eye(2).ravel()                  # P(B = a | A = a) = 1
    noisy = np.array([[0.9, 0.1], [0.2, 0.8]]).ravel()
    xor = np.array([[[1, 0], [0, 1]], [[0, 1], [1, 0]]], float).ravel()   # C = A xor B'
    vals = [pa, copy, noisy, xor]
    pot = cpt.cpt_potentials(card, cliques, fams, vals)
    assert np.count_nonzero(pot[0] == 0) > 0 and np.count_nonzero(pot[1] == 0) > 0
    # C = 0  <=>  B' = A; P(C=0) = 0.3*0.9 + 0.7*0.8
    pc0 = 0.3 * 0.9 + 0.7 * 0.8
    r = hugin.propagate(card, cliques, parent, pot, {})
    assert abs(r.log_z) < 1e-15 and r.marginals[3][0] == pytest.approx(pc0, rel=1e-14)
    r = hugin.propagate(card, cliques, parent, pot, {3: 0})
    assert r.marginals[1][0] == pytest.approx(0.3 * 0.9 / pc0, rel=1e-14)   # B = A, given C = 0
    for ev in ({3: 1}, {1: 1, 3: 0}, {}):
        r = hugin.propagate(card, cliques, parent, pot, ev)
        lz, m = brute.brute_force(card, fams, vals, ev)
        assert abs(r.log_z - lz) <= 1e-13 and max_marg_err(r.marginals, m) < 1e-13
    # B must equal A: observing A = 0 and B = 1 has probability zero
    with pytest.raises(hugin.ZeroEvidence):
        hugin.propagate(card, cliques, parent, pot, {0: 0, 1: 1})
