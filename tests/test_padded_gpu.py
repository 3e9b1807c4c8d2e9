"""Case lanes on trees whose cardinalities are not all powers of two.  Such a
tree is propagated over a padded copy: every cardinality is raised to the
next power of two, and the added states have zero potential in every clique,
so the joint on the original states, P(e) and every marginal are unchanged
(Eq. 1).  The checks run through the C ABI against the FP64 oracle on the
original tree, element by element, at the FP32 tolerances (max relative
error 1e-5 on normalised marginals and on log Z).  They cover mixed and
ternary cardinalities (ragged slabs, a case offset), an evidence state that
is valid in the padded copy but not in the tree, P(e) = 0 in one lane, tables
rewritten by the CPT initialisation (the padded copy follows them), the
width autotuner's choice, and the switch that turns padding off."""
import numpy as np
import pytest

from oracle import cpt, hugin
from paper_1202_3777_gb300 import synth
from parity_util import TOL, logz_ok, marg_errors, split_marginals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def jt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1202_3777_gb300 import build
    build.build()
    from paper_1202_3777_gb300 import jt as mod
    return mod


@pytest.fixture
def lanes(monkeypatch):
    monkeypatch.setenv("JT_CASE_BLOCK", "32")
    monkeypatch.delenv("JT_PAD_CARDS", raising=False)


def _propagate(jt, tree, ev, first=0):
    n = ev.shape[0]
    h = jt.jt_load_synth(tree, compute=jt.JT_F32, max_cases=first + n)
    jt.jt_set_evidence_dense(h, first, ev)
    jt.jt_propagate(h, first, n)
    return h


def _check(jt, h, tree, ev, idx, first=0, pot=None):
    n = ev.shape[0]
    st = jt.jt_get_status(h, first, n)
    lz = jt.jt_get_log_evidence(h, first, n)
    m = jt.jt_get_marginals(h, first, n)
    worst = 0.0
    for i in idx:
        assert st[i] == jt.JT_OK, (i, st[i])
        e = hugin.evidence_dict(*synth.case_from_row(ev[i]))
        ref = hugin.propagate_tree(tree, e) if pot is None else \
            hugin.propagate(tree.card, tree.cliques, tree.parent, pot, e)
        assert logz_ok(lz[i], ref.log_z, "f32"), (i, lz[i], ref.log_z)
        worst = max(worst, marg_errors(split_marginals(m[i], tree.card), ref.marginals, "f32"))
    assert worst <= TOL["f32"], worst


def _padded_lanes(jt, h, first, n):
    sch = jt.jt_get_schedule(h, first, n)
    assert sch["case_block"] == 32 and sch["padded"], sch


def test_ternary_tree_ragged_slabs(jt, lanes):
    """The 32-clique tree of 5 ternary variables per clique (243 entries,
    1024 padded): 40 cases from case 3, so the second slab is ragged."""
    t = synth.small_tree().as_dtype(np.float32)
    ev = synth.evidence_matrix(t, 40, (0.02, 0.25), 500)
    h = _propagate(jt, t, ev, first=3)
    _padded_lanes(jt, h, 3, 40)
    _check(jt, h, t, ev, range(40), first=3)
    h.free()


def test_batched_tree_mixed_cardinalities(jt, lanes):
    """The 256-clique tree of cardinalities 2-4 (2.19M entries, 5.28M
    padded), 64 cases with 10% of the variables observed; a sample spread
    over both slabs."""
    t = synth.batched_tree().as_dtype(np.float32)
    ev = synth.evidence_matrix(t, 64, 0.10, 900)
    h = _propagate(jt, t, ev)
    _padded_lanes(jt, h, 0, 64)
    _check(jt, h, t, ev, [0, 17, 31, 32, 50, 63])
    h.free()


@pytest.mark.parametrize("seed", range(4))
def test_random_trees_with_odd_cardinalities(jt, lanes, seed):
    """Cardinalities 3, 4, 6 and 7 (padded to 4 or 8; cliques of 3-5
    variables, so every padded table has at least 64 entries), 33 cases (a
    slab of one case)."""
    t = synth.random_small_tree(seed, n_cliques=6 + seed, card_choices=(3, 4, 6, 7), k_range=(3, 5),
                                max_states=1e30).as_dtype(np.float32)
    ev = synth.evidence_matrix(t, 33, (0.0, 0.4), 70 + seed)
    h = _propagate(jt, t, ev)
    _padded_lanes(jt, h, 0, 33)
    _check(jt, h, t, ev, range(33))
    h.free()


def test_state_valid_only_in_the_padded_copy(jt, lanes):
    """Device-side dense evidence with state 3 on a ternary variable: the
    padded copy has a fourth state, but the kernel checks the tree's own
    cardinality, so that case alone reports JT_ERR_INVALID_ARG; a case whose
    evidence has P(e) = 0 reports JT_ERR_ZERO_EVIDENCE; the others match the
    oracle."""
    import torch
    t = synth.small_tree()
    pot = t.pot.copy()
    off = t.pot_off
    v0 = int(t.cliques[4][0])
    pot[off[4]:off[5]].reshape([3] * 5)[2] = 0.0
    t0 = t.with_pot(pot).as_dtype(np.float32)
    ev = synth.evidence_matrix(t0, 36, 0.05, 800)
    ev[:, v0] = -1
    ev[5, :] = -1
    ev[5, v0] = 2                     # P(e) = 0
    bad = ev.copy()
    bad[9, 11] = 3                    # beyond cardinality 3, within the padded 4
    h = jt.jt_load_synth(t0, compute=jt.JT_F32, max_cases=36)
    jt.jt_set_evidence_dense(h, 0, torch.from_numpy(bad).cuda(), stream=torch.cuda.current_stream())
    jt.jt_propagate(h, 0, 36)
    _padded_lanes(jt, h, 0, 36)
    st = jt.jt_get_status(h, 0, 36)
    assert st[9] == jt.JT_ERR_INVALID_ARG and st[5] == jt.JT_ERR_ZERO_EVIDENCE, st
    ok = [i for i in range(36) if i not in (5, 9)]
    _check(jt, h, t0, ev, ok[::5] + [35])
    h.free()


def test_padded_copy_follows_cpt_initialisation(jt, lanes):
    """A tree loaded without tables, then initialised from the CPTs of a
    network on the device: propagations over the padded copy use the new
    tables (the oracle runs on the CPT products)."""
    t = synth.random_small_tree(3, n_cliques=7, card_choices=(3, 4), k_range=(3, 5), max_states=1e30)
    fams, vals = synth.bn_for_tree(t, 12, max_parents=3)
    ref = cpt.cpt_potentials(t.card, t.cliques, fams, vals)
    h = jt.jt_load_tree(t.card, t.cliques, t.parent, None, compute=jt.JT_F32, max_cases=40)
    jt.jt_init_from_cpts(h, fams, vals)
    ev = synth.evidence_matrix(t, 40, (0.0, 0.3), 61)
    jt.jt_set_evidence_dense(h, 0, ev)
    jt.jt_propagate(h, 0, 40)
    _padded_lanes(jt, h, 0, 40)
    _check(jt, h, t, ev, range(0, 40, 3), pot=ref)
    # a normalised network: P(no evidence) = 1
    jt.jt_set_evidence(h, 0, np.zeros(0, np.int32), np.zeros(0, np.int32))
    jt.jt_propagate(h, 0, 40)
    assert abs(jt.jt_get_log_evidence(h, 0, 1)[0]) <= TOL["f32"]
    h.free()


def test_width_choice_includes_padded_lanes(jt, monkeypatch):
    """Without JT_CASE_BLOCK the first propagation of a 64-case range times
    the padded case lanes beside the case blocks, keeps the fastest, and
    the result matches the oracle."""
    monkeypatch.delenv("JT_CASE_BLOCK", raising=False)
    monkeypatch.delenv("JT_PAD_CARDS", raising=False)
    t = synth.small_tree().as_dtype(np.float32)
    ev = synth.evidence_matrix(t, 64, 0.05, 810)
    h = _propagate(jt, t, ev)
    sch = jt.jt_get_schedule(h, 0, 64)
    assert 32 in sch["candidate_ms"] and 8 in sch["candidate_ms"], sch
    assert sch["padded"] == (sch["case_block"] == 32), sch
    _check(jt, h, t, ev, [0, 21, 42, 63])
    h.free()


def test_padding_switched_off(jt, monkeypatch):
    """JT_PAD_CARDS=0: no padded copy, so forced case lanes fall back to the
    8-case blocks, with the same results."""
    monkeypatch.setenv("JT_CASE_BLOCK", "32")
    monkeypatch.setenv("JT_PAD_CARDS", "0")
    t = synth.small_tree().as_dtype(np.float32)
    ev = synth.evidence_matrix(t, 40, 0.05, 820)
    h = _propagate(jt, t, ev)
    sch = jt.jt_get_schedule(h, 0, 40)
    assert sch["case_block"] == 8 and not sch["padded"], sch
    _check(jt, h, t, ev, [0, 39])
    h.free()
