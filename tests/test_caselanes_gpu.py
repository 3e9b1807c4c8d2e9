"""Case-lane schedules (32 evidence cases per work item, one per lane of
every warp; FP32, power-of-two cliques) against the FP64 oracle, element by
element, through the C ABI.

They exercise what is particular to that schedule: case-minor windows and
message slabs, ragged last slabs (lanes with no case), the per-lane evidence
masks on digits inside a block at every level (entry, vector of 4, tile of 32,
above the tile), evidence on digits above the block (a zero block factor),
evidence carried by input messages, block-constant inputs and outputs, empty
separators, calibrated tables, P(e) = 0 in one lane, and windows left over by
other kernels.  Tolerances as for every FP32 result: max relative error 1e-5
on normalised marginals and on log Z."""
import numpy as np
import pytest

from oracle import hugin
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


def _f32(tree):
    return tree.as_dtype(np.float32)


def _run(jt, tree, cases, flags=0, expect_lanes=True):
    h = jt.jt_load_synth(tree, compute=jt.JT_F32, max_cases=len(cases), flags=flags)
    for i, (v, s) in enumerate(cases):
        jt.jt_set_evidence(h, i, v, s)
    jt.jt_propagate(h, 0, len(cases))
    if expect_lanes:
        assert jt.jt_get_schedule(h, 0, len(cases))["case_block"] == 32
    lz = jt.jt_get_log_evidence(h, 0, len(cases))
    m = jt.jt_get_marginals(h, 0, len(cases))
    st = jt.jt_get_status(h, 0, len(cases))
    return lz, [split_marginals(m[i], tree.card) for i in range(len(cases))], st, h


def _check(tree, cases, lz, margs, idx):
    worst = 0.0
    for i in idx:
        ref = hugin.propagate_tree(tree, hugin.evidence_dict(*cases[i]))
        assert logz_ok(lz[i], ref.log_z, "f32"), (i, lz[i], ref.log_z)
        worst = max(worst, marg_errors(margs[i], ref.marginals, "f32"))
    assert worst <= TOL["f32"], worst
    return worst


def _pow2_tree(seed, n_cliques):
    return _f32(synth.random_small_tree(seed, n_cliques=n_cliques, card_choices=(2, 4, 8), k_range=(5, 7),
                                        allow_empty_sep=True, max_states=1e30))


@pytest.mark.parametrize("seed", range(12))
def test_pow2_random_trees(jt, lanes, seed):
    """Random trees of cardinalities 2, 4 and 8 (digits of 1-3 bits, so
    observed digits land on every mask level), empty separators, up to 40%
    of the variables observed; 40 cases: a full slab and a ragged one."""
    t = _pow2_tree(seed, 4 + seed)
    ev = synth.evidence_matrix(t, 40, (0.0, 0.4), 100 + seed)
    cases = [synth.case_from_row(r) for r in ev]
    lz, m, st, _ = _run(jt, t, cases)
    assert np.all(st == jt.JT_OK), st
    _check(t, cases, lz, m, range(len(cases)))


def test_reduced_large_clique_three_slabs(jt, lanes):
    """12 cliques of 4^8 entries: several blocks per clique and several
    chunks per block; 70 cases = two full slabs and a ragged third."""
    t = _f32(synth.large_clique_tree(seed=5, n_cliques=12, n_vars_per=8, card=4, max_depth=4))
    ev = synth.evidence_matrix(t, 70, 0.10, 300)
    cases = [synth.case_from_row(r) for r in ev]
    lz, m, st, _ = _run(jt, t, cases)
    assert np.all(st == jt.JT_OK)
    _check(t, cases, lz, m, range(len(cases)))


@pytest.mark.parametrize("name,n,idx", [("large_clique", 40, [0, 13, 31, 32, 39]),
                                        ("high_card", 33, [0, 16, 31, 32])])
def test_full_size_configs(jt, lanes, name, n, idx):
    """The 64 x 4^10 and 48 x 32^4 trees at full size, with the workloads'
    evidence, a sample of cases spread over both slabs."""
    w = synth.WORKLOADS[name]
    t = _f32(w["build"]())
    cases = [synth.workload_evidence(name, t, 500 + i) for i in range(n)]
    lz, m, st, _ = _run(jt, t, cases)
    assert np.all(st == jt.JT_OK)
    _check(t, cases, lz, m, idx)


def test_lanes_equal_one_case_at_a_time(jt, monkeypatch):
    """Each case's result is the same inside a 35-case case-lane propagation
    and propagated alone (one case per work item)."""
    t = _f32(synth.large_clique_tree(seed=9, n_cliques=10, n_vars_per=8, card=4, max_depth=4))
    ev = synth.evidence_matrix(t, 35, 0.10, 11)
    cases = [synth.case_from_row(r) for r in ev]
    monkeypatch.setenv("JT_CASE_BLOCK", "32")
    lz_b, m_b, _, _ = _run(jt, t, cases)
    h = jt.jt_load_synth(t, compute=jt.JT_F32, max_cases=len(cases))
    for i, (v, s) in enumerate(cases):
        jt.jt_set_evidence(h, i, v, s)
        jt.jt_propagate(h, i, 1)
    lz_1 = jt.jt_get_log_evidence(h, 0, len(cases))
    m_1 = jt.jt_get_marginals(h, 0, len(cases))
    for i in range(len(cases)):
        assert abs(lz_b[i] - lz_1[i]) <= 1e-5 * max(1, abs(lz_1[i]))
        assert marg_errors(m_b[i], split_marginals(m_1[i], t.card), "f32") <= 1e-5


def test_calibrated_cliques(jt, lanes):
    """Materialised cliques of a case-lane propagation equal the oracle's
    calibrated tables P(x_C | e), in the first and the ragged slab."""
    t = _pow2_tree(3, 7)
    ev = synth.evidence_matrix(t, 33, (0.0, 0.3), 7)
    cases = [synth.case_from_row(r) for r in ev]
    lz, m, st, h = _run(jt, t, cases, flags=jt.JT_MATERIALIZE_CLIQUES)
    sizes = t.table_sizes()
    worst = 0.0
    for i in (0, 17, 32):
        ref = hugin.propagate_tree(t, hugin.evidence_dict(*cases[i]))
        for c in range(t.n_cliques):
            g = jt.jt_get_clique(h, i, c, int(sizes[c]))
            worst = max(worst, marg_errors([g], [ref.cliques[c]], "f32"))
    assert worst <= TOL["f32"], worst


def test_zero_evidence_in_one_lane(jt, lanes):
    """P(e) = 0 for one case of a slab: that lane reports
    JT_ERR_ZERO_EVIDENCE and log Z = -inf; the other lanes match the oracle."""
    t = _pow2_tree(5, 6)
    pot = t.pot.astype(np.float64).copy()
    off = t.pot_off
    c = 1
    v = int(t.cliques[c][0])
    shape = [int(t.card[x]) for x in t.cliques[c]]
    pot[off[c]:off[c + 1]].reshape(shape)[1] = 0.0    # every entry with v = 1
    t0 = _f32(t.with_pot(pot))
    ev = synth.evidence_matrix(t0, 36, (0.0, 0.2), 8)
    ev[5, :] = -1
    ev[5, v] = 1
    cases = [synth.case_from_row(r) for r in ev]
    lz, m, st, _ = _run(jt, t0, cases)
    zero = [i for i in range(len(cases)) if ev[i, v] == 1]   # case 5, and any other that observes v = 1
    assert 5 in zero
    for i in zero:
        assert st[i] == jt.JT_ERR_ZERO_EVIDENCE and lz[i] == float("-inf"), (i, st[i], lz[i])
    others = [i for i in range(len(cases)) if i not in zero]
    assert len(others) >= 24 and all(st[i] == jt.JT_OK for i in others), st
    _check(t0, cases, lz, m, others)


def test_results_do_not_depend_on_stale_shared_memory(jt, lanes):
    """An FP64 propagation first leaves its own values (NaN and Inf bit
    patterns as FP32) in every SM's shared memory; the case-lane results,
    with a ragged slab, still match the oracle and repeat."""
    big = synth.high_card_tree().as_dtype(np.float64)
    hb = jt.jt_load_synth(big, compute=jt.JT_F64, max_cases=8)
    jt.jt_set_evidence_dense(hb, 0, synth.evidence_matrix(big, 8, 0.05, 3))
    t = _pow2_tree(8, 9)
    ev = synth.evidence_matrix(t, 37, (0.0, 0.3), 9)
    cases = [synth.case_from_row(r) for r in ev]
    first = None
    for rep in range(4):
        jt.jt_propagate(hb, 0, 8)
        lz, m, st, h = _run(jt, t, cases)
        h.free()
        assert np.all(st == jt.JT_OK)
        if first is None:
            first = lz
            _check(t, cases, lz, m, [0, 5, 31, 32, 36])
        else:
            assert np.all(np.abs(lz - first) <= 1e-6 * np.maximum(1.0, np.abs(first)))
    hb.free()


def test_width_choice_includes_case_lanes(jt, monkeypatch):
    """Without JT_CASE_BLOCK a 64-case range of a power-of-two tree times the
    case-lane schedule among the others; whichever wins, results match."""
    monkeypatch.delenv("JT_CASE_BLOCK", raising=False)
    t = _f32(synth.large_clique_tree(seed=5, n_cliques=12, n_vars_per=8, card=4, max_depth=4))
    ev = synth.evidence_matrix(t, 64, 0.10, 21)
    cases = [synth.case_from_row(r) for r in ev]
    lz, m, st, h = _run(jt, t, cases, expect_lanes=False)
    assert jt.jt_get_schedule(h, 0, 64)["case_block"] in (1, 4, 8, 32)
    _check(t, cases, lz, m, [0, 31, 63])
