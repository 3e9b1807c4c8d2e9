"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: max relative error 1e-5 on normalised marginals in FP32 and
1e-12 in FP64; log Z within the same relative bound.  FP32 runs feed the
oracle the same FP32-rounded potentials the GPU holds."""
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


@pytest.fixture(params=["0", "1", "4", "8", "32"])
def case_block(request, monkeypatch):
    """Propagations pick one case per work item, blocks of 4 or 8, 32 cases
    on the lanes of a warp, or the whole tree per CTA by timing them on
    first use; these tests pin each schedule in turn so all stay covered (32
    falls back to 8 on trees that case lanes do not apply to, 0 to 8 -- or to
    one case per item for a single case -- on trees too large for one CTA)."""
    monkeypatch.setenv("JT_CASE_BLOCK", request.param)
    return int(request.param)


def _prep(tree, prec):
    return tree.as_dtype(np.float32) if prec == "f32" else tree.as_dtype(np.float64)


def _run_cases(jt, tree, prec, cases, flags=0, batch=True):
    """Propagate every case (list of (vars, states)) and return
    (logz array, list of marginal lists, handle)."""
    comp = jt.JT_F32 if prec == "f32" else jt.JT_F64
    h = jt.jt_load_synth(tree, compute=comp, max_cases=len(cases), flags=flags)
    for i, (v, s) in enumerate(cases):
        jt.jt_set_evidence(h, i, v, s)
    if batch:
        jt.jt_propagate(h, 0, len(cases))
    else:
        for i in range(len(cases)):
            jt.jt_propagate(h, i, 1)
    lz = jt.jt_get_log_evidence(h, 0, len(cases))
    m = jt.jt_get_marginals(h, 0, len(cases))
    st = jt.jt_get_status(h, 0, len(cases))
    assert np.all(st == jt.JT_OK), st
    return lz, [split_marginals(m[i], tree.card) for i in range(len(cases))], h


def _check(tree, cases, lz, margs, prec, idx=None):
    worst = 0.0
    for i in (range(len(cases)) if idx is None else idx):
        ref = hugin.propagate_tree(tree, hugin.evidence_dict(*cases[i]))
        assert logz_ok(lz[i], ref.log_z, prec), (i, lz[i], ref.log_z)
        worst = max(worst, marg_errors(margs[i], ref.marginals, prec))
    assert worst <= TOL[prec], worst
    return worst


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_small_tree(jt, case_block, prec):
    t = _prep(synth.small_tree(), prec)
    cases = [synth.random_evidence(t, 4, s) for s in range(5)] + [(np.zeros(0, np.int32),) * 2]
    lz, m, _ = _run_cases(jt, t, prec, cases)
    _check(t, cases, lz, m, prec)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_brute_force_variant(jt, case_block, prec):
    t = _prep(synth.small_brute_tree(), prec)
    cases = [synth.random_evidence(t, k, k) for k in range(4)]
    lz, m, _ = _run_cases(jt, t, prec, cases)
    _check(t, cases, lz, m, prec)


@pytest.mark.parametrize("seed", range(16))
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_random_small_trees(jt, case_block, seed, prec):
    """Random cardinalities 2-5, empty separators, separator variables in any
    position of the listed order."""
    t = _prep(synth.random_small_tree(seed, n_cliques=3 + seed % 9, allow_empty_sep=True,
                                      k_range=(1, 5), max_states=1e30), prec)
    cases = [synth.random_evidence(t, (seed + j) % 4, seed * 10 + j) for j in range(3)]
    lz, m, _ = _run_cases(jt, t, prec, cases)
    _check(t, cases, lz, m, prec)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_batched_tree_ragged_batch(jt, case_block, prec):
    """256-clique tree with mixed cardinalities; 37 cases (a ragged last
    case block), compared on a sample of cases."""
    t = _prep(synth.batched_tree(), prec)
    ev = synth.evidence_matrix(t, 37, 0.10, 4000)
    cases = [synth.case_from_row(r) for r in ev]
    lz, m, _ = _run_cases(jt, t, prec, cases)
    _check(t, cases, lz, m, prec, idx=[0, 7, 8, 21, 36])


def test_batched_equals_one_at_a_time(jt, case_block):
    """Each case's result is the same alone and inside a batch."""
    t = _prep(synth.batched_tree(n_cliques=64), "f32")
    ev = synth.evidence_matrix(t, 19, 0.10, 77)
    cases = [synth.case_from_row(r) for r in ev]
    lz_b, m_b, _ = _run_cases(jt, t, "f32", cases, batch=True)
    lz_1, m_1, _ = _run_cases(jt, t, "f32", cases, batch=False)
    for i in range(len(cases)):
        assert abs(lz_b[i] - lz_1[i]) <= 1e-5 * max(1, abs(lz_1[i]))
        assert marg_errors(m_b[i], m_1[i], "f32") <= 1e-5


@pytest.mark.parametrize("builder", ["large_clique", "high_card"])
def test_reduced_large_configs(jt, case_block, builder):
    """Smaller members of the large-clique families: several tiles per
    clique and ragged tails, FP32 and FP64."""
    if builder == "large_clique":
        t = synth.large_clique_tree(seed=5, n_cliques=12, n_vars_per=8, card=4, max_depth=4)
    else:
        t = synth.high_card_tree(seed=5, n_cliques=10, card=12)
    for prec in ("f32", "f64"):
        tp = _prep(t, prec)
        cases = [synth.random_evidence(tp, 3, s) for s in range(3)]
        lz, m, _ = _run_cases(jt, tp, prec, cases)
        _check(tp, cases, lz, m, prec)


@pytest.mark.parametrize("name", ["large_clique", "high_card"])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_full_size_configs(jt, case_block, name, prec):
    """64 x 2^20 and 48 x 2^20 entry trees at the sizes the benchmark runs."""
    w = synth.WORKLOADS[name]
    t = _prep(w["build"](), prec)
    cases = [synth.workload_evidence(name, t, 7), synth.workload_evidence(name, t, 8)]
    lz, m, _ = _run_cases(jt, t, prec, cases, batch=(prec == "f32"))
    _check(t, cases, lz, m, prec)


def test_binary_serving_tree(jt, case_block):
    t = _prep(synth.binary_serving_tree(), "f32")
    ev = synth.evidence_matrix(t, 9, (0.01, 0.20), 99)
    cases = [synth.case_from_row(r) for r in ev]
    lz, m, _ = _run_cases(jt, t, "f32", cases)
    _check(t, cases, lz, m, "f32", idx=[0, 4, 8])


def test_results_do_not_depend_on_stale_shared_memory(jt, monkeypatch):
    """A propagation reads no shared memory it did not write: an FP64
    propagation first leaves its own values (NaN and Inf bit patterns as
    FP32) in every SM's shared memory, and ragged case blocks of tiny cliques
    (lanes past the block end, two-entry windows) must still give the
    oracle's results."""
    monkeypatch.setenv("JT_CASE_BLOCK", "8")   # the case-block schedule (ragged: 9 cases)
    big = _prep(synth.high_card_tree(), "f64")
    hb = jt.jt_load_synth(big, compute=jt.JT_F64, max_cases=16)
    jt.jt_set_evidence_dense(hb, 0, synth.evidence_matrix(big, 16, 0.05, 3))
    t = _prep(synth.binary_serving_tree(), "f32")
    ev = synth.evidence_matrix(t, 9, (0.01, 0.20), 99)
    cases = [synth.case_from_row(r) for r in ev]
    first = None
    for rep in range(8):
        jt.jt_propagate(hb, 0, 16)
        lz, m, h = _run_cases(jt, t, "f32", cases)
        h.free()
        if first is None:
            first = (lz, m)
            _check(t, cases, lz, m, "f32", idx=[0, 5, 8])
        else:
            assert np.all(np.abs(lz - first[0]) <= 1e-6 * np.maximum(1.0, np.abs(first[0])))
    hb.free()


def test_case_block_choice_by_timing(jt, monkeypatch):
    """Without JT_CASE_BLOCK the first multi-case propagation of a range
    times the schedules and keeps one: the results match the oracle and
    later propagations of the range reuse the choice (same results up to the
    order of atomic additions)."""
    monkeypatch.delenv("JT_CASE_BLOCK", raising=False)
    t = _prep(synth.small_tree(), "f32")
    ev = synth.evidence_matrix(t, 12, 0.10, 5)
    cases = [synth.case_from_row(r) for r in ev]
    lz, m, h = _run_cases(jt, t, "f32", cases)
    _check(t, cases, lz, m, "f32", idx=[0, 11])
    jt.jt_propagate(h, 0, len(cases))
    lz2 = jt.jt_get_log_evidence(h, 0, len(cases))
    assert np.all(np.abs(lz2 - lz) <= 1e-6 * np.maximum(1.0, np.abs(lz)))
    h.free()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_calibrated_cliques(jt, prec):
    """Materialised cliques equal the oracle's calibrated tables P(x_C | e)."""
    t = _prep(synth.small_tree(), prec)
    cases = [synth.random_evidence(t, 4, 3)]
    lz, m, h = _run_cases(jt, t, prec, cases, flags=jt.JT_MATERIALIZE_CLIQUES)
    ref = hugin.propagate_tree(t, hugin.evidence_dict(*cases[0]))
    sizes = t.table_sizes()
    worst = 0.0
    for c in range(t.n_cliques):
        g = jt.jt_get_clique(h, 0, c, int(sizes[c]))
        worst = max(worst, marg_errors([g], [ref.cliques[c]], prec))
    assert worst <= TOL[prec]


def test_zero_evidence_reported(jt):
    """P(e) = 0: status JT_ERR_ZERO_EVIDENCE, log Z = -inf, other cases of
    the batch unaffected."""
    t = synth.small_brute_tree()
    pot = t.pot.copy()
    off = t.pot_off
    v = int(t.cliques[2][0])
    pot[off[2]:off[3]].reshape([3] * 5)[1] = 0.0
    t0 = t.with_pot(pot)
    h = jt.jt_load_synth(t0, compute=jt.JT_F64, max_cases=2)
    jt.jt_set_evidence(h, 0, [v], [1])
    jt.jt_set_evidence(h, 1, [v], [0])
    jt.jt_propagate(h, 0, 2)
    st = jt.jt_get_status(h, 0, 2)
    assert st[0] == jt.JT_ERR_ZERO_EVIDENCE and st[1] == jt.JT_OK
    assert jt.jt_log_evidence(h, 0) == float("-inf")
    with pytest.raises(jt.JtError) as e:
        jt.jt_get_marginal(h, 0, 0, 3)
    assert e.value.status == jt.JT_ERR_ZERO_EVIDENCE
    ref = hugin.propagate_tree(t0, {v: 0})
    assert abs(jt.jt_log_evidence(h, 1) - ref.log_z) < 1e-12 * max(1, abs(ref.log_z))


def test_zero_separator_entries(jt):
    """Zeros that make separator entries 0 while P(e) > 0 (the 0/0 := 0
    rule) give the oracle's answer."""
    t = synth.small_brute_tree()
    pot = t.pot.copy()
    off = t.pot_off
    s = hugin.separator(t.cliques[1], t.cliques[int(t.parent[1])])
    tab = pot[off[1]:off[2]].reshape([3] * 5)
    idx = [slice(None)] * 5
    idx[list(t.cliques[1]).index(s[0])] = 0
    tab[tuple(idx)] = 0.0
    t0 = t.with_pot(pot)
    for prec in ("f32", "f64"):
        tp = _prep(t0, prec)
        cases = [(np.zeros(0, np.int32), np.zeros(0, np.int32)), synth.random_evidence(tp, 2, 4)]
        lz, m, _ = _run_cases(jt, tp, prec, cases)
        _check(tp, cases, lz, m, prec)


def test_state_errors(jt):
    t = synth.small_tree()
    h = jt.jt_load_synth(t, compute=jt.JT_F64, max_cases=2)
    with pytest.raises(jt.JtError) as e:
        jt.jt_log_evidence(h, 0)
    assert e.value.status == jt.JT_ERR_STATE
    with pytest.raises(jt.JtError) as e:
        jt.jt_set_evidence(h, 0, [3, 3], [0, 1])
    assert e.value.status == jt.JT_ERR_INVALID_ARG
    with pytest.raises(jt.JtError) as e:
        jt.jt_set_evidence(h, 0, [3], [7])
    assert e.value.status == jt.JT_ERR_INVALID_ARG
    with pytest.raises(jt.JtError) as e:
        jt.jt_propagate(h, 1, 2)
    assert e.value.status == jt.JT_ERR_INVALID_ARG
    with pytest.raises(jt.JtError) as e:
        jt.jt_get_clique(h, 0, 0, 243)
    assert e.value.status == jt.JT_ERR_STATE
    # device-side range check of dense evidence: a bad state marks only that case
    ev = np.full((2, t.n_vars), -1, np.int16)
    jt.jt_set_evidence_dense(h, 0, ev)
    jt.jt_propagate(h, 0, 2)
    assert list(jt.jt_get_status(h, 0, 2)) == [jt.JT_OK, jt.JT_OK]


def test_evidence_replacement_and_reuse(jt):
    """Re-setting evidence and propagating again gives the new answer (no
    state leaks between propagations)."""
    t = synth.small_tree()
    h = jt.jt_load_synth(t, compute=jt.JT_F64, max_cases=1)
    for s in range(3):
        v, st = synth.random_evidence(t, 3 + s, 50 + s)
        jt.jt_set_evidence(h, 0, v, st)
        jt.jt_propagate(h, 0, 1)
        ref = hugin.propagate_tree(t, hugin.evidence_dict(v, st))
        assert abs(jt.jt_log_evidence(h, 0) - ref.log_z) < 1e-12 * max(1, abs(ref.log_z))
        for var in (0, 40, 97):
            g = jt.jt_get_marginal(h, 0, var, int(t.card[var]))
            assert np.allclose(g, ref.marginals[var], rtol=1e-12, atol=0)
