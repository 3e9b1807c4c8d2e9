"""Whole-tree schedules (one CTA per evidence case, the case's messages in
shared memory, levels separated by CTA barriers) against the FP64 oracle,
element by element, through the C ABI: FP64 and FP32, a single case (the
latency path), more cases than the grid holds (CTAs loop over cases), mixed
and power-of-two cardinalities, empty separators, P(e) = 0 and an
out-of-range evidence state in one case of a batch.  Tolerances 1e-5 (FP32)
and 1e-12 (FP64) relative on normalised marginals and log Z."""
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
def whole(monkeypatch):
    monkeypatch.setenv("JT_CASE_BLOCK", "0")


def _run(jt, tree, prec, ev, first=0):
    comp = jt.JT_F32 if prec == "f32" else jt.JT_F64
    tp = tree.as_dtype(np.float32 if prec == "f32" else np.float64)
    n = ev.shape[0]
    h = jt.jt_load_synth(tp, compute=comp, max_cases=first + n)
    jt.jt_set_evidence_dense(h, first, ev)
    jt.jt_propagate(h, first, n)
    assert jt.jt_get_schedule(h, first, n)["case_block"] == 0
    st = jt.jt_get_status(h, first, n)
    lz = jt.jt_get_log_evidence(h, first, n)
    m = jt.jt_get_marginals(h, first, n)
    return tp, h, st, lz, m


def _check(jt, tp, ev, st, lz, m, prec, idx):
    worst = 0.0
    for i in idx:
        assert st[i] == jt.JT_OK, (i, st[i])
        ref = hugin.propagate_tree(tp, hugin.evidence_dict(*synth.case_from_row(ev[i])))
        assert logz_ok(lz[i], ref.log_z, prec), (i, lz[i], ref.log_z)
        worst = max(worst, marg_errors(split_marginals(m[i], tp.card), ref.marginals, prec))
    assert worst <= TOL[prec], worst


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_small_tree_one_case(jt, whole, prec):
    t = synth.small_tree()
    ev = synth.evidence_matrix(t, 1, 0.05, 12)
    tp, h, st, lz, m = _run(jt, t, prec, ev)
    _check(jt, tp, ev, st, lz, m, prec, [0])
    h.free()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_brute_force_variant(jt, whole, prec):
    t = synth.small_brute_tree()
    ev = synth.evidence_matrix(t, 4, (0.0, 0.4), 21)
    tp, h, st, lz, m = _run(jt, t, prec, ev)
    _check(jt, tp, ev, st, lz, m, prec, range(4))
    h.free()


def test_more_cases_than_ctas(jt, whole):
    """700 cases of the 32-clique tree: every CTA propagates several cases
    in turn, reusing its shared memory; a sample spread over the range,
    starting at a case offset."""
    t = synth.small_tree()
    ev = synth.evidence_matrix(t, 700, 0.05, 300)
    tp, h, st, lz, m = _run(jt, t, "f32", ev, first=5)
    assert np.all(st == jt.JT_OK)
    _check(jt, tp, ev, st, lz, m, "f32", [0, 1, 151, 152, 303, 304, 607, 608, 699])
    h.free()


def test_binary_serving_tree(jt, whole):
    t = synth.binary_serving_tree()
    ev = synth.evidence_matrix(t, 24, (0.01, 0.20), 44)
    tp, h, st, lz, m = _run(jt, t, "f32", ev)
    _check(jt, tp, ev, st, lz, m, "f32", [0, 11, 23])
    h.free()


@pytest.mark.parametrize("seed", range(8))
def test_random_small_trees(jt, whole, seed):
    """Mixed cardinalities (2-5; the generic key path) and powers of two
    (the shift path), empty separators, FP64."""
    if seed % 2:
        t = synth.random_small_tree(seed, n_cliques=4 + seed, card_choices=(2, 4, 8), k_range=(2, 5),
                                    allow_empty_sep=True, max_states=1e30)
    else:
        t = synth.random_small_tree(seed, n_cliques=4 + seed, allow_empty_sep=True, k_range=(1, 5),
                                    max_states=1e30)
    ev = synth.evidence_matrix(t, 6, (0.0, 0.4), 60 + seed)
    tp, h, st, lz, m = _run(jt, t, "f64", ev)
    _check(jt, tp, ev, st, lz, m, "f64", range(6))
    h.free()


def test_zero_evidence_and_bad_state_in_a_batch(jt, whole):
    """One case has P(e) = 0, another an evidence state beyond its
    variable's cardinality (device-side dense evidence is range-checked by
    the kernel); each is reported for its own case and the others match the
    oracle."""
    import torch
    t = synth.small_brute_tree()
    pot = t.pot.copy()
    off = t.pot_off
    v = int(t.cliques[2][0])
    pot[off[2]:off[3]].reshape([3] * 5)[1] = 0.0
    t0 = t.with_pot(pot)
    ev = np.full((4, t0.n_vars), -1, np.int16)
    ev[1, v] = 1                      # P(e) = 0
    ev[2, 0] = 2
    ev[3, 5] = 0
    h = jt.jt_load_synth(t0, compute=jt.JT_F64, max_cases=4)
    bad = ev.copy()
    bad[2, 0] = 7                     # beyond cardinality 3
    jt.jt_set_evidence_dense(h, 0, torch.from_numpy(bad).cuda(), stream=torch.cuda.current_stream())
    jt.jt_propagate(h, 0, 4)
    assert jt.jt_get_schedule(h, 0, 4)["case_block"] == 0
    st = jt.jt_get_status(h, 0, 4)
    assert list(st) == [jt.JT_OK, jt.JT_ERR_ZERO_EVIDENCE, jt.JT_ERR_INVALID_ARG, jt.JT_OK]
    lz = jt.jt_get_log_evidence(h, 0, 4)
    m = jt.jt_get_marginals(h, 0, 4)
    _check(jt, t0, ev, st, lz, m, "f64", [0, 3])
    h.free()


def test_single_case_choice_by_timing(jt, monkeypatch):
    """Without JT_CASE_BLOCK a one-case propagation of a small tree times
    the whole-tree and the one-case-per-item schedules and keeps one; both
    timings are reported and the result matches the oracle."""
    monkeypatch.delenv("JT_CASE_BLOCK", raising=False)
    t = synth.small_tree()
    ev = synth.evidence_matrix(t, 1, 0.05, 13)
    h = jt.jt_load_synth(t, compute=jt.JT_F64, max_cases=1)
    jt.jt_set_evidence_dense(h, 0, ev)
    jt.jt_propagate(h, 0, 1)
    sch = jt.jt_get_schedule(h, 0, 1)
    assert sch["case_block"] in (0, 1) and set(sch["candidate_ms"]) == {0, 1}, sch
    _check(jt, t, ev, jt.jt_get_status(h, 0, 1), jt.jt_get_log_evidence(h, 0, 1), jt.jt_get_marginals(h, 0, 1),
           "f64", [0])
    h.free()
