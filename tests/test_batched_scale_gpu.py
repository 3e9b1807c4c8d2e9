"""Batched evidence at its stated size: 4096 independent evidence cases on
the resident 256-clique tree (6-9 variables of cardinality 2-4 per clique,
separators of 2-5 variables, 10% of the variables observed per case, case
seed = base seed + case id), FP32, in one persistent propagation launch
(the schedule's width chosen by timing on first use), compared element by
element with the FP64 oracle on a spread sample of cases: the first and last
cases, the edges of case blocks, and cases spread over the range.  Ranges of
4093 cases end in a ragged case block and a ragged slab of case lanes."""
import numpy as np
import pytest

from oracle import hugin
from paper_1202_3777_gb300 import synth
from parity_util import TOL, logz_ok, marg_errors, split_marginals

pytestmark = pytest.mark.gpu

N = 4096


@pytest.fixture(scope="module")
def jt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1202_3777_gb300 import build
    build.build()
    from paper_1202_3777_gb300 import jt as mod
    return mod


@pytest.fixture(scope="module")
def loaded(jt):
    t = synth.batched_tree().as_dtype(np.float32)
    ev = synth.evidence_matrix(t, N, synth.WORKLOADS["batched"]["frac"], 4000)
    h = jt.jt_load_synth(t, compute=jt.JT_F32, max_cases=N)
    jt.jt_set_evidence_dense(h, 0, ev)
    yield t, ev, h
    h.free()


def _sample(n):
    rng = np.random.default_rng(11)
    edge = [0, 1, 7, 8, 31, 32, n // 2 - 1, n // 2, n - 9, n - 8, n - 2, n - 1]
    spread = rng.choice(n, size=16, replace=False).tolist()
    return sorted(set(i for i in edge + spread if 0 <= i < n))


def _check(jt, t, ev, h, first, n):
    st = jt.jt_get_status(h, first, n)
    assert np.all(st == jt.JT_OK), np.nonzero(st)[0][:10]
    lz = jt.jt_get_log_evidence(h, first, n)
    m = jt.jt_get_marginals(h, first, n)
    worst = 0.0
    for i in _sample(n):
        ref = hugin.propagate_tree(t, hugin.evidence_dict(*synth.case_from_row(ev[first + i])))
        assert logz_ok(lz[i], ref.log_z, "f32"), (i, lz[i], ref.log_z)
        worst = max(worst, marg_errors(split_marginals(m[i], t.card), ref.marginals, "f32"))
    assert worst <= TOL["f32"], worst
    return worst


def test_4096_cases_one_launch(jt, loaded, monkeypatch):
    monkeypatch.delenv("JT_CASE_BLOCK", raising=False)
    t, ev, h = loaded
    jt.jt_propagate(h, 0, N)
    sch = jt.jt_get_schedule(h, 0, N)
    # case lanes run over the tree's power-of-two padded copy (cardinality 3)
    assert sch["case_block"] in (1, 4, 8, 32) and sch["grid"] <= 152 * 2
    assert sch["padded"] == (sch["case_block"] == 32), sch
    _check(jt, t, ev, h, 0, N)
    # a second propagation of the range replays the recorded graph
    jt.jt_propagate(h, 0, N)
    _check(jt, t, ev, h, 0, N)


def test_ragged_last_case_block(jt, loaded, monkeypatch):
    monkeypatch.setenv("JT_CASE_BLOCK", "8")
    t, ev, h = loaded
    jt.jt_propagate(h, 0, N - 3)
    assert jt.jt_get_schedule(h, 0, N - 3)["case_block"] == 8
    _check(jt, t, ev, h, 0, N - 3)


def test_ragged_last_slab_padded_lanes(jt, loaded, monkeypatch):
    """4091 cases (a range not recorded before: a range keeps the schedule of
    its first propagation), so the last slab holds 27 cases."""
    monkeypatch.setenv("JT_CASE_BLOCK", "32")
    t, ev, h = loaded
    jt.jt_propagate(h, 0, N - 5)
    sch = jt.jt_get_schedule(h, 0, N - 5)
    assert sch["case_block"] == 32 and sch["padded"], sch
    _check(jt, t, ev, h, 0, N - 5)
