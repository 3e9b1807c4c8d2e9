"""Block sizes tuned per clique-size class.  The first timed propagation of a
range, after choosing its schedule width, searches a shift of the block-size
target for each clique-size class present (tables of < 2^14, < 2^18 and more
entries): halved, doubled, and once more in a direction that helps.  Later
ranges of the same tree and width reuse the shifts.  Whatever the shifts,
the schedule computes Eq. 1-3 over Algorithms 2-4, so results match the
FP64 oracle at the FP32 tolerances (max relative error 1e-5 on normalised
marginals and on log Z)."""
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
def auto(monkeypatch):
    monkeypatch.delenv("JT_CASE_BLOCK", raising=False)
    monkeypatch.delenv("JT_BLOCK_TUNE", raising=False)


def _tree():
    # 8 cliques of 4^8 entries (2^16: the middle size class), separators of 4-6 variables
    return synth.large_clique_tree(n_cliques=8, n_vars_per=8).as_dtype(np.float32)


def _check(jt, h, t, ev, first, idx):
    n = ev.shape[0]
    st = jt.jt_get_status(h, first, n)
    lz = jt.jt_get_log_evidence(h, first, n)
    m = jt.jt_get_marginals(h, first, n)
    for i in idx:
        assert st[i] == jt.JT_OK, (i, st[i])
        ref = hugin.propagate_tree(t, hugin.evidence_dict(*synth.case_from_row(ev[i])))
        assert logz_ok(lz[i], ref.log_z, "f32"), (i, lz[i], ref.log_z)
        assert marg_errors(split_marginals(m[i], t.card), ref.marginals, "f32") <= TOL["f32"]


def test_tuned_schedule_matches_the_oracle_and_is_reused(jt, auto):
    t = _tree()
    ev = synth.evidence_matrix(t, 20, 0.05, 930)
    h = jt.jt_load_synth(t, compute=jt.JT_F32, max_cases=20)
    jt.jt_set_evidence_dense(h, 0, ev)
    # one case: the one-case schedule, tuned
    jt.jt_propagate(h, 0, 1)
    s1 = jt.jt_get_schedule(h, 0, 1)
    assert s1["case_block"] == 1 and len(s1["block_shift"]) == 3, s1
    assert all(-2 <= x <= 2 for x in s1["block_shift"]), s1
    assert s1["block_shift"][0] == 0 and s1["block_shift"][2] == 0, s1   # only the 2^16 class is present
    _check(jt, h, t, ev[:1], 0, [0])
    # another one-case range of the same tree: the same shifts, no new search
    jt.jt_propagate(h, 7, 1)
    s2 = jt.jt_get_schedule(h, 7, 1)
    assert s2["case_block"] == 1 and s2["block_shift"] == s1["block_shift"], (s1, s2)
    _check(jt, h, t, ev[7:8], 7, [0])
    # a batch: its own width, tuned for that width
    jt.jt_propagate(h, 0, 20)
    s3 = jt.jt_get_schedule(h, 0, 20)
    assert all(-2 <= x <= 2 for x in s3["block_shift"]), s3
    _check(jt, h, t, ev, 0, [0, 9, 19])
    h.free()


def test_tuning_switched_off(jt, monkeypatch):
    monkeypatch.delenv("JT_CASE_BLOCK", raising=False)
    monkeypatch.setenv("JT_BLOCK_TUNE", "0")
    t = _tree()
    ev = synth.evidence_matrix(t, 3, 0.05, 931)
    h = jt.jt_load_synth(t, compute=jt.JT_F32, max_cases=3)
    jt.jt_set_evidence_dense(h, 0, ev)
    jt.jt_propagate(h, 0, 3)
    assert jt.jt_get_schedule(h, 0, 3)["block_shift"] == [0, 0, 0]
    _check(jt, h, t, ev, 0, [0, 2])
    h.free()
