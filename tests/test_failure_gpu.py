"""Failure path of the persistent propagation kernels, in the allowed form:
no fault, trap or unbounded wait on the GPU.  A host-side hook
(JT_FAULT_UNMET_DEPENDENCY=1, read when a case range's graph is recorded)
makes one work item wait for a block that never finishes; with a short wait
limit (JT_WAIT_LIMIT_MS=20) that item's bounded wait gives up, every other
role of every CTA stops at its next wait, and the host reports
JT_ERR_TIMEOUT.  The context stays usable: the next propagation of the same
tree matches the oracle."""
import time

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


def _trees():
    pow2 = synth.random_small_tree(3, n_cliques=7, card_choices=(2, 4, 8), k_range=(5, 7), allow_empty_sep=True,
                                   max_states=1e30)
    return {
        "one-case": (synth.small_tree(), "1", 1),                    # one case per work item, FP64
        "case-block": (synth.batched_tree(n_cliques=48), "8", 9),   # 8-case blocks, FP64
        "case-lanes": (pow2.as_dtype(np.float32), "32", 33),        # 32 cases on the lanes, FP32
    }


@pytest.mark.parametrize("kind", ["one-case", "case-block", "case-lanes"])
def test_wait_timeout_reported_and_recovered(jt, monkeypatch, kind):
    tree, width, n = _trees()[kind]
    comp = jt.JT_F32 if kind == "case-lanes" else jt.JT_F64
    h = jt.jt_load_synth(tree, compute=comp, max_cases=2 * n)
    ev = synth.evidence_matrix(tree, 2 * n, 0.10, 40)
    jt.jt_set_evidence_dense(h, 0, ev)
    monkeypatch.setenv("JT_CASE_BLOCK", width)
    monkeypatch.setenv("JT_WAIT_LIMIT_MS", "20")
    monkeypatch.setenv("JT_FAULT_UNMET_DEPENDENCY", "1")
    t0 = time.time()
    jt.jt_propagate(h, 0, n)
    with pytest.raises(jt.JtError) as e:
        jt.jt_get_status(h, 0, n)
    assert e.value.status == jt.JT_ERR_TIMEOUT
    assert time.time() - t0 < 30
    # the next propagation (another case range: a graph recorded without the
    # hook) runs normally on the same tree and context
    monkeypatch.delenv("JT_FAULT_UNMET_DEPENDENCY")
    monkeypatch.delenv("JT_WAIT_LIMIT_MS")
    jt.jt_propagate(h, n, n)
    st = jt.jt_get_status(h, n, n)
    assert np.all(st == jt.JT_OK), st
    if kind == "case-lanes":
        assert jt.jt_get_schedule(h, n, n)["case_block"] == 32
    prec = "f32" if comp == jt.JT_F32 else "f64"
    lz = jt.jt_get_log_evidence(h, n, n)
    m = jt.jt_get_marginals(h, n, n)
    worst = 0.0
    for i in (0, n - 1):
        ref = hugin.propagate_tree(tree, hugin.evidence_dict(*synth.case_from_row(ev[n + i])))
        assert logz_ok(lz[i], ref.log_z, prec), (lz[i], ref.log_z)
        worst = max(worst, marg_errors(split_marginals(m[i], tree.card), ref.marginals, prec))
    assert worst <= TOL[prec], worst
    h.free()
