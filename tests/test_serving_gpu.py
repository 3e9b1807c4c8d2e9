"""The serving loop (continuous batching over resident trees): every query's
result is the same served in the mix as propagated alone, within the FP32
tolerance (1e-5 relative on marginals and log Z), and matches the FP64
oracle on a sample."""
import numpy as np
import pytest

from oracle import hugin
from paper_1202_3777_gb300 import synth
from parity_util import TOL, logz_ok, marg_errors, split_marginals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1202_3777_gb300 import build
    build.build()
    from paper_1202_3777_gb300 import jt, serve
    return jt, serve


def _trees():
    return {
        "small": synth.small_tree().as_dtype(np.float32),
        "binary": synth.binary_serving_tree().as_dtype(np.float32),
        "large": synth.large_clique_tree(seed=5, n_cliques=10, n_vars_per=8, card=4, max_depth=4).as_dtype(np.float32),
        "highcard": synth.high_card_tree(seed=5, n_cliques=8, card=12).as_dtype(np.float32),
    }


def test_results_alone_equal_results_in_the_mix(mods):
    jt, serve = mods
    trees = _trees()
    srv = serve.Server(trees, budget_bytes=8 << 30, max_batch=16)
    srv.warm_up()
    rng = np.random.default_rng(11)
    names = list(trees)
    arrivals, t = [], 0.0
    for qid in range(80):
        name = names[rng.integers(len(names))]
        tr = trees[name]
        ev = synth.evidence_matrix(tr, 1, (0.01, 0.20), 5000 + qid)[0]
        t += rng.exponential(2e-4)
        arrivals.append((t, serve.Query(qid, name, ev)))
    done = srv.run_arrivals(arrivals)
    assert len(done) == 80 and all(q.status == jt.JT_OK for q in done)
    # several queries shared a batch (continuous batching happened) ...
    assert max(q.batch for q in done) > 1, [q.batch for q in done]
    # ... and batches of different trees ran on the GPU at the same time
    # (their propagation kernels' spans on the global timer intersect)
    assert serve.overlapping_pairs(srv.spans) >= 1, srv.spans
    srv.free()
    alone = {n: jt.jt_load_synth(tr, compute=jt.JT_F32, max_cases=1) for n, tr in trees.items()}
    for q in sorted(done, key=lambda q: q.qid):
        h = alone[q.tree]
        jt.jt_set_evidence_dense(h, 0, q.states[None, :])
        jt.jt_propagate(h, 0, 1)
        m = jt.jt_get_marginals(h, 0, 1)[0]
        lz = float(jt.jt_get_log_evidence(h, 0, 1)[0])
        card = trees[q.tree].card
        assert abs(q.log_z - lz) <= TOL["f32"] * max(1.0, abs(lz)), (q.qid, q.log_z, lz)
        assert marg_errors(split_marginals(q.marginals, card), split_marginals(m, card), "f32") <= TOL["f32"]
    for h in alone.values():
        h.free()
    # and the oracle agrees on a sample
    for q in sorted(done, key=lambda q: q.qid)[:6]:
        tr = trees[q.tree]
        ref = hugin.propagate_tree(tr, hugin.evidence_dict(*synth.case_from_row(q.states)))
        assert logz_ok(q.log_z, ref.log_z, "f32")
        assert marg_errors(split_marginals(q.marginals, tr.card), ref.marginals, "f32") <= TOL["f32"]


def test_latency_summary(mods):
    jt, serve = mods
    qs = [serve.Query(i, "a", np.zeros(1, np.int16), arrival=0.0, done=0.001 * (i + 1)) for i in range(100)]
    s = serve.latency_summary(qs, {"a": 1000})
    assert abs(s["p50_ms"] - 50.5) < 1e-6 and abs(s["p99_ms"] - 99.01) < 1e-6
    assert abs(s["clique_entries_per_s"] - 1000 * 100 / 0.1) < 1e-3


def test_capped_propagation_matches_full_grid(mods):
    """jt_propagate_ctas on 1, 7 and 76 SMs gives the full-grid results (the
    schedule's items are the same; fewer CTAs take them in the same queue
    order), and each kernel's span on the global timer is reported."""
    jt, serve = mods
    t = synth.large_clique_tree(seed=5, n_cliques=10, n_vars_per=8, card=4, max_depth=4).as_dtype(np.float32)
    h = jt.jt_load_synth(t, compute=jt.JT_F32, max_cases=16)
    jt.jt_set_evidence_dense(h, 0, synth.evidence_matrix(t, 16, 0.1, 31))
    jt.jt_propagate(h, 0, 16)
    lz0, m0 = jt.jt_get_log_evidence(h, 0, 16), jt.jt_get_marginals(h, 0, 16)
    s0, e0 = jt.jt_get_kernel_span(h)
    assert e0 > s0
    for cap in (1, 7, 76):
        jt.jt_propagate_ctas(h, 0, 16, cap)
        assert np.all(jt.jt_get_status(h, 0, 16) == jt.JT_OK)
        lz, m = jt.jt_get_log_evidence(h, 0, 16), jt.jt_get_marginals(h, 0, 16)
        assert np.all(np.abs(lz - lz0) <= 1e-5 * np.maximum(1.0, np.abs(lz0)))
        for i in range(16):
            assert marg_errors(split_marginals(m[i], t.card), split_marginals(m0[i], t.card), "f32") <= 1e-5
        s, e = jt.jt_get_kernel_span(h)
        assert e > s > e0
    with pytest.raises(jt.JtError) as err:
        jt.jt_propagate_ctas(h, 0, 16, -1)
    assert err.value.status == jt.JT_ERR_INVALID_ARG
    h.free()
