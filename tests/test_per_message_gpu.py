"""The paper's per-message propagation (Algorithm 1 with index-mapping
tables, naive and interleaved layouts) against the FP64 oracle through the C
ABI: log Z, marginals and the calibrated cliques, FP32 and FP64."""
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


def _run(jt, tree, prec, cases, layout):
    comp = jt.JT_F32 if prec == "f32" else jt.JT_F64
    h = jt.jt_load_synth(tree, compute=comp, max_cases=len(cases), flags=jt.JT_MATERIALIZE_CLIQUES)
    for i, (v, s) in enumerate(cases):
        jt.jt_set_evidence(h, i, v, s)
    for i in range(len(cases)):
        jt.jt_propagate_per_message(h, i, layout)
    lz = jt.jt_get_log_evidence(h, 0, len(cases))
    m = jt.jt_get_marginals(h, 0, len(cases))
    assert np.all(jt.jt_get_status(h, 0, len(cases)) == jt.JT_OK)
    return h, lz, [split_marginals(m[i], tree.card) for i in range(len(cases))]


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_small_tree(jt, layout, prec):
    t = synth.small_tree().as_dtype(np.float32 if prec == "f32" else np.float64)
    cases = [synth.random_evidence(t, 4, s) for s in range(3)] + [(np.zeros(0, np.int32),) * 2]
    h, lz, m = _run(jt, t, prec, cases, layout)
    for i, c in enumerate(cases):
        ref = hugin.propagate_tree(t, hugin.evidence_dict(*c))
        assert logz_ok(lz[i], ref.log_z, prec), (i, lz[i], ref.log_z)
        assert marg_errors(m[i], ref.marginals, prec) <= TOL[prec]
    # the calibrated cliques of the last case
    ref = hugin.propagate_tree(t, hugin.evidence_dict(*cases[-1]))
    sizes = t.table_sizes()
    for c in range(t.n_cliques):
        g = jt.jt_get_clique(h, len(cases) - 1, c, int(sizes[c]))
        assert marg_errors([g], [ref.cliques[c]], prec) <= TOL[prec]
    h.free()


@pytest.mark.parametrize("seed", range(6))
def test_random_small_trees(jt, seed):
    """Random cardinalities 2-5 and empty separators."""
    t = synth.random_small_tree(seed, n_cliques=3 + seed % 9, allow_empty_sep=True, k_range=(1, 5),
                                max_states=1e30).as_dtype(np.float64)
    cases = [synth.random_evidence(t, (seed + j) % 4, seed * 10 + j) for j in range(2)]
    h, lz, m = _run(jt, t, "f64", cases, seed % 2)
    for i, c in enumerate(cases):
        ref = hugin.propagate_tree(t, hugin.evidence_dict(*c))
        assert logz_ok(lz[i], ref.log_z, "f64")
        assert marg_errors(m[i], ref.marginals, "f64") <= TOL["f64"]
    h.free()


def test_layouts_agree_on_a_large_clique_tree(jt):
    """A smaller member of the large-clique family (several thousand entries
    per separator list): both layouts give the oracle's answer."""
    t = synth.large_clique_tree(seed=5, n_cliques=12, n_vars_per=8, card=4, max_depth=4).as_dtype(np.float32)
    cases = [synth.random_evidence(t, 3, 11)]
    ref = hugin.propagate_tree(t, hugin.evidence_dict(*cases[0]))
    for layout in (0, 1):
        h, lz, m = _run(jt, t, "f32", cases, layout)
        assert logz_ok(lz[0], ref.log_z, "f32")
        assert marg_errors(m[0], ref.marginals, "f32") <= TOL["f32"]
        h.free()


def test_needs_materialised_cliques_and_a_valid_layout(jt):
    t = synth.small_tree().as_dtype(np.float32)
    h = jt.jt_load_synth(t, compute=jt.JT_F32, max_cases=1)
    with pytest.raises(jt.JtError):
        jt.jt_propagate_per_message(h, 0, 1)
    h.free()
    h = jt.jt_load_synth(t, compute=jt.JT_F32, max_cases=1, flags=jt.JT_MATERIALIZE_CLIQUES)
    with pytest.raises(jt.JtError):
        jt.jt_propagate_per_message(h, 0, 2)
    h.free()
