"""Propagation over trees whose small separators were merged away (the
remedy of Sec. 5), through the C ABI: the merged tree is loaded without
tables, its tables are built on the device from the original clique tables
(the initialisation kernel), and every marginal and log Z match the FP64
oracle on the ORIGINAL tree."""
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


CASES = {
    # card 3, separators of 9 entries: 32 cliques -> 22
    "small-32x243": (lambda: synth.small_tree(), 10, 3 ** 8),
    # binary, separators of 2-8 entries: 64 cliques -> 42
    "binary-64": (lambda: synth.binary_serving_tree(n_cliques=64), 8, 1 << 8),
}


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("name", list(CASES))
def test_merged_tree_matches_the_original(jt, name, prec):
    from paper_1202_3777_gb300.merge import load_merged
    build, min_sep, cap = CASES[name]
    tree = build()
    comp = jt.JT_F32 if prec == "f32" else jt.JT_F64
    pot = tree.pot.astype(np.float32).astype(np.float64) if prec == "f32" else tree.pot
    cases = [synth.random_evidence(tree, k, 60 + k) for k in (0, 2, 4)]
    h, m = load_merged(tree.card, tree.cliques, tree.parent, pot, min_sep, cap, compute=comp,
                       max_cases=len(cases))
    assert len(m.cliques) < tree.n_cliques
    for i, (v, s) in enumerate(cases):
        jt.jt_set_evidence(h, i, v, s)
    jt.jt_propagate(h, 0, len(cases))
    lz = jt.jt_get_log_evidence(h, 0, len(cases))
    mg = jt.jt_get_marginals(h, 0, len(cases))
    assert np.all(jt.jt_get_status(h, 0, len(cases)) == jt.JT_OK)
    off = tree.pot_off
    tables = [pot[off[c]:off[c + 1]] for c in range(tree.n_cliques)]
    for i, (v, s) in enumerate(cases):
        r = hugin.propagate(tree.card, tree.cliques, tree.parent, tables, hugin.evidence_dict(v, s))
        assert logz_ok(lz[i], r.log_z, prec), (i, lz[i], r.log_z)
        assert marg_errors(split_marginals(mg[i], tree.card), r.marginals, prec) <= TOL[prec]
