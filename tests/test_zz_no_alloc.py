"""The allocation-free clique read-out (jt_get_clique_noalloc) against the
existing read-out (jt_get_clique), through the C ABI.

jt_get_clique_noalloc exists for callers that must not allocate device
memory (a component that owns the device's memory through a fixed arena, or
a serving path that forbids allocation): it writes into the caller's device
buffer and reduces through a scratch array that lives in the library.  That
array is shared by every call and keeps the previous call's contents, so the
checks below make several calls in a row, with tables of one and of several
partial-sum blocks, and check the size limit.  This file runs last (it is
collected after the other test files) and needs nothing from them."""
import numpy as np
import pytest

from paper_1202_3777_gb300 import synth
from parity_util import TOL, marg_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1202_3777_gb300 import build
    build.build()
    from paper_1202_3777_gb300 import jt as mod
    return mod, torch


def _materialised(jt, tree, prec, n_cases):
    comp = jt.JT_F32 if prec == "f32" else jt.JT_F64
    tp = tree.as_dtype(np.float32 if prec == "f32" else np.float64)
    h = jt.jt_load_synth(tp, compute=comp, max_cases=n_cases, flags=jt.JT_MATERIALIZE_CLIQUES)
    for i in range(n_cases):
        jt.jt_set_evidence(h, i, *synth.random_evidence(tp, 3, 40 + i))
    jt.jt_propagate(h, 0, n_cases)
    assert np.all(jt.jt_get_status(h, 0, n_cases) == jt.JT_OK)
    return tp, h


def _compare(jt, torch, tp, h, calls, prec):
    sizes = tp.table_sizes()
    stream = torch.cuda.current_stream()
    for case, clique in calls:
        n = int(sizes[clique])
        ref = jt.jt_get_clique(h, case, clique, n)
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        jt.jt_get_clique_noalloc(h, case, clique, out, stream=stream)
        stream.synchronize()
        got = out.cpu().numpy()
        assert marg_errors([got], [ref], prec) <= TOL[prec], (case, clique)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_noalloc_matches_get_clique_small(env, prec):
    """One partial-sum block per table; consecutive calls on different
    cases and cliques."""
    jt, torch = env
    tp, h = _materialised(jt, synth.small_tree(), prec, 2)
    _compare(jt, torch, tp, h, [(0, 3), (1, 3), (0, 17), (1, 0)], prec)
    h.free()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_noalloc_matches_get_clique_multiblock(env, prec):
    """Tables of 4^8 = 65,536 entries: sixteen partial sums per call; a
    smaller table after a larger one leaves stale partials behind, which
    must not leak into its sum."""
    jt, torch = env
    tree = synth.large_clique_tree(seed=5, n_cliques=6, n_vars_per=8, card=4, max_depth=3)
    tp, h = _materialised(jt, tree, prec, 1)
    _compare(jt, torch, tp, h, [(0, 0), (0, 5), (0, 0)], prec)
    h.free()
    # a 243-entry table right after the 65,536-entry ones
    tp2, h2 = _materialised(jt, synth.small_tree(), prec, 1)
    _compare(jt, torch, tp2, h2, [(0, 4), (0, 4)], prec)
    h2.free()


def test_noalloc_rejects_tables_above_limit(env):
    """A clique of 2^23 entries exceeds the 4,194,304-entry limit."""
    jt, torch = env
    card = np.full(23, 2, np.int32)
    pot = np.full(1 << 23, 0.5, np.float32)
    h = jt.jt_load_tree(card, [np.arange(23)], [-1], pot, compute=jt.JT_F32, max_cases=1,
                        flags=jt.JT_MATERIALIZE_CLIQUES)
    out = torch.zeros(1 << 23, dtype=torch.float64, device="cuda")
    with pytest.raises(jt.JtError) as e:
        jt.jt_get_clique_noalloc(h, 0, 0, out)
    assert e.value.status == jt.JT_ERR_UNSUPPORTED
    assert "4194304" in jt.jt_last_error()
    h.free()


def test_noalloc_on_a_side_stream_is_ordered_with_propagations(env):
    """A read-out on a stream of its own, issued right after a propagation
    and followed at once by the next propagation (new evidence) on the
    propagation's stream, with no host synchronisation in between, reads the
    table of the first propagation: the read-out waits for the propagation
    that wrote the table, and the next propagation waits for the read-out
    before it rewrites it."""
    jt, torch = env
    tree = synth.large_clique_tree(seed=5, n_cliques=6, n_vars_per=8, card=4, max_depth=3)
    tp, h = _materialised(jt, tree, "f32", 1)
    clique = 3
    n = int(tp.table_sizes()[clique])
    ref1 = jt.jt_get_clique(h, 0, clique, n)
    main = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    jt.jt_propagate(h, 0, 1, main)                      # same evidence: rewrites the same table
    jt.jt_get_clique_noalloc(h, 0, clique, out, stream=side)
    jt.jt_set_evidence(h, 0, *synth.random_evidence(tp, 5, 999))
    jt.jt_propagate(h, 0, 1, main)                      # new evidence: a different table
    side.synchronize()
    assert marg_errors([out.cpu().numpy()], [ref1], "f32") <= TOL["f32"]
    ref2 = jt.jt_get_clique(h, 0, clique, n)
    assert np.max(np.abs(ref2 - ref1)) > 1e-6              # the second propagation did change it
    h.free()


def test_noalloc_allocates_no_device_memory(env):
    """After a first call (which looks up the scratch array's address),
    further read-outs change neither the device's free memory
    (cudaMemGetInfo) nor the memory torch has allocated."""
    jt, torch = env
    tp, h = _materialised(jt, synth.small_tree(), "f64", 1)
    n = int(tp.table_sizes()[5])
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    jt.jt_get_clique_noalloc(h, 0, 5, out, stream=stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for c in (5, 7, 5, 11):
        jt.jt_get_clique_noalloc(h, 0, c, out, stream=stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == alloc0
    h.free()
