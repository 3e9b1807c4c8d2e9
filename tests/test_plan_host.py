"""The propagation planner on the host (no GPU): ``tests/plan_check.cpp``
links the library's planner (csrc/jt_plan.cpp), builds the schedules of a
tree for one case, 4- and 8-case blocks, and checks what the persistent
kernel relies on: every block of every stage is one work item per case
block, the dependencies are those of Algorithms 2-4, and no item waits for
a block queued after it.  Run on the workloads, on merged trees (high
fan-out), on trees with empty separators and on the separator sweep.  The
whole-tree plan (one CTA per case) must pack its level indices so that they
unpack to its arrays, and order every collect stage before its parent's.
Schedules planned with the block targets halved or doubled (the block-size
autotuner's search space) must satisfy the same invariants.

Trees with cardinalities other than powers of two also get the padded plan
(every cardinality raised to a power of two, the added states impossible):
its case-lane schedules are checked the same way, its evidence limits and
output rows must be the original tree's, every tile a stage marks for
skipping must hold only added-state entries, and every padded table entry,
decoded from its own digits, must map to the original entry with the same
digits, or be a hole exactly where a digit is an added state."""
import os
import shutil
import subprocess

import pytest

from paper_1202_3777_gb300 import synth
from paper_1202_3777_gb300.merge import merge_small_separators

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.isdir(CUDA_INC):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("plan") / "plan_check")
    csrc = os.path.join(ROOT, "paper_1202_3777_gb300", "csrc")
    cmd = ["g++", "-std=c++17", "-O2", "-I", csrc, "-I", os.path.join(ROOT, "include"), "-I", CUDA_INC,
           os.path.join(ROOT, "tests", "plan_check.cpp"), os.path.join(csrc, "jt_plan.cpp"), "-o", exe, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def _run(exe, card, cliques, parent, *extra):
    words = [len(card), *[int(x) for x in card], len(cliques)]
    for c in cliques:
        words += [len(c), *[int(v) for v in c]]
    words += [int(x) for x in parent]
    r = subprocess.run([exe, *extra], input=" ".join(map(str, words)), capture_output=True, text=True)
    return r.returncode, r.stdout.strip().splitlines()


TREES = {
    "small": lambda: synth.small_tree(),
    "large-clique": lambda: synth.large_clique_tree(),
    "high-card": lambda: synth.high_card_tree(),
    "batched": lambda: synth.batched_tree(),
    "binary-serving": lambda: synth.binary_serving_tree(),
    "sep-sweep-4^1": lambda: synth.separator_sweep_tree(1, k=8),
    "sep-sweep-4^7": lambda: synth.separator_sweep_tree(7, k=8),
    "empty-separators": lambda: synth.random_small_tree(7, n_cliques=9, allow_empty_sep=True, max_states=1 << 40),
}


# trees whose cliques all have power-of-two cardinalities and >= 32 entries:
# the case-lane schedule (32 cases per work item) must plan them
CASE_LANE_TREES = {"large-clique", "high-card", "sep-sweep-4^1", "sep-sweep-4^7"}
# trees with other cardinalities whose padded plan the case lanes must plan
PADDED_TREES = {"small", "batched"}
# trees the whole-tree schedule (one CTA per case) must plan
WHOLE_TREE_TREES = {"small", "binary-serving", "empty-separators"}


def _pow2(t):
    return all(int(c) & (int(c) - 1) == 0 for c in t.card)


@pytest.mark.parametrize("name", list(TREES))
def test_schedules_of_the_workloads(checker, name):
    t = TREES[name]()
    rc, lines = _run(checker, t.card, t.cliques, t.parent)
    assert rc == 0, lines
    base = [ln for ln in lines if ln.startswith("cb=")]
    assert len(base) == 6, lines
    for ln in base:
        if ln.startswith("cb=32 ") and name not in CASE_LANE_TREES:
            assert " OK " in ln or " UNSUPPORTED " in ln, ln
        else:
            assert " OK " in ln, ln
    tune = [ln for ln in lines if ln.startswith("tune ")]
    assert tune and all(" OK " in ln for ln in tune), lines
    small = [ln for ln in lines if ln.startswith("small ")]
    assert len(small) == 1 and (" OK " in small[0] or (name not in WHOLE_TREE_TREES and " UNSUPPORTED " in small[0])), \
        lines
    pad = [ln for ln in lines if ln.startswith("pad")]
    if _pow2(t):
        assert not pad, lines
    else:
        assert len(pad) == 3 and pad[-1].startswith("padmap OK"), lines
        for ln in pad[:2]:
            assert " OK " in ln or (name not in PADDED_TREES and " UNSUPPORTED " in ln), ln


def test_planted_hole_tile_mistake_is_caught(checker):
    """A stage's first added-state digit given one state too few: tiles at
    the digit's last real state are then marked as holes, and hold entries
    that are not."""
    t = synth.small_tree()
    rc, lines = _run(checker, t.card, t.cliques, t.parent, "plant-holes")
    assert rc == 1 and any(ln.startswith("pad cb=32") and "marked as holes" in ln for ln in lines), lines


def test_planted_padding_mistake_is_caught(checker):
    """Two digits' strides swapped in the padding map: some padded entry then
    maps to an original entry with other digits."""
    t = synth.small_tree()
    rc, lines = _run(checker, t.card, t.cliques, t.parent, "plant-pad")
    assert rc == 1 and any(ln.startswith("padmap FAIL") for ln in lines), lines


def test_planted_chunk_key_mistake_is_caught(checker):
    """Every one-case port of the large-clique tree claimed to keep its key
    over the iterations of a chunk: the consumers would then gather and
    reduce a thread's four vectors under one key, and the check must see a
    port whose key changes inside a chunk."""
    t = synth.large_clique_tree()
    rc, lines = _run(checker, t.card, t.cliques, t.parent, "plant-inchunk")
    one = [ln for ln in lines if ln.startswith("cb=1 ")]
    assert rc == 1 and one and all("varies inside a chunk" in ln for ln in one), lines


@pytest.mark.parametrize("min_sep,cap", [(8, 1 << 8), (16, 1 << 10), (1 << 20, 1 << 12)])
def test_schedules_of_merged_trees(checker, min_sep, cap):
    t = synth.binary_serving_tree()
    m = merge_small_separators(t.card, t.cliques, t.parent, min_sep, cap)
    rc, lines = _run(checker, t.card, m.cliques, m.parent)
    assert rc == 0, lines
    for ln in lines:
        assert " OK " in ln or ((ln.startswith("cb=32 ") or ln.startswith("small ")) and " UNSUPPORTED " in ln), ln


@pytest.mark.parametrize("plant,what", [("plant-order", "queued after"), ("plant-repeat", "block")])
def test_planted_schedule_mistakes_are_caught(checker, plant, what):
    t = synth.small_tree()
    rc, lines = _run(checker, t.card, t.cliques, t.parent, plant)
    planned = [ln for ln in lines if " UNSUPPORTED " not in ln and not ln.startswith(("padmap", "small ", "tune "))]
    assert rc == 1 and len(planned) >= 4 and all(" FAIL " in ln and what in ln for ln in planned), lines

