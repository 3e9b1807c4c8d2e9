"""The C-ABI library loads, exports every entry point declared in
include/jt.h, and rejects malformed trees before touching the GPU
(validation runs on the host).  CPU only: no compute call is made."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def jt():
    from paper_1202_3777_gb300 import build
    build.build()
    from paper_1202_3777_gb300 import jt as mod
    return mod


def _declared():
    src = open(os.path.join(ROOT, "include", "jt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(jt_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(jt):
    declared = _declared()
    assert "jt_load_tree" in declared and "jt_propagate" in declared
    for name in declared:
        assert hasattr(jt._lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", jt.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (jt_[a-z_]+)", out))
    assert set(declared) <= exported
    assert set(jt.exported_symbols()) <= set(declared)


def test_strerror(jt):
    assert jt.jt_strerror(jt.JT_OK) == "ok"
    assert "junction" in jt.jt_strerror(jt.JT_ERR_NOT_A_JUNCTION_TREE)
    assert jt.jt_strerror(99) == "unknown status"


def _tiny():
    card = [2, 3, 2]
    cliques = [[0, 1], [1, 2]]
    parent = [-1, 0]
    pot = np.full(6 + 6, 0.5)
    return card, cliques, parent, pot


@pytest.mark.parametrize("mutate,code", [
    (lambda c, q, p, x: (c, [[0, 1], [1, 2], [0, 2]], [-1, 0, 1], np.full(16, .5)), "NOT_A_JUNCTION_TREE"),
    (lambda c, q, p, x: (c, [[0, 1], [1, 2], [2]], [-1, 2, 1], np.full(14, .5)), "NOT_A_JUNCTION_TREE"),
    (lambda c, q, p, x: (c, [[0, 0], [1, 2]], p, np.full(10, .5)), "NOT_A_JUNCTION_TREE"),
    (lambda c, q, p, x: (c, q, [1, -1], x), "NOT_A_JUNCTION_TREE"),
    (lambda c, q, p, x: ([2, 3, 2, 2], q, p, x), "NOT_A_JUNCTION_TREE"),     # variable in no clique
    (lambda c, q, p, x: ([1, 3, 2], q, p, np.full(9, .5)), "INVALID_ARG"),    # card < 2
    (lambda c, q, p, x: (c, [[0, 1], [1, 5]], p, x), "INVALID_ARG"),          # bad var id
    (lambda c, q, p, x: (c, q, p, np.concatenate([x[:-1], [-1.0]])), "INVALID_ARG"),
    (lambda c, q, p, x: (c, q, p, np.concatenate([x[:-1], [np.nan]])), "INVALID_ARG"),
    (lambda c, q, p, x: (c, q, p, np.concatenate([x[:-1], [np.inf]])), "INVALID_ARG"),
    (lambda c, q, p, x: ([2] * 40, [list(range(40))], [-1], np.zeros(1)), "UNSUPPORTED"),
])
def test_validation_errors(jt, mutate, code):
    args = mutate(*_tiny())
    assert jt.raw_load_status(*args) == getattr(jt, "JT_ERR_" + code)
    assert jt.jt_last_error() != ""


def test_bad_descriptor_fields(jt):
    c, q, p, x = _tiny()
    assert jt.raw_load_status(c, q, p, x, max_cases=0) == jt.JT_ERR_INVALID_ARG
    assert jt.raw_load_status(c, q, p, x, flags=0x80) == jt.JT_ERR_INVALID_ARG
    assert jt.raw_load_status(c, q, p, x, compute=7) == jt.JT_ERR_INVALID_ARG


def test_tree_without_tables_is_still_validated(jt):
    """potentials = NULL (tables start at one, for jt_init_from_cpts) skips
    only the value checks: the structure is validated before any device
    work."""
    c, q, p, x = _tiny()
    assert jt.raw_load_status(c, [[0, 1], [1, 2], [0, 2]], [-1, 0, 1], None) == jt.JT_ERR_NOT_A_JUNCTION_TREE
    assert jt.raw_load_status([1, 3, 2], q, p, None) == jt.JT_ERR_INVALID_ARG


def test_initialisation_entry_points_reject_a_null_tree(jt):
    import ctypes as C
    d = jt.jt_cpt_desc(0, None, None, None, None)
    assert jt._lib.jt_init_from_cpts(None, C.byref(d), None, None) == jt.JT_ERR_INVALID_ARG
    out = np.zeros(4)
    assert jt._lib.jt_get_potential(None, 0, out.ctypes.data_as(C.c_void_p)) == jt.JT_ERR_INVALID_ARG


def test_plain_c_program_links_and_runs(jt, tmp_path):
    """The header is C99 (no C++ in the ABI): a C program that takes the
    address of every declared entry point compiles with warnings as errors,
    links against libjt.so and runs the calls that need no GPU."""
    import shutil
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    src = os.path.join(ROOT, "tests", "abi_consumer.c")
    body = open(src).read()
    for name in _declared():
        assert f"(any_fn){name}," in body or f"(any_fn){name}\n" in body, name
    libdir = os.path.dirname(jt.LIB)
    exe = str(tmp_path / "abi_consumer")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), src,
           "-o", exe, "-L", libdir, "-ljt", f"-Wl,-rpath,{libdir}", "-Wl,--allow-shlib-undefined"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert r.stdout.startswith("c-abi ok")
