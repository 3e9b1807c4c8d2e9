"""ctypes binding of libjt (include/jt.h): the same entry points, with numpy
arrays marshalled to plain pointers.  No arithmetic of the method happens
here; every step of a propagation runs in the library's CUDA kernels.

Importing this module loads ``_build/libjt.so`` and raises if it is missing
(build it with ``python -m paper_1202_3777_gb300.build`` or
``__graft_entry__.build()``); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from .build import LIB

if not os.path.exists(LIB):
    raise ImportError(f"libjt.so not built ({LIB}); run paper_1202_3777_gb300.build.build()")
_lib = C.CDLL(LIB)

# status codes (jt_status)
JT_OK = 0
JT_ERR_INVALID_ARG = 1
JT_ERR_NOT_A_JUNCTION_TREE = 2
JT_ERR_OOM = 3
JT_ERR_ZERO_EVIDENCE = 4
JT_ERR_TIMEOUT = 5
JT_ERR_CUDA = 6
JT_ERR_STATE = 7
JT_ERR_UNSUPPORTED = 8
JT_F32 = 0
JT_F64 = 1
JT_MATERIALIZE_CLIQUES = 0x1


class JtError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.jt_strerror(status).decode()
        detail = _lib.jt_last_error().decode()
        super().__init__(f"{where}: {msg} ({detail})" if detail else f"{where}: {msg}")


class jt_tree_desc(C.Structure):
    _fields_ = [
        ("n_vars", C.c_int32),
        ("card", C.POINTER(C.c_int32)),
        ("n_cliques", C.c_int32),
        ("clique_off", C.POINTER(C.c_int64)),
        ("clique_vars", C.POINTER(C.c_int32)),
        ("parent", C.POINTER(C.c_int32)),
        ("potentials", C.c_void_p),
        ("potentials_dtype", C.c_int),
        ("compute", C.c_int),
        ("max_cases", C.c_int32),
        ("flags", C.c_uint32),
    ]


class jt_tree_info(C.Structure):
    _fields_ = [
        ("n_vars", C.c_int32), ("n_cliques", C.c_int32), ("depth", C.c_int32),
        ("entries", C.c_int64), ("work_per_case", C.c_int64), ("marginal_len", C.c_int64),
        ("device_bytes", C.c_int64), ("case_bytes", C.c_int64), ("max_cases", C.c_int32), ("compute", C.c_int),
        ("flags", C.c_uint32),
    ]


class jt_schedule_info(C.Structure):
    _fields_ = [
        ("case_block", C.c_int32), ("n_items", C.c_int32), ("grid", C.c_int32), ("smem_bytes", C.c_int32),
        ("window_entries", C.c_int32), ("padded", C.c_int32), ("block_shift", C.c_int8 * 4),
        ("reserved", C.c_int32),
        ("candidate_ms", C.c_float * 5),
    ]


class jt_cpt_desc(C.Structure):
    _fields_ = [
        ("n_cpts", C.c_int32),
        ("fam_off", C.POINTER(C.c_int32)),
        ("fam_vars", C.POINTER(C.c_int32)),
        ("values", C.POINTER(C.c_double)),
        ("home", C.POINTER(C.c_int32)),
    ]


_vp = C.c_void_p
_i32 = C.c_int32
_sig = {
    "jt_load_tree": (C.c_int, [C.POINTER(jt_tree_desc), _vp, C.POINTER(_vp)]),
    "jt_set_evidence": (C.c_int, [_vp, _i32, _i32, _vp, _vp]),
    "jt_set_evidence_dense": (C.c_int, [_vp, _i32, _i32, _vp, _i32, _vp]),
    "jt_propagate": (C.c_int, [_vp, _i32, _i32, _vp]),
    "jt_profile_propagate": (C.c_int, [_vp, _i32, _i32, _vp, _vp, _i32, C.POINTER(_i32)]),
    "jt_get_marginal": (C.c_int, [_vp, _i32, _i32, _vp]),
    "jt_log_evidence": (C.c_int, [_vp, _i32, _vp]),
    "jt_get_marginals": (C.c_int, [_vp, _i32, _i32, _vp, _i32, _vp]),
    "jt_get_log_evidence": (C.c_int, [_vp, _i32, _i32, _vp, _i32, _vp]),
    "jt_get_status": (C.c_int, [_vp, _i32, _i32, _vp]),
    "jt_get_clique": (C.c_int, [_vp, _i32, _i32, _vp]),
    "jt_get_clique_noalloc": (C.c_int, [_vp, _i32, _i32, _vp, _vp]),
    "jt_propagate_per_message": (C.c_int, [_vp, _i32, _i32, _vp, C.POINTER(C.c_float)]),
    "jt_init_from_cpts": (C.c_int, [_vp, C.POINTER(jt_cpt_desc), _vp, C.POINTER(C.c_float)]),
    "jt_get_potential": (C.c_int, [_vp, _i32, _vp]),
    "jt_get_info": (C.c_int, [_vp, C.POINTER(jt_tree_info)]),
    "jt_get_schedule": (C.c_int, [_vp, _i32, _i32, C.POINTER(jt_schedule_info)]),
    "jt_propagate_ctas": (C.c_int, [_vp, _i32, _i32, _i32, _vp]),
    "jt_get_kernel_span": (C.c_int, [_vp, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    "jt_free": (None, [_vp]),
    "jt_strerror": (C.c_char_p, [C.c_int]),
    "jt_last_error": (C.c_char_p, []),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def exported_symbols():
    """Names bound from the library (all must resolve)."""
    return sorted(_sig)


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(st: int, where: str, ok=(JT_OK,)):
    if st not in ok:
        raise JtError(st, where)
    return st


def _stream(stream) -> Optional[int]:
    """Accept None, an int handle, or an object with ``cuda_stream``
    (a torch.cuda.Stream)."""
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Tree:
    """A loaded tree (handle owner).  Methods are the C entry points."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep
        info = jt_tree_info()
        _check(_lib.jt_get_info(handle, C.byref(info)), "jt_get_info")
        self.info = info
        self.n_vars = info.n_vars
        self.marginal_len = info.marginal_len

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "handle", None):
            _lib.jt_free(self.handle)
            self.handle = None


def jt_load_tree(card, cliques, parent, potentials, compute: int = JT_F32, max_cases: int = 1,
                 flags: int = 0, stream=None) -> Tree:
    """Load a tree given as numpy arrays / lists: ``card`` [n_vars],
    ``cliques`` (list of variable arrays, table order), ``parent`` [n]
    (parent[0] = -1), ``potentials`` (concatenated tables, float64 or
    float32; None: every table starts at one, for jt_init_from_cpts)."""
    card = np.ascontiguousarray(card, dtype=np.int32)
    cl = [np.asarray(c, dtype=np.int32) for c in cliques]
    off = np.concatenate([[0], np.cumsum([len(c) for c in cl])]).astype(np.int64)
    flat = np.ascontiguousarray(np.concatenate(cl) if cl else np.zeros(0, np.int32), dtype=np.int32)
    par = np.ascontiguousarray(parent, dtype=np.int32)
    if potentials is None:
        pot = None
    else:
        pot = np.ascontiguousarray(potentials)
    if pot is not None and all(0 <= int(v) < len(card) for c in cl for v in c) and len(cl) and max(len(c) for c in cl) <= 32:
        need = sum(int(np.prod([int(card[v]) for v in c], dtype=np.float64)) for c in cl)
        if pot.size < need:
            raise ValueError(f"potentials hold {pot.size} entries, the tables need {need}")
    if pot is None:
        pdt = JT_F64
    elif pot.dtype == np.float32:
        pdt = JT_F32
    else:
        pot = np.ascontiguousarray(pot, dtype=np.float64)
        pdt = JT_F64
    d = jt_tree_desc(len(card), card.ctypes.data_as(C.POINTER(C.c_int32)), len(cl),
                     off.ctypes.data_as(C.POINTER(C.c_int64)), flat.ctypes.data_as(C.POINTER(C.c_int32)),
                     par.ctypes.data_as(C.POINTER(C.c_int32)), None if pot is None else pot.ctypes.data_as(C.c_void_p), pdt,
                     compute, max_cases, flags)
    h = C.c_void_p()
    _check(_lib.jt_load_tree(C.byref(d), _stream(stream), C.byref(h)), "jt_load_tree")
    return Tree(h, None)


def jt_load_synth(tree, compute: int = JT_F32, max_cases: int = 1, flags: int = 0, stream=None) -> Tree:
    """Load a ``synth.Tree``."""
    return jt_load_tree(tree.card, tree.cliques, tree.parent, tree.pot, compute, max_cases, flags, stream)


def jt_set_evidence(t: Tree, case_id: int, vars_, states):
    v = np.ascontiguousarray(vars_, dtype=np.int32)
    s = np.ascontiguousarray(states, dtype=np.int32)
    if v.shape != s.shape:
        raise ValueError("vars and states differ in length")
    _check(_lib.jt_set_evidence(t.handle, case_id, len(v), _ptr(v), _ptr(s)), "jt_set_evidence")


def jt_set_evidence_dense(t: Tree, first_case: int, states, stream=None):
    """``states``: int16 [n_cases, n_vars] numpy array (host), or a torch
    int16 CUDA tensor (device)."""
    if hasattr(states, "data_ptr") and getattr(states, "is_cuda", False):
        n = int(states.shape[0])
        _check(_lib.jt_set_evidence_dense(t.handle, first_case, n, C.c_void_p(states.data_ptr()), 1,
                                          _stream(stream)), "jt_set_evidence_dense")
        return
    a = np.ascontiguousarray(states, dtype=np.int16)
    _check(_lib.jt_set_evidence_dense(t.handle, first_case, a.shape[0], _ptr(a), 0, _stream(stream)),
           "jt_set_evidence_dense")


def jt_propagate(t: Tree, first_case: int = 0, n_cases: int = 1, stream=None):
    _check(_lib.jt_propagate(t.handle, first_case, n_cases, _stream(stream)), "jt_propagate")


def jt_profile_propagate(t: Tree, first_case: int = 0, n_cases: int = 1, stream=None) -> np.ndarray:
    """Device times (ms) of one propagation: [propagation kernel,
    finalisation]."""
    n = C.c_int32(0)
    buf = np.zeros(2, dtype=np.float32)
    _check(_lib.jt_profile_propagate(t.handle, first_case, n_cases, _stream(stream), _ptr(buf), len(buf),
                                     C.byref(n)), "jt_profile_propagate")
    return buf[:n.value]


def jt_get_marginal(t: Tree, case_id: int, var: int, card: int) -> np.ndarray:
    out = np.empty(card, dtype=np.float64)
    _check(_lib.jt_get_marginal(t.handle, case_id, var, _ptr(out)), "jt_get_marginal")
    return out


def jt_log_evidence(t: Tree, case_id: int = 0) -> float:
    out = np.zeros(1, dtype=np.float64)
    st = _lib.jt_log_evidence(t.handle, case_id, _ptr(out))
    _check(st, "jt_log_evidence", ok=(JT_OK, JT_ERR_ZERO_EVIDENCE))
    return float(out[0])


def jt_get_marginals(t: Tree, first_case: int, n_cases: int, out=None, stream=None):
    """Host: returns float64 [n_cases, marginal_len].  Device: pass a torch
    float64 CUDA tensor as ``out``; the copy is only enqueued."""
    if out is not None and hasattr(out, "data_ptr") and getattr(out, "is_cuda", False):
        _check(_lib.jt_get_marginals(t.handle, first_case, n_cases, C.c_void_p(out.data_ptr()), 1,
                                     _stream(stream)), "jt_get_marginals")
        return out
    res = np.empty((n_cases, t.marginal_len), dtype=np.float64)
    _check(_lib.jt_get_marginals(t.handle, first_case, n_cases, _ptr(res), 0, _stream(stream)),
           "jt_get_marginals")
    return res


def jt_get_log_evidence(t: Tree, first_case: int, n_cases: int, out=None, stream=None):
    if out is not None and hasattr(out, "data_ptr") and getattr(out, "is_cuda", False):
        _check(_lib.jt_get_log_evidence(t.handle, first_case, n_cases, C.c_void_p(out.data_ptr()), 1,
                                        _stream(stream)), "jt_get_log_evidence")
        return out
    res = np.empty(n_cases, dtype=np.float64)
    _check(_lib.jt_get_log_evidence(t.handle, first_case, n_cases, _ptr(res), 0, _stream(stream)),
           "jt_get_log_evidence")
    return res


def jt_get_status(t: Tree, first_case: int, n_cases: int) -> np.ndarray:
    res = np.empty(n_cases, dtype=np.int32)
    _check(_lib.jt_get_status(t.handle, first_case, n_cases, _ptr(res)), "jt_get_status")
    return res


def jt_get_clique(t: Tree, case_id: int, clique: int, size: int) -> np.ndarray:
    out = np.empty(size, dtype=np.float64)
    _check(_lib.jt_get_clique(t.handle, case_id, clique, _ptr(out)), "jt_get_clique")
    return out


def jt_get_clique_noalloc(t: Tree, case_id: int, clique: int, out, stream=None):
    """Allocation-free read-out into ``out``, a torch float64 CUDA tensor of
    the clique's size (enqueued only)."""
    _check(_lib.jt_get_clique_noalloc(t.handle, case_id, clique, C.c_void_p(out.data_ptr()), _stream(stream)),
           "jt_get_clique_noalloc")
    return out


def jt_propagate_per_message(t: Tree, case_id: int, layout: int = 1, stream=None) -> float:
    """The paper's per-message propagation (Algorithm 1 with index-mapping
    tables, layout 0 naive / 1 interleaved) for one case; returns its device
    time in ms (the tree needs JT_MATERIALIZE_CLIQUES)."""
    ms = C.c_float(0.0)
    _check(_lib.jt_propagate_per_message(t.handle, case_id, layout, _stream(stream), C.byref(ms)),
           "jt_propagate_per_message")
    return float(ms.value)


def jt_init_from_cpts(t: Tree, families, tables, home=None, stream=None) -> float:
    """Overwrite the tree's clique tables with the product of the CPTs homed
    in each (Algorithm 4's initialisation, on the device).  ``families[i]``
    lists CPT i's variables in its table order, ``tables[i]`` is that table
    (flattened), ``home`` optionally names each CPT's clique.  Returns the
    device time of the initialisation kernel in ms."""
    fams = [np.ascontiguousarray(f, dtype=np.int32) for f in families]
    off = np.concatenate([[0], np.cumsum([len(f) for f in fams])]).astype(np.int32)
    flat = np.ascontiguousarray(np.concatenate(fams) if fams else np.zeros(0, np.int32), dtype=np.int32)
    vals = np.ascontiguousarray(np.concatenate([np.ravel(x) for x in tables]) if len(tables) else np.zeros(0),
                                dtype=np.float64)
    hm = None if home is None else np.ascontiguousarray(home, dtype=np.int32)
    d = jt_cpt_desc(len(fams), off.ctypes.data_as(C.POINTER(C.c_int32)), flat.ctypes.data_as(C.POINTER(C.c_int32)),
                    vals.ctypes.data_as(C.POINTER(C.c_double)),
                    None if hm is None else hm.ctypes.data_as(C.POINTER(C.c_int32)))
    ms = C.c_float(0.0)
    _check(_lib.jt_init_from_cpts(t.handle, C.byref(d), _stream(stream), C.byref(ms)), "jt_init_from_cpts")
    return float(ms.value)


def jt_get_potential(t: Tree, clique: int, size: int) -> np.ndarray:
    """Resident (uncalibrated) table of ``clique`` in its listed order."""
    out = np.empty(size, dtype=np.float64)
    _check(_lib.jt_get_potential(t.handle, clique, _ptr(out)), "jt_get_potential")
    return out


def jt_get_schedule(t: Tree, first_case: int, n_cases: int) -> dict:
    """The schedule the case range's propagations use (after its first
    jt_propagate): cases per work item, work items, grid, shared memory."""
    info = jt_schedule_info()
    _check(_lib.jt_get_schedule(t.handle, first_case, n_cases, C.byref(info)), "jt_get_schedule")
    return {"case_block": info.case_block, "n_items": info.n_items, "grid": info.grid,
            "smem_bytes": info.smem_bytes, "window_entries": info.window_entries, "padded": bool(info.padded),
            "block_shift": [int(x) for x in info.block_shift[:3]],
            "candidate_ms": {w: float(info.candidate_ms[i]) for i, w in enumerate((32, 8, 4, 1, 0))
                             if info.candidate_ms[i] >= 0}}


def jt_propagate_ctas(t: Tree, first_case: int, n_cases: int, max_ctas: int, stream=None):
    """jt_propagate holding at most max_ctas SMs (0: all), so propagations of
    several trees on their own streams can run side by side."""
    _check(_lib.jt_propagate_ctas(t.handle, first_case, n_cases, max_ctas, _stream(stream)), "jt_propagate_ctas")


def jt_get_kernel_span(t: Tree):
    """(start_ns, end_ns) of the tree's last propagation kernel on the GPU's
    global timer."""
    a, b = C.c_uint64(), C.c_uint64()
    _check(_lib.jt_get_kernel_span(t.handle, C.byref(a), C.byref(b)), "jt_get_kernel_span")
    return int(a.value), int(b.value)


def jt_free(t: Tree):
    t.free()


def jt_strerror(status: int) -> str:
    return _lib.jt_strerror(status).decode()


def jt_last_error() -> str:
    return _lib.jt_last_error().decode()


def raw_load_status(card, cliques, parent, potentials, compute=JT_F32, max_cases=1, flags=0):
    """Status code of jt_load_tree without raising (for validation tests);
    frees the tree if it loaded."""
    try:
        t = jt_load_tree(card, cliques, parent, potentials, compute, max_cases, flags)
    except JtError as e:
        return e.status
    t.free()
    return JT_OK
