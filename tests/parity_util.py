"""Shared helpers for the GPU parity tests: run a case through the C ABI
and compare with the FP64 oracle using the tolerance the method states
(max relative error 1e-5 on normalised marginals in FP32, 1e-12 in FP64)."""
import numpy as np

TOL = {"f32": 1e-5, "f64": 1e-12}
FLOOR = {"f32": 1e-30, "f64": 1e-290}


def marg_errors(gpu, ref, prec):
    """Max relative error over entries >= floor; entries the oracle makes
    exactly zero (excluded by evidence) must be exactly zero; entries below
    the floor need absolute error <= floor."""
    floor = FLOOR[prec]
    worst = 0.0
    for g, o in zip(gpu, ref):
        g = np.asarray(g, float)
        o = np.asarray(o, float)
        assert g.shape == o.shape
        assert np.all(np.isfinite(g)), "non-finite marginal"
        zero = o == 0.0
        assert np.all(g[zero] == 0.0), "evidence-excluded state is not exactly zero"
        big = o >= floor
        if big.any():
            worst = max(worst, float(np.max(np.abs(g[big] - o[big]) / o[big])))
        small = ~big & ~zero
        if small.any():
            assert float(np.max(np.abs(g[small] - o[small]))) <= floor
    return worst


def split_marginals(flat, card):
    out, o = [], 0
    for k in card:
        out.append(flat[o:o + int(k)])
        o += int(k)
    return out


def logz_ok(g, o, prec):
    return abs(g - o) <= TOL[prec] * max(1.0, abs(o))
