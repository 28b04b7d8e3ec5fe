"""Shared helpers for the GPU parity tests: build the CUDA-path problem and
its oracle twin from the same seeded workload description."""
import numpy as np

import synth
from oracle import stokes


def problem_spec(dim, p, n_el, disc="TH"):
    n = (n_el,) * dim if np.isscalar(n_el) else tuple(n_el)
    return dict(dim=dim, p=p, n_el=n, disc=disc)


def knots_of(spec):
    return [synth.open_uniform_knots(n, spec["p"]) for n in spec["n_el"]]


def oracle_problem(spec, nu=1.0):
    return stokes.build(knots_of(spec), spec["p"], spec["disc"], nu=nu)


def gpu_problem(spec, **kw):
    import paper_1712_00403_gb300 as fd
    disc = fd.TH if spec["disc"] == "TH" else fd.RT
    return fd.Stokes(knots_of(spec), spec["p"], disc=disc, **kw)


def max_rel(a, b):
    """Element-wise relative error of a against b: max |a - b| / max |b|,
    so that every entry, not only the norm, is held to the bar."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return float(np.abs(a - b).max() / np.abs(b).max())
