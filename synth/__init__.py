"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

Holds workload definitions (sizes, degrees, seeds) and random draws only; none
of the method's arithmetic lives here. Knot vectors are inputs of the setup
call: open, uniform, interior multiplicity p - alpha with alpha = p - 1.
"""
import numpy as np

# Named workloads. "n_el" is per direction; p = pressure degree.
WORKLOADS = {
    # 2D unit square, Taylor-Hood, p=2, 16x16 elements, FP64 FD, MINRES 1e-8, seed 1
    "square_th_p2_16": dict(dim=2, disc="TH", p=2, n_el=(16, 16), seeds=[1]),
    # 3D unit cube, Taylor-Hood, p=3, 64^3 elements, 16 right-hand sides, seeds 200..215
    "cube_th_p3_64": dict(dim=3, disc="TH", p=3, n_el=(64, 64, 64), seeds=list(range(200, 216))),
    # 3D unit cube, Taylor-Hood, p=3, 40^3 elements, 16 right-hand sides (profiling-sized case:
    # 1,673,830 DoF, 214 MB per 16-vector block, larger than L2)
    "cube_th_p3_40": dict(dim=3, disc="TH", p=3, n_el=(40, 40, 40), seeds=list(range(200, 216))),
    # 3D mapped cube (sine bump map, variable viscosity), p=3, 32^3 elements, seeds 300..303
    "mapped_th_p3_32": dict(dim=3, disc="TH", p=3, n_el=(32, 32, 32), seeds=list(range(300, 304)),
                            geometry="sine_bump"),
    # the mapped cube at 16^3 elements (profiling-sized: about 1.8e8 nonzeros, a few GB on the device)
    "mapped_th_p3_16": dict(dim=3, disc="TH", p=3, n_el=(16, 16, 16), seeds=list(range(300, 304)),
                            geometry="sine_bump"),
    # the same mapped cube at 64^3 elements (6,740,830 DoF, 32.8 M quadrature points): sized for the
    # matrix-free operator (its CSR would hold about 1.1e10 nonzeros)
    "mapped_th_p3_64": dict(dim=3, disc="TH", p=3, n_el=(64, 64, 64), seeds=list(range(300, 304)),
                            geometry="sine_bump"),
    # the eighth of a thick annulus (radii 1 and 2, height 1, nu = 1) in polar form, p=3, 32^3 elements
    "annulus_th_p3_32": dict(dim=3, disc="TH", p=3, n_el=(32, 32, 32), seeds=list(range(300, 304)),
                             geometry="annulus"),
    # 64 independent unit-cube TH instances, p ~ U{2..6}, elements per direction ~ U{16..96}
    # (instance draw seed 400, right-hand side seeds 401..464)
    "batched_64": dict(kind="batched", count=64, seed=400, rhs_seed0=401),
    # Poisson arrivals of mixed requests (see serving_requests)
    "serving": dict(kind="serving", rates=[50, 200, 1000, 2000], per_rate=48, seed=500, mix_seed=550),
}


def open_uniform_knots(n_el, p, alpha=None):
    """[0]*(p+1), interior j/n_el repeated (p - alpha) times, [1]*(p+1)."""
    alpha = p - 1 if alpha is None else alpha
    mult = p - alpha
    knots = [0.0] * (p + 1)
    for j in range(1, n_el):
        knots += [j / n_el] * mult
    knots += [1.0] * (p + 1)
    return np.array(knots, dtype=np.float64)


def knots_for(workload):
    w = WORKLOADS[workload] if isinstance(workload, str) else workload
    return [open_uniform_knots(n, w["p"]) for n in w["n_el"]]


def rhs(seed, block_sizes):
    """Right-hand side i.i.d. N(0,1) from numpy.random.default_rng(seed); the
    last (pressure) block has its arithmetic mean removed so that the
    right-hand side is orthogonal to the constant-pressure kernel."""
    rng = np.random.default_rng(seed)
    b = rng.standard_normal(int(sum(block_sizes)))
    npres = block_sizes[-1]
    b[-npres:] -= b[-npres:].mean()
    return b


def random_vector(seed, n):
    return np.random.default_rng(seed).standard_normal(n)


def batched_instances(seed=400, count=64, p_range=(2, 6), nel_range=(16, 96)):
    """Independent unit-cube Taylor-Hood instances: p ~ U{2..6}, elements per
    direction ~ U{16..96} independently per direction."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        p = int(rng.integers(p_range[0], p_range[1] + 1))
        n_el = tuple(int(v) for v in rng.integers(nel_range[0], nel_range[1] + 1, size=3))
        out.append(dict(dim=3, disc="TH", p=p, n_el=n_el))
    return out


def serving_requests(rate_index, rate, count, seed=500, mix_seed=550, nel3=(16, 96)):
    """Poisson arrival times (rate per second, stream seeded seed + rate_index) and a
    50/50 mix of 3D Taylor-Hood instances (p ~ U{2..6}, elements per direction ~
    U{nel3}) and 2D instances (Taylor-Hood or Raviart-Thomas with equal odds,
    p ~ U{2..8}, elements per direction ~ U{32..256}); instance draws from the
    stream seeded mix_seed + rate_index."""
    rng_t = np.random.default_rng(seed + rate_index)
    t = np.cumsum(rng_t.exponential(1.0 / rate, size=count))
    rng = np.random.default_rng(mix_seed + rate_index)
    out = []
    for k in range(count):
        if rng.random() < 0.5:
            p = int(rng.integers(2, 7))
            n_el = tuple(int(v) for v in rng.integers(nel3[0], nel3[1] + 1, size=3))
            out.append(dict(t=float(t[k]), dim=3, disc="TH", p=p, n_el=n_el, seed=int(rng.integers(1 << 30))))
        else:
            p = int(rng.integers(2, 9))
            n_el = tuple(int(v) for v in rng.integers(32, 257, size=2))
            disc = "TH" if rng.random() < 0.5 else "RT"
            out.append(dict(t=float(t[k]), dim=2, disc=disc, p=p, n_el=n_el, seed=int(rng.integers(1 << 30))))
    return out
