"""Seeded synthetic inputs shaped like the workloads the method is measured on.

This module holds none of the method's arithmetic: it only draws points,
vectors and row samples.  The CUDA path's tests and benchmark and the oracle
both take their inputs from here, so the two sides see identical data.

Recipe (numpy PCG64 via default_rng, FP64 on the host):
  * points i.i.d. uniform in [0, 1)^3; targets seed 1, sources seed 2;
  * x complex with i.i.d. N(0, 1) real and imaginary parts, seed 3
    (drawn as an (N, 2) standard-normal array: column 0 real, column 1 imag);
  * sampled rows: distinct indices, seed 4, sorted ascending;
  * the tensor grid of Sect. 4: coordinates (2n - 1) 2^-k - 1, n = 1 .. 2^k,
    in [-1, 1]^3, 8^k points, x fastest.
"""
import numpy as np

SEED_TARGETS = 1
SEED_SOURCES = 2
SEED_X = 3
SEED_ROWS = 4

# Named workloads: point count, wave number, tree depth, Chebyshev order
# (nodes per axis), root cube [0, 1]^3, eta2 = 5, l_hf by the default rule.
# The "paper-grid" workloads are the setting of Sect. 4 / Table 1: the 8^k
# tensor grid in [-1, 1]^3 as targets and sources (P_S = P_T), kappa =
# 0.1 2^k, n_max = 512 (depth k - 3, 512 points per leaf), m = 4.
WORKLOADS = {
    "uniform-8k-k16-d4-o4": dict(n=8192, kappa=16.0, depth=4, order=4),
    "uniform-1M-k64-d6-o5": dict(n=1 << 20, kappa=64.0, depth=6, order=5),
    "uniform-4M-k128-d7-o6": dict(n=1 << 22, kappa=128.0, depth=7, order=6),
    "paper-grid-k6": dict(n=8 ** 6, kappa=6.4, depth=10, order=5, grid=6, n_max=512),
    "paper-grid-k7": dict(n=8 ** 7, kappa=12.8, depth=10, order=5, grid=7, n_max=512),
}


def uniform_points(n, seed):
    """n points i.i.d. uniform in [0, 1)^3, shape (n, 3), float64."""
    return np.random.default_rng(seed).random((int(n), 3))


def complex_normal(n, seed=SEED_X, nrhs=None):
    """Complex vector(s) with i.i.d. N(0,1) real and imaginary parts.

    nrhs=None: shape (n,).  Otherwise shape (nrhs, n): one row per right-hand
    side, drawn one after the other from the same generator.
    """
    rng = np.random.default_rng(seed)
    if nrhs is None:
        z = rng.standard_normal((int(n), 2))
        return z[:, 0] + 1j * z[:, 1]
    out = np.empty((int(nrhs), int(n)), dtype=np.complex128)
    for r in range(int(nrhs)):
        z = rng.standard_normal((int(n), 2))
        out[r] = z[:, 0] + 1j * z[:, 1]
    return out


def sample_rows(n, count, seed=SEED_ROWS):
    """`count` distinct row indices in [0, n), sorted ascending."""
    count = min(int(count), int(n))
    return np.sort(np.random.default_rng(seed).choice(int(n), count, replace=False)).astype(np.int64)


def tensor_grid(k):
    """The 8^k points of Sect. 4 in [-1, 1]^3 (x fastest)."""
    g = (2.0 * np.arange(1, 2 ** k + 1) - 1.0) * 2.0 ** (-k) - 1.0
    zz, yy, xx = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)


def workload(name):
    """(targets, sources, x, params) of a named workload; params also holds
    the root cube ("root": (lo, side)) and n_max."""
    w = dict(WORKLOADS[name])
    if "grid" in w:
        t = tensor_grid(w["grid"])
        s = t
        w["root"] = ((-1.0, -1.0, -1.0), 2.0)
    else:
        t = uniform_points(w["n"], SEED_TARGETS)
        s = uniform_points(w["n"], SEED_SOURCES)
        w["root"] = ((0.0, 0.0, 0.0), 1.0)
        w.setdefault("n_max", 0)
    x = complex_normal(w["n"], SEED_X)
    return t, s, x, w
