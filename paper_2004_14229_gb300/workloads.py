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
    in [-1, 1]^3, 8^k points, x fastest;
  * batches of independent problems (batch_problems): problem i draws from
    default_rng(100 + i), in order, N log-uniform in [N_lo, N_hi] (rounded),
    kappa log-uniform in [k_lo, k_hi], targets, sources, then nrhs complex
    vectors (as complex_normal); the distribution cycles uniform in [0,1)^3,
    Gaussian about (0.5)^3 with sigma 0.15 (redrawn until inside [0,1)^3),
    and a shell about (0.5)^3 with uniform direction and radius
    volume-uniform in [0.45, 0.5].  Tree depth: ceil(log8(N / 64)), at least
    1, the depth at which Alg. 1 with n_max = 64 stops on uniform points.
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
    "uniform-256k-k64-d5-o6": dict(n=1 << 18, kappa=64.0, depth=5, order=6),
    "paper-grid-k6": dict(n=8 ** 6, kappa=6.4, depth=10, order=5, grid=6, n_max=512),
    "paper-grid-k7": dict(n=8 ** 7, kappa=12.8, depth=10, order=5, grid=7, n_max=512),
    "paper-grid-k8": dict(n=8 ** 8, kappa=25.6, depth=10, order=5, grid=8, n_max=512),
    "paper-grid-k9": dict(n=8 ** 9, kappa=51.2, depth=10, order=5, grid=9, n_max=512),
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


SEED_BATCH = 100
BATCH_KINDS = ("uniform", "gaussian", "shell")


def _points(rng, n, kind):
    if kind == "uniform":
        return rng.random((n, 3))
    if kind == "gaussian":
        out = np.empty((0, 3))
        while out.shape[0] < n:
            z = 0.5 + 0.15 * rng.standard_normal((n, 3))
            z = z[np.all((z >= 0.0) & (z < 1.0), axis=1)]
            out = np.concatenate([out, z])
        return out[:n]
    if kind == "shell":
        d = rng.standard_normal((n, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        a, b = 0.45, 0.5
        r = (a ** 3 + rng.random(n) * (b ** 3 - a ** 3)) ** (1.0 / 3.0)
        return 0.5 + r[:, None] * d
    raise ValueError(kind)


def batch_problems(nprob=64, n_range=(1e4, 1e6), kappa_range=(8.0, 256.0), nrhs=16, seed0=SEED_BATCH):
    """Independent problems: list of dicts (targets, sources, kappa, max_depth,
    kind, x of shape (nrhs, N) complex128)."""
    out = []
    for i in range(int(nprob)):
        rng = np.random.default_rng(seed0 + i)
        n = int(round(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1])))))
        kappa = float(np.exp(rng.uniform(np.log(kappa_range[0]), np.log(kappa_range[1]))))
        kind = BATCH_KINDS[i % 3]
        t = _points(rng, n, kind)
        s = _points(rng, n, kind)
        x = np.empty((int(nrhs), n), dtype=np.complex128)
        for r in range(int(nrhs)):
            z = rng.standard_normal((n, 2))
            x[r] = z[:, 0] + 1j * z[:, 1]
        depth = max(1, int(np.ceil(np.log(n / 64.0) / np.log(8.0))))
        out.append(dict(targets=t, sources=s, kappa=kappa, max_depth=depth, kind=kind, x=x))
    return out


SEED_SELECTOR = 7


def selector_init(seed=SEED_SELECTOR):
    """Initial parameters of the 4 -> 64 -> 64 -> 64 -> 2 selector network
    (8770 float32, layout of include/dfdm.h): Glorot-uniform weights, zero
    biases, drawn layer by layer from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((64, 4), (64, 64), (64, 64), (2, 64)):
        a = np.sqrt(6.0 / (fan_in + fan_out))
        parts.append(rng.uniform(-a, a, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def selector_problems(count, seed0=200, n_range=(2000, 8000), kappa_range=(2.0, 48.0), depths=(3,)):
    """Small problems on which the method measures its own error for the
    selector's training data: problem i has tree depth d = depths[i % len(depths)]
    and draws from default_rng(seed0 + i), in order, N log-uniform in
    n_range x 8^(d - 3) (the same points per leaf box at every depth), kappa
    log-uniform in the i-th of `count` equal log-intervals of kappa_range (so
    the problems cover the range), targets, sources (uniform in [0,1)^3), one
    complex vector."""
    out = []
    lk0, lk1 = np.log(kappa_range[0]), np.log(kappa_range[1])
    for i in range(int(count)):
        rng = np.random.default_rng(seed0 + i)
        depth = int(depths[i % len(depths)])
        scale = 8.0 ** (depth - 3)
        n = int(round(np.exp(rng.uniform(np.log(n_range[0] * scale), np.log(n_range[1] * scale)))))
        kappa = float(np.exp(lk0 + (i + rng.uniform()) * (lk1 - lk0) / count))
        t = rng.random((n, 3))
        s = rng.random((n, 3))
        z = rng.standard_normal((n, 2))
        out.append(dict(targets=t, sources=s, kappa=kappa, max_depth=depth, x=z[:, 0] + 1j * z[:, 1]))
    return out
