"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the interpolation method: it only draws point
sets, sampled fields and target sets.  Every draw uses numpy's
``default_rng(seed)``; seeds are 1000 + workload index, held-out targets use the
workload seed + 500.

Workloads (points in [0,1]^2):
  * ``uniform_tps``  n = 1,500 i.i.d. uniform points, f = sin(4x)cos(3y) + 0.5x^2,
                     500 uniform held-out targets (k = 2).
  * ``cubic_mix``    n = 100,000 from 20 equal-weight isotropic Gaussians
                     (sigma = 0.02, centres U[0.1,0.9]^2), truncated to the unit
                     square by redrawing; f = 5 Gaussian bumps + a linear trend (k = 3).
  * ``tps_1m``       n = 1,048,576: 943,718 uniform + 104,858 points in 50
                     clusters (sigma = 0.005, centres U[0.05,0.95]^2, truncated),
                     f = exp(-8((x-.3)^2+(y-.6)^2)) + sin(10xy), 10,000 targets (k = 2).
The paper's own experiments use Sobol/uniform points and public data that are not
available here; these sets stand in for them with the same shapes and mixes.

Streams of independent requests (``serving_requests``: n log-uniform in [1,000, 500,000],
k in {1, 2, 3}, uniform or clustered points, bump-sum fields; ``batch_jobs``: k in {4, 5},
n log-uniform in [2,000, 200,000], the Franke function of Sec. 3.3) and Poisson arrival
times (``poisson_arrivals``) feed the serving and batched forms.
"""
from __future__ import annotations

import numpy as np


def uniform(n: int, rng) -> np.ndarray:
    return rng.random((n, 2))


def _truncated_normal_cloud(n: int, centre, sigma: float, rng) -> np.ndarray:
    out = np.empty((0, 2))
    while out.shape[0] < n:
        p = centre + sigma * rng.standard_normal((2 * (n - out.shape[0]) + 8, 2))
        p = p[(p >= 0.0).all(axis=1) & (p <= 1.0).all(axis=1)]
        out = np.concatenate([out, p])
    return out[:n]


def gaussian_mixture(n: int, n_comp: int, sigma: float, lo: float, hi: float, rng) -> np.ndarray:
    centres = lo + (hi - lo) * rng.random((n_comp, 2))
    counts = np.full(n_comp, n // n_comp)
    counts[: n - counts.sum()] += 1
    parts = [_truncated_normal_cloud(int(c), centres[i], sigma, rng) for i, c in enumerate(counts)]
    return np.concatenate(parts)


def f_uniform_tps(p: np.ndarray) -> np.ndarray:
    return np.sin(4 * p[:, 0]) * np.cos(3 * p[:, 1]) + 0.5 * p[:, 0] ** 2


def f_tps_1m(p: np.ndarray) -> np.ndarray:
    return np.exp(-8 * ((p[:, 0] - 0.3) ** 2 + (p[:, 1] - 0.6) ** 2)) + np.sin(10 * p[:, 0] * p[:, 1])


def bump_field(rng, n_bumps: int = 5):
    a = rng.uniform(-1, 1, n_bumps)
    c = rng.random((n_bumps, 2))
    s = rng.uniform(0.05, 0.2, n_bumps)
    b = rng.uniform(-1, 1, 3)

    def f(p):
        out = b[0] + b[1] * p[:, 0] + b[2] * p[:, 1]
        for i in range(n_bumps):
            d2 = (p[:, 0] - c[i, 0]) ** 2 + (p[:, 1] - c[i, 1]) ** 2
            out = out + a[i] * np.exp(-d2 / (2 * s[i] ** 2))
        return out

    return f


def f_sec32(p: np.ndarray) -> np.ndarray:
    """Test function of Sec. 3.2 (oscillation plus a C^0 cusp)."""
    x, y = p[:, 0], p[:, 1]
    return np.cos(30 * x + 0.8) * np.sin(30 * y - 2.1) + 5 * np.exp(-5 * np.sqrt((x - 0.25) ** 2 + (y - 0.75) ** 2))


def workload(name: str, n: int | None = None, n_targets: int | None = None, seed: int | None = None):
    """Return dict(points, f, targets, k, meta) for a named workload.  `n`
    overrides the point count (same recipe), for scaled-down parity cases; `seed`
    overrides the recipe's seed (another draw of the same workload)."""
    if name == "uniform_tps":
        seed = 1000 if seed is None else seed
        n = 1500 if n is None else n
        nt = 500 if n_targets is None else n_targets
        rng = np.random.default_rng(seed)
        pts = uniform(n, rng)
        f = f_uniform_tps(pts)
        k = 2
    elif name == "cubic_mix":
        seed = 1001 if seed is None else seed
        n = 100_000 if n is None else n
        nt = 1000 if n_targets is None else n_targets
        rng = np.random.default_rng(seed)
        pts = gaussian_mixture(n, 20, 0.02, 0.1, 0.9, rng)
        f = bump_field(rng)(pts)
        k = 3
    elif name == "tps_1m":
        seed = 1002 if seed is None else seed
        n = 1_048_576 if n is None else n
        nt = 10_000 if n_targets is None else n_targets
        rng = np.random.default_rng(seed)
        n_cl = int(round(0.1 * n))
        pts = np.concatenate([uniform(n - n_cl, rng), gaussian_mixture(n_cl, 50, 0.005, 0.05, 0.95, rng)])
        f = f_tps_1m(pts)
        k = 2
    else:
        raise KeyError(name)
    trng = np.random.default_rng(seed + 500)
    targets = uniform(nt, trng)
    return {"points": np.ascontiguousarray(pts), "f": np.ascontiguousarray(f), "targets": targets,
            "k": k, "seed": seed, "name": name}


def franke(p: np.ndarray) -> np.ndarray:
    """The Franke function as Sec. 3.3 states it: sum_j w_j exp(-(9x - c_j)' L_j (9x - c_j))
    with w = (0.75, 0.75, 0.5, -0.2), c = (2,2), (-1,-1), (7,3), (4,7), and diagonal
    L_1 = L_3 = I/4, L_2 = diag(1/49, 1/10), L_4 = I."""
    x, y = 9 * p[:, 0], 9 * p[:, 1]
    return (0.75 * np.exp(-((x - 2) ** 2 + (y - 2) ** 2) / 4) + 0.75 * np.exp(-(x + 1) ** 2 / 49 - (y + 1) ** 2 / 10)
            + 0.5 * np.exp(-((x - 7) ** 2 + (y - 3) ** 2) / 4) - 0.2 * np.exp(-(x - 4) ** 2 - (y - 7) ** 2))


def _geometry(n: int, clustered: bool, rng) -> np.ndarray:
    if clustered:
        return gaussian_mixture(n, 10, 0.02, 0.1, 0.9, rng)
    return uniform(n, rng)


def serving_requests(count: int, seed: int = 1004, n_lo: int = 1000, n_hi: int = 500_000, n_targets: int = 100):
    """Independent interpolation requests: n log-uniform in [n_lo, n_hi], k uniform in
    {1, 2, 3} (minimal polynomial block), uniform or clustered points (even odds), a
    bump-sum field with a linear trend, n_targets uniform targets.  Returns a list of
    dicts(points, f, targets, k)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        k = int(rng.integers(1, 4))
        pts = _geometry(n, bool(rng.integers(0, 2)), rng)
        f = bump_field(rng)(pts)
        out.append({"points": np.ascontiguousarray(pts), "f": np.ascontiguousarray(f),
                    "targets": uniform(n_targets, rng), "k": k})
    return out


def sobol(n: int, seed: int) -> np.ndarray:
    """The first n points of a scrambled 2D Sobol sequence on [0,1]^2 (Sec. 3.3 samples
    its points from a Sobol sequence)."""
    import warnings

    from scipy.stats import qmc

    with warnings.catch_warnings():
        warnings.simplefilter("ignore")  # n need not be a power of two
        return qmc.Sobol(d=2, scramble=True, seed=seed).random(n)


def batch_jobs(count: int = 64, seed: int = 1003, n_lo: int = 2000, n_hi: int = 200_000, n_targets: int = 100):
    """Independent higher-order jobs as in Sec. 3.3: k in {4, 5} (quadratic block), n
    log-uniform in [n_lo, n_hi], points from a scrambled Sobol sequence on [0,1]^2 (one
    scramble per job), the Franke function, n_targets uniform targets."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        k = int(rng.integers(4, 6))
        pts = sobol(n, int(rng.integers(0, 2**31)))
        out.append({"points": np.ascontiguousarray(pts), "f": franke(pts), "targets": uniform(n_targets, rng),
                    "k": k})
    return out


def poisson_arrivals(count: int, rate: float, seed: int = 1005) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate (requests per second)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, count))
