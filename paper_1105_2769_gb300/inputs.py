"""Seeded synthetic point sets shaped like the paper's workloads.

This module only draws coordinates. It holds none of the three-body
arithmetic, so both the CPU oracle's tests and the GPU path may use it
without sharing any of the method's code.

Distributions:
  * uniform in a cube (the paper's "uniform" set, Section 6, and the
    exhaustive-kernel workloads at N = 512, 32 768 and 65 536);
  * an isotropic Gaussian mixture (the multi-tree workload, N = 2^20);
  * uniform in the unit ball and on a thin spherical shell (the paper's
    "ball" and "annulus" sets, Section 6; the annulus is read as a shell
    because Section 7 calls it a lower-dimensional manifold).

Every set may be rejection-resampled so that no two points are closer
than ``d_min``; the Axilrod-Teller potential is singular at zero
distance, so a minimum separation keeps every sum finite.

Rejection rule (deterministic for a given seed): all candidates are drawn
at once; every pair closer than ``d_min`` rejects the point with the
larger index; rejected points are redrawn from their own component and
checked against the accepted points (a conflict rejects the new point)
and against each other (the larger index loses). The loop ends when a
round rejects nothing, so the result has every pairwise distance
>= d_min.
"""
from __future__ import annotations

import numpy as np

try:  # scipy is on both the build host and the GPU host
    from scipy.spatial import cKDTree as _KDTree
except Exception:  # pragma: no cover - fallback keeps the module importable
    _KDTree = None


def _conflict_pairs(pts: np.ndarray, d_min: float) -> np.ndarray:
    """All index pairs (i < j) with |p_i - p_j| < d_min, as an (M, 2) array."""
    if len(pts) < 2 or d_min <= 0.0:
        return np.zeros((0, 2), dtype=np.int64)
    if _KDTree is not None:
        tree = _KDTree(pts)
        # query_pairs uses <= r; shrink r by one ulp-ish factor so the test
        # is the strict "closer than d_min".
        pairs = tree.query_pairs(d_min * (1.0 - 1e-12), output_type="ndarray")
        if pairs.size == 0:
            return np.zeros((0, 2), dtype=np.int64)
        pairs = np.sort(pairs.astype(np.int64), axis=1)
        d = np.linalg.norm(pts[pairs[:, 0]] - pts[pairs[:, 1]], axis=1)
        return pairs[d < d_min]
    # Plain cell-grid search (no scipy): cells of side d_min, 27 neighbours.
    cell = np.floor(pts / d_min).astype(np.int64)
    cell -= cell.min(axis=0)
    dims = cell.max(axis=0) + 3
    key = ((cell[:, 0] + 1) * dims[1] + (cell[:, 1] + 1)) * dims[2] + (cell[:, 2] + 1)
    order = np.argsort(key, kind="stable")
    skey = key[order]
    out = []
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                nkey = key + (dx * dims[1] + dy) * dims[2] + dz
                lo = np.searchsorted(skey, nkey, "left")
                hi = np.searchsorted(skey, nkey, "right")
                cnt = hi - lo
                for r in range(int(cnt.max(initial=0))):
                    has = cnt > r
                    i = np.nonzero(has)[0]
                    j = order[lo[has] + r]
                    keep = i < j
                    i, j = i[keep], j[keep]
                    d = np.linalg.norm(pts[i] - pts[j], axis=1)
                    m = d < d_min
                    if m.any():
                        out.append(np.stack([i[m], j[m]], axis=1))
    if not out:
        return np.zeros((0, 2), dtype=np.int64)
    return np.unique(np.concatenate(out), axis=0)


def rsa_resample(pts: np.ndarray, d_min: float, redraw, max_rounds: int = 100000):
    """Enforce a minimum pairwise distance by rejection and redraw.

    ``redraw(idx)`` returns fresh candidates (len(idx), 3) for the given
    point indices. Returns (points, total_rejections)."""
    pts = np.array(pts, dtype=np.float64, copy=True)
    n = len(pts)
    pairs = _conflict_pairs(pts, d_min)
    bad = np.unique(pairs[:, 1]) if pairs.size else np.zeros(0, np.int64)
    rejections = int(bad.size)
    rounds = 0
    while bad.size:
        rounds += 1
        if rounds > max_rounds:
            raise RuntimeError("rejection resampling did not converge")
        pts[bad] = redraw(bad)
        is_new = np.zeros(n, dtype=bool)
        is_new[bad] = True
        pairs = _conflict_pairs(pts, d_min)
        if pairs.size == 0:
            break
        i, j = pairs[:, 0], pairs[:, 1]
        ni, nj = is_new[i], is_new[j]
        rej = []
        # old-new conflicts reject the new point
        rej.append(j[~ni & nj])
        rej.append(i[ni & ~nj])
        # new-new conflicts reject the larger index (j > i)
        rej.append(j[ni & nj])
        bad = np.unique(np.concatenate(rej))
        rejections += int(bad.size)
    return pts, rejections


def uniform_cube(n: int, side: float, d_min: float, seed: int, return_stats=False):
    """n points i.i.d. uniform in [0, side]^3, resampled to min distance d_min."""
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.0, side, size=(n, 3))
    pts, rej = rsa_resample(pts, d_min, lambda idx: rng.uniform(0.0, side, size=(len(idx), 3)))
    return (pts, {"rejections": rej}) if return_stats else pts


def gaussian_mixture(n: int, n_comp: int, centre_box: float, sigma_lo: float,
                     sigma_hi: float, d_min: float, seed: int, return_stats=False):
    """Equal-weight isotropic Gaussian mixture.

    Centres ~ U[0, centre_box]^3, sigma ~ U[sigma_lo, sigma_hi]; point m
    belongs to component m % n_comp (equal weights)."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, centre_box, size=(n_comp, 3))
    sigmas = rng.uniform(sigma_lo, sigma_hi, size=n_comp)
    comp = np.arange(n) % n_comp

    def draw(idx):
        c = comp[idx]
        return centres[c] + sigmas[c, None] * rng.standard_normal(size=(len(idx), 3))

    pts = draw(np.arange(n))
    pts, rej = rsa_resample(pts, d_min, draw)
    stats = {"rejections": rej, "centres": centres, "sigmas": sigmas}
    return (pts, stats) if return_stats else pts


def unit_ball(n: int, d_min: float, seed: int):
    """n points uniform inside the unit ball (the paper's "ball" set)."""
    rng = np.random.default_rng(seed)

    def draw(idx):
        m = len(idx)
        v = rng.standard_normal(size=(m, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        r = rng.uniform(0.0, 1.0, size=m) ** (1.0 / 3.0)
        return v * r[:, None]

    pts = draw(np.arange(n))
    return rsa_resample(pts, d_min, draw)[0]


def spherical_shell(n: int, r_in: float, r_out: float, d_min: float, seed: int):
    """n points uniform in the shell r_in <= |x| <= r_out (the "annulus" set)."""
    rng = np.random.default_rng(seed)

    def draw(idx):
        m = len(idx)
        v = rng.standard_normal(size=(m, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        u = rng.uniform(0.0, 1.0, size=m)
        r = (r_in ** 3 + u * (r_out ** 3 - r_in ** 3)) ** (1.0 / 3.0)
        return v * r[:, None]

    pts = draw(np.arange(n))
    return rsa_resample(pts, d_min, draw)[0]


def random_weights(n: int, seed: int) -> np.ndarray:
    """Seeded cotangent weights g (for vector-Jacobian products), N(0,1)."""
    return np.random.default_rng(seed).standard_normal(n)


def sample_indices(n: int, m: int, seed: int) -> np.ndarray:
    """m distinct particle indices in [0, n), sorted (seeded subsample)."""
    rng = np.random.default_rng(seed)
    m = min(m, n)
    return np.sort(rng.choice(n, size=m, replace=False)).astype(np.int64)


# Named workloads (sizes and distributions of the paper-shaped configurations).
def workload(name: str, return_stats: bool = False):
    """Return the point set of a named workload.

    exh64_n512      : N=512, U[0,1]^3, d_min 0.01, seed 1
    exh32_n32768    : N=32 768, U[0,32]^3, d_min 0.5, seed 2
    gmm_n1048576    : N=2^20, 64-component GMM (centres U[0,100]^3,
                      sigma U[0.5,3]), d_min 0.05, seed 3
    forces_n65536   : N=65 536, U[0,32]^3, d_min 0.5, seed 4
    gmm4_n65536     : N=65 536 from the same generator as gmm_n1048576 with 4
                      components (16 384 points each, as there) in a cube of
                      side 100 (4/64)^(1/3), so component density and
                      per-component structure match the 2^20 set; seed 3
    gmm16_n262144   : the same with 16 components (262 144 points) in a cube
                      of side 100 (16/64)^(1/3); seed 3
    gmm32_n524288   : the same with 32 components (524 288 points) in a cube
                      of side 100 (32/64)^(1/3); seed 3
    """
    if name == "exh64_n512":
        r = uniform_cube(512, 1.0, 0.01, 1, return_stats=True)
    elif name == "exh32_n32768":
        r = uniform_cube(32768, 32.0, 0.5, 2, return_stats=True)
    elif name == "gmm_n1048576":
        r = gaussian_mixture(1 << 20, 64, 100.0, 0.5, 3.0, 0.05, 3, return_stats=True)
    elif name == "forces_n65536":
        r = uniform_cube(65536, 32.0, 0.5, 4, return_stats=True)
    elif name == "gmm4_n65536":
        r = gaussian_mixture(65536, 4, 100.0 * (4 / 64) ** (1 / 3), 0.5, 3.0, 0.05, 3,
                             return_stats=True)
    elif name == "gmm16_n262144":
        r = gaussian_mixture(1 << 18, 16, 100.0 * (16 / 64) ** (1 / 3), 0.5, 3.0, 0.05, 3,
                             return_stats=True)
    elif name == "gmm32_n524288":
        r = gaussian_mixture(1 << 19, 32, 100.0 * (32 / 64) ** (1 / 3), 0.5, 3.0, 0.05, 3,
                             return_stats=True)
    else:
        raise KeyError(name)
    return r if return_stats else r[0]


def min_pair_distance(pts: np.ndarray) -> float:
    """Smallest pairwise distance (for checking the resampling)."""
    if _KDTree is None or len(pts) < 2:
        d = np.linalg.norm(pts[:, None, :] - pts[None, :, :], axis=-1)
        d[np.diag_indices(len(pts))] = np.inf
        return float(d.min())
    dd, _ = _KDTree(pts).query(pts, k=2)
    return float(dd[:, 1].min())
