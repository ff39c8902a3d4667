"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only draws random numbers and post-processes label arrays
(boundary noise, compaction).  It holds none of the method's arithmetic:
converting drawn physical parameters to linear parameters, rasterising a
diagram and everything after that is done separately by the CUDA library
and by the oracle.

All draws use numpy's PCG64 bit generator seeded explicitly, so every input
is reproducible on any machine.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20260520


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def power_params(seed: int, N: int, dim: int = 2, w_max: float = 0.05):
    """Sites uniform in [-1,1]^dim and weights uniform in (0, w_max)."""
    g = rng(seed)
    y = g.uniform(-1.0, 1.0, size=(N, dim))
    w = g.uniform(0.0, w_max, size=N)
    return y, w


def apd_params(seed: int, N: int, dim: int = 2, lam=(0.5, 2.0), w_max: float = 0.05):
    """Sites, weights and SPD anisotropy matrices R diag(lambda) R^T with
    lambda log-uniform in ``lam`` and R Haar-distributed (QR of a Gaussian
    matrix with the sign of diag(R) fixed)."""
    g = rng(seed)
    y = g.uniform(-1.0, 1.0, size=(N, dim))
    w = g.uniform(0.0, w_max, size=N)
    A = np.empty((N, dim, dim))
    for i in range(N):
        Z = g.standard_normal((dim, dim))
        Q, R = np.linalg.qr(Z)
        Q = Q * np.sign(np.diag(R))[None, :]
        lam_i = np.exp(g.uniform(np.log(lam[0]), np.log(lam[1]), size=dim))
        A[i] = (Q * lam_i[None, :]) @ Q.T
    return y, w, A


def poly_params(seed: int, N: int, dim: int, K: int, sigma: float | None = None):
    """Sites uniform in [-1,1]^dim and an [N, K] array of normal draws
    N(0, sigma^2), sigma = 1/(2N) by default.  A degree-d polynomial diagram
    is built by each side from these: the coefficients of total degree <= 1
    come from the sites (a power diagram with zero weights) and the rest are
    the normal draws.  The spread 1/(2N) keeps the perturbation comparable to
    the power-diagram cost differences inside a cell (about 4/N), so nearly
    all N grains stay non-empty (485 of 500 at N = 500) while about 18% of
    the pixels change label relative to the Voronoi diagram of the sites;
    with unit spread only about 85 of 500 grains would be non-empty."""
    g = rng(seed)
    y = g.uniform(-1.0, 1.0, size=(N, dim))
    s = 1.0 / (2.0 * N) if sigma is None else float(sigma)
    z = s * g.standard_normal((N, K))
    return y, z


def random_theta(seed: int, N: int, K: int, scale: float = 1.0):
    return scale * rng(seed).standard_normal((N, K))


def random_labels(seed: int, P: int, N: int):
    return rng(seed).integers(0, N, size=P, dtype=np.int32)


def boundary_noise(labels, shape, prob: float, seed: int):
    """Label noise on grain boundaries.

    A boundary pixel is one with an axis neighbour (4 in 2-D, 6 in 3-D) of a
    different label.  Independently with probability ``prob`` each boundary
    pixel takes the label of one of its differing neighbours, chosen
    uniformly.  Decisions are made on the clean input; the result is a copy.
    ``labels`` is flat with axis 1 fastest and ``shape`` = (n1, n2[, n3]).
    """
    g = rng(seed)
    shape = tuple(int(s) for s in shape)
    lab = np.asarray(labels, dtype=np.int32).reshape(shape[::-1])  # [.., n2, n1]
    nd = lab.ndim
    cand = []
    for ax in range(nd):
        for sh in (+1, -1):
            nb = np.roll(lab, sh, axis=ax)
            valid = np.ones_like(lab, dtype=bool)
            idx = [slice(None)] * nd
            idx[ax] = 0 if sh == +1 else -1
            valid[tuple(idx)] = False
            cand.append(np.where(valid & (nb != lab), nb, -1))
    cand = np.stack(cand, axis=-1)  # [..., 2*nd]
    n_diff = (cand >= 0).sum(axis=-1)
    is_bd = n_diff > 0
    flip = is_bd & (g.random(lab.shape) < prob)
    pick = g.random(lab.shape)
    out = lab.copy()
    fi = np.nonzero(flip)
    if fi[0].size:
        c = cand[fi]                       # [F, 2*nd]
        nd_ = n_diff[fi]
        r = np.minimum((pick[fi] * nd_).astype(np.int64), nd_ - 1)
        order = np.argsort(c < 0, axis=1, kind="stable")  # differing first
        cs = np.take_along_axis(c, order, axis=1)
        out[fi] = cs[np.arange(cs.shape[0]), r]
    return out.reshape(-1)


def compact(labels):
    """Relabel to 0..N_eff-1 keeping the order of the used labels (empty
    grains have no maximiser, so generated maps drop them).  Returns
    (labels, N_eff, used) where used[new] = old."""
    lab = np.asarray(labels, dtype=np.int32)
    used = np.unique(lab)
    remap = np.full(int(used.max()) + 1, -1, dtype=np.int32)
    remap[used] = np.arange(used.size, dtype=np.int32)
    return remap[lab], int(used.size), used


def batched_shapes(seed: int, n_maps: int, side=(128, 1024), grains=(20, 2000)):
    """Per-map (n1, n2, N) for a batch of 2-D maps: sides and grain counts
    uniform integers in the given closed ranges."""
    g = rng(seed)
    n1 = g.integers(side[0], side[1] + 1, size=n_maps)
    n2 = g.integers(side[0], side[1] + 1, size=n_maps)
    N = g.integers(grains[0], grains[1] + 1, size=n_maps)
    return [(int(a), int(b), int(c)) for a, b, c in zip(n1, n2, N)]
