"""The tile bounds behind the tensor-core pass 1's block skipping.

Inside a pixel tile (16 x 8 pixels in 2-D, 8 x 4 x 4 in 3-D) a feature
moves away from its value at the tile's centre pixel by at most
D_k = sum_a alpha_a (alpha_a + 1) / 2 * h_a, from |P_m| <= 1 and
|P_m'| <= m (m + 1) / 2 on [-1, 1] (h_a: the largest offset from the centre
pixel along axis a).  Pass 1 leaves a block out only when these bounds put
all its logits far below the tile's reference logit, so the bound must
hold; here it is checked against the oracle's own features on whole tiles
of several grids, including the extreme tiles at the domain's corners.
"""
import numpy as np
import pytest

import oracle as O

TILE = {2: (16, 8), 3: (8, 4, 4)}


def exps(dim, d):
    # the graded order of the multi-indices (as the oracle's basis)
    out = []
    for g in range(d + 1):
        if dim == 2:
            for a1 in range(g, -1, -1):
                out.append((a1, g - a1))
        else:
            for a1 in range(g, -1, -1):
                for a2 in range(g - a1, -1, -1):
                    out.append((a1, a2, g - a1 - a2))
    return np.array(out)


def tile_points(shape, t0):
    dim = len(shape)
    ts = TILE[dim]
    axes = [-1.0 + (2.0 * np.arange(t0[a] * ts[a], (t0[a] + 1) * ts[a]) + 1.0) / shape[a] for a in range(dim)]
    c = [-1.0 + (2.0 * (t0[a] * ts[a] + ts[a] // 2) + 1.0) / shape[a] for a in range(dim)]
    pts = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, dim)
    return pts, np.array([c])


@pytest.mark.parametrize("shape,d", [((64, 48), 4), ((1024, 1024), 4), ((32, 16), 6), ((40, 24, 16), 2),
                                     ((48, 40, 32), 3), ((256, 256, 256), 3)])
def test_feature_moves_within_bound(shape, d):
    dim = len(shape)
    ts = TILE[dim]
    A = exps(dim, d)
    assert A.shape[0] == O.K(dim, d)
    h = np.array([ts[a] / shape[a] for a in range(dim)])
    D = (A * (A + 1) / 2 * h).sum(1)
    ntile = [shape[a] // ts[a] for a in range(dim)]
    rng = np.random.default_rng(7)
    corners = [tuple(0 for _ in range(dim)), tuple(n - 1 for n in ntile), tuple([0] + [n - 1 for n in ntile[1:]])]
    picks = corners + [tuple(int(rng.integers(0, n)) for n in ntile) for _ in range(20)]
    worst = 0.0
    for t0 in picks:
        pts, c = tile_points(shape, t0)
        E = O.features(O.Grid(coords=pts), d)
        Ec = O.features(O.Grid(coords=c), d)
        dev = np.abs(E - Ec).max(0)
        assert np.all(dev <= D * (1 + 1e-12) + 1e-15), (t0, dev, D)
        worst = max(worst, float((dev / np.where(D > 0, D, 1)).max()))
    # the bound is not vacuous: some feature comes within a factor 4 of it
    assert worst > 0.25
