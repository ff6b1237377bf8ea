"""Pins for the oracle's phase assembly: the reliability-sorting unwrapper of Herraez et al. (2002)
that the paper applies to its local phases (Sec. 3). Each test checks it against something other
than itself: exact recovery of smooth phase maps, numpy's 1-D unwrap, a closed form of the
reliability, and an independent maximum spanning tree (networkx) integrated edge by edge.
"""
import numpy as np
import pytest

import oracle as O

TWO_PI = 2 * np.pi


def _wrapf(a):
    return ((np.asarray(a, dtype=np.float64) + np.pi) % TWO_PI - np.pi).astype(np.float32)


def _k_offset_constant(k, k_ref, mask):
    d = (k - k_ref)[mask]
    return d.size > 0 and np.all(d == d[0])


@pytest.mark.parametrize("seed", range(4))
def test_unwrap_smooth_maps_exact(seed):
    """A map whose neighbour steps stay below pi is recovered exactly, up to one 2 pi multiple."""
    rng = np.random.default_rng(seed)
    H, W = 33 + seed, 47
    y, x = np.mgrid[0:H, 0:W]
    a, b, c = rng.uniform(-0.02, 0.02, 3)
    phi = a * (x - 20) ** 2 + b * (y - 10) ** 2 + c * x * y + 0.4 * np.sin(x / 4.0 + y / 7.0) + rng.uniform(-3, 3)
    u, k, n = O.unwrap(_wrapf(phi))
    assert n == 1
    t = (u - phi) / TWO_PI
    assert np.abs(t - np.round(t[0, 0])).max() < 1e-5


def test_unwrap_single_row_is_numpy_unwrap():
    rng = np.random.default_rng(1)
    steps = rng.uniform(-2.5, 2.5, 300)
    phi = np.cumsum(steps)
    w = _wrapf(phi)[None, :]
    u, k, n = O.unwrap(w)
    ref = np.unwrap(w[0].astype(np.float64))
    assert n == 1
    t = (u[0] - ref) / TWO_PI
    assert np.all(np.abs(t - np.round(t[0])) < 1e-9)


def test_reliability_closed_form_quadratic():
    """phi = a x^2 + b y^2 has second differences H = 2a, V = 2b, D1 = D2 = 2a + 2b (in the order the
    method takes them), so R = 1 / sqrt(4a^2 + 4b^2 + 2 (2a + 2b)^2) at every interior pixel."""
    a, b = 0.031, -0.017
    y, x = np.mgrid[0:30, 0:30]  # every step (diagonals too) stays below pi
    R = O.unwrap_reliability(_wrapf(a * x ** 2 + b * y ** 2))
    exp = 1.0 / np.sqrt(4 * a * a + 4 * b * b + 2 * (2 * a + 2 * b) ** 2)
    assert np.abs(R[1:-1, 1:-1] / exp - 1).max() < 2e-3
    # the frame's border has no second difference: least reliable
    assert (R[0, :] == 0).all() and (R[-1, :] == 0).all() and (R[:, 0] == 0).all() and (R[:, -1] == 0).all()


def test_reliability_missing_values():
    w = _wrapf(np.random.default_rng(2).uniform(-3, 3, (12, 14)))
    w[5, 6] = np.nan
    R = O.unwrap_reliability(w)
    assert np.isnan(R[5, 6])
    assert (R[4:7, 5:8][~np.isnan(R[4:7, 5:8])] == 0).all()  # neighbours of a missing value
    assert (R[8:11, 2:12] > 0).all()


def test_unwrap_missing_column_splits_components():
    H, W = 20, 31
    y, x = np.mgrid[0:H, 0:W]
    phi = 0.45 * x + 0.2 * y
    w = _wrapf(phi)
    w[:, 15] = np.nan
    u, k, n = O.unwrap(w)
    assert n == 2
    assert np.isnan(u[:, 15]).all()
    for sl in (np.s_[:, :15], np.s_[:, 16:]):
        t = (u[sl] - phi[sl]) / TWO_PI
        assert np.abs(t - np.round(t[0, 0])).max() < 1e-5


def _mst_integration(w):
    """Independent reference: maximum spanning tree of the pixel grid (networkx, Kruskal) under the
    method's edge order (reliability descending, then edge index 2 (i W + j) + (0 right, 1 down)
    ascending, given to networkx as a rank so ties are decided the same way), then the 2 pi jumps
    integrated from a root along the tree."""
    nx = pytest.importorskip("networkx")
    H, W = w.shape
    R = O.unwrap_reliability(w)
    edges = []
    for i in range(H):
        for j in range(W):
            if j + 1 < W:
                edges.append((np.float32(R[i, j] + R[i, j + 1]), 2 * (i * W + j), (i, j), (i, j + 1)))
            if i + 1 < H:
                edges.append((np.float32(R[i, j] + R[i + 1, j]), 2 * (i * W + j) + 1, (i, j), (i + 1, j)))
    order = sorted(range(len(edges)), key=lambda t: (-float(edges[t][0]), edges[t][1]))
    G = nx.Graph()
    for rank, t in enumerate(order):
        G.add_edge(edges[t][2], edges[t][3], weight=-rank)  # a smaller rank is a heavier edge
    T = nx.maximum_spanning_tree(G, algorithm="kruskal")
    k = np.zeros((H, W), dtype=np.int64)
    for p, q in nx.bfs_edges(T, (0, 0)):
        d = np.float32(w[q]) - np.float32(w[p])
        k[q] = k[p] + (-1 if d > np.float32(np.pi) else (1 if d <= -np.float32(np.pi) else 0))
    return k


@pytest.mark.parametrize("seed", range(3))
def test_unwrap_is_max_spanning_tree_integration(seed):
    """Herraez's merge order is Kruskal's: on a noisy map with residues (where the result depends on
    the order) the oracle equals integration along the maximum spanning tree."""
    rng = np.random.default_rng(10 + seed)
    H, W = 11, 13
    y, x = np.mgrid[0:H, 0:W]
    phi = 0.6 * x - 0.4 * y + rng.normal(0, 1.1, (H, W))
    w = _wrapf(phi)
    u, k, n = O.unwrap(w)
    kr = _mst_integration(w)
    assert _k_offset_constant(k.astype(np.int64), kr, np.ones_like(k, dtype=bool))


def test_unwrap_transpose():
    rng = np.random.default_rng(4)
    y, x = np.mgrid[0:15, 0:18]
    w = _wrapf(0.5 * x + 0.3 * y + rng.normal(0, 1.0, (15, 18)))
    u1, k1, _ = O.unwrap(w)
    u2, k2, _ = O.unwrap(np.ascontiguousarray(w.T))
    assert _k_offset_constant(k1.T.astype(np.int64), k2.astype(np.int64), np.ones_like(k2, dtype=bool))
