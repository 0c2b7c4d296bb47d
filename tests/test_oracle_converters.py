"""Pins of the oracle's mesh and point-cloud converters (App. A.4):
sigma_k = (d_k / 2)^2 / log(1 / zeta) on the diagonal of Sigma_k, d_k the
mean length of the edges at vertex k (mesh) or the mean distance to the m
nearest points (point cloud).  Checked against closed forms of regular
shapes and against scipy's k-d tree for the nearest points."""
import math

import numpy as np
import pytest

import oracle


def _iso(d, zeta):
    s = (d / 2.0) ** 2 / math.log(1.0 / zeta)
    return np.array([1 / s, 0, 0, 1 / s, 0, 1 / s])


@pytest.mark.parametrize("zeta", [0.2, 0.5, 0.8])
def test_equilateral_triangle(zeta):
    a = 0.7
    V = np.array([[0, 0, 0], [a, 0, 0], [a / 2, a * math.sqrt(3) / 2, 0]])
    means, P = oracle.mesh_to_gaussians(V, [[0, 1, 2]], zeta)
    np.testing.assert_array_equal(means, V)
    for k in range(3):
        np.testing.assert_allclose(P[k], _iso(a, zeta), rtol=1e-12)


def test_tetrahedron_three_equal_edges_per_vertex():
    a = 1.3
    V = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) * (a / math.sqrt(8))
    F = [[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]]
    _, P = oracle.mesh_to_gaussians(V, F, 0.5)
    for k in range(4):
        np.testing.assert_allclose(P[k], _iso(a, 0.5), rtol=1e-12)


def test_shared_edge_counted_once():
    """A square of two triangles: the diagonal's end vertices average two sides
    and the diagonal; counting the shared diagonal twice would differ."""
    h = 0.5
    V = np.array([[0, 0, 0], [h, 0, 0], [h, h, 0], [0, h, 0]], float)
    _, P = oracle.mesh_to_gaussians(V, [[0, 1, 2], [0, 2, 3]], 0.5)
    np.testing.assert_allclose(P[0], _iso((2 * h + h * math.sqrt(2)) / 3, 0.5), rtol=1e-12)
    np.testing.assert_allclose(P[1], _iso(h, 0.5), rtol=1e-12)


def test_grid_interior_vertex():
    """Regular grid triangulated along one diagonal: an interior vertex has four
    axis edges h and two diagonals h sqrt 2."""
    n, h = 5, 0.2
    xs, ys = np.meshgrid(np.arange(n) * h, np.arange(n) * h, indexing="ij")
    V = np.stack([xs.ravel(), ys.ravel(), np.zeros(n * n)], 1)
    vid = lambda i, j: i * n + j
    F = []
    for i in range(n - 1):
        for j in range(n - 1):
            F += [[vid(i, j), vid(i + 1, j), vid(i + 1, j + 1)], [vid(i, j), vid(i + 1, j + 1), vid(i, j + 1)]]
    _, P = oracle.mesh_to_gaussians(V, F, 0.5)
    np.testing.assert_allclose(P[vid(2, 2)], _iso(h * (4 + 2 * math.sqrt(2)) / 6, 0.5), rtol=1e-12)
    # flattened along the normal (+-z for a flat mesh): P = diag(1/s, 1/s, 1/(f s))
    f = 0.25
    _, Pf = oracle.mesh_to_gaussians(V, F, 0.5, flatten=f)
    s = 1.0 / P[vid(2, 2)][0]
    np.testing.assert_allclose(Pf[vid(2, 2)], [1 / s, 0, 0, 1 / s, 0, 1 / (f * s)], rtol=1e-12, atol=1e-12)


def test_flatten_follows_a_tilted_normal():
    """Rotate a flat patch: the flattened inverse covariance is the rotated one."""
    h = 0.3
    V = np.array([[0, 0, 0], [h, 0, 0], [0, h, 0], [h, h, 0]], float)
    F = [[0, 1, 3], [0, 3, 2]]
    c, s_ = math.cos(0.7), math.sin(0.7)
    Rx = np.array([[1, 0, 0], [0, c, -s_], [0, s_, c]])
    _, P0 = oracle.mesh_to_gaussians(V, F, 0.5, flatten=0.1)
    _, P1 = oracle.mesh_to_gaussians(V @ Rx.T, F, 0.5, flatten=0.1)
    unpack = lambda p: np.array([[p[0], p[1], p[2]], [p[1], p[3], p[4]], [p[2], p[4], p[5]]])
    for k in range(4):
        np.testing.assert_allclose(unpack(P1[k]), Rx @ unpack(P0[k]) @ Rx.T, rtol=1e-10, atol=1e-10)


def test_point_lattice_six_neighbours():
    h = 0.1
    g = np.arange(5) * h
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    _, P = oracle.points_to_gaussians(X, m=6, zeta=0.5)
    centre = 2 * 25 + 2 * 5 + 2
    np.testing.assert_allclose(P[centre], _iso(h, 0.5), rtol=1e-12)


def test_points_match_kdtree():
    spatial = pytest.importorskip("scipy.spatial")
    X = np.random.default_rng(3).uniform(-1, 1, (300, 3))
    for m in (1, 4, 9):
        _, P = oracle.points_to_gaussians(X, m=m, zeta=0.5)
        dist, _ = spatial.cKDTree(X).query(X, k=m + 1)
        d = dist[:, 1:].mean(1)
        s = (d / 2) ** 2 / math.log(2.0)
        np.testing.assert_allclose(P[:, 0], 1 / s, rtol=1e-12)
        np.testing.assert_allclose(P[:, 1], 0.0)
