"""Mesh and point-cloud converters (App. A.4) through the C ABI against the
FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2205_15401_gb300 import scenes

from gpu_util import lib_ready, r32, to_dev
from parity import rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-5  # relative per tensor: FP32 edge lengths and sums


@pytest.mark.parametrize("flatten", [0.0, 0.3])
@pytest.mark.parametrize("zeta", [0.2, 0.5])
def test_sphere_mesh(flatten, zeta):
    voge = lib_ready()
    V, F = scenes.uv_sphere(12, 24, 1.0, seed=1, jitter=0.05)
    means, P = voge.voge_mesh_to_gaussians(to_dev(V), to_dev(F, torch.int32), zeta, flatten)
    torch.cuda.synchronize()
    wm, wP = oracle.mesh_to_gaussians(r32(V), F, zeta, flatten=flatten if flatten > 0 else None)
    np.testing.assert_array_equal(means.cpu().numpy(), V)
    assert rel_err(P.cpu().numpy(), wP) <= TOL


def test_bad_faces_are_skipped_and_lone_vertices_have_no_size():
    voge = lib_ready()
    V, F = scenes.uv_sphere(6, 8)
    V = np.concatenate([V, [[3.0, 0.0, 0.0]]]).astype(np.float32)  # a vertex on no face
    bad = np.array([[0, 0, 1], [1, 2, len(V) + 5], [-1, 2, 3]], np.int32)
    Fb = np.concatenate([F, bad]).astype(np.int32)
    _, P = voge.voge_mesh_to_gaussians(to_dev(V), to_dev(Fb, torch.int32), 0.5, 0.0)
    torch.cuda.synchronize()
    _, wP = oracle.mesh_to_gaussians(r32(V), F, 0.5)  # the valid faces only
    P = P.cpu().numpy()
    assert np.all(np.isnan(P[-1])) and np.all(np.isnan(wP[-1]))
    assert rel_err(P[:-1], wP[:-1]) <= TOL


@pytest.mark.parametrize("m", [1, 4, 9, 20, 32])
def test_point_cloud(m):
    voge = lib_ready()
    X = r32(np.random.default_rng(m).uniform(-1, 1, (3001, 3)))
    means, P = voge.voge_points_to_gaussians(to_dev(X), m, 0.5)
    torch.cuda.synchronize()
    _, wP = oracle.points_to_gaussians(X, m=m, zeta=0.5)
    np.testing.assert_array_equal(means.cpu().numpy(), X)
    assert rel_err(P.cpu().numpy(), wP) <= TOL


def test_converted_mesh_renders():
    """A converted sphere goes straight into the renderer."""
    voge = lib_ready()
    V, F = scenes.uv_sphere(16, 32, 1.0)
    means, P = voge.voge_mesh_to_gaussians(to_dev(V), to_dev(F, torch.int32), 0.5, 0.3)
    attr = torch.ones((V.shape[0], 3), device="cuda")
    R, T = voge.voge_pose_to_RT(np.array([0.3, 0.2, 4.0, 0.0]))
    cam = {"R": R, "T": T, "F": 64.0, "Ox": 32.0, "Oy": 32.0, "H": 64, "W": 64}
    img, w, idx = voge.Renderer([cam], V.shape[0], 3, K=20, tau=1.0, thresh=0.01).forward(means, P, attr)
    torch.cuda.synchronize()
    img = img.cpu().numpy()
    assert np.isfinite(img).all() and img.max() > 0.5  # the sphere covers the image centre


def test_bad_arguments():
    voge = lib_ready()
    lib = voge.lib()
    assert lib.voge_points_to_gaussians(10, 0, 0.5, None, None, None, None) == -1
    assert lib.voge_points_to_gaussians(10, 10, 0.5, None, None, None, None) == -1
    assert lib.voge_points_to_gaussians(10, 3, 1.5, None, None, None, None) == -1
    assert lib.voge_mesh_to_gaussians(4, 1, None, None, 0.5, -1.0, None, None, None, 0, None) == -1
    assert lib.voge_mesh_workspace_bytes(-1, 3) == 0
