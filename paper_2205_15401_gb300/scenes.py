"""Seeded synthetic scenes shaped like the paper's workloads.

This module only draws inputs: Gaussian centres, inverse covariances,
attributes and camera poses.  It holds none of the renderer's arithmetic and
is the one module that both the CUDA path (bench, tests) and the FP64 oracle
(tests) read.  Camera poses are returned as (azimuth, elevation, distance,
roll); turning a pose into (R, T) is the renderer's own step and each side
does it itself.

Workloads (the paper's datasets are not available; these stand in for them):
  plain_64        1 x 64^2, f=64, camera at the origin looking +z, N=128
                  ellipsoids, means U([-1,1]^2 x [3,5]), covariance R diag(s^2) Rᵀ,
                  s ~ lognormal(ln 0.08, 0.3) per axis, RGB U[0,1], tau=1, K=all,
                  no threshold.
  posefit_256     1 x 256^2, f=256, pose azim U(-pi,pi), elev U(-pi/6,pi/3),
                  dist 4, roll U(-0.1,0.1); N=4000 isotropic (s=0.03) Gaussians on
                  a superquadric shell (semi-axes 1.0/0.6/0.4, exponents
                  U(0.5,1.5)); C=128 N(0,1) features, unit-normalised rows; K=20,
                  eta=1e-3 (stands in for the PASCAL3D+ feature pose fitting).
  fit_8x512       8 x 512^2, f=512, 8 cameras on a Fibonacci view sphere of
                  radius 4 looking at the origin; N=50,000 anisotropic Gaussians
                  on a unit sphere with 0.02 radial noise, s ~ lognormal(ln 0.01,
                  0.4) per axis; RGB U[0,1]; K=20, eta=0.01 (stands in for the
                  multi-view shape-fitting meshes of 2.5k-34k vertices).
  large_1024      1 x 1024^2, f=1024, camera at the origin; N=500,000, means
                  U([-2,2]^3) + (0,0,6), s ~ lognormal(ln 0.005, 0.5) per axis;
                  C=16 N(0,1); K=32, eta=1e-4 (stands in for the 438k-point
                  bridge point cloud).
  serving stream  Poisson arrivals (mean 2 ms); N ~ U[1k,100k] (fit_8x512
                  generator), side in {128,256,512}, C in {3,16,128},
                  K in {10,20,32}.
"""
from __future__ import annotations

import math

import numpy as np


def random_rotations(rng, n):
    """Uniform random rotations: QR of a Gaussian matrix with the sign fixed."""
    A = rng.standard_normal((n, 3, 3))
    Q, Rm = np.linalg.qr(A)
    d = np.sign(np.diagonal(Rm, axis1=1, axis2=2))
    d[d == 0] = 1.0
    Q = Q * d[:, None, :]
    det = np.linalg.det(Q)
    Q[det < 0, :, 0] *= -1.0
    return Q


def inverse_covariance(rot, scales):
    """P = R diag(1/s^2) Rᵀ packed as (xx, xy, xz, yy, yz, zz), float32."""
    P = np.einsum("nij,nj,nkj->nik", rot, 1.0 / scales.astype(np.float64) ** 2, rot)
    out = np.stack([P[:, 0, 0], P[:, 0, 1], P[:, 0, 2], P[:, 1, 1], P[:, 1, 2], P[:, 2, 2]], 1)
    return np.ascontiguousarray(out.astype(np.float32))


def _identity_camera(H, W, F):
    return {"R": np.eye(3, dtype=np.float32), "T": np.zeros(3, np.float32), "F": float(F), "Ox": W / 2.0,
            "Oy": H / 2.0, "H": int(H), "W": int(W)}


def plain_64(seed=0, N=128):
    rng = np.random.default_rng(seed)
    means = np.concatenate([rng.uniform(-1, 1, (N, 2)), rng.uniform(3, 5, (N, 1))], 1).astype(np.float32)
    rot = random_rotations(rng, N)
    s = np.exp(rng.normal(math.log(0.08), 0.3, (N, 3)))
    attr = rng.uniform(0, 1, (N, 3)).astype(np.float32)
    return {"name": "plain_64", "means": means, "inv_cov": inverse_covariance(rot, s), "attr": attr,
            "cameras": [_identity_camera(64, 64, 64)], "poses": None, "H": 64, "W": 64, "F": 64.0,
            "tau": 1.0, "K": 0, "eta": 0.0}


def _superquadric(rng, N, axes, e1, e2):
    eta = rng.uniform(-math.pi / 2, math.pi / 2, N)
    om = rng.uniform(-math.pi, math.pi, N)

    def spow(x, e):
        return np.sign(x) * np.abs(x) ** e

    x = axes[0] * spow(np.cos(eta), e1) * spow(np.cos(om), e2)
    y = axes[1] * spow(np.cos(eta), e1) * spow(np.sin(om), e2)
    z = axes[2] * spow(np.sin(eta), e1)
    return np.stack([x, y, z], 1)


def posefit_256(seed=0, N=4000, C=128):
    rng = np.random.default_rng(seed)
    e1, e2 = rng.uniform(0.5, 1.5, 2)
    means = _superquadric(rng, N, (1.0, 0.6, 0.4), e1, e2).astype(np.float32)
    s = np.full((N, 3), 0.03)
    rot = np.broadcast_to(np.eye(3), (N, 3, 3))
    attr = rng.standard_normal((N, C))
    attr = (attr / np.linalg.norm(attr, axis=1, keepdims=True)).astype(np.float32)
    pose = np.array([[rng.uniform(-math.pi, math.pi), rng.uniform(-math.pi / 6, math.pi / 3), 4.0,
                      rng.uniform(-0.1, 0.1)]])
    return {"name": "posefit_256", "means": means, "inv_cov": inverse_covariance(rot, s), "attr": attr,
            "cameras": None, "poses": pose, "H": 256, "W": 256, "F": 256.0, "tau": 1.0, "K": 20, "eta": 1e-3}


def fibonacci_poses(n, dist=4.0):
    """n camera poses (azim, elev, dist, roll) on a Fibonacci sphere."""
    golden = math.pi * (3.0 - math.sqrt(5.0))
    out = []
    for i in range(n):
        y = 1.0 - (2.0 * i + 1.0) / n
        out.append([(i * golden) % (2 * math.pi) - math.pi, math.asin(y), dist, 0.0])
    return np.array(out)


def fit_8x512(seed=0, N=50_000, B=8, side=512, C=3, K=20):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((N, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    means = (d * (1.0 + 0.02 * rng.standard_normal((N, 1)))).astype(np.float32)
    rot = random_rotations(rng, N)
    s = np.exp(rng.normal(math.log(0.01), 0.4, (N, 3)))
    attr = rng.uniform(0, 1, (N, C)).astype(np.float32)
    target_means = (means + 0.01 * rng.standard_normal((N, 3))).astype(np.float32)
    target_attr = (attr + 0.1 * rng.standard_normal((N, C))).astype(np.float32)
    return {"name": "fit_8x512", "means": means, "inv_cov": inverse_covariance(rot, s), "attr": attr,
            "target_means": target_means, "target_attr": target_attr, "cameras": None,
            "poses": fibonacci_poses(B), "H": side, "W": side, "F": float(side), "tau": 1.0, "K": K, "eta": 0.01}


def large_1024(seed=0, N=500_000, C=16):
    rng = np.random.default_rng(seed)
    means = (rng.uniform(-2, 2, (N, 3)) + np.array([0.0, 0.0, 6.0])).astype(np.float32)
    rot = random_rotations(rng, N)
    s = np.exp(rng.normal(math.log(0.005), 0.5, (N, 3)))
    attr = rng.standard_normal((N, C)).astype(np.float32)
    return {"name": "large_1024", "means": means, "inv_cov": inverse_covariance(rot, s), "attr": attr,
            "cameras": [_identity_camera(1024, 1024, 1024)], "poses": None, "H": 1024, "W": 1024, "F": 1024.0,
            "tau": 1.0, "K": 32, "eta": 1e-4}


def two_cuboids(gap, occludee_shift=(0.0, 0.0, 0.0), side=128, n=6):
    """Occlusion-reasoning scene (the two-cuboid setup of Sec. 4): a red
    occluder 1 x 1 x 0.6 scale units centred on the optical axis at depth 6,
    and a blue 1 x 1 x 1 occludee `gap` units behind it, moved by
    `occludee_shift`.  Each cuboid is an n x n x m grid of axis-aligned
    Gaussians spaced like its cells.  Returns the scene dict with "parts":
    index ranges of the occluder and the occludee."""
    def box(centre, size, m):
        axes = [np.linspace(-0.5, 0.5, k) * sz for k, sz in zip((n, n, m), size)]
        g = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3) + np.asarray(centre)
        s = np.array([sz / k for sz, k in zip(size, (n, n, m))]) * 0.6
        return g, np.tile(s, (g.shape[0], 1))
    a_m, a_s = box((0.0, 0.0, 6.0), (1.0, 1.0, 0.6), 3)
    b_c = np.array([0.0, 0.0, 6.0 + 0.3 + gap + 0.5]) + np.asarray(occludee_shift, dtype=np.float64)
    b_m, b_s = box(b_c, (1.0, 1.0, 1.0), n)
    means = np.concatenate([a_m, b_m]).astype(np.float32)
    scales = np.concatenate([a_s, b_s])
    rot = np.tile(np.eye(3), (means.shape[0], 1, 1))
    attr = np.concatenate([np.tile([1.0, 0.0, 0.0], (a_m.shape[0], 1)), np.tile([0.0, 0.0, 1.0], (b_m.shape[0], 1))])
    na = a_m.shape[0]
    return {"name": "two_cuboids", "means": means, "inv_cov": inverse_covariance(rot, scales),
            "attr": attr.astype(np.float32), "cameras": [_identity_camera(side, side, side)], "poses": None,
            "H": side, "W": side, "F": float(side), "tau": 1.0, "K": 32, "eta": 1e-3,
            "parts": {"occluder": (0, na), "occludee": (na, means.shape[0])}}


def uv_sphere(n_lat=12, n_lon=24, radius=1.0, seed=None, jitter=0.0):
    """Triangle mesh of a sphere: poles plus n_lat - 1 rings of n_lon vertices
    (float32 vertices, int32 faces); `jitter` moves the vertices radially."""
    verts = [[0.0, 0.0, radius]]
    for i in range(1, n_lat):
        th = math.pi * i / n_lat
        for j in range(n_lon):
            ph = 2 * math.pi * j / n_lon
            verts.append([radius * math.sin(th) * math.cos(ph), radius * math.sin(th) * math.sin(ph),
                          radius * math.cos(th)])
    verts.append([0.0, 0.0, -radius])
    verts = np.array(verts)
    if jitter > 0:
        verts *= 1.0 + jitter * np.random.default_rng(seed).uniform(-1, 1, (len(verts), 1))
    ring = lambda i, j: 1 + (i - 1) * n_lon + (j % n_lon)
    last = len(verts) - 1
    faces = [[0, ring(1, j), ring(1, j + 1)] for j in range(n_lon)]
    for i in range(1, n_lat - 1):
        for j in range(n_lon):
            faces += [[ring(i, j), ring(i + 1, j), ring(i + 1, j + 1)], [ring(i, j), ring(i + 1, j + 1), ring(i, j + 1)]]
    faces += [[ring(n_lat - 1, j), last, ring(n_lat - 1, j + 1)] for j in range(n_lon)]
    return verts.astype(np.float32), np.array(faces, np.int32)


def serving_stream(seed=0, duration_s=10.0, mean_gap_s=0.002):
    """Request descriptors for the Poisson serving workload."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(mean_gap_s)
        if t > duration_s:
            break
        out.append({"t": t, "N": int(rng.integers(1000, 100_001)), "side": int(rng.choice([128, 256, 512])),
                    "C": int(rng.choice([3, 16, 128])), "K": int(rng.choice([10, 20, 32])),
                    "seed": int(rng.integers(0, 2**31 - 1))})
    return out


def cameras(scene, pose_to_RT):
    """Camera dicts for a scene; poses go through the caller's pose_to_RT.

    R and T are rounded to float32, the precision the renderer takes them in."""
    if scene.get("cameras") is not None:
        return [dict(c) for c in scene["cameras"]]
    out = []
    for pose in scene["poses"]:
        R, T = pose_to_RT(pose)
        out.append({"R": np.asarray(R, np.float32).reshape(3, 3), "T": np.asarray(T, np.float32).reshape(3),
                    "F": scene["F"], "Ox": scene["W"] / 2.0, "Oy": scene["H"] / 2.0, "H": scene["H"],
                    "W": scene["W"]})
    return out


SCENES = {"plain_64": plain_64, "posefit_256": posefit_256, "fit_8x512": fit_8x512, "large_1024": large_1024}
