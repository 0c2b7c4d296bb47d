"""Pins of the oracle's analytic backward and camera pose against finite differences."""
import math

import numpy as np
import pytest

import oracle
from paper_2205_15401_gb300 import scenes


def small_scene(seed=0, N=12, C=2):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((N, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    means = 0.3 * d
    rot = scenes.random_rotations(rng, N)
    s = rng.uniform(0.06, 0.15, (N, 3))
    P = np.einsum("nij,nj,nkj->nik", rot, 1 / s**2, rot)
    P6 = np.stack([P[:, 0, 0], P[:, 0, 1], P[:, 0, 2], P[:, 1, 1], P[:, 1, 2], P[:, 2, 2]], 1)
    attr = rng.uniform(-1, 1, (N, C))
    poses = np.array([[0.3, 0.2, 2.0, 0.05], [-1.1, -0.3, 2.2, -0.02]])
    cams = []
    for p in poses:
        R, T = oracle.pose_to_RT(p)
        cams.append({"R": R, "T": T, "F": 14.0, "Ox": 7.0, "Oy": 7.0, "H": 14, "W": 14})
    return cams, means, P6, attr, rng


def loss(cams, means, P6, attr, pix, idx, G, tau):
    return float((oracle.fine(cams, means, P6, attr, tau, pix, idx, nthreads=1)["image"] * G).sum())


def fd_check(fn, x, analytic, rel_h=1e-6, n_probe=None, rng=None):
    flat = x.reshape(-1)
    ids = range(flat.size) if n_probe is None else rng.choice(flat.size, n_probe, replace=False)
    num, ana = [], []
    for i in ids:
        h = rel_h * max(1.0, abs(flat[i]))
        old = flat[i]
        flat[i] = old + h
        fp = fn()
        flat[i] = old - h
        fm = fn()
        flat[i] = old
        num.append((fp - fm) / (2 * h))
        ana.append(analytic.reshape(-1)[i])
    num, ana = np.array(num), np.array(ana)
    err = np.linalg.norm(num - ana) / max(np.linalg.norm(num), 1e-30)
    return err, num, ana


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_central_differences(seed):
    cams, means, P6, attr, rng = small_scene(seed)
    tau, K, eta = 1.3, 6, 0.01
    fwd = oracle.render(cams, means, P6, attr, K=K, tau=tau, eta=eta)
    pix, idx = fwd["pix"], fwd["idx"]
    assert (fwd["count"] >= 2).sum() > 20
    G = rng.standard_normal(fwd["image"].shape)
    g = oracle.render_bwd(cams, means, P6, attr, tau, pix, idx, G, nthreads=1)

    def f():
        return loss(cams, means, P6, attr, pix, idx, G, tau)

    for name, x, ana in [("means", means, g["g_means"]), ("inv_cov", P6, g["g_inv_cov"]), ("attr", attr, g["g_attr"])]:
        err, num, _ = fd_check(f, x, ana)
        assert np.linalg.norm(num) > 1e-6, name
        assert err < 1e-6, (name, err)
    for v in range(2):
        R = cams[v]["R"]
        err, num, _ = fd_check(f, R, g["g_R"][v])
        assert err < 1e-6, ("R", v, err)
        T = cams[v]["T"]
        err, num, _ = fd_check(f, T, g["g_T"][v])
        assert err < 1e-6, ("T", v, err)


def test_pose_to_RT_is_a_look_at():
    rng = np.random.default_rng(3)
    for _ in range(20):
        a, e, d, r = rng.uniform(-math.pi, math.pi), rng.uniform(-1.2, 1.2), rng.uniform(1, 8), rng.uniform(-0.5, 0.5)
        R, T = oracle.pose_to_RT([a, e, d, r])
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-14)
        Cw = d * np.array([math.cos(e) * math.sin(a), math.sin(e), math.cos(e) * math.cos(a)])
        np.testing.assert_allclose(R @ Cw + T, 0, atol=1e-12)      # camera centre
        np.testing.assert_allclose(T, [0, 0, d], atol=1e-12)        # origin on the optical axis at depth d
        # world up projects to image "up" (negative camera y) when there is no roll
        R0, _ = oracle.pose_to_RT([a, e, d, 0.0])
        assert (R0 @ np.array([0, 1.0, 0]))[1] < 0
        assert abs((R0 @ np.array([0, 1.0, 0]))[0]) < 1e-12


def test_pose_identity_case():
    R, T = oracle.pose_to_RT([0.0, 0.0, 3.0, 0.0])
    np.testing.assert_allclose(R, np.diag([1.0, -1.0, -1.0]), atol=1e-15)
    np.testing.assert_allclose(T, [0, 0, 3.0], atol=1e-15)


def test_pose_grad_matches_central_differences():
    rng = np.random.default_rng(4)
    for _ in range(10):
        pose = np.array([rng.uniform(-3, 3), rng.uniform(-1, 1), rng.uniform(2, 6), rng.uniform(-0.3, 0.3)])
        dR, dT = rng.standard_normal((3, 3)), rng.standard_normal(3)
        g = oracle.pose_grad(pose, dR, dT)
        for q in range(4):
            h = 1e-6
            pp, pm = pose.copy(), pose.copy()
            pp[q] += h
            pm[q] -= h
            Rp, Tp = oracle.pose_to_RT(pp)
            Rm, Tm = oracle.pose_to_RT(pm)
            num = ((Rp - Rm) * dR).sum() / (2 * h) + ((Tp - Tm) * dT).sum() / (2 * h)
            assert g[q] == pytest.approx(num, rel=1e-7, abs=1e-9)


def test_occluded_gaussian_receives_gradient():
    """A kernel behind an opaque one still gets gradient (the occlusion-reasoning claim, Sec. 4.3)."""
    cam = {"R": np.eye(3), "T": np.zeros(3), "F": 10.0, "Ox": 5.0, "Oy": 5.0, "H": 10, "W": 10}
    v = 1 / 0.2**2
    P6 = np.array([[v, 0, 0, v, 0, v], [v, 0, 0, v, 0, v]])
    means = np.array([[0.0, 0.0, 2.0], [0.05, 0.0, 3.0]])  # index 1 is behind index 0
    attr = np.array([[0.0], [1.0]])
    tau = 4.0  # the front kernel passes about e^{-4} of the light at its centre
    fwd = oracle.render([cam], means, P6, attr, K=0, tau=tau, eta=0.0)
    G = np.ones_like(fwd["image"])
    g = oracle.render_bwd([cam], means, P6, attr, tau, fwd["pix"], fwd["idx"], G)
    assert abs(g["g_means"][1, 0]) > 1e-3  # moving the hidden kernel sideways changes the image
    assert abs(g["g_attr"][1, 0]) > 1e-3
    assert abs(g["g_means"][0, 0]) > 1e-3  # and so does moving the occluder


def test_both_gradient_paths_contribute():
    """Gradient flows through T(l_k) and through e^{q_k} (the ablation of Table 4 blocks either)."""
    cam = {"R": np.eye(3), "T": np.zeros(3), "F": 10.0, "Ox": 5.0, "Oy": 5.0, "H": 10, "W": 10}
    v = 1 / 0.2**2
    P6 = np.array([[v, 0, 0, v, 0, v], [v, 0, 0, v, 0, v]])
    means = np.array([[0.0, 0.0, 2.0], [0.05, 0.0, 2.02]])
    attr = np.array([[0.0], [1.0]])  # only the back kernel is visible in the loss
    fwd = oracle.render([cam], means, P6, attr, K=0, tau=1.0, eta=0.0)
    G = np.ones_like(fwd["image"])
    g = oracle.render_bwd([cam], means, P6, attr, 1.0, fwd["pix"], fwd["idx"], G)
    # the front kernel has colour 0: its gradient comes only through the back kernel's T
    assert np.abs(g["g_means"][0]).max() > 1e-4
    # the back kernel's own peak density a drives a gradient on its inverse covariance
    assert np.abs(g["g_inv_cov"][1]).max() > 1e-7
