"""Occlusion reasoning of two objects (the two-cuboid experiment of Sec. 4):
the occludee sits 1.5 or 5 scale units behind the occluder, mostly hidden,
and only its location is optimised against a target image where it shows
beside the occluder.  The gradient on the hidden object has to come through
the volume blending of Eq. 7.

Checks: the GPU's gradient on the occludee's translation equals the FP64
oracle's, points towards the target, and a short optimisation moves the
occludee most of the way there."""
import numpy as np
import pytest
import torch

import oracle
from paper_2205_15401_gb300 import scenes

from gpu_util import lib_ready, r32, to_dev
from parity import rel_err

pytestmark = pytest.mark.gpu

TARGET_X, START_X = 0.6, 0.15


def _scene(gap, x):
    sc = scenes.two_cuboids(gap, occludee_shift=(x, 0.0, 0.0))
    cams = scenes.cameras(sc, oracle.pose_to_RT)
    return sc, cams


def _loss_and_grad(voge, R, means, inv_cov, attr, target, lo, hi):
    img, w, idx = R.forward(means, inv_cov, attr)
    g = torch.empty_like(img)
    loss = torch.zeros(1, device="cuda")
    voge.voge_mse_grad(img, target, g, loss)
    gm = torch.zeros_like(means)
    R.backward(means, inv_cov, attr, idx, g, gm, None, None, None, weights=w)
    return float(loss), gm[lo:hi].sum(0)


@pytest.mark.parametrize("gap", [1.5, 5.0])
def test_hidden_object_gradient_matches_oracle_and_points_to_target(gap):
    voge = lib_ready()
    sc, cams = _scene(gap, START_X)
    tsc, _ = _scene(gap, TARGET_X)
    lo, hi = sc["parts"]["occludee"]
    K, eta = sc["K"], sc["eta"]
    m64, p64, a64 = (sc[k].astype(np.float64) for k in ("means", "inv_cov", "attr"))
    target = oracle.render(cams, tsc["means"].astype(np.float64), p64, a64, K=K, tau=1.0, eta=eta)["image"]
    R = voge.Renderer(cams, m64.shape[0], 3, K=K, tau=1.0, thresh=eta)
    means, inv_cov, attr = to_dev(sc["means"]), to_dev(sc["inv_cov"]), to_dev(sc["attr"])
    _, gt = _loss_and_grad(voge, R, means, inv_cov, attr, to_dev(r32(target)), lo, hi)
    torch.cuda.synchronize()
    # the oracle's gradient on the same inputs (its own lists and image)
    ref = oracle.render(cams, m64, p64, a64, K=K, tau=1.0, eta=eta)
    g_img = 2.0 * (ref["image"] - r32(target)) / ref["image"].size
    want = oracle.render_bwd(cams, m64, p64, a64, 1.0, ref["pix"], ref["idx"], g_img)["g_means"][lo:hi].sum(0)
    got = gt.cpu().numpy()
    assert rel_err(got, want) <= 1e-3, (got, want)
    assert got[0] < 0.0  # moving the occludee towards +x (the target) lowers the loss
    assert abs(got[0]) > 10.0 * max(abs(got[1]), 1e-12)  # mostly along x, the direction it is off by


@pytest.mark.parametrize("gap", [1.5, 5.0])
def test_optimising_the_hidden_object_reaches_the_target(gap):
    voge = lib_ready()
    sc, cams = _scene(gap, START_X)
    tsc, _ = _scene(gap, TARGET_X)
    lo, hi = sc["parts"]["occludee"]
    R = voge.Renderer(cams, sc["means"].shape[0], 3, K=sc["K"], tau=1.0, thresh=sc["eta"])
    means, inv_cov, attr = to_dev(sc["means"]), to_dev(sc["inv_cov"]), to_dev(sc["attr"])
    target, _, _ = R.forward(to_dev(tsc["means"]), inv_cov, attr)
    target = target.clone()
    base = means.clone()
    t = torch.zeros(3, device="cuda")  # translation of the occludee
    m1, v1 = torch.zeros(3, device="cuda"), torch.zeros(3, device="cuda")
    lr, b1, b2 = 0.02, 0.9, 0.999
    loss0 = None
    for step in range(1, 61):
        means.copy_(base)
        means[lo:hi] += t
        loss, g = _loss_and_grad(voge, R, means, inv_cov, attr, target, lo, hi)
        loss0 = loss if loss0 is None else loss0
        m1 = b1 * m1 + (1 - b1) * g
        v1 = b2 * v1 + (1 - b2) * g * g
        t = t - lr * (m1 / (1 - b1 ** step)) / (torch.sqrt(v1 / (1 - b2 ** step)) + 1e-12)
    torch.cuda.synchronize()
    x = START_X + float(t[0])
    assert abs(x - TARGET_X) < 0.25 * abs(START_X - TARGET_X), x
    assert loss < 0.1 * loss0
