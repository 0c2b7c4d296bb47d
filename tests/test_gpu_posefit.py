"""Feature-level render-and-compare pose fitting (Sec. 4.1 use): many start
poses as the views of one render call, fitted together."""
import numpy as np
import pytest
import torch

import oracle
from paper_2205_15401_gb300 import scenes
from paper_2205_15401_gb300.posefit import PoseFitter

from gpu_util import lib_ready, r32, to_dev
from parity import rel_err

pytestmark = pytest.mark.gpu


def _setup(side=64, C=16, seed=0):
    voge = lib_ready()
    sc = scenes.posefit_256(seed=seed, N=4000, C=C)
    true = sc["poses"][0]
    m, p, a = to_dev(sc["means"]), to_dev(sc["inv_cov"]), to_dev(sc["attr"])
    R, T = voge.voge_pose_to_RT(true)
    cam = {"R": R, "T": T, "F": float(side), "Ox": side / 2, "Oy": side / 2, "H": side, "W": side}
    target = voge.Renderer([cam], sc["means"].shape[0], C, K=20, tau=1.0, thresh=1e-3).forward(m, p, a)[0].clone()
    return voge, sc, true, (m, p, a), target


def test_starts_near_the_truth_converge_and_the_best_is_found():
    voge, sc, true, (m, p, a), target = _setup()
    rng = np.random.default_rng(7)
    scale = np.array([0.3, 0.15, 0.3, 0.05])
    near = true + rng.uniform(-1, 1, (6, 4)) * scale
    far = true + rng.uniform(-1, 1, (2, 4)) * np.array([2.5, 0.8, 1.0, 0.3])
    fitter = PoseFitter(m, p, a, target, 64, 64, 64.0, np.concatenate([far, near]), lr=0.02)
    losses0 = fitter.view_losses().cpu().numpy()
    best, losses = fitter.run(150)
    err = np.abs(best - true)
    assert err[0] < 0.01 and err[1] < 0.01 and err[2] < 0.02 and err[3] < 0.01, err
    assert losses.min() < 1e-3 * losses0[2:].min()
    # the near starts all ended at the truth
    final = fitter.poses.cpu().numpy()[2:]
    assert np.abs(final[:, :2] - true[:2]).max() < 0.01


def test_pose_gradient_of_a_fitting_step_matches_oracle():
    """dL/d(azimuth, elevation, distance, roll) of each start, from one
    forward/backward of the fitter's batch, against the FP64 oracle."""
    voge = lib_ready()
    side, C = 40, 8
    sc = scenes.posefit_256(seed=3, N=1500, C=C)
    true = sc["poses"][0]
    starts = true + np.array([[0.1, -0.05, 0.2, 0.02], [-0.15, 0.04, -0.1, -0.03]])
    m64, p64, a64 = (sc[k].astype(np.float64) for k in ("means", "inv_cov", "attr"))
    cam_of = lambda pose: dict(zip(("R", "T"), oracle.pose_to_RT(pose)), F=float(side), Ox=side / 2, Oy=side / 2,
                               H=side, W=side)
    tgt = r32(oracle.render([cam_of(true)], m64, p64, a64, K=20, tau=1.0, eta=1e-3)["image"])
    fitter = PoseFitter(to_dev(sc["means"]), to_dev(sc["inv_cov"]), to_dev(sc["attr"]), to_dev(tgt), side, side,
                        float(side), starts, lr=0.0)
    fitter.renderer.set_cameras(fitter._cameras(starts))
    image, w, idx = fitter.renderer.forward(fitter.means, fitter.inv_cov, fitter.attr, out=fitter.out)
    fitter.loss.zero_()
    voge.voge_mse_grad(image, fitter.target, fitter.g_image, fitter.loss)
    fitter.g_cam.zero_()
    fitter.renderer.backward(fitter.means, fitter.inv_cov, fitter.attr, idx, fitter.g_image, grad_cam=fitter.g_cam,
                             weights=w)
    voge.voge_pose_grad(fitter.poses, fitter.g_cam, fitter.g_pose)
    torch.cuda.synchronize()
    got = fitter.g_pose.cpu().numpy()
    cams = [cam_of(s) for s in starts]
    ref = oracle.render(cams, m64, p64, a64, K=20, tau=1.0, eta=1e-3)
    n = ref["image"].size
    g_img = 2.0 * (ref["image"] - np.tile(tgt, (2, 1))) / n
    bwd = oracle.render_bwd(cams, m64, p64, a64, 1.0, ref["pix"], ref["idx"], g_img)
    for b in range(2):
        want = oracle.pose_grad(starts[b], bwd["g_R"][b], bwd["g_T"][b])
        assert rel_err(got[b], want) <= 2e-3, (b, got[b], want)
