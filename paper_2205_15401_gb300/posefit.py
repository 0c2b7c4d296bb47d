"""Render-and-compare pose estimation on feature maps (the pose-fitting use of
Sec. 4.1): the object's Gaussians carry features, an observed feature map is
compared with renders, and the camera pose (azimuth, elevation, distance,
roll) is fitted by gradient descent through the renderer.

Many start poses are fitted at once: they are the views of one render call,
so one forward, one MSE, one backward, one pose-gradient and one Adam launch
advance all of them.  Only the library's kernels do arithmetic; this module
orders the calls (the camera matrices of the current poses are set on the
host between steps, as the render call takes them from there).
"""
from __future__ import annotations

import numpy as np
import torch

from . import voge


class PoseFitter:
    """Fits B start poses of one scene against one observed feature map.

    means [N][3], inv_cov [N][6], attr [N][C]: the scene (device, float32).
    target [H*W][C]: the observed feature map (device, float32).
    starts: B x 4 start poses (azimuth, elevation, distance, roll), radians.
    """

    def __init__(self, means, inv_cov, attr, target, H, W, F, starts, K=20, tau=1.0, thresh=1e-3, lr=0.05,
                 device="cuda"):
        self.means, self.inv_cov, self.attr = means, inv_cov, attr
        self.H, self.W, self.F = int(H), int(W), float(F)
        starts = np.asarray(starts, dtype=np.float32).reshape(-1, 4)
        self.B = starts.shape[0]
        self.N, self.C = means.shape[0], attr.shape[1]
        self.device = torch.device(device)
        self.poses = torch.tensor(starts, device=self.device)
        self.renderer = voge.Renderer(self._cameras(starts), self.N, self.C, K=K, tau=tau, thresh=thresh,
                                      device=self.device)
        self.out = self.renderer.alloc_outputs()
        P = self.H * self.W
        assert target.shape == (P, self.C)
        self.target = target.repeat(self.B, 1).contiguous()  # every view compares with the same observation
        self.g_image = torch.empty_like(self.out[0])
        self.loss = torch.zeros(1, device=self.device)
        self.g_cam = torch.zeros((self.B, 12), device=self.device)
        self.g_pose = torch.zeros((self.B, 4), device=self.device)
        self.m = torch.zeros((self.B, 4), device=self.device)
        self.v = torch.zeros((self.B, 4), device=self.device)
        self.lr = float(lr)
        self.steps = 0

    def _cameras(self, poses):
        cams = []
        for p in np.asarray(poses, dtype=np.float64).reshape(-1, 4):
            R, T = voge.voge_pose_to_RT(p)
            cams.append({"R": R, "T": T, "F": self.F, "Ox": self.W / 2.0, "Oy": self.H / 2.0, "H": self.H,
                         "W": self.W})
        return cams

    def step(self):
        """One fitting step of every start: render, MSE, backward to the
        cameras, chain to the pose parameters, Adam.  Returns the summed loss
        (a device scalar; reading it synchronises)."""
        self.renderer.set_cameras(self._cameras(self.poses.cpu().numpy()))
        image, weights, index = self.renderer.forward(self.means, self.inv_cov, self.attr, out=self.out)
        self.loss.zero_()
        voge.voge_mse_grad(image, self.target, self.g_image, self.loss)
        self.g_cam.zero_()
        self.renderer.backward(self.means, self.inv_cov, self.attr, index, self.g_image, grad_cam=self.g_cam,
                               weights=weights)
        voge.voge_pose_grad(self.poses, self.g_cam, self.g_pose)
        self.steps += 1
        voge.voge_adam_step(self.poses, self.g_pose, self.m, self.v, self.lr, self.steps)
        return self.loss

    def view_losses(self):
        """Mean squared feature error of each start at its current pose."""
        self.renderer.set_cameras(self._cameras(self.poses.cpu().numpy()))
        image, _, _ = self.renderer.forward(self.means, self.inv_cov, self.attr, out=self.out)
        P = self.H * self.W
        losses = torch.zeros(self.B, device=self.device)
        for b in range(self.B):
            sl = slice(b * P, (b + 1) * P)
            voge.voge_mse_grad(image[sl], self.target[sl], self.g_image[sl], losses[b:b + 1])
        return losses

    def run(self, steps):
        """`steps` fitting steps, then (best pose [4] on the host, per-start losses [B])."""
        for _ in range(steps):
            self.step()
        losses = self.view_losses().cpu().numpy()
        best = int(np.argmin(losses))
        return self.poses[best].cpu().numpy().astype(np.float64), losses
