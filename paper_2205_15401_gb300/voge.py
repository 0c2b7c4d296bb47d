"""Python binding of libvoge.so: argument marshalling only.

Every function named ``voge_*`` mirrors the C entry point of the same name in
``include/voge.h``: it converts torch tensors to device pointers, the current
torch stream to a ``cudaStream_t`` and camera dicts to ``voge_camera``
structs, and calls the library.  There is no fallback: if ``libvoge.so`` has
not been built, or a call fails, a RuntimeError is raised.

On top of the binding sit ``Renderer`` (workspace management) and
``VoGERender`` (a ``torch.autograd.Function`` whose forward is
``voge_render_fwd`` and whose backward is ``voge_render_bwd_w``; it saves the
per-pixel index lists and weights).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import threading

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libvoge.so")
CHECKED_LIB_PATH = os.path.join(_PKG, "libvoge_checked.so")
_lock = threading.Lock()
_libs = {}
_use_checked = False

VOGE_OK = 0
VOGE_FLAG_PLAIN = 1
VOGE_FLAG_REUSE_PROJECTION = 2
VOGE_FLAG_SPLIT_FORWARD = 4


class voge_camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("T", ctypes.c_float * 3), ("F", ctypes.c_float),
                ("Ox", ctypes.c_float), ("Oy", ctypes.c_float), ("H", ctypes.c_int32), ("W", ctypes.c_int32)]


class voge_trace_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class voge_alu_peaks(ctypes.Structure):
    _fields_ = [("fma_tflops", ctypes.c_double), ("ex2_tops", ctypes.c_double), ("fwd_gpairs", ctypes.c_double),
                ("bwd_gpairs", ctypes.c_double), ("ms", ctypes.c_double * 4), ("sms", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class voge_render_stats_t(ctypes.Structure):
    _fields_ = [("traces", ctypes.c_int64), ("entries", ctypes.c_int64), ("pairs", ctypes.c_int64)]


class voge_params(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int32), ("N", ctypes.c_int32), ("C", ctypes.c_int32), ("K", ctypes.c_int32),
                ("tau", ctypes.c_float), ("thresh", ctypes.c_float), ("flags", ctypes.c_int32),
                ("bin_capacity", ctypes.c_int32)]


def lib():
    """Load libvoge.so (built in-tree), or libvoge_checked.so inside
    checked_library(); raises if it is missing."""
    path = CHECKED_LIB_PATH if _use_checked else LIB_PATH
    with _lock:
        if path not in _libs:
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with paper_2205_15401_gb300.build.build()")
            L = ctypes.CDLL(path)
            vp, P = ctypes.c_void_p, ctypes.POINTER
            L.voge_version.restype = ctypes.c_int
            L.voge_strerror.restype = ctypes.c_char_p
            L.voge_strerror.argtypes = [ctypes.c_int]
            L.voge_list_length.argtypes = [P(voge_params)]
            L.voge_list_length.restype = ctypes.c_int
            L.voge_workspace_bytes.argtypes = [P(voge_camera), P(voge_params)]
            L.voge_workspace_bytes.restype = ctypes.c_size_t
            L.voge_render_fwd.argtypes = [P(voge_camera), P(voge_params), vp, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
            L.voge_render_fwd.restype = ctypes.c_int
            L.voge_render_stats.argtypes = [vp, P(voge_render_stats_t), vp]
            L.voge_render_stats.restype = ctypes.c_int
            L.voge_render_fine.argtypes = [P(voge_camera), P(voge_params), vp, vp, vp, vp, vp, vp, vp, ctypes.c_size_t,
                                           vp]
            L.voge_render_fine.restype = ctypes.c_int
            L.voge_render_bwd.argtypes = [P(voge_camera), P(voge_params), vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                          ctypes.c_size_t, vp]
            L.voge_render_bwd.restype = ctypes.c_int
            L.voge_render_bwd_w.argtypes = [P(voge_camera), P(voge_params), vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                            vp, ctypes.c_size_t, vp]
            L.voge_render_bwd_w.restype = ctypes.c_int
            L.voge_sample.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp, vp, vp, vp, vp,
                                      vp]
            L.voge_sample.restype = ctypes.c_int
            L.voge_mesh_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int32]
            L.voge_mesh_workspace_bytes.restype = ctypes.c_size_t
            L.voge_mesh_to_gaussians.argtypes = [ctypes.c_int32, ctypes.c_int32, vp, vp, ctypes.c_float,
                                                 ctypes.c_float, vp, vp, vp, ctypes.c_size_t, vp]
            L.voge_mesh_to_gaussians.restype = ctypes.c_int
            L.voge_points_to_gaussians.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_float, vp, vp, vp, vp]
            L.voge_points_to_gaussians.restype = ctypes.c_int
            L.voge_pose_to_RT.argtypes = [P(ctypes.c_double), P(ctypes.c_float), P(ctypes.c_float)]
            L.voge_pose_to_RT.restype = None
            L.voge_pose_grad.argtypes = [vp, vp, vp, ctypes.c_int32, vp]
            L.voge_pose_grad.restype = ctypes.c_int
            L.voge_mse_grad.argtypes = [vp, vp, ctypes.c_int64, vp, vp, vp]
            L.voge_mse_grad.restype = ctypes.c_int
            L.voge_adam_step.argtypes = [vp, vp, vp, vp, ctypes.c_int64, ctypes.c_float, ctypes.c_float,
                                         ctypes.c_float, ctypes.c_float, ctypes.c_int32, vp]
            L.voge_adam_step.restype = ctypes.c_int
            L.voge_render_fwd_static.argtypes = [P(voge_camera), P(voge_params), vp, vp, vp, vp, vp, vp, vp]
            L.voge_render_fwd_static.restype = ctypes.c_int
            L.voge_trace_enable.argtypes = [ctypes.c_int]
            L.voge_trace_enable.restype = ctypes.c_int
            L.voge_trace_read.argtypes = [P(voge_trace_entry), ctypes.c_int]
            L.voge_trace_read.restype = ctypes.c_int
            L.voge_trace_reset.restype = None
            L.voge_measure_alu_peaks.argtypes = [P(voge_alu_peaks), vp]
            L.voge_measure_alu_peaks.restype = ctypes.c_int
            _libs[path] = L
    return _libs[path]


@contextlib.contextmanager
def checked_library():
    """Within the block every binding call goes to libvoge_checked.so (built by
    build.build(checked=True)): the tile kernels check their gather and
    scatter indices, and a failed check raises (VOGE_ERR_CHECK)."""
    global _use_checked
    prev = _use_checked
    _use_checked = True
    try:
        yield
    finally:
        _use_checked = prev


def _check(rc, what):
    if rc != VOGE_OK:
        raise RuntimeError(f"{what} failed: {lib().voge_strerror(rc).decode()} ({rc})")


def _ptr(t, dtype=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_cameras(cams):
    """List of dicts (R 3x3, T 3, F, Ox, Oy, H, W) -> ctypes array of voge_camera."""
    arr = (voge_camera * len(cams))()
    for v, c in enumerate(cams):
        R = np.asarray(c["R"], dtype=np.float32).reshape(9)
        T = np.asarray(c["T"], dtype=np.float32).reshape(3)
        for q in range(9):
            arr[v].R[q] = float(R[q])
        for q in range(3):
            arr[v].T[q] = float(T[q])
        arr[v].F, arr[v].Ox, arr[v].Oy = float(c["F"]), float(c["Ox"]), float(c["Oy"])
        arr[v].H, arr[v].W = int(c["H"]), int(c["W"])
    return arr


def make_params(B, N, C, K, tau, thresh, flags=0, bin_capacity=0):
    return voge_params(int(B), int(N), int(C), int(K), float(tau), float(thresh), int(flags), int(bin_capacity))


# ----------------------------------------------------------------- C ABI ---
def voge_version():
    return int(lib().voge_version())


def voge_list_length(params):
    return int(lib().voge_list_length(ctypes.byref(params)))


def voge_workspace_bytes(cams, params):
    n = lib().voge_workspace_bytes(cams, ctypes.byref(params))
    if n == 0:
        raise RuntimeError("voge_workspace_bytes: invalid cameras or parameters")
    return int(n)


def voge_render_fwd(cams, params, means, inv_cov, attr, image, weights, index, workspace, stream=None):
    f32, i32 = torch.float32, torch.int32
    rc = lib().voge_render_fwd(cams, ctypes.byref(params), _ptr(means, f32), _ptr(inv_cov, f32), _ptr(attr, f32),
                               _ptr(image, f32), _ptr(weights, f32), _ptr(index, i32), _ptr(workspace),
                               workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "voge_render_fwd")


def voge_render_stats(workspace, stream=None):
    """Counts of the last forward pass run in ``workspace``: a dict of
    traces (coarse-pass Gaussian-ray traces), entries and pairs."""
    st = voge_render_stats_t()
    _check(lib().voge_render_stats(_ptr(workspace), ctypes.byref(st), _stream(stream)), "voge_render_stats")
    return {"traces": int(st.traces), "entries": int(st.entries), "pairs": int(st.pairs)}


def voge_render_fine(cams, params, means, inv_cov, attr, index, image, weights, workspace, stream=None):
    """Fine pass (Eq. 7-8) over given per-pixel lists ``index`` [P][L]."""
    f32, i32 = torch.float32, torch.int32
    rc = lib().voge_render_fine(cams, ctypes.byref(params), _ptr(means, f32), _ptr(inv_cov, f32), _ptr(attr, f32),
                                _ptr(index, i32), _ptr(image, f32), _ptr(weights, f32), _ptr(workspace),
                                workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "voge_render_fine")


def voge_render_bwd(cams, params, means, inv_cov, attr, index, grad_image, grad_means, grad_inv_cov, grad_attr,
                    grad_cam, workspace, stream=None):
    f32, i32 = torch.float32, torch.int32
    rc = lib().voge_render_bwd(cams, ctypes.byref(params), _ptr(means, f32), _ptr(inv_cov, f32), _ptr(attr, f32),
                               _ptr(index, i32), _ptr(grad_image, f32), _ptr(grad_means, f32),
                               _ptr(grad_inv_cov, f32), _ptr(grad_attr, f32), _ptr(grad_cam, f32),
                               _ptr(workspace), workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "voge_render_bwd")


def voge_render_bwd_w(cams, params, means, inv_cov, attr, index, weights, grad_image, grad_means, grad_inv_cov,
                      grad_attr, grad_cam, workspace, stream=None):
    """voge_render_bwd taking the forward's weights (or None to recompute them)."""
    f32, i32 = torch.float32, torch.int32
    rc = lib().voge_render_bwd_w(cams, ctypes.byref(params), _ptr(means, f32), _ptr(inv_cov, f32), _ptr(attr, f32),
                                 _ptr(index, i32), _ptr(weights, f32), _ptr(grad_image, f32), _ptr(grad_means, f32),
                                 _ptr(grad_inv_cov, f32), _ptr(grad_attr, f32), _ptr(grad_cam, f32),
                                 _ptr(workspace), workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "voge_render_bwd_w")


def voge_sample(index, weights, features, N, alpha=None, wsum=None, stream=None):
    """Neural sampler (Sec. 3.4 Eq. 10): (alpha [N][C], wsum [N]) from the
    renderer's index [P][L] / weights [P][L] and per-pixel features [P][C]."""
    f32, i32 = torch.float32, torch.int32
    P, L = index.shape
    C = features.shape[1]
    if alpha is None:
        alpha = torch.empty((N, C), dtype=f32, device=features.device)
    if wsum is None:
        wsum = torch.empty((N,), dtype=f32, device=features.device)
    rc = lib().voge_sample(P, L, N, C, _ptr(index, i32), _ptr(weights, f32), _ptr(features, f32), _ptr(alpha, f32),
                           _ptr(wsum, f32), _stream(stream))
    _check(rc, "voge_sample")
    return alpha, wsum


def voge_mesh_to_gaussians(verts, faces, zeta=0.5, flatten=0.0, stream=None):
    """Mesh converter (App. A.4): (means [V][3], inv_cov [V][6]) on the device."""
    f32, i32 = torch.float32, torch.int32
    V, F = verts.shape[0], faces.shape[0]
    means = torch.empty((V, 3), dtype=f32, device=verts.device)
    inv_cov = torch.empty((V, 6), dtype=f32, device=verts.device)
    nbytes = lib().voge_mesh_workspace_bytes(V, F)
    ws = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=verts.device)
    _check(lib().voge_mesh_to_gaussians(V, F, _ptr(verts, f32), _ptr(faces, i32), float(zeta), float(flatten),
                                        _ptr(means, f32), _ptr(inv_cov, f32), _ptr(ws), ws.numel(), _stream(stream)),
           "voge_mesh_to_gaussians")
    return means, inv_cov


def voge_points_to_gaussians(points, m=4, zeta=0.5, stream=None):
    """Point-cloud converter (App. A.4): (means [V][3], inv_cov [V][6]) on the device."""
    f32 = torch.float32
    V = points.shape[0]
    means = torch.empty((V, 3), dtype=f32, device=points.device)
    inv_cov = torch.empty((V, 6), dtype=f32, device=points.device)
    _check(lib().voge_points_to_gaussians(V, int(m), float(zeta), _ptr(points, f32), _ptr(means, f32),
                                          _ptr(inv_cov, f32), _stream(stream)), "voge_points_to_gaussians")
    return means, inv_cov


def voge_render_fwd_static(cams, params, means, inv_cov, attr, image, weights, index, stream=None):
    """voge_render_fwd without a workspace argument (library-held workspace; see include/voge.h)."""
    f32, i32 = torch.float32, torch.int32
    rc = lib().voge_render_fwd_static(cams, ctypes.byref(params), _ptr(means, f32), _ptr(inv_cov, f32),
                                      _ptr(attr, f32), _ptr(image, f32), _ptr(weights, f32), _ptr(index, i32),
                                      _stream(stream))
    _check(rc, "voge_render_fwd_static")


def voge_pose_to_RT(pose):
    p = (ctypes.c_double * 4)(*[float(x) for x in np.asarray(pose, dtype=np.float64).reshape(4)])
    R = (ctypes.c_float * 9)()
    T = (ctypes.c_float * 3)()
    lib().voge_pose_to_RT(p, R, T)
    return np.array(R[:], np.float32).reshape(3, 3), np.array(T[:], np.float32)


def voge_pose_grad(pose, grad_cam, grad_pose, stream=None):
    B = pose.shape[0]
    f32 = torch.float32
    _check(lib().voge_pose_grad(_ptr(pose, f32), _ptr(grad_cam, f32), _ptr(grad_pose, f32), B, _stream(stream)),
           "voge_pose_grad")


def voge_mse_grad(image, target, grad_image, loss, stream=None):
    f32 = torch.float32
    _check(lib().voge_mse_grad(_ptr(image, f32), _ptr(target, f32), image.numel(), _ptr(grad_image, f32),
                               _ptr(loss, f32), _stream(stream)), "voge_mse_grad")


def voge_adam_step(param, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    f32 = torch.float32
    _check(lib().voge_adam_step(_ptr(param, f32), _ptr(grad, f32), _ptr(m, f32), _ptr(v, f32), param.numel(),
                                float(lr), float(beta1), float(beta2), float(eps), int(step), _stream(stream)),
           "voge_adam_step")


def voge_trace_enable(on=True):
    return bool(lib().voge_trace_enable(1 if on else 0))


def voge_trace_read():
    """{kernel name: (launches, total device ms)} accumulated since the last reset."""
    buf = (voge_trace_entry * 64)()
    n = lib().voge_trace_read(buf, 64)
    return {buf[q].name.decode(): (int(buf[q].launches), float(buf[q].total_ms)) for q in range(min(n, 64))}


def voge_trace_reset():
    lib().voge_trace_reset()


def voge_measure_alu_peaks(stream=None):
    """Measured arithmetic ceilings of the current GPU (register-only loops on
    every SM, about 0.2 s): FP32 FMA TFLOP/s, MUFU ex2 rate (10^12/s), and the
    forward and backward pair terms of Eq. 7 in 10^9 pairs/s."""
    out = voge_alu_peaks()
    _check(lib().voge_measure_alu_peaks(ctypes.byref(out), _stream(stream)), "voge_measure_alu_peaks")
    return {"fma_tflops": out.fma_tflops, "ex2_tops": out.ex2_tops, "fwd_gpairs": out.fwd_gpairs,
            "bwd_gpairs": out.bwd_gpairs, "ms": list(out.ms), "sms": int(out.sms)}


# -------------------------------------------------------------- helpers ---
def cameras_from_poses(poses, F, H, W):
    """Camera dicts for poses (azim, elev, dist, roll) through voge_pose_to_RT."""
    out = []
    for p in np.asarray(poses, dtype=np.float64).reshape(-1, 4):
        R, T = voge_pose_to_RT(p)
        out.append({"R": R, "T": T, "F": float(F), "Ox": W / 2.0, "Oy": H / 2.0, "H": int(H), "W": int(W)})
    return out


class Renderer:
    """Cameras + parameters + a cached device workspace for repeated renders."""

    def __init__(self, cams, N, C, K=20, tau=1.0, thresh=0.01, flags=0, bin_capacity=0, device="cuda"):
        self.cam_list = list(cams)
        self.cams = make_cameras(self.cam_list)
        self.params = make_params(len(self.cam_list), N, C, K, tau, thresh, flags, bin_capacity)
        self.L = voge_list_length(self.params)
        self.pixels = sum(int(c["H"]) * int(c["W"]) for c in self.cam_list)
        self.device = torch.device(device)
        nbytes = voge_workspace_bytes(self.cams, self.params)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)

    def set_cameras(self, cams):
        self.cam_list = list(cams)
        assert len(self.cam_list) == self.params.B
        self.cams = make_cameras(self.cam_list)
        nbytes = voge_workspace_bytes(self.cams, self.params)
        if nbytes > self.workspace.numel():
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)

    def alloc_outputs(self):
        P, C, L = self.pixels, self.params.C, self.L
        image = torch.empty((P, C), dtype=torch.float32, device=self.device)
        weights = torch.empty((P, max(L, 1)), dtype=torch.float32, device=self.device)
        index = torch.empty((P, max(L, 1)), dtype=torch.int32, device=self.device)
        return image, weights, index

    def forward(self, means, inv_cov, attr, out=None, flags=None):
        image, weights, index = out if out is not None else self.alloc_outputs()
        params = self.params if flags is None else make_params(self.params.B, self.params.N, self.params.C,
                                                               self.params.K, self.params.tau, self.params.thresh,
                                                               flags, self.params.bin_capacity)
        voge_render_fwd(self.cams, params, means, inv_cov, attr, image, weights, index, self.workspace)
        return image, weights, index

    def fine(self, means, inv_cov, attr, index, image=None, weights=None):
        """Fine pass alone over given lists index [P][L] (voge_render_fine)."""
        if image is None:
            image = torch.empty((self.pixels, self.params.C), dtype=torch.float32, device=self.device)
        voge_render_fine(self.cams, self.params, means, inv_cov, attr, index, image, weights, self.workspace)
        return image, weights

    def backward(self, means, inv_cov, attr, index, grad_image, grad_means=None, grad_inv_cov=None, grad_attr=None,
                 grad_cam=None, reuse_projection=False, weights=None):
        """Accumulate gradients.  ``weights``: the forward's weights output for
        the same ``index`` (skips recomputing W), or None."""
        params = self.params
        if reuse_projection:
            params = make_params(params.B, params.N, params.C, params.K, params.tau, params.thresh,
                                 params.flags | VOGE_FLAG_REUSE_PROJECTION, params.bin_capacity)
        if weights is None:
            voge_render_bwd(self.cams, params, means, inv_cov, attr, index, grad_image, grad_means, grad_inv_cov,
                            grad_attr, grad_cam, self.workspace)
        else:
            voge_render_bwd_w(self.cams, params, means, inv_cov, attr, index, weights, grad_image, grad_means,
                              grad_inv_cov, grad_attr, grad_cam, self.workspace)


class VoGERender(torch.autograd.Function):
    """image = VoGERender.apply(means, inv_cov, attr, renderer, cam_grad_holder).

    Gradients flow to means [N,3], inv_cov [N,6] and attr [N,C].  If
    ``cam_grad_holder`` is a tensor of shape [B,12], dL/d(R,T) of each view is
    accumulated into it during backward (for pose fitting)."""

    @staticmethod
    def forward(ctx, means, inv_cov, attr, renderer, cam_grad=None):
        means, inv_cov, attr = means.contiguous(), inv_cov.contiguous(), attr.contiguous()
        image, weights, index = renderer.forward(means, inv_cov, attr)
        ctx.renderer = renderer
        ctx.cam_grad = cam_grad
        ctx.save_for_backward(means, inv_cov, attr, index, weights)
        ctx.mark_non_differentiable(weights, index)
        return image, weights, index

    @staticmethod
    def backward(ctx, grad_image, grad_w=None, grad_i=None):
        means, inv_cov, attr, index, weights = ctx.saved_tensors
        r = ctx.renderer
        gm = torch.zeros_like(means) if ctx.needs_input_grad[0] else None
        gp = torch.zeros_like(inv_cov) if ctx.needs_input_grad[1] else None
        ga = torch.zeros_like(attr) if ctx.needs_input_grad[2] else None
        if grad_image is None:
            return gm, gp, ga, None, None
        r.backward(means, inv_cov, attr, index, grad_image.contiguous(), gm, gp, ga, ctx.cam_grad, weights=weights)
        return gm, gp, ga, None, None


def render(means, inv_cov, attr, renderer, cam_grad=None):
    """Differentiable render; returns (image [P,C], weights [P,L], index [P,L])."""
    return VoGERender.apply(means, inv_cov, attr, renderer, cam_grad)


# --------------------------------------------------------------- serving ---
class voge_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_slots", ctypes.c_int32), ("max_queue", ctypes.c_int32),
                ("use_graphs", ctypes.c_int32), ("batching", ctypes.c_int32), ("inflight_ticks", ctypes.c_int32),
                ("max_tick_gaussians", ctypes.c_int64), ("max_tick_pixels", ctypes.c_int64),
                ("mem_budget_bytes", ctypes.c_size_t)]


class voge_request(ctypes.Structure):
    _fields_ = [("cam", voge_camera), ("scene", ctypes.c_int32), ("N", ctypes.c_int32), ("C", ctypes.c_int32),
                ("K", ctypes.c_int32), ("tau", ctypes.c_float), ("thresh", ctypes.c_float),
                ("means", ctypes.c_void_p), ("inv_cov", ctypes.c_void_p), ("attr", ctypes.c_void_p),
                ("target", ctypes.c_void_p), ("image", ctypes.c_void_p), ("grad_means", ctypes.c_void_p),
                ("grad_inv_cov", ctypes.c_void_p), ("grad_attr", ctypes.c_void_p), ("grad_cam", ctypes.c_void_p),
                ("loss", ctypes.c_void_p)]


class voge_request_timing(ctypes.Structure):
    _fields_ = [("submit_us", ctypes.c_double), ("admit_us", ctypes.c_double), ("start_us", ctypes.c_double),
                ("done_us", ctypes.c_double), ("tick", ctypes.c_int32), ("status", ctypes.c_int32)]


class voge_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("ticks", ctypes.c_int64), ("requests_in_ticks", ctypes.c_int64),
                ("graphs_captured", ctypes.c_int64), ("queued", ctypes.c_int64), ("resident", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


def _server_lib():
    L = lib()
    if not getattr(L, "_server_bound", False):
        P, vp = ctypes.POINTER, ctypes.c_void_p
        L.voge_server_create.argtypes = [P(voge_server_config), P(vp)]
        L.voge_server_create.restype = ctypes.c_int
        L.voge_server_submit.argtypes = [vp, P(voge_request), P(ctypes.c_uint64)]
        L.voge_server_submit.restype = ctypes.c_int
        L.voge_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_int32, P(voge_request_timing)]
        L.voge_server_wait.restype = ctypes.c_int
        L.voge_server_get_stats.argtypes = [vp, P(voge_server_stats)]
        L.voge_server_get_stats.restype = ctypes.c_int
        L.voge_server_add_scene.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, vp, vp, vp, P(ctypes.c_int32)]
        L.voge_server_add_scene.restype = ctypes.c_int
        L.voge_server_remove_scene.argtypes = [vp, ctypes.c_int32]
        L.voge_server_remove_scene.restype = ctypes.c_int
        L.voge_server_pause.argtypes = [vp, ctypes.c_int32]
        L.voge_server_pause.restype = ctypes.c_int
        L.voge_server_destroy.argtypes = [vp]
        L.voge_server_destroy.restype = ctypes.c_int
        L._server_bound = True
    return L


def _host_ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"] and t.dtype == np.float32
        return ctypes.c_void_p(t.ctypes.data)
    assert isinstance(t, torch.Tensor) and not t.is_cuda and t.is_contiguous() and t.dtype == torch.float32
    return ctypes.c_void_p(t.data_ptr())


class Server:
    """voge_server_* through ctypes.  Host arrays of a request (numpy float32 or
    CPU torch tensors, preferably pinned) are kept referenced until its wait."""

    def __init__(self, mem_budget_bytes=8 << 30, max_slots=64, use_graphs=True, batching=True, inflight_ticks=2,
                 max_tick_gaussians=0, max_tick_pixels=0, max_queue=0, device=None):
        L = _server_lib()
        dev = torch.cuda.current_device() if device is None else int(device)
        cfg = voge_server_config(dev, int(max_slots), int(max_queue), int(bool(use_graphs)), int(bool(batching)),
                                 int(inflight_ticks), int(max_tick_gaussians), int(max_tick_pixels),
                                 int(mem_budget_bytes))
        h = ctypes.c_void_p()
        _check(L.voge_server_create(ctypes.byref(cfg), ctypes.byref(h)), "voge_server_create")
        self.h = h
        self.keep = {}

    def add_scene(self, means, inv_cov, attr):
        m, p, a = (np.ascontiguousarray(x, dtype=np.float32) for x in (means, inv_cov, attr))
        sid = ctypes.c_int32()
        _check(_server_lib().voge_server_add_scene(self.h, m.shape[0], a.shape[1], _host_ptr(m), _host_ptr(p),
                                                     _host_ptr(a), ctypes.byref(sid)), "voge_server_add_scene")
        return int(sid.value)

    def remove_scene(self, sid):
        return int(_server_lib().voge_server_remove_scene(self.h, int(sid)))

    def submit(self, cam, target, K, tau=1.0, thresh=0.01, scene=-1, means=None, inv_cov=None, attr=None,
               outputs=None):
        """outputs: dict of host buffers image / grad_means / grad_inv_cov / grad_attr / grad_cam / loss."""
        outputs = outputs or {}
        req = voge_request()
        req.cam = make_cameras([cam])[0]
        req.scene = int(scene)
        if scene < 0:
            req.N, req.C = int(means.shape[0]), int(attr.shape[1])
        req.K, req.tau, req.thresh = int(K), float(tau), float(thresh)
        req.means, req.inv_cov, req.attr = _host_ptr(means), _host_ptr(inv_cov), _host_ptr(attr)
        req.target = _host_ptr(target)
        for k in ("image", "grad_means", "grad_inv_cov", "grad_attr", "grad_cam", "loss"):
            setattr(req, k, _host_ptr(outputs.get(k)))
        t = ctypes.c_uint64()
        rc = _server_lib().voge_server_submit(self.h, ctypes.byref(req), ctypes.byref(t))
        if rc != VOGE_OK:
            return rc, None
        self.keep[int(t.value)] = (target, means, inv_cov, attr, outputs)
        return rc, int(t.value)

    def wait(self, ticket, timeout_ms=-1):
        tm = voge_request_timing()
        rc = _server_lib().voge_server_wait(self.h, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(tm))
        if rc != -5:  # VOGE_ERR_TIMEOUT keeps the ticket alive
            self.keep.pop(ticket, None)
        return rc, {"submit_us": tm.submit_us, "admit_us": tm.admit_us, "start_us": tm.start_us,
                    "done_us": tm.done_us, "tick": tm.tick, "status": tm.status}

    def pause(self, paused=True):
        _check(_server_lib().voge_server_pause(self.h, int(bool(paused))), "voge_server_pause")

    def stats(self):
        st = voge_server_stats()
        _check(_server_lib().voge_server_get_stats(self.h, ctypes.byref(st)), "voge_server_get_stats")
        return {k: int(getattr(st, k)) for k, _ in voge_server_stats._fields_ if k != "pad"}

    def close(self):
        if self.h:
            _server_lib().voge_server_destroy(self.h)
            self.h = None
            self.keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
