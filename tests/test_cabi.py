"""The C ABI library builds, loads and exports every symbol include/voge.h declares.

These run on the CPU: no call here launches a kernel.  The host-only entry
points (sizes, errors, camera pose) are checked for their values.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def voge():
    from paper_2205_15401_gb300 import build

    build.build()
    from paper_2205_15401_gb300 import voge as v

    v.lib()
    return v


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(voge_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(voge):
    names = declared_symbols()
    assert "voge_render_fwd" in names and "voge_render_bwd" in names
    L = voge.lib()
    for n in names:
        assert hasattr(L, n), f"libvoge.so does not export {n}"
        assert isinstance(getattr(L, n), ctypes._CFuncPtr)


def test_library_is_built_for_sm103a():
    from paper_2205_15401_gb300 import build

    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_version_and_errors(voge):
    assert voge.voge_version() >= 100
    L = voge.lib()
    for code in range(0, -9, -1):
        assert len(L.voge_strerror(code)) > 0


def _cams(B=2, H=64, W=48):
    return [{"R": np.eye(3), "T": np.zeros(3), "F": 50.0, "Ox": W / 2, "Oy": H / 2, "H": H, "W": W} for _ in range(B)]


def test_list_length_and_workspace(voge):
    cams = voge.make_cameras(_cams())
    p = voge.make_params(2, 100, 3, 20, 1.0, 0.01)
    assert voge.voge_list_length(p) == 20
    assert voge.voge_list_length(voge.make_params(2, 10, 3, 20, 1.0, 0.01)) == 10
    assert voge.voge_list_length(voge.make_params(2, 100, 3, 0, 1.0, 0.01)) == 100
    n1 = voge.voge_workspace_bytes(cams, p)
    n2 = voge.voge_workspace_bytes(cams, voge.make_params(2, 1000, 3, 20, 1.0, 0.01))
    assert 0 < n1 < n2
    with pytest.raises(RuntimeError):
        voge.voge_workspace_bytes(cams, voge.make_params(2, 100, 3, 20, -1.0, 0.01))  # tau must be > 0
    bad = voge.make_cameras(_cams(H=0))
    with pytest.raises(RuntimeError):
        voge.voge_workspace_bytes(bad, p)


def test_invalid_arguments_rejected_without_launch(voge):
    """Argument checks run before any CUDA call: a NULL workspace is VOGE_ERR_WORKSPACE, bad sizes VOGE_ERR_ARG."""
    L = voge.lib()
    cams = voge.make_cameras(_cams())
    p = voge.make_params(2, 100, 3, 20, 1.0, 0.01)
    fake = ctypes.c_void_p(256)
    rc = L.voge_render_fwd(cams, ctypes.byref(p), fake, fake, fake, fake, None, fake, None, 0, None)
    assert rc == -2
    p_bad = voge.make_params(0, 100, 3, 20, 1.0, 0.01)
    rc = L.voge_render_fwd(cams, ctypes.byref(p_bad), fake, fake, fake, fake, None, fake, fake, 1 << 30, None)
    assert rc == -1
    rc = L.voge_render_bwd(cams, ctypes.byref(p), fake, fake, fake, fake, None, None, None, None, None, None, 0, None)
    assert rc == -1  # grad_image missing
    # fine pass on given lists
    rc = L.voge_render_fine(cams, ctypes.byref(p), fake, fake, fake, fake, fake, None, None, 0, None)
    assert rc == -2  # no workspace
    rc = L.voge_render_fine(cams, ctypes.byref(p), fake, fake, fake, fake, None, None, fake, 1 << 30, None)
    assert rc == -1  # no image
    rc = L.voge_render_fine(cams, ctypes.byref(p_bad), fake, fake, fake, fake, fake, None, fake, 1 << 30, None)
    assert rc == -1
    st = voge.voge_render_stats_t()
    assert L.voge_render_stats(None, ctypes.byref(st), None) == -1  # no workspace
    assert L.voge_render_stats(fake, None, None) == -1  # no output
    assert L.voge_render_stats(ctypes.c_void_p(260), ctypes.byref(st), None) == -1  # misaligned workspace
    p_long = voge.make_params(2, 100, 3, 40, 1.0, 0.01)
    rc = L.voge_render_fine(cams, ctypes.byref(p_long), fake, fake, fake, fake, fake, None, fake, 1 << 30, None)
    assert rc == -4  # lists longer than 32: VOGE_ERR_UNSUPPORTED, before any CUDA call


def test_helper_entry_points_check_arguments_before_any_cuda_call(voge):
    """Every entry point validates its sizes and pointers on the host before it
    touches CUDA: invalid calls return VOGE_ERR_ARG (-1) and empty ones VOGE_OK
    (0), here on a machine without a GPU."""
    L = voge.lib()
    S = voge._server_lib()
    fake = ctypes.c_void_p(256)
    # neural sampler (Eq. 10)
    assert L.voge_sample(-1, 3, 4, 2, None, None, None, None, None, None) == -1  # negative pixel count
    assert L.voge_sample(10, 3, 4, 0, None, None, None, None, None, None) == -1  # no channels
    assert L.voge_sample(10, 3, 4, 2, None, None, None, None, None, None) == -1  # missing buffers
    assert L.voge_sample(10, 3, 0, 2, fake, fake, fake, None, None, None) == 0   # no kernels: nothing to do
    # converters (App. A.4)
    assert L.voge_points_to_gaussians(10, 0, 0.5, None, None, None, None) == -1  # m < 1
    assert L.voge_points_to_gaussians(10, 10, 0.5, None, None, None, None) == -1  # m >= V
    assert L.voge_points_to_gaussians(10, 3, 1.5, None, None, None, None) == -1  # zeta outside (0, 1)
    assert L.voge_mesh_to_gaussians(4, 1, None, None, 0.5, -1.0, None, None, None, 0, None) == -1  # flatten < 0
    assert L.voge_mesh_to_gaussians(4, 1, fake, None, 0.5, 0.0, fake, fake, fake, 1 << 20, None) == -1  # no faces
    # pose gradient, loss gradient and optimiser
    assert L.voge_pose_grad(None, None, None, -1, None) == -1
    assert L.voge_pose_grad(None, None, None, 0, None) == 0
    assert L.voge_mse_grad(None, None, -1, None, None, None) == -1
    assert L.voge_mse_grad(None, None, 0, None, None, None) == 0
    assert L.voge_adam_step(fake, fake, fake, fake, 10, 0.1, 0.9, 0.999, 1e-8, 0, None) == -1  # step < 1
    assert L.voge_adam_step(None, None, None, None, 10, 0.1, 0.9, 0.999, 1e-8, 1, None) == -1  # missing buffers
    # serving: configurations and handles
    cfg = voge.voge_server_config(device=0, max_slots=4, mem_budget_bytes=1024)  # below the 1 MiB minimum
    out = ctypes.c_void_p()
    assert S.voge_server_create(ctypes.byref(cfg), ctypes.byref(out)) == -1
    cfg = voge.voge_server_config(device=0, max_slots=0, mem_budget_bytes=64 << 20)  # no slot
    assert S.voge_server_create(ctypes.byref(cfg), ctypes.byref(out)) == -1
    ticket = ctypes.c_uint64()
    assert S.voge_server_submit(None, None, ctypes.byref(ticket)) == -1
    assert S.voge_server_wait(None, 1, 0, None) == -1
    assert S.voge_server_pause(None, 1) == -1
    assert S.voge_server_remove_scene(None, 0) == -1
    assert S.voge_server_destroy(None) == -1
    assert L.voge_measure_alu_peaks(None, None) == -1


def test_pose_to_RT_matches_oracle(voge):
    rng = np.random.default_rng(0)
    for _ in range(50):
        pose = [rng.uniform(-3.1, 3.1), rng.uniform(-1.3, 1.3), rng.uniform(1, 8), rng.uniform(-0.5, 0.5)]
        R, T = voge.voge_pose_to_RT(pose)
        Ro, To = oracle.pose_to_RT(pose)
        np.testing.assert_allclose(R, Ro, atol=2e-7)
        np.testing.assert_allclose(T, To, atol=1e-6)
