"""The no-allocation forward entry point, checked against voge_render_fwd.

voge_render_fwd_static serves callers that cannot allocate device memory where
they render (a real-time loop whose device memory budget is fixed up front, a
program without an allocator of its own): it uses a workspace held inside the
library instead of one the caller passes.  Its results must equal those of the
ordinary entry point, call after call, although every call shares (and
reuses) that one library-held workspace, left behind by calls of other shapes
and other code paths.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL_IMAGE = 1e-4  # the image tolerance of the parity tests


def _scene(seed, N, side, B):
    import oracle
    from paper_2205_15401_gb300 import scenes

    sc = scenes.fit_8x512(seed=seed, N=N, B=B, side=side)
    cams = scenes.cameras(sc, oracle.pose_to_RT)
    inv_cov = (sc["inv_cov"] / 16.0).astype(np.float32)  # wider kernels at these small sizes
    return cams, sc["means"], inv_cov, sc["attr"]


def _voge():
    from paper_2205_15401_gb300 import build

    build.build()
    from paper_2205_15401_gb300 import voge

    return voge


def _static_equals_workspace_path(voge, seed, N, side, B, K, eta, flags=0):
    cams, means, inv_cov, attr = _scene(seed, N, side, B)
    r = voge.Renderer(cams, N, 3, K=K, tau=1.0, thresh=eta, flags=flags)
    assert voge.voge_workspace_bytes(r.cams, r.params) <= (32 << 20)
    m, p, a = (torch.tensor(x, device="cuda") for x in (means, inv_cov, attr))
    img_ref, w_ref, idx_ref = r.forward(m, p, a)
    img, w, idx = r.alloc_outputs()
    img.fill_(-7.0)
    w.fill_(-7.0)
    idx.fill_(-7)
    voge.voge_render_fwd_static(r.cams, r.params, m, p, a, img, w, idx)
    torch.cuda.synchronize()
    L = r.L
    assert torch.equal(idx[:, :L], idx_ref[:, :L])
    assert float((img - img_ref).abs().max()) <= TOL_IMAGE
    assert float((w[:, :L] - w_ref[:, :L]).abs().max()) <= TOL_IMAGE
    assert int((idx_ref[:, :L] >= 0).sum()) > 0


def test_static_workspace_matches_workspace_path_twice():
    """Two calls in a row of different shapes on the tiled register-list path."""
    voge = _voge()
    for seed, N, side, B, K, eta in [(21, 3000, 96, 2, 20, 0.01), (22, 1200, 64, 3, 8, 0.02)]:
        _static_equals_workspace_path(voge, seed, N, side, B, K, eta)


def test_static_workspace_generic_and_plain_paths():
    """The layouts that use the shared array differently: the generic path
    (lists longer than 32, per-pixel lists kept in the workspace) and the
    plain comparator (no tile counters cleared), each right after a call of
    another shape and path left its contents behind."""
    voge = _voge()
    from paper_2205_15401_gb300.voge import VOGE_FLAG_PLAIN

    _static_equals_workspace_path(voge, 23, 2500, 80, 2, 20, 0.01)
    _static_equals_workspace_path(voge, 24, 300, 48, 2, 40, 0.01)  # generic: K > 32
    _static_equals_workspace_path(voge, 25, 200, 40, 1, 0, 0.0)  # generic: K = all, no threshold
    _static_equals_workspace_path(voge, 26, 800, 56, 2, 16, 0.01, flags=VOGE_FLAG_PLAIN)
    _static_equals_workspace_path(voge, 27, 1500, 72, 3, 20, 0.01)  # back on the tiled path


def test_static_workspace_rejects_oversize_request():
    voge = _voge()
    cams = voge.make_cameras([{"R": np.eye(3), "T": np.zeros(3), "F": 512.0, "Ox": 256.0, "Oy": 256.0, "H": 512,
                               "W": 512}] * 8)
    params = voge.make_params(8, 500_000, 3, 20, 1.0, 0.01)
    assert voge.voge_workspace_bytes(cams, params) > (32 << 20)
    fake = ctypes.c_void_p(256)
    rc = voge.lib().voge_render_fwd_static(cams, ctypes.byref(params), fake, fake, fake, fake, fake, fake, None)
    assert rc == -2  # VOGE_ERR_WORKSPACE, nothing launched
