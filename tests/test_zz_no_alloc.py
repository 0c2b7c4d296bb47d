"""The no-allocation forward entry point, checked against voge_render_fwd.

voge_render_fwd_static serves callers that cannot allocate device memory where
they render (a host callback, a real-time loop with a fixed memory budget, a
program without an allocator of its own): it uses a workspace held inside the
library instead of one the caller passes.  Its results must equal those of the
ordinary entry point, call after call, although every call shares (and
reuses) that one library-held workspace.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _scene(seed, N, side, B):
    import oracle
    from paper_2205_15401_gb300 import scenes

    sc = scenes.fit_8x512(seed=seed, N=N, B=B, side=side)
    cams = scenes.cameras(sc, oracle.pose_to_RT)
    inv_cov = (sc["inv_cov"] / 16.0).astype(np.float32)  # wider kernels at these small sizes
    return cams, sc["means"], inv_cov, sc["attr"]


def test_static_workspace_matches_workspace_path_twice():
    from paper_2205_15401_gb300 import build

    build.build()
    from paper_2205_15401_gb300 import voge

    tol_image = 1e-4  # the image tolerance of the parity tests
    for seed, N, side, B, K, eta in [(21, 3000, 96, 2, 20, 0.01), (22, 1200, 64, 3, 8, 0.02)]:
        cams, means, inv_cov, attr = _scene(seed, N, side, B)
        r = voge.Renderer(cams, N, 3, K=K, tau=1.0, thresh=eta)
        assert voge.voge_workspace_bytes(r.cams, r.params) <= (32 << 20)
        m, p, a = (torch.tensor(x, device="cuda") for x in (means, inv_cov, attr))
        img_ref, w_ref, idx_ref = r.forward(m, p, a)
        img, w, idx = r.alloc_outputs()
        img.fill_(-7.0)
        idx.fill_(-7)
        voge.voge_render_fwd_static(r.cams, r.params, m, p, a, img, w, idx)
        torch.cuda.synchronize()
        L = r.L
        assert torch.equal(idx[:, :L], idx_ref[:, :L])
        assert float((img - img_ref).abs().max()) <= tol_image
        assert float((w[:, :L] - w_ref[:, :L]).abs().max()) <= tol_image
        assert int((idx_ref[:, :L] >= 0).sum()) > 0


def test_static_workspace_rejects_oversize_request():
    from paper_2205_15401_gb300 import build

    build.build()
    from paper_2205_15401_gb300 import voge

    cams = voge.make_cameras([{"R": np.eye(3), "T": np.zeros(3), "F": 512.0, "Ox": 256.0, "Oy": 256.0, "H": 512,
                               "W": 512}] * 8)
    params = voge.make_params(8, 500_000, 3, 20, 1.0, 0.01)
    assert voge.voge_workspace_bytes(cams, params) > (32 << 20)
    fake = ctypes.c_void_p(256)
    rc = voge.lib().voge_render_fwd_static(cams, ctypes.byref(params), fake, fake, fake, fake, fake, fake, None)
    assert rc == -2  # VOGE_ERR_WORKSPACE, nothing launched
