"""Helpers shared by the GPU tests: run the CUDA path through the C ABI."""
import numpy as np
import torch

import oracle
from paper_2205_15401_gb300 import build, scenes


def lib_ready():
    build.build()
    from paper_2205_15401_gb300 import voge

    voge.lib()
    return voge


def r32(x):
    """Round to float32 and back: the values the CUDA path actually sees."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def to_dev(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def gpu_forward(cams, means, inv_cov, attr, K, tau, eta, flags=0, bin_capacity=0):
    voge = lib_ready()
    for x in (means, inv_cov, attr):
        assert np.array_equal(np.asarray(x, np.float64), r32(x)), "inputs must be float32 values"
    N, C = means.shape[0], attr.shape[1]
    r = voge.Renderer(cams, N, C, K=K, tau=tau, thresh=eta, flags=flags, bin_capacity=bin_capacity)
    m, p, a = to_dev(means), to_dev(inv_cov), to_dev(attr)
    image, weights, index = r.forward(m, p, a)
    torch.cuda.synchronize()
    return r, (m, p, a), image.cpu().numpy(), weights.cpu().numpy()[:, : r.L], index.cpu().numpy()[:, : r.L]


def gpu_backward(r, dev_inputs, index_np, grad_image_np, want_cam=True, weights_np=None):
    m, p, a = dev_inputs
    gm, gp, ga = torch.zeros_like(m), torch.zeros_like(p), torch.zeros_like(a)
    gc = torch.zeros((r.params.B, 12), device="cuda") if want_cam else None
    idx = to_dev(index_np, torch.int32)
    w = None if weights_np is None else to_dev(np.ascontiguousarray(weights_np), torch.float32)
    r.backward(m, p, a, idx, to_dev(grad_image_np), gm, gp, ga, gc, weights=w)
    torch.cuda.synchronize()
    out = {"g_means": gm.cpu().numpy(), "g_inv_cov": gp.cpu().numpy(), "g_attr": ga.cpu().numpy()}
    if want_cam:
        gcn = gc.cpu().numpy()
        out["g_R"] = gcn[:, :9].reshape(-1, 3, 3)
        out["g_T"] = gcn[:, 9:]
    return out


def scene_inputs(sc):
    cams = scenes.cameras(sc, oracle.pose_to_RT)
    return cams, sc["means"].astype(np.float64), sc["inv_cov"].astype(np.float64), sc["attr"].astype(np.float64)


def pixel_rows(cams, pix):
    """Global pixel row of each (view, row, col)."""
    base = np.cumsum([0] + [c["H"] * c["W"] for c in cams])[:-1]
    W = np.array([c["W"] for c in cams])
    return base[pix[:, 0]] + pix[:, 1] * W[pix[:, 0]] + pix[:, 2]


def sample_pixels(cams, n, seed=0, covered_from=None):
    rng = np.random.default_rng(seed)
    allp = oracle.all_pixels(cams)
    sel = rng.choice(allp.shape[0], size=min(n, allp.shape[0]), replace=False)
    return np.ascontiguousarray(allp[np.sort(sel)])
