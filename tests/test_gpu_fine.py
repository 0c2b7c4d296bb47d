"""The fine pass alone (voge_render_fine, Eq. 7-8) on given lists, and the
split forward (selection kernel, then the fine kernel) against the fused one.

Random lists exercise the fine pass independently of the selection: any
order, short and empty lists, a list ended early by -1.  Tolerances are those
of tests/parity.py (1e-4 absolute on image and weights).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2205_15401_gb300 import scenes

from gpu_util import gpu_forward, lib_ready, pixel_rows, r32, sample_pixels, scene_inputs, to_dev
from parity import TOL_IMAGE

pytestmark = pytest.mark.gpu


def _random_lists(rng, P, L, N, fill=0.8):
    """[P][L] lists of distinct kernels in random order, each of random length
    (about `fill` of the pixels non-empty), -1 padded."""
    idx = np.full((P, L), -1, np.int32)
    lens = np.where(rng.uniform(size=P) < fill, rng.integers(1, L + 1, P), 0)
    for p in range(P):
        if lens[p]:
            idx[p, : lens[p]] = rng.choice(N, size=lens[p], replace=False)
    return idx


def _fine_gpu(cams, m, p, a, idx, K, tau, with_weights=True):
    voge = lib_ready()
    N, C = m.shape[0], a.shape[1]
    r = voge.Renderer(cams, N, C, K=K, tau=tau, thresh=0.01)
    assert r.L == idx.shape[1]
    w = torch.full((r.pixels, r.L), -7.0, device="cuda") if with_weights else None
    img = torch.full((r.pixels, C), -7.0, device="cuda")
    r.fine(to_dev(m), to_dev(p), to_dev(a), to_dev(idx, torch.int32), img, w)
    torch.cuda.synchronize()
    return img.cpu().numpy(), (w.cpu().numpy() if with_weights else None)


def _near_scene(seed, N, C, cams_hw):
    """Kernels around the rays of every view (so that random lists see real
    overlap in depth) with moderate sizes."""
    rng = np.random.default_rng(seed)
    means = r32(np.concatenate([rng.uniform(-0.6, 0.6, (N, 2)), rng.uniform(3.0, 3.4, (N, 1))], 1))
    inv_cov = r32(scenes.inverse_covariance(scenes.random_rotations(rng, N),
                                            np.exp(rng.normal(np.log(0.05), 0.4, (N, 3)))))
    attr = r32(rng.standard_normal((N, C)))
    cams = [{"R": np.eye(3), "T": np.zeros(3), "F": float(max(h, w)), "Ox": w / 2, "Oy": h / 2, "H": h, "W": w}
            for h, w in cams_hw]
    return cams, means, inv_cov, attr


@pytest.mark.parametrize("K,C", [(8, 3), (16, 5), (20, 3), (20, 128), (24, 16), (32, 16), (32, 1)])
def test_fine_random_lists_match_oracle(K, C):
    cams, m, p, a = _near_scene(100 + K + C, 300, C, [(37, 53), (16, 16), (24, 40)])
    pix = oracle.all_pixels(cams)
    idx = _random_lists(np.random.default_rng(K * 7 + C), pix.shape[0], K, 300)
    idx[3, 2:] = -1
    idx[4, 1] = -1  # a -1 ends the list: later entries are ignored
    img, w = _fine_gpu(cams, m, p, a, idx, K, tau=0.8)
    cut = idx.copy()
    for q in range(cut.shape[0]):
        neg = np.nonzero(cut[q] < 0)[0]
        if neg.size:
            cut[q, neg[0]:] = -1
    ref = oracle.fine(cams, m, p, a, 0.8, pix, cut)
    assert np.abs(img - ref["image"]).max() <= TOL_IMAGE
    assert np.abs(w - ref["weights"]).max() <= TOL_IMAGE
    assert np.abs(ref["weights"]).max() > 0.05


def test_fine_without_weights_and_empty_lists():
    cams, m, p, a = _near_scene(7, 200, 3, [(20, 20)])
    idx = np.full((400, 12), -1, np.int32)
    img, _ = _fine_gpu(cams, m, p, a, idx, 12, tau=1.0, with_weights=False)
    assert np.abs(img).max() == 0.0


def test_split_forward_equals_fused():
    """The split forward (selection kernel, then the fine kernel) gives the
    fused kernel's lists bit for bit, and its image and weights (the same
    arithmetic per pixel)."""
    from paper_2205_15401_gb300.voge import VOGE_FLAG_SPLIT_FORWARD

    for K, args in [(20, dict(seed=6, N=8000, B=3, side=200)), (32, dict(seed=8, N=6000, B=2, side=120)),
                    (8, dict(seed=9, N=3000, B=2, side=90)), (24, dict(seed=10, N=4000, B=1, side=130))]:
        sc = scenes.fit_8x512(**args)
        cams, m, p, a = scene_inputs(sc)
        _, _, img_f, w_f, idx_f = gpu_forward(cams, m, p, a, K, 1.0, 0.01)
        _, _, img_s, w_s, idx_s = gpu_forward(cams, m, p, a, K, 1.0, 0.01, flags=VOGE_FLAG_SPLIT_FORWARD)
        np.testing.assert_array_equal(idx_s, idx_f)
        np.testing.assert_array_equal(img_s, img_f)
        np.testing.assert_array_equal(w_s, w_f)


def test_fine_on_fit_8x512_lists():
    """Full size: the fine pass over the forward's own lists of the 8-view
    512^2 scene reproduces the forward's image and weights, and the oracle's
    Eq. 7-8 on 6000 sampled pixels."""
    sc = scenes.fit_8x512(seed=0)
    cams, m, p, a = scene_inputs(sc)
    r, dev, img, w, idx = gpu_forward(cams, m, p, a, 20, 1.0, 0.01)
    img2, w2 = _fine_gpu(cams, m, p, a, idx, 20, tau=1.0)
    np.testing.assert_array_equal(idx.shape, w2.shape)
    assert np.abs(img2 - img).max() <= 1e-6 and np.abs(w2 - w).max() <= 1e-6
    pix = sample_pixels(cams, 6000, seed=2)
    rows = pixel_rows(cams, pix)
    ref = oracle.fine(cams, m, p, a, 1.0, pix, idx[rows])
    assert np.abs(img2[rows] - ref["image"]).max() <= TOL_IMAGE
    assert np.abs(w2[rows] - ref["weights"]).max() <= TOL_IMAGE


def test_fine_on_large_1024_lists():
    """Full size, 1024^2 with 500,000 kernels, C = 16, K = 32: the fine pass
    over the forward's lists against the oracle on 2500 sampled pixels."""
    sc = scenes.large_1024(seed=0)
    cams, m, p, a = scene_inputs(sc)
    r, dev, img, w, idx = gpu_forward(cams, m, p, a, 32, 1.0, 1e-4)
    img2, w2 = _fine_gpu(cams, m, p, a, idx, 32, tau=1.0)
    assert np.abs(img2 - img).max() <= 1e-6
    pix = sample_pixels(cams, 2500, seed=4)
    rows = pixel_rows(cams, pix)
    ref = oracle.fine(cams, m, p, a, 1.0, pix, idx[rows])
    assert np.abs(img2[rows] - ref["image"]).max() <= TOL_IMAGE
    assert np.abs(w2[rows] - ref["weights"]).max() <= TOL_IMAGE


def test_render_stats_counts_match_the_lists():
    """voge_render_stats: the kept entries and the fine pass's pairs equal the
    counts of the index output exactly; the coarse pass traced at least every
    kept entry, and the tiled path (depth-sorted, with early exit) traced no
    more candidates than the plain path, which tests every Gaussian."""
    voge = lib_ready()
    from paper_2205_15401_gb300.voge import VOGE_FLAG_PLAIN

    sc = scenes.fit_8x512(seed=31, N=6000, B=2, side=160)
    cams, m, p, a = scene_inputs(sc)
    traced = {}
    for flags in (0, VOGE_FLAG_PLAIN):
        r = voge.Renderer(cams, m.shape[0], 3, K=20, tau=1.0, thresh=0.01, flags=flags)
        img, w, idx = r.forward(to_dev(m), to_dev(p), to_dev(a))
        st = voge.voge_render_stats(r.workspace)
        n = (idx[:, : r.L] >= 0).sum(1).to(torch.int64)
        assert st["entries"] == int(n.sum()) > 0
        assert st["pairs"] == int((n * n).sum())
        assert st["traces"] >= st["entries"]
        traced[flags] = st["traces"]
    assert traced[0] <= traced[VOGE_FLAG_PLAIN]
