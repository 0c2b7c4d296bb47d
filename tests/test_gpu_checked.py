"""The checked library (libvoge_checked.so, -DVOGE_CHECKED) on the GPU.

Every tile-kernel path -- fused and split forward, each list capacity, the
generic path for lists longer than 32, the plain comparator, narrow and wide
attributes, ragged views -- runs through the checked library on small
parity cases: no index check fails (a failure raises, VOGE_ERR_CHECK), the
forward's lists, weights and image equal the normal build's bit for bit, and
the gradients agree to the rounding that atomics leave (1e-5 relative).
No input here is out of range: the checks are exercised on valid work."""
import numpy as np
import pytest
import torch

from paper_2205_15401_gb300 import scenes

from gpu_util import gpu_backward, gpu_forward, lib_ready, r32, scene_inputs, to_dev
from parity import rel_err

pytestmark = pytest.mark.gpu


def _ragged(seed=70):
    rng = np.random.default_rng(seed)
    N = 300
    means = r32(np.concatenate([rng.uniform(-1, 1, (N, 2)), rng.uniform(3, 5, (N, 1))], 1))
    inv_cov = r32(scenes.inverse_covariance(scenes.random_rotations(rng, N),
                                            np.exp(rng.normal(np.log(0.08), 0.3, (N, 3)))))
    attr = r32(rng.uniform(0, 1, (N, 5)))
    cams = [{"R": np.eye(3), "T": np.zeros(3), "F": 40.0, "Ox": 26.5, "Oy": 18.5, "H": 37, "W": 53},
            {"R": np.eye(3), "T": np.zeros(3), "F": 33.0, "Ox": 14.5, "Oy": 30.5, "H": 61, "W": 29}]
    return cams, means, inv_cov, attr


def _cases():
    from paper_2205_15401_gb300.voge import VOGE_FLAG_PLAIN, VOGE_FLAG_SPLIT_FORWARD

    small = scene_inputs(scenes.fit_8x512(seed=71, N=2000, B=2, side=72))
    small = (small[0], small[1], small[2] / 16.0, small[3])
    wide = scene_inputs(scenes.fit_8x512(seed=72, N=1500, B=1, side=64, C=16))
    wide = (wide[0], wide[1], wide[2] / 16.0, wide[3])
    dense = scene_inputs(scenes.plain_64(seed=73))
    return [("K20 fused", small, 20, 0.01, 0), ("K20 split", small, 20, 0.01, VOGE_FLAG_SPLIT_FORWARD),
            ("K8", small, 8, 0.01, 0), ("K24", small, 24, 0.01, 0), ("K32 split", small, 32, 0.01,
                                                                       VOGE_FLAG_SPLIT_FORWARD),
            ("K40 generic", small, 40, 0.01, 0), ("plain", small, 16, 0.01, VOGE_FLAG_PLAIN),
            ("C16 K32", wide, 32, 0.005, 0), ("dense K=all", dense, 0, 0.0, 0),
            ("ragged C5", _ragged(), 12, 0.005, 0)]


@pytest.mark.parametrize("case", range(10))
def test_checked_library_runs_clean_and_matches(case):
    from paper_2205_15401_gb300 import build
    from paper_2205_15401_gb300 import voge

    lib_ready()
    build.build(checked=True)
    name, (cams, m, p, a), K, eta, flags = _cases()[case]
    g = np.random.default_rng(case).standard_normal((sum(c["H"] * c["W"] for c in cams), a.shape[1]))
    out = {}
    for checked in (False, True):
        ctx = voge.checked_library() if checked else _null()
        with ctx:
            r, dev, img, w, idx = gpu_forward(cams, m, p, a, K, 1.0, eta, flags=flags)
            grads = gpu_backward(r, dev, idx, g, weights_np=w)
            grads_rw = gpu_backward(r, dev, idx, g)
        out[checked] = (img, w, idx, grads, grads_rw)
    n_img, n_w, n_idx, n_g, n_grw = out[False]
    c_img, c_w, c_idx, c_g, c_grw = out[True]
    np.testing.assert_array_equal(c_idx, n_idx, err_msg=name)
    np.testing.assert_array_equal(c_img, n_img, err_msg=name)
    np.testing.assert_array_equal(c_w, n_w, err_msg=name)
    assert (n_idx >= 0).sum() > 0, name
    for k in n_g:
        assert rel_err(c_g[k], n_g[k]) <= 1e-5, (name, k)
        assert rel_err(c_grw[k], n_grw[k]) <= 1e-5, (name, k)


class _null:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False
