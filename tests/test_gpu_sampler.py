"""Neural sampler (Sec. 3.4 Eq. 10) through the C ABI against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2205_15401_gb300 import scenes

from gpu_util import gpu_forward, lib_ready, r32, scene_inputs, to_dev
from parity import rel_err

pytestmark = pytest.mark.gpu

TOL_SAMPLE = 1e-4  # relative (per tensor); FP32 sums over up to a few hundred pixels per kernel


def _synthetic_lists(rng, P, L, N, holes=True):
    idx = rng.integers(0, N, (P, L)).astype(np.int32)
    n = rng.integers(0, L + 1, P)
    for p in range(P):
        idx[p, n[p]:] = -1
    if holes:  # empty slots inside lists and indices past N are skipped too
        idx[rng.random((P, L)) < 0.05] = -1
        idx[rng.random((P, L)) < 0.01] = N + 3
    W = r32(rng.uniform(0.0, 1.0, (P, L)))
    return idx, W


@pytest.mark.parametrize("C", [1, 3, 4, 16, 128])
def test_synthetic_lists_match_oracle(C):
    voge = lib_ready()
    rng = np.random.default_rng(100 + C)
    P, L, N = 3001, 13, 257  # ragged against warps and 16-byte rows
    idx, W = _synthetic_lists(rng, P, L, N)
    phi = r32(rng.standard_normal((P, C)))
    alpha, wsum = voge.voge_sample(to_dev(idx, torch.int32), to_dev(W), to_dev(phi), N)
    torch.cuda.synchronize()
    want_a, want_w = oracle.sample(idx, W, phi, N)
    assert rel_err(wsum.cpu().numpy(), want_w) <= TOL_SAMPLE
    assert rel_err(alpha.cpu().numpy(), want_a) <= TOL_SAMPLE
    unseen = want_w == 0
    assert np.all(alpha.cpu().numpy()[unseen] == 0)


def test_rendered_lists_match_oracle_render():
    """GPU render -> GPU sampler against oracle render -> oracle sampler."""
    voge = lib_ready()
    sc = scenes.fit_8x512(seed=31, N=700, B=2, side=48)
    cams, m, p, a = scene_inputs(sc)
    p = p / 16.0
    r, dev, img, w, idx = gpu_forward(cams, m, p, a, 20, 1.0, 0.01)
    phi = r32(np.random.default_rng(32).standard_normal((img.shape[0], 16)))
    alpha, wsum = voge.voge_sample(to_dev(np.ascontiguousarray(idx), torch.int32), to_dev(np.ascontiguousarray(w)),
                                   to_dev(phi), m.shape[0])
    torch.cuda.synchronize()
    ref = oracle.render(cams, m, p, a, K=20, tau=1.0, eta=0.01)
    want_a, want_w = oracle.sample(ref["idx"], ref["weights"], phi, m.shape[0])
    assert (want_w > 0).sum() > 100
    assert rel_err(wsum.cpu().numpy(), want_w) <= TOL_SAMPLE
    assert rel_err(alpha.cpu().numpy(), want_a) <= 1e-3  # lists equal up to ties; weights to 1e-4


def test_empty_inputs():
    voge = lib_ready()
    N, C = 9, 4
    idx = torch.full((5, 3), -1, dtype=torch.int32, device="cuda")
    W = torch.zeros((5, 3), device="cuda")
    phi = torch.ones((5, C), device="cuda")
    alpha, wsum = voge.voge_sample(idx, W, phi, N)
    torch.cuda.synchronize()
    assert float(alpha.abs().max()) == 0.0 and float(wsum.abs().max()) == 0.0
    # no pixels at all
    alpha, wsum = voge.voge_sample(idx[:0], W[:0], phi[:0], N)
    torch.cuda.synchronize()
    assert float(alpha.abs().max()) == 0.0


def test_full_size_properties():
    """8 views of 512x512 with the benchmark's lists: constant features sample
    back exactly, and the sampler is linear in the features."""
    voge = lib_ready()
    sc = scenes.fit_8x512(seed=0)
    cams = scenes.cameras(sc, oracle.pose_to_RT)
    N, C = sc["means"].shape[0], 16
    R = voge.Renderer(cams, N, sc["attr"].shape[1], K=20, tau=1.0, thresh=0.01)
    m, p, a = (torch.tensor(sc[k], device="cuda") for k in ("means", "inv_cov", "attr"))
    _, w, idx = R.forward(m, p, a)
    P = idx.shape[0]
    c = torch.tensor(np.linspace(-1.0, 2.0, C, dtype=np.float32), device="cuda")
    alpha, wsum = voge.voge_sample(idx, w, c.repeat(P, 1).contiguous(), N)
    seen = wsum > 0
    assert int(seen.sum()) > N // 2
    torch.testing.assert_close(alpha[seen], c.repeat(int(seen.sum()), 1), rtol=2e-5, atol=2e-6)
    if int((~seen).sum()):
        assert float(alpha[~seen].abs().max()) == 0.0
    g = torch.Generator(device="cuda").manual_seed(5)
    f1 = torch.randn((P, C), device="cuda", generator=g)
    f2 = torch.randn((P, C), device="cuda", generator=g)
    a1, _ = voge.voge_sample(idx, w, f1, N)
    a2, _ = voge.voge_sample(idx, w, f2, N)
    a12, _ = voge.voge_sample(idx, w, (2.0 * f1 - 3.0 * f2).contiguous(), N)
    torch.cuda.synchronize()
    assert rel_err((a12).cpu().numpy(), (2.0 * a1 - 3.0 * a2).cpu().numpy()) <= 1e-5


def test_bad_arguments():
    voge = lib_ready()
    lib = voge.lib()
    assert lib.voge_sample(-1, 3, 4, 2, None, None, None, None, None, None) == -1
    assert lib.voge_sample(10, 3, 4, 0, None, None, None, None, None, None) == -1
    assert lib.voge_sample(10, 3, 4, 2, None, None, None, None, None, None) == -1
