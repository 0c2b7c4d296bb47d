"""CUDA path vs the FP64 oracle, through the C ABI, on seeded synthetic scenes.

Sizes span several tiles and ragged tails; the four workload shapes are run
at full size (sampled pixels where the full image would take the oracle too
long).  Tolerances are those of tests/parity.py.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2205_15401_gb300 import scenes

from gpu_util import gpu_backward, gpu_forward, lib_ready, pixel_rows, r32, sample_pixels, scene_inputs, to_dev
from parity import TOL_GRAD, check_forward, check_grads, rel_err

pytestmark = pytest.mark.gpu


def _run_full(cams, means, inv_cov, attr, K, tau, eta, **kw):
    r, dev, img, w, idx = gpu_forward(cams, means, inv_cov, attr, K, tau, eta, **kw)
    res = check_forward(img, w, idx, cams, means, inv_cov, attr, K, tau, eta)
    return r, dev, img, w, idx, res


def test_plain_64_all_kernels_no_threshold():
    """64^2, N=128, K = all, eta = 0 (the plain forward workload)."""
    sc = scenes.plain_64(seed=0)
    cams, m, p, a = scene_inputs(sc)
    *_, res = _run_full(cams, m, p, a, K=0, tau=1.0, eta=0.0)
    assert res["covered"] > 2000


@pytest.mark.parametrize("K", [1, 5, 8, 12, 16, 20, 24, 27, 32, 40])
def test_plain_64_list_lengths(K):
    """Every register-list capacity and the generic path (K > 32)."""
    sc = scenes.plain_64(seed=1)
    cams, m, p, a = scene_inputs(sc)
    *_, res = _run_full(cams, m, p, a, K=K, tau=1.0, eta=0.01)
    assert res["covered"] > 1000


def test_posefit_256_full_image():
    """256^2, N=4000 on a superquadric shell, C=128, K=20, eta=1e-3, every pixel."""
    sc = scenes.posefit_256(seed=0)
    cams, m, p, a = scene_inputs(sc)
    *_, res = _run_full(cams, m, p, a, K=20, tau=1.0, eta=1e-3)
    assert res["covered"] > 5000


def test_fit_8x512_sampled_pixels():
    """8 x 512^2, N=50,000, K=20, eta=0.01 at full size; 6000 sampled pixels checked."""
    sc = scenes.fit_8x512(seed=0)
    cams, m, p, a = scene_inputs(sc)
    r, dev, img, w, idx = gpu_forward(cams, m, p, a, 20, 1.0, 0.01)
    pix = sample_pixels(cams, 6000, seed=1)
    rows = pixel_rows(cams, pix)
    res = check_forward(img[rows], w[rows], idx[rows], cams, m, p, a, 20, 1.0, 0.01, pix=pix)
    assert res["covered"] > 800


def test_fit_8x512_gradients_sampled():
    """Backward at full size with the loss gradient on sampled pixels only."""
    sc = scenes.fit_8x512(seed=2)
    cams, m, p, a = scene_inputs(sc)
    r, dev, img, w, idx = gpu_forward(cams, m, p, a, 20, 1.0, 0.01)
    pix = sample_pixels(cams, 3000, seed=3)
    rows = pixel_rows(cams, pix)
    g = np.zeros_like(img)
    g[rows] = np.random.default_rng(4).standard_normal((rows.size, img.shape[1]))
    got = gpu_backward(r, dev, idx, g)
    want = oracle.render_bwd(cams, m, p, a, 1.0, pix, idx[rows], g[rows])
    check_grads(got, want)


def test_fit_8x512_gradients_dense_with_forward_weights():
    """The backward the fitting step runs (voge_render_bwd_w, W_k read from
    the forward) at full size, with a loss gradient on every pixel, so every
    kept entry's reductions take part; norm and per-element bounds."""
    sc = scenes.fit_8x512(seed=2)
    cams, m, p, a = scene_inputs(sc)
    r, dev, img, w, idx = gpu_forward(cams, m, p, a, 20, 1.0, 0.01)
    g = r32(np.random.default_rng(4).standard_normal(img.shape))
    got = gpu_backward(r, dev, idx, g, weights_np=w)
    want = oracle.render_bwd(cams, m, p, a, 1.0, oracle.all_pixels(cams), idx, g)
    check_grads(got, want)


def test_large_1024_gradients_sampled():
    """1024^2, N=500,000, C=16, K=32 at full size, the loss gradient on 4000
    sampled pixels; both backward forms (with and without the forward's W)."""
    sc = scenes.large_1024(seed=0)
    cams, m, p, a = scene_inputs(sc)
    r, dev, img, w, idx = gpu_forward(cams, m, p, a, 32, 1.0, 1e-4)
    pix = sample_pixels(cams, 4000, seed=7)
    rows = pixel_rows(cams, pix)
    g = np.zeros_like(img)
    g[rows] = r32(np.random.default_rng(8).standard_normal((rows.size, img.shape[1])))
    want = oracle.render_bwd(cams, m, p, a, 1.0, pix, idx[rows], g[rows])
    for weights in (None, w):
        check_grads(gpu_backward(r, dev, idx, g, weights_np=weights), want)


def test_large_1024_sampled_pixels():
    """1024^2, N=500,000 in a box, C=16, K=32, eta=1e-4 at full size; 2500 sampled pixels."""
    sc = scenes.large_1024(seed=0)
    cams, m, p, a = scene_inputs(sc)
    r, dev, img, w, idx = gpu_forward(cams, m, p, a, 32, 1.0, 1e-4)
    pix = sample_pixels(cams, 2500, seed=5)
    rows = pixel_rows(cams, pix)
    res = check_forward(img[rows], w[rows], idx[rows], cams, m, p, a, 32, 1.0, 1e-4, pix=pix)
    assert res["covered"] > 1500


def test_tiled_equals_plain_bit_exact():
    """Tile binning (with sorting and early exit) changes no bit of any output."""
    sc = scenes.fit_8x512(seed=6, N=8000, B=3, side=200)
    cams, m, p, a = scene_inputs(sc)
    from paper_2205_15401_gb300.voge import VOGE_FLAG_PLAIN

    _, _, img_t, w_t, idx_t = gpu_forward(cams, m, p, a, 20, 1.0, 0.01)
    _, _, img_p, w_p, idx_p = gpu_forward(cams, m, p, a, 20, 1.0, 0.01, flags=VOGE_FLAG_PLAIN)
    np.testing.assert_array_equal(idx_t, idx_p)
    np.testing.assert_array_equal(img_t, img_p)
    np.testing.assert_array_equal(w_t, w_p)


def _centres_per_tile(cam, means, tile_w=16, tile_h=16):
    """Projected centres per 16x16 tile: a lower bound of each tile's candidate count."""
    X = means @ np.asarray(cam["R"]).T + np.asarray(cam["T"])
    z = X[:, 2]
    u = cam["F"] * X[:, 0] / z + cam["Ox"]
    v = cam["F"] * X[:, 1] / z + cam["Oy"]
    ok = (z > 0) & (u >= 0) & (u < cam["W"]) & (v >= 0) & (v < cam["H"])
    tiles = (v[ok] // tile_h).astype(int) * ((cam["W"] + tile_w - 1) // tile_w) + (u[ok] // tile_w).astype(int)
    return np.bincount(tiles)


@pytest.mark.parametrize("N,lo", [(1000, 128), (2500, 512), (6000, 1024), (12000, 2048)])
def test_long_tile_lists_sorted_exactly(N, lo):
    """Tiles with hundreds to thousands of candidates (every sort size class,
    and lists past the sorted maximum) give the same bits as no binning."""
    sc = scenes.fit_8x512(seed=21, N=N, B=1, side=64)
    cams, m, p, a = scene_inputs(sc)
    assert _centres_per_tile(cams[0], m).max() > lo
    from paper_2205_15401_gb300.voge import VOGE_FLAG_PLAIN

    _, _, img_t, w_t, idx_t = gpu_forward(cams, m, p, a, 20, 1.0, 0.01)
    _, _, img_p, w_p, idx_p = gpu_forward(cams, m, p, a, 20, 1.0, 0.01, flags=VOGE_FLAG_PLAIN)
    np.testing.assert_array_equal(idx_t, idx_p)
    np.testing.assert_array_equal(img_t, img_p)
    np.testing.assert_array_equal(w_t, w_p)


def test_bin_overflow_falls_back_exactly():
    sc = scenes.posefit_256(seed=3, N=3000, C=4)
    cams, m, p, a = scene_inputs(sc)
    _, _, img0, w0, idx0 = gpu_forward(cams, m, p, a, 20, 1.0, 1e-3)
    _, _, img1, w1, idx1 = gpu_forward(cams, m, p, a, 20, 1.0, 1e-3, bin_capacity=1)
    np.testing.assert_array_equal(idx0, idx1)
    np.testing.assert_array_equal(img0, img1)


# ----------------------------------------------------------- edge cases ---
def _cam(H, W, F, R=None, T=None):
    return {"R": np.eye(3) if R is None else R, "T": np.zeros(3) if T is None else T, "F": F, "Ox": W / 2,
            "Oy": H / 2, "H": H, "W": W}


def test_empty_scene():
    lib_ready()
    from paper_2205_15401_gb300 import voge

    cams = [_cam(20, 30, 20.0)]
    r = voge.Renderer(cams, 0, 3, K=4, tau=1.0, thresh=0.01)
    img, w, idx = r.alloc_outputs()
    img.fill_(7.0)
    z = torch.zeros((0, 3), device="cuda")
    r.forward(z, torch.zeros((0, 6), device="cuda"), z, out=(img, w, idx))
    torch.cuda.synchronize()
    assert float(img.abs().max()) == 0.0


def test_ragged_sizes_and_mixed_views():
    """Views of different, non-multiple-of-16 sizes in one call."""
    rng = np.random.default_rng(7)
    N = 300
    means = r32(np.concatenate([rng.uniform(-1, 1, (N, 2)), rng.uniform(3, 5, (N, 1))], 1))
    inv_cov = r32(scenes.inverse_covariance(scenes.random_rotations(rng, N),
                                            np.exp(rng.normal(np.log(0.08), 0.3, (N, 3)))))
    attr = r32(rng.uniform(0, 1, (N, 2)))
    c, s = np.cos(0.1), np.sin(0.1)
    R2 = np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])  # small turn about the vertical axis
    cams = [_cam(37, 53, 40.0), _cam(16, 16, 18.0), _cam(61, 29, 33.0, R=r32(R2), T=r32([0.1, -0.1, 0.2]))]
    *_, res = _run_full(cams, means, inv_cov, attr, K=12, tau=0.7, eta=0.005)
    assert res["covered"] > 500


def test_threshold_rejects_everything():
    sc = scenes.plain_64(seed=2, N=50)
    cams, m, p, a = scene_inputs(sc)
    _, _, img, w, idx = gpu_forward(cams, m, p, a, 8, 1.0, 0.99999)
    ref = oracle.render(cams, m, p, a, K=8, tau=1.0, eta=0.99999)
    assert (ref["count"] == 0).all()
    assert (idx == -1).all() and np.abs(img).max() == 0.0


def test_list_longer_than_scene():
    sc = scenes.plain_64(seed=3, N=6)
    cams, m, p, a = scene_inputs(sc)
    *_, res = _run_full(cams, m, p, a, K=20, tau=1.0, eta=0.0)  # K > N: every candidate


def test_gaussians_behind_and_around_camera():
    """Kernels behind the camera are never kept; a kernel enclosing the camera is kept where e^{q} > eta."""
    rng = np.random.default_rng(8)
    means = r32([[0.0, 0.0, -2.0], [0.1, 0.0, 0.3], [0.2, -0.1, 3.0], [0.0, 0.1, 4.0]])
    s = np.array([[0.3, 0.3, 0.3], [0.8, 0.8, 0.8], [0.2, 0.1, 0.3], [0.3, 0.4, 0.2]])
    inv_cov = r32(scenes.inverse_covariance(scenes.random_rotations(rng, 4), s))
    attr = r32(rng.uniform(0, 1, (4, 3)))
    cams = [_cam(40, 40, 30.0)]
    r, dev, img, w, idx, res = _run_full(cams, means, inv_cov, attr, K=4, tau=1.0, eta=0.01)
    assert not (idx == 0).any()
    assert (idx == 1).any()


def test_nearly_flat_gaussians():
    """Flattened ellipsoids (axis ratio 20:1), the 2D-ellipse limit of App. A.3 / Fig. 11."""
    rng = np.random.default_rng(9)
    N = 200
    means = r32(np.concatenate([rng.uniform(-0.8, 0.8, (N, 2)), rng.uniform(3, 4, (N, 1))], 1))
    s = np.stack([rng.uniform(0.05, 0.1, N), rng.uniform(0.05, 0.1, N), np.full(N, 0.004)], 1)
    inv_cov = r32(scenes.inverse_covariance(scenes.random_rotations(rng, N), s))
    attr = r32(rng.uniform(0, 1, (N, 3)))
    cams = [_cam(48, 48, 48.0)]
    *_, res = _run_full(cams, means, inv_cov, attr, K=8, tau=1.0, eta=0.01)
    assert res["covered"] > 500


# ------------------------------------------------------------ gradients ---
@pytest.mark.parametrize("K,eta", [(8, 0.01), (20, 0.001), (24, 0.001), (32, 0.01), (0, 0.0)])
def test_backward_small_scene(K, eta):
    sc = scenes.fit_8x512(seed=11, N=500, B=2, side=40)
    cams, m, p, a = scene_inputs(sc)
    p = p / 16.0  # wider kernels at this small size
    r, dev, img, w, idx = gpu_forward(cams, m, p, a, K, 1.0, eta)
    g = np.random.default_rng(12).standard_normal(img.shape)
    got = gpu_backward(r, dev, idx, g)
    want = oracle.render_bwd(cams, m, p, a, 1.0, oracle.all_pixels(cams), idx, g)
    check_grads(got, want)


@pytest.mark.parametrize("C", [1, 2, 3, 5, 8, 16])
@pytest.mark.parametrize("K", [16, 32])
def test_backward_attribute_widths(C, K):
    """Every way the attribute gradient is gathered (slots of the camera-space
    sums for C <= 3, one reduction per channel, warp rows for C >= 8) in a
    class with and one without the shared-memory W buffer."""
    sc = scenes.fit_8x512(seed=40 + C, N=400, B=2, side=36, C=C)
    cams, m, p, a = scene_inputs(sc)
    p = p / 16.0
    r, dev, img, w, idx = gpu_forward(cams, m, p, a, K, 1.0, 0.005)
    g = np.random.default_rng(41).standard_normal(img.shape)
    got = gpu_backward(r, dev, idx, g)
    want = oracle.render_bwd(cams, m, p, a, 1.0, oracle.all_pixels(cams), idx, g)
    check_grads(got, want)


@pytest.mark.parametrize("K", [16, 20, 32])
def test_backward_with_forward_weights(K):
    """voge_render_bwd_w (W_k from the forward) gives the gradients of the
    recomputing backward and of the oracle."""
    sc = scenes.fit_8x512(seed=50 + K, N=600, B=2, side=40)
    cams, m, p, a = scene_inputs(sc)
    p = p / 16.0
    r, dev, img, w, idx = gpu_forward(cams, m, p, a, K, 1.0, 0.005)
    g = np.random.default_rng(51).standard_normal(img.shape)
    with_w = gpu_backward(r, dev, idx, g, weights_np=w)
    without = gpu_backward(r, dev, idx, g)
    want = oracle.render_bwd(cams, m, p, a, 1.0, oracle.all_pixels(cams), idx, g)
    for k in ("g_means", "g_inv_cov", "g_attr", "g_R", "g_T"):
        assert rel_err(with_w[k], without[k]) <= 1e-4, k
    check_grads(with_w, want)


def test_backward_attribute_gradient_alone():
    """Asking for the attribute gradient only (narrow attributes are folded in
    by the finalize step) gives the same values as asking for everything."""
    voge = lib_ready()
    sc = scenes.fit_8x512(seed=60, N=500, B=3, side=40)
    cams, m, p, a = scene_inputs(sc)
    p = p / 16.0
    r, dev, img, w, idx = gpu_forward(cams, m, p, a, 20, 1.0, 0.005)
    g = to_dev(np.random.default_rng(61).standard_normal(img.shape))
    mm, pp, aa = dev
    i = to_dev(idx, torch.int32)
    ga_only = torch.zeros_like(aa)
    r.backward(mm, pp, aa, i, g, None, None, ga_only, None)
    gm, gp, ga, gc = torch.zeros_like(mm), torch.zeros_like(pp), torch.zeros_like(aa), torch.zeros((3, 12), device="cuda")
    r.backward(mm, pp, aa, i, g, gm, gp, ga, gc)
    torch.cuda.synchronize()
    assert float(ga.abs().max()) > 0
    assert rel_err(ga_only.cpu().numpy(), ga.cpu().numpy()) <= 1e-5


def test_backward_posefit_features():
    """C=128 features, K=20: attribute and camera gradients of the pose-fitting workload."""
    sc = scenes.posefit_256(seed=4, N=1500)
    sc["H"] = sc["W"] = 96
    sc["F"] = 96.0
    cams, m, p, a = scene_inputs(sc)
    r, dev, img, w, idx = gpu_forward(cams, m, p, a, 20, 1.0, 1e-3)
    g = np.random.default_rng(13).standard_normal(img.shape)
    got = gpu_backward(r, dev, idx, g)
    want = oracle.render_bwd(cams, m, p, a, 1.0, oracle.all_pixels(cams), idx, g)
    check_grads(got, want)


def test_reuse_projection_matches():
    sc = scenes.fit_8x512(seed=14, N=400, B=2, side=32)
    cams, m, p, a = scene_inputs(sc)
    p = p / 16.0
    r, dev, img, w, idx = gpu_forward(cams, m, p, a, 8, 1.0, 0.01)
    g = np.random.default_rng(15).standard_normal(img.shape)
    mm, pp, aa = dev
    out = []
    for reuse in (False, True):
        if reuse:
            r.forward(mm, pp, aa)
        gm, gp, ga = torch.zeros_like(mm), torch.zeros_like(pp), torch.zeros_like(aa)
        r.backward(mm, pp, aa, to_dev(idx, torch.int32), to_dev(g), gm, gp, ga, None, reuse_projection=reuse)
        torch.cuda.synchronize()
        out.append([gm.cpu().numpy(), gp.cpu().numpy(), ga.cpu().numpy()])
    for x, y in zip(out[0], out[1]):
        assert rel_err(x, y) < 1e-5


def test_packed_backward_with_the_forwards_record_of_live_row_pairs():
    """The fitting step's backward (forward weights, C <= 3, K <= 20: the packed
    form) over the forward's own lists with the projection reused takes the
    forward's record of which 16 x 2-pixel row pairs kept an entry.  Its
    gradients match the oracle and a backward that finds those row pairs itself
    (the lists copied, or the projection recomputed), on ragged views whose
    edges cut tiles and row pairs."""
    voge = lib_ready()
    rng = np.random.default_rng(22)
    N = 1200
    means = r32(np.concatenate([rng.uniform(-1, 1, (N, 2)), rng.uniform(3, 5, (N, 1))], 1))
    inv_cov = r32(scenes.inverse_covariance(scenes.random_rotations(rng, N),
                                            np.exp(rng.normal(np.log(0.06), 0.3, (N, 3)))))
    attr = r32(rng.uniform(0, 1, (N, 3)))
    cams = [{"R": np.eye(3), "T": np.zeros(3), "F": 45.0, "Ox": 30.5, "Oy": 21.5, "H": 43, "W": 61},
            {"R": np.eye(3), "T": np.zeros(3), "F": 38.0, "Ox": 17.5, "Oy": 33.5, "H": 67, "W": 35}]
    r = voge.Renderer(cams, N, 3, K=20, tau=1.0, thresh=0.005)
    m, p, a = to_dev(means), to_dev(inv_cov), to_dev(attr)
    img, w, idx = r.forward(m, p, a)
    g = to_dev(np.random.default_rng(23).standard_normal(tuple(img.shape)))

    def run(index, weights, reuse):
        gm, gp, ga = torch.zeros_like(m), torch.zeros_like(p), torch.zeros_like(a)
        gc = torch.zeros((2, 12), device="cuda")
        r.backward(m, p, a, index, g, gm, gp, ga, gc, reuse_projection=reuse, weights=weights)
        torch.cuda.synchronize()
        gcn = gc.cpu().numpy()
        return {"g_means": gm.cpu().numpy(), "g_inv_cov": gp.cpu().numpy(), "g_attr": ga.cpu().numpy(),
                "g_R": gcn[:, :9].reshape(-1, 3, 3), "g_T": gcn[:, 9:]}

    own = run(idx, w, True)
    copied = run(idx.clone(), w.clone(), True)
    r.forward(m, p, a, out=(img, w, idx))
    recomputed = run(idx, w, False)
    L = r.L
    want = oracle.render_bwd(cams, means, inv_cov, attr, 1.0, oracle.all_pixels(cams),
                             idx.cpu().numpy()[:, :L], g.cpu().numpy())
    check_grads(own, want)
    for other in (copied, recomputed):
        for k in own:
            assert rel_err(other[k], own[k]) <= 1e-5, k


def test_pose_gradient_kernel():
    voge = lib_ready()
    rng = np.random.default_rng(16)
    poses = r32(np.stack([rng.uniform(-3, 3, 5), rng.uniform(-1, 1, 5), rng.uniform(2, 6, 5),
                          rng.uniform(-0.3, 0.3, 5)], 1))
    gcam = r32(rng.standard_normal((5, 12)))
    gp = torch.zeros((5, 4), device="cuda")
    voge.voge_pose_grad(to_dev(poses), to_dev(gcam), gp)
    torch.cuda.synchronize()
    for v in range(5):
        want = oracle.pose_grad(poses[v], gcam[v, :9].reshape(3, 3), gcam[v, 9:])
        np.testing.assert_allclose(gp[v].cpu().numpy(), want, rtol=2e-5, atol=2e-5)


def test_mse_grad_kernel():
    voge = lib_ready()
    rng = np.random.default_rng(17)
    x, y = r32(rng.standard_normal(10007)), r32(rng.standard_normal(10007))
    g = torch.zeros(10007, device="cuda")
    loss = torch.zeros(1, device="cuda")
    voge.voge_mse_grad(to_dev(x), to_dev(y), g, loss)
    torch.cuda.synchronize()
    assert float(loss) == pytest.approx(np.mean((x - y) ** 2), rel=1e-5)
    np.testing.assert_allclose(g.cpu().numpy(), 2 * (x - y) / x.size, rtol=1e-5, atol=1e-9)


@pytest.mark.parametrize("n,off", [(10007, 0), (4096, 1)])
def test_mse_grad_kernel_sizes_and_alignment(n, off):
    """The four-wide path, its tail, and unaligned views (scalar path)."""
    voge = lib_ready()
    rng = np.random.default_rng(19)
    x, y = r32(rng.standard_normal(n + off)), r32(rng.standard_normal(n + off))
    xd, yd = to_dev(x)[off:], to_dev(y)[off:]
    g = torch.zeros(n + off, device="cuda")[off:]
    loss = torch.zeros(1, device="cuda")
    voge.voge_mse_grad(xd, yd, g, loss)
    torch.cuda.synchronize()
    d = (x[off:] - y[off:]).astype(np.float64)
    assert float(loss) == pytest.approx(np.mean(d ** 2), rel=1e-5)
    np.testing.assert_allclose(g.cpu().numpy(), 2 * d / n, rtol=1e-5, atol=1e-9)


@pytest.mark.parametrize("n,off", [(10007, 0), (4096, 1)])
def test_adam_step_matches_formula(n, off):
    """voge_adam_step against Adam's update written out in FP64 (Kingma & Ba,
    Algorithm 1, bias-corrected), over three steps; the gradient is zeroed."""
    voge = lib_ready()
    rng = np.random.default_rng(23)
    x0 = rng.standard_normal(n + off).astype(np.float32)
    xd = to_dev(x0)
    md, vd = torch.zeros(n + off, device="cuda"), torch.zeros(n + off, device="cuda")
    xr, mr, vr = x0[off:].astype(np.float64), np.zeros(n), np.zeros(n)
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-8
    for step in (1, 2, 3):
        g = r32(rng.standard_normal(n + off))
        gd = to_dev(g)
        voge.voge_adam_step(xd[off:], gd[off:], md[off:], vd[off:], lr, step, b1, b2, eps)
        gg = g[off:].astype(np.float64)
        mr = b1 * mr + (1 - b1) * gg
        vr = b2 * vr + (1 - b2) * gg * gg
        xr = xr - lr * (mr / (1 - b1 ** step)) / (np.sqrt(vr / (1 - b2 ** step)) + eps)
        torch.cuda.synchronize()
        assert float(gd[off:].abs().max()) == 0.0
    np.testing.assert_allclose(xd[off:].cpu().numpy(), xr, rtol=1e-5, atol=1e-6)


def test_autograd_function_matches_direct_backward():
    voge = lib_ready()
    sc = scenes.fit_8x512(seed=18, N=300, B=1, side=32)
    cams, m, p, a = scene_inputs(sc)
    p = p / 16.0
    r = voge.Renderer(cams, m.shape[0], 3, K=8, tau=1.0, thresh=0.01)
    mt, pt, at = (to_dev(x).requires_grad_() for x in (m, p, a))
    img, w, idx = voge.render(mt, pt, at, r)
    g = torch.randn_like(img)
    (img * g).sum().backward()
    got = gpu_backward(r, (mt.detach(), pt.detach(), at.detach()), idx.cpu().numpy()[:, : r.L], g.cpu().numpy(),
                       want_cam=False)
    assert rel_err(mt.grad.cpu().numpy(), got["g_means"]) < 1e-5
    assert rel_err(at.grad.cpu().numpy(), got["g_attr"]) < 1e-5
