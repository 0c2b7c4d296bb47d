"""Serving: results are the same alone and in the mix, plus admission and timeout paths."""
import numpy as np
import pytest
import torch

import oracle
from paper_2205_15401_gb300 import scenes

from gpu_util import lib_ready, to_dev
from parity import TOL_GRAD, TOL_IMAGE, rel_err

pytestmark = pytest.mark.gpu


def _requests(seed, n):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n):
        N = int(rng.integers(300, 3000))
        side = int(rng.choice([32, 48, 80]))
        C = int(rng.choice([3, 16]))
        K = int(rng.choice([10, 20, 32]))
        sc = scenes.fit_8x512(seed=seed * 100 + q, N=N, B=1, side=side, C=C)
        cam = scenes.cameras(sc, oracle.pose_to_RT)[0]
        out.append({"cam": cam, "means": sc["means"], "inv_cov": (sc["inv_cov"] / 16.0).astype(np.float32),
                    "attr": sc["attr"], "K": K, "thresh": 0.01,
                    "target": rng.uniform(0, 1, (side * side, C)).astype(np.float32)})
    return out


def _alone_via_api(r):
    voge = lib_ready()
    N, C = r["means"].shape[0], r["attr"].shape[1]
    R = voge.Renderer([r["cam"]], N, C, K=r["K"], tau=1.0, thresh=r["thresh"])
    m, p, a, tgt = to_dev(r["means"]), to_dev(r["inv_cov"]), to_dev(r["attr"]), to_dev(r["target"])
    img, w, idx = R.forward(m, p, a)
    g = torch.empty_like(img)
    loss = torch.zeros(1, device="cuda")
    voge.voge_mse_grad(img, tgt, g, loss)
    gm, gp, ga = torch.zeros_like(m), torch.zeros_like(p), torch.zeros_like(a)
    gc = torch.zeros((1, 12), device="cuda")
    R.backward(m, p, a, idx, g, gm, gp, ga, gc)
    torch.cuda.synchronize()
    return {"image": img.cpu().numpy(), "loss": float(loss), "grad_means": gm.cpu().numpy(),
            "grad_inv_cov": gp.cpu().numpy(), "grad_attr": ga.cpu().numpy(), "grad_cam": gc.cpu().numpy()[0]}


def _outputs(r):
    N, C = r["means"].shape[0], r["attr"].shape[1]
    P = r["cam"]["H"] * r["cam"]["W"]
    pin = lambda *s: torch.zeros(s, dtype=torch.float32).pin_memory()
    return {"image": pin(P, C), "grad_means": pin(N, 3), "grad_inv_cov": pin(N, 6), "grad_attr": pin(N, C),
            "grad_cam": pin(12), "loss": pin(1)}


def _compare(got, want):
    assert np.abs(got["image"].numpy() - want["image"]).max() <= TOL_IMAGE
    assert float(got["loss"][0]) == pytest.approx(want["loss"], rel=1e-5, abs=1e-9)
    for k in ("grad_means", "grad_inv_cov", "grad_attr", "grad_cam"):
        assert rel_err(got[k].numpy(), want[k]) <= TOL_GRAD, k


@pytest.mark.parametrize("graphs", [True, False])
def test_results_in_the_mix_equal_alone(graphs):
    voge = lib_ready()
    reqs = _requests(1, 10)
    alone = [_alone_via_api(r) for r in reqs]
    srv = voge.Server(mem_budget_bytes=1 << 30, max_slots=16, use_graphs=graphs, batching=True, inflight_ticks=2)
    outs, tickets = [], []
    for q, r in enumerate(reqs):
        if q == 3:
            srv.pause(True)  # the rest is admitted meanwhile and starts as one mixed tick
        o = _outputs(r)
        rc, t = srv.submit(r["cam"], r["target"], r["K"], thresh=r["thresh"], means=r["means"],
                           inv_cov=r["inv_cov"], attr=r["attr"], outputs=o)
        assert rc == 0
        outs.append(o)
        tickets.append(t)
    srv.pause(False)
    for t in tickets:
        rc, tm = srv.wait(t, 60_000)
        assert rc == 0, rc
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs)
    assert st["requests_in_ticks"] > st["ticks"]  # at least one tick ran several requests together
    for o, w in zip(outs, alone):
        _compare(o, w)


def test_one_request_per_tick_equals_api():
    voge = lib_ready()
    reqs = _requests(2, 4)
    srv = voge.Server(mem_budget_bytes=1 << 30, max_slots=4, use_graphs=False, batching=False, inflight_ticks=1)
    for r in reqs:
        o = _outputs(r)
        rc, t = srv.submit(r["cam"], r["target"], r["K"], thresh=r["thresh"], means=r["means"],
                           inv_cov=r["inv_cov"], attr=r["attr"], outputs=o)
        assert rc == 0
        assert srv.wait(t, 60_000)[0] == 0
        _compare(o, _alone_via_api(r))
    assert srv.stats()["ticks"] == len(reqs)
    srv.close()


def test_resident_scene_equals_inline():
    voge = lib_ready()
    r = _requests(3, 1)[0]
    srv = voge.Server(mem_budget_bytes=1 << 30, max_slots=4)
    sid = srv.add_scene(r["means"], r["inv_cov"], r["attr"])
    o1, o2 = _outputs(r), _outputs(r)
    _, t1 = srv.submit(r["cam"], r["target"], r["K"], thresh=r["thresh"], scene=sid, outputs=o1)
    _, t2 = srv.submit(r["cam"], r["target"], r["K"], thresh=r["thresh"], means=r["means"], inv_cov=r["inv_cov"],
                       attr=r["attr"], outputs=o2)
    assert srv.wait(t1, 60_000)[0] == 0 and srv.wait(t2, 60_000)[0] == 0
    assert srv.remove_scene(sid) == 0
    srv.close()
    np.testing.assert_array_equal(o1["image"].numpy(), o2["image"].numpy())
    assert rel_err(o1["grad_means"].numpy(), o2["grad_means"].numpy()) < 1e-5


def test_admission_refusal_and_timeout():
    voge = lib_ready()
    srv = voge.Server(mem_budget_bytes=96 << 20, max_slots=2, max_tick_gaussians=1 << 16, max_tick_pixels=1 << 18)
    big = _requests(4, 1)[0]
    cam = dict(big["cam"], H=2048, W=2048, Ox=1024.0, Oy=1024.0)
    rc, _ = srv.submit(cam, np.zeros((2048 * 2048, big["attr"].shape[1]), np.float32), big["K"],
                       means=big["means"], inv_cov=big["inv_cov"], attr=big["attr"])
    assert rc == -6  # VOGE_ERR_ADMISSION: can never fit this server
    r = _requests(5, 1)[0]
    o = _outputs(r)
    rc, t = srv.submit(r["cam"], r["target"], r["K"], means=r["means"], inv_cov=r["inv_cov"], attr=r["attr"],
                       outputs=o)
    assert rc == 0
    rc0, _ = srv.wait(t, 0)
    assert rc0 in (0, -5)  # done already, or VOGE_ERR_TIMEOUT with the ticket still valid
    if rc0 == -5:
        assert srv.wait(t, 60_000)[0] == 0
    srv.close()


def test_served_request_matches_oracle():
    voge = lib_ready()
    r = _requests(6, 1)[0]
    r["cam"] = dict(r["cam"])
    o = _outputs(r)
    srv = voge.Server(mem_budget_bytes=1 << 30, max_slots=2)
    _, t = srv.submit(r["cam"], r["target"], r["K"], thresh=r["thresh"], means=r["means"], inv_cov=r["inv_cov"],
                      attr=r["attr"], outputs=o)
    assert srv.wait(t, 60_000)[0] == 0
    srv.close()
    cams = [r["cam"]]
    m, p, a = (r[k].astype(np.float64) for k in ("means", "inv_cov", "attr"))
    ref = oracle.render(cams, m, p, a, K=r["K"], tau=1.0, eta=r["thresh"])
    img = o["image"].numpy()
    assert np.abs(img - ref["image"]).max() <= 1e-4
    n = img.size
    g_img = 2.0 * (ref["image"] - r["target"].astype(np.float64)) / n
    want = oracle.render_bwd(cams, m, p, a, 1.0, ref["pix"], ref["idx"], g_img)
    assert rel_err(o["grad_means"].numpy(), want["g_means"]) <= TOL_GRAD
    assert rel_err(o["grad_attr"].numpy(), want["g_attr"]) <= TOL_GRAD
