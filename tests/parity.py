"""Parity checks of the CUDA path against the FP64 oracle.

Tolerances:
  image, weights     1e-4 absolute against the oracle's Eq. 7-8 evaluated in
                     FP64 on the GPU's own lists
  index lists        identical, except where the FP32 decision may differ from
                     the FP64 one: two kept kernels with |l_a - l_b| <=
                     1e-6 max(1, |l|) (tie in l), a kernel with |a - eta| <=
                     1e-5 eta (at the threshold: the FP32 qt carries a relative
                     error of a few ulp times qt <= 2 ln(1/eta) <= 18.5, i.e.
                     below 5e-6 in a), or either of those at the K-th place
  gradients          ||g - g_ref|| / ||g_ref|| <= 1e-3 per tensor, and per
                     element |g - g_ref| <= 1e-3 (|g_ref| + 1e-3 max|g_ref|)
                     (lists frozen: no gradient flows through the selection)
"""
import os

import numpy as np

import oracle

TOL_IMAGE = 1e-4
TOL_GRAD = 1e-3
TOL_L = 1e-6
TOL_ETA = 1e-5


def _pixel_candidates(cams, means, inv_cov, attr, tau, pix):
    """Every kernel with M_z > 0, b > 0, l > 0 for the given pixels, sorted by (l, index)."""
    r = oracle.render(cams, means, inv_cov, attr, K=0, tau=tau, eta=0.0, pix=pix)
    return r


def check_lists(gpu_idx, ref, cams, means, inv_cov, attr, K, tau, eta):
    """Validate the GPU lists against the oracle's.  Returns the number of pixels
    whose list differs (each such difference must be an allowed tie)."""
    gpu_idx = np.asarray(gpu_idx)
    ref_idx = ref["idx"]
    assert gpu_idx.shape == ref_idx.shape, (gpu_idx.shape, ref_idx.shape)
    diff = np.nonzero((gpu_idx != ref_idx).any(1))[0]
    if diff.size == 0:
        return 0
    assert diff.size <= max(3, 2e-3 * gpu_idx.shape[0]), f"{diff.size} of {gpu_idx.shape[0]} lists differ"
    full = _pixel_candidates(cams, means, inv_cov, attr, tau, ref["pix"][diff])
    for q, p in enumerate(diff):
        n = full["count"][q]
        lv = {int(g): float(l) for g, l in zip(full["idx"][q, :n], full["l"][q, :n])}
        av = {int(g): float(a) for g, a in zip(full["idx"][q, :n], full["a"][q, :n])}
        got = [int(g) for g in gpu_idx[p] if g >= 0]
        want = [int(g) for g in ref_idx[p] if g >= 0]
        for g in got:
            assert g in lv, f"pixel {p}: GPU kept kernel {g} that is not a candidate"
            if eta > 0:
                assert av[g] > eta * (1 - TOL_ETA), f"pixel {p}: kernel {g} below threshold ({av[g]})"
        for x, y in zip(got[:-1], got[1:]):
            assert lv[x] <= lv[y] + TOL_L * max(1.0, abs(lv[y])), f"pixel {p}: GPU list not sorted by l"
        kth = lv[want[-1]] if want else 0.0
        for g in set(got) ^ set(want):
            at_thr = eta > 0 and abs(av[g] - eta) <= TOL_ETA * eta
            at_k = abs(lv[g] - kth) <= TOL_L * max(1.0, abs(kth)) or (
                len(got) == len(want) and abs(lv[g] - lv[got[-1]]) <= TOL_L * max(1.0, abs(lv[got[-1]])))
            assert at_thr or at_k, f"pixel {p}: kernel {g} differs and is not at a tie (l={lv[g]}, a={av[g]})"
        if set(got) == set(want):  # same set, different order: must be an l tie
            for x, y in zip(got, want):
                if x != y:
                    assert abs(lv[x] - lv[y]) <= TOL_L * max(1.0, abs(lv[x])), f"pixel {p}: order differs"
    return int(diff.size)


# (test, lists differing at allowed ties, lists compared) of every forward check
# and (test, tensor, relative error, per-element excess) of every gradient
# check in the session; conftest prints them at the end of the run
LIST_DIFFS = []
# (test, worst |image - oracle|, worst |W - oracle|) of each forward check
FWD_ERRS = []
GRAD_STATS = []


def check_forward(image, weights, index, cams, means, inv_cov, attr, K, tau, eta, pix=None, ref=None):
    """Full forward parity on the pixels `pix` (all if None).  image/weights/index: numpy rows for those pixels."""
    if ref is None:
        ref = oracle.render(cams, means, inv_cov, attr, K=K, tau=tau, eta=eta, pix=pix, culled=eta > 0)
    n_diff = check_lists(index, ref, cams, means, inv_cov, attr, K, tau, eta)
    LIST_DIFFS.append((os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0], n_diff, int(ref["idx"].shape[0])))
    fine = oracle.fine(cams, means, inv_cov, attr, tau, ref["pix"], index)
    err_img = np.abs(image - fine["image"]).max() if image.size else 0.0
    err_w = np.abs(weights - fine["weights"]).max() if weights is not None and weights.size else 0.0
    FWD_ERRS.append((os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0], float(err_img), float(err_w)))
    assert err_img <= TOL_IMAGE, f"image error {err_img}"
    assert err_w <= TOL_IMAGE, f"weight error {err_w}"
    return {"ref": ref, "n_diff": n_diff, "err_image": float(err_img), "covered": int((ref["count"] > 0).sum())}


def rel_err(got, want):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    return float(np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-30))


def elem_excess(got, want, tol=TOL_GRAD):
    """Largest |g - g_ref| / (tol (|g_ref| + tol max|g_ref|)) over the elements:
    at most 1 when every element is inside the per-element bound."""
    got = np.asarray(got, np.float64).reshape(-1)
    want = np.asarray(want, np.float64).reshape(-1)
    if want.size == 0:
        return 0.0
    bound = tol * (np.abs(want) + tol * np.abs(want).max())
    return float((np.abs(got - want) / np.maximum(bound, 1e-300)).max())


def check_grads(got, want, keys=("g_means", "g_inv_cov", "g_attr", "g_R", "g_T"), tol=TOL_GRAD):
    """Gradient parity of each tensor: the norm bound and the per-element bound.
    Returns {key: (relative norm error, per-element excess)}."""
    out = {}
    for k in keys:
        assert np.linalg.norm(want[k]) > 0, f"{k}: reference gradient is zero"
        rel, exc = rel_err(got[k], want[k]), elem_excess(got[k], want[k], tol)
        out[k] = (rel, exc)
        GRAD_STATS.append((os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0], k, rel, exc))
        assert rel <= tol, f"{k}: relative error {rel}"
        assert exc <= 1.0, f"{k}: an element exceeds its bound by {exc:.3g}x"
    return out
