"""Pins of the oracle's neural sampler (Sec. 3.4 Eq. 10) on the CPU.

alpha_k = sum_p W_pk phi_p / sum_p W_pk, the sum over the pixels whose kept
list holds k.  The pins below do not re-run the oracle's loop: a worked
example by hand, a dense matrix form of the same definition, closed forms
(constant features, one pixel per kernel), and invariants (linearity in phi,
invariance to scaling a kernel's weights).
"""
import numpy as np
import pytest

import oracle
from paper_2205_15401_gb300 import scenes


def test_worked_example_by_hand():
    # pixel 0 keeps kernels 0 (W = 0.5) and 1 (W = 0.25); pixel 1 keeps kernel 1 (W = 0.75).
    # phi_0 = (1, 2), phi_1 = (3, 4).
    # kernel 0: 0.5 (1, 2) / 0.5 = (1, 2)
    # kernel 1: (0.25 (1, 2) + 0.75 (3, 4)) / (0.25 + 0.75) = (2.5, 3.5)
    # kernel 2: kept by no pixel -> 0 (reading C-17), wsum 0
    idx = np.array([[0, 1], [1, -1]], np.int32)
    W = np.array([[0.5, 0.25], [0.75, 0.0]])
    phi = np.array([[1.0, 2.0], [3.0, 4.0]])
    alpha, wsum = oracle.sample(idx, W, phi, 3)
    np.testing.assert_array_equal(alpha, [[1.0, 2.0], [2.5, 3.5], [0.0, 0.0]])
    np.testing.assert_array_equal(wsum, [0.5, 1.0, 0.0])


def _lists(seed=0, N=40, side=24, K=6):
    sc = scenes.plain_64(seed=seed, N=N)
    cams = [dict(scenes.cameras(sc, oracle.pose_to_RT)[0], H=side, W=side, Ox=side / 2, Oy=side / 2, F=side)]
    ref = oracle.render(cams, sc["means"].astype(np.float64), sc["inv_cov"].astype(np.float64),
                        sc["attr"].astype(np.float64), K=K, tau=1.0, eta=1e-3)
    return ref["idx"], ref["weights"], N


def test_matches_dense_matrix_form():
    """The same definition as matrix products: alpha = (Wᵀ Phi) / (Wᵀ 1)."""
    idx, W, N = _lists()
    P, L = idx.shape
    phi = np.random.default_rng(1).standard_normal((P, 5))
    dense = np.zeros((P, N))
    for p in range(P):
        for k in range(L):
            if idx[p, k] >= 0:
                dense[p, idx[p, k]] += W[p, k]
    den = dense.sum(0)
    want = np.where(den[:, None] > 0, (dense.T @ phi) / np.where(den > 0, den, 1.0)[:, None], 0.0)
    alpha, wsum = oracle.sample(idx, W, phi, N)
    assert (den > 0).sum() > 10
    np.testing.assert_allclose(wsum, den, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(alpha, want, rtol=1e-12, atol=1e-14)


def test_constant_features_come_back():
    """phi_p = c everywhere: every kept kernel samples exactly c."""
    idx, W, N = _lists(seed=2)
    c = np.array([0.3, -1.5, 2.0])
    alpha, wsum = oracle.sample(idx, W, np.tile(c, (idx.shape[0], 1)), N)
    seen = wsum > 0
    assert seen.sum() > 10
    np.testing.assert_allclose(alpha[seen], np.tile(c, (seen.sum(), 1)), rtol=1e-13)
    np.testing.assert_array_equal(alpha[~seen], 0.0)


def test_kernel_kept_by_one_pixel_takes_its_feature():
    idx = np.array([[2], [0], [1]], np.int32)
    W = np.array([[0.3], [0.9], [1e-6]])
    phi = np.arange(9.0).reshape(3, 3)
    alpha, _ = oracle.sample(idx, W, phi, 3)
    np.testing.assert_allclose(alpha, phi[[1, 2, 0]], rtol=1e-13)


def test_linear_in_features_and_blind_to_weight_scale():
    idx, W, N = _lists(seed=3)
    rng = np.random.default_rng(4)
    P = idx.shape[0]
    f1, f2 = rng.standard_normal((P, 4)), rng.standard_normal((P, 4))
    a1, _ = oracle.sample(idx, W, f1, N)
    a2, _ = oracle.sample(idx, W, f2, N)
    a12, _ = oracle.sample(idx, W, 2.0 * f1 - 3.0 * f2, N)
    np.testing.assert_allclose(a12, 2.0 * a1 - 3.0 * a2, rtol=1e-10, atol=1e-12)
    # scaling all weights by s leaves alpha unchanged and scales wsum by s
    a3, w3 = oracle.sample(idx, 7.5 * W, f1, N)
    _, w1 = oracle.sample(idx, W, f1, N)
    np.testing.assert_allclose(a3, a1, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(w3, 7.5 * w1, rtol=1e-13)


@pytest.mark.parametrize("bad", [-1, -7])
def test_empty_slots_are_skipped(bad):
    idx = np.array([[bad, 0], [0, bad]], np.int32)
    W = np.array([[5.0, 1.0], [3.0, 9.0]])
    phi = np.array([[1.0], [2.0]])
    alpha, wsum = oracle.sample(idx, W, phi, 1)
    np.testing.assert_allclose(alpha, [[(1.0 * 1.0 + 3.0 * 2.0) / 4.0]])
    np.testing.assert_allclose(wsum, [4.0])
