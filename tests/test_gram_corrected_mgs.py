"""The identity behind the FP32 Arnoldi iteration: for any computed (not exactly orthonormal)
basis v_1..v_j, the modified Gram-Schmidt coefficients of Fig. 2,
    h_k = v_k . (w - sum_{i<k} h_i v_i),
equal the forward substitution h_k = c_k - sum_{i<k} G_ki h_i with c_k = v_k . w and the
Gram matrix G_ki = v_k . v_i.  Checked in FP64 on bases with a controlled loss of
orthogonality, against sequential MGS; classical Gram-Schmidt (dropping G) must differ."""
import numpy as np
import pytest


def mgs_coefficients(V, w):
    w = w.copy()
    h = np.zeros(V.shape[1])
    for k in range(V.shape[1]):
        h[k] = V[:, k] @ w
        w -= h[k] * V[:, k]
    return h, w


def gram_corrected_coefficients(V, w):
    c = V.T @ w
    G = V.T @ V
    h = np.zeros_like(c)
    for k in range(len(c)):
        h[k] = c[k] - G[k, :k] @ h[:k]
    return h, w - V @ h


@pytest.mark.parametrize("j,loss", [(5, 1e-8), (20, 1e-6), (31, 1e-3)])
def test_forward_substitution_gives_the_mgs_coefficients(j, loss):
    rng = np.random.default_rng(j)
    n = 400
    Q, _ = np.linalg.qr(rng.standard_normal((n, j)))
    V = Q + loss * rng.standard_normal((n, j))          # a basis that is not orthonormal
    w = rng.standard_normal(n) * 3.0 + V @ rng.standard_normal(j)
    h_mgs, w_mgs = mgs_coefficients(V, w)
    h_gc, w_gc = gram_corrected_coefficients(V, w)
    assert np.allclose(h_gc, h_mgs, rtol=1e-11, atol=1e-11 * np.abs(h_mgs).max())
    assert np.linalg.norm(w_gc - w_mgs) <= 1e-10 * np.linalg.norm(w)
    # classical Gram-Schmidt keeps c_k: it differs by about the loss of orthogonality
    h_cgs = V.T @ w
    assert np.abs(h_cgs - h_mgs).max() > 0.1 * loss * np.abs(h_mgs).max()
