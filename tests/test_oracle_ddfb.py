"""Pins of the oracle's DDFB denoiser (Sec. II-B, Example 2: unrolled dual
forward-backward), independent of the oracle's own arithmetic:

* W_k against the library conv2d (1 -> P channels, zero "same" padding) and
  W_k^* against the library conv_transpose2d, asymmetric filters;
* linear regime (hard-tanh and both projections inactive): D(v) equals the
  recursion u_0 = A_K v, u_k = u_{k-1} + gamma_k A_k (v - A_k^T u_{k-1}),
  D = v - gamma_K A_K^T u_{K-1}, with dense matrices A_k built from the library
  convolution; this fixes the order of the layers, the initial dual variable
  and where each gamma enters;
* identity analysis operator (P = 1, a 1 x 1 unit filter) with many layers:
  the dual forward-backward iteration converges to the proximal point of
  ht |x| + iota_[0,1], i.e. clip(soft(v, ht), 0, 1).
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fnn


@pytest.mark.parametrize("ny,nx,P,ks", [(7, 9, 4, 3), (12, 5, 3, 5), (1, 6, 2, 3)])
def test_analysis_operator_and_adjoint_match_library(orc, ny, nx, P, ks):
    rng = np.random.default_rng(ny * 10 + ks)
    wk = rng.standard_normal((P, ks, ks))
    v = rng.standard_normal((ny, nx))
    u = rng.standard_normal((P, ny, nx))
    wt = torch.from_numpy(wk[:, None])                     # [P][1][ks][ks]
    ref_W = Fnn.conv2d(torch.from_numpy(v)[None, None], wt, padding=ks // 2)[0].numpy()
    ref_Wt = Fnn.conv_transpose2d(torch.from_numpy(u)[None], wt, padding=ks // 2)[0, 0].numpy()
    np.testing.assert_allclose(orc.ddfb_W(v, wk), ref_W, rtol=0, atol=1e-12)
    np.testing.assert_allclose(orc.ddfb_Wt(u, wk), ref_Wt, rtol=0, atol=1e-12)


def _dense(wk, ny, nx):
    """Matrix of the 1 -> P zero-padded convolution, from the library conv2d."""
    n = ny * nx
    E = torch.from_numpy(np.eye(n).reshape(n, 1, ny, nx))
    cols = Fnn.conv2d(E, torch.from_numpy(wk[:, None]), padding=wk.shape[-1] // 2)
    return cols.reshape(n, -1).numpy().T                     # [(P ny nx), n]


def test_linear_regime_matches_dense_recursion(orc):
    ny, nx, P, K = 6, 7, 3, 4
    rng = np.random.default_rng(3)
    w = 0.02 * rng.standard_normal((K, P, 3, 3))
    gam = np.array([0.7, 1.1, 0.9, 0.6])
    v = rng.uniform(0.3, 0.7, (ny, nx))
    net = orc.Ddfb(w, gam, ht=1e6)
    got = orc.ddfb_denoise(v, net)
    A = [_dense(w[k], ny, nx) for k in range(K)]
    vv = v.ravel()
    u = A[K - 1] @ vv
    for k in range(K - 1):
        s = vv - A[k].T @ u
        assert (s > 0).all() and (s < 1).all()           # the projection is inactive
        u = u + gam[k] * (A[k] @ s)
    ref = vv - gam[K - 1] * (A[K - 1].T @ u)
    assert (ref > 0).all() and (ref < 1).all()
    np.testing.assert_allclose(got.ravel(), ref, rtol=0, atol=1e-13)


def test_identity_operator_converges_to_clipped_soft_threshold(orc):
    rng = np.random.default_rng(5)
    v = rng.uniform(-0.5, 1.5, (9, 11))
    ht = 0.2
    K = 80
    net = orc.Ddfb(np.ones((K, 1, 1, 1)), np.ones(K), ht)
    got = orc.ddfb_denoise(v, net)
    soft = np.sign(v) * np.maximum(np.abs(v) - ht, 0.0)
    np.testing.assert_allclose(got, np.clip(soft, 0, 1), rtol=0, atol=1e-12)
