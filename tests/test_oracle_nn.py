"""Pins for the FP64 oracle of the learned preconditioner (CPU only).

Against: a brute-force seven-fold loop for the 3x3x3 convolution; central
finite differences for every gradient; positive homogeneity of a bias-free
ReLU network; the zero network reducing to Jacobi.
"""
import numpy as np
import pytest

from oracle import nn


def brute_conv(a, W):
    X, Y, Z, Cin = a.shape
    out = np.zeros((X, Y, Z, W.shape[1]))
    for i in range(X):
        for j in range(Y):
            for k in range(Z):
                for t in range(27):
                    dx, dy, dz = t % 3 - 1, (t // 3) % 3 - 1, t // 9 - 1
                    ii, jj, kk = i + dx, j + dy, k + dz
                    if 0 <= ii < X and 0 <= jj < Y and 0 <= kk < Z:
                        for o in range(W.shape[1]):
                            for c in range(Cin):
                                out[i, j, k, o] += W[t, o, c] * a[ii, jj, kk, c]
    return out


def masks(shape, seed=0):
    rng = np.random.default_rng(seed)
    dof = (rng.random(shape) < 0.8).astype(float)
    free = dof * (rng.random(shape) < 0.9)
    return dof, free


def test_tap_order():
    assert nn.TAPS[0] == (-1, -1, -1) and nn.TAPS[13] == (0, 0, 0) and nn.TAPS[26] == (1, 1, 1)
    assert nn.TAPS[1] == (0, -1, -1)  # x fastest


def test_conv_matches_brute_force():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((4, 3, 5, 2))
    W = rng.standard_normal((27, 3, 2))
    assert np.allclose(nn.conv3d(a, W), brute_conv(a, W), atol=1e-12)


def test_conv_backward_finite_differences():
    rng = np.random.default_rng(2)
    a = rng.standard_normal((3, 4, 3, 2))
    W = rng.standard_normal((27, 3, 2))
    g = rng.standard_normal((3, 4, 3, 3))
    ga, gW = nn.conv3d_backward(a, W, g)
    h = 1e-6
    for _ in range(10):
        idx = tuple(rng.integers(0, s) for s in a.shape)
        e = np.zeros_like(a)
        e[idx] = h
        fd = (np.sum(g * nn.conv3d(a + e, W)) - np.sum(g * nn.conv3d(a - e, W))) / (2 * h)
        assert np.isclose(ga[idx], fd, rtol=1e-7, atol=1e-9)
        idw = tuple(rng.integers(0, s) for s in W.shape)
        e = np.zeros_like(W)
        e[idw] = h
        fd = (np.sum(g * nn.conv3d(a, W + e)) - np.sum(g * nn.conv3d(a, W - e))) / (2 * h)
        assert np.isclose(gW[idw], fd, rtol=1e-7, atol=1e-9)


def test_network_backward_finite_differences():
    shape = (4, 4, 3)
    dof, free = masks(shape, 3)
    rng = np.random.default_rng(4)
    x = free[..., None] * rng.standard_normal(shape + (3,))
    Ws = nn.init_weights(5)
    gy = rng.standard_normal(shape + (3,))
    y, cache = nn.network(x, Ws, dof, free)
    gWs, _ = nn.network_backward(cache, gy, Ws, dof, free)
    h = 1e-6
    for l in range(3):
        for _ in range(6):
            idw = tuple(rng.integers(0, s) for s in Ws[l].shape)
            Wp = [W.copy() for W in Ws]
            Wm = [W.copy() for W in Ws]
            Wp[l][idw] += h
            Wm[l][idw] -= h
            fd = (np.sum(gy * nn.network(x, Wp, dof, free)[0]) - np.sum(gy * nn.network(x, Wm, dof, free)[0])) / (2 * h)
            assert np.isclose(gWs[l][idw], fd, rtol=1e-5, atol=1e-8), (l, idw)


def test_positive_homogeneity_and_masks():
    shape = (5, 4, 4)
    dof, free = masks(shape, 6)
    rng = np.random.default_rng(7)
    x = free[..., None] * rng.standard_normal(shape + (3,))
    Ws = nn.init_weights(8)
    y1, _ = nn.network(x, Ws, dof, free)
    y2, _ = nn.network(3.7 * x, Ws, dof, free)
    assert np.allclose(y2, 3.7 * y1, atol=1e-12)
    assert np.all(y1[free == 0] == 0)


def test_zero_network_is_jacobi():
    shape = (4, 4, 4)
    dof, free = masks(shape, 9)
    rng = np.random.default_rng(10)
    r = free[..., None] * rng.standard_normal(shape + (3,))
    dinv = free[..., None] * rng.uniform(0.5, 2.0, shape + (3,))
    Ws = [np.zeros_like(W) for W in nn.init_weights(0)]
    z, _ = nn.precondition(r, dinv, Ws, dof, free)
    assert np.allclose(z, dinv * r)


def test_loss_gradient_finite_differences():
    shape = (3, 3, 3)
    dof, free = masks(shape, 11)
    n = int(np.prod(shape)) * 3
    rng = np.random.default_rng(12)
    Mr = rng.standard_normal((n, n))
    Hm = Mr @ Mr.T + n * np.eye(n)
    fmask = np.repeat(free.reshape(-1), 3)
    Hm = Hm * np.outer(fmask, fmask) + np.diag(1 - fmask)

    def hvp(v):
        return (fmask * (Hm @ (fmask * v.reshape(-1)))).reshape(v.shape)

    dinv = free[..., None] / np.diag(Hm).reshape(shape + (3,))
    r = free[..., None] * rng.standard_normal(shape + (3,))
    e = free[..., None] * rng.standard_normal(shape + (3,))
    Ws = nn.init_weights(13)
    L, gWs = nn.loss_and_grad(r, e, dinv, Ws, dof, free, hvp)
    h = 1e-6
    for l in range(3):
        for _ in range(4):
            idw = tuple(rng.integers(0, s) for s in Ws[l].shape)
            Wp = [W.copy() for W in Ws]
            Wm = [W.copy() for W in Ws]
            Wp[l][idw] += h
            Wm[l][idw] -= h
            fd = (nn.loss_and_grad(r, e, dinv, Wp, dof, free, hvp)[0] -
                  nn.loss_and_grad(r, e, dinv, Wm, dof, free, hvp)[0]) / (2 * h)
            assert np.isclose(gWs[l][idw], fd, rtol=1e-5, atol=1e-9), (l, idw)


def test_loss_is_zero_for_an_exact_preconditioner_and_scale_free():
    """With H diagonal, Jacobi (zero network) is the exact inverse: the H-cosine is 1.  The loss
    depends only on the direction of z: positive homogeneity of the network makes it invariant to
    the scale of r, and it is bounded by [0, 2]."""
    shape = (4, 3, 3)
    dof, free = masks(shape, 14)
    rng = np.random.default_rng(15)
    hdiag = free[..., None] * rng.uniform(1.0, 3.0, shape + (3,)) + (1 - free[..., None])

    def hvp(v):
        return free[..., None] * hdiag * v

    dinv = free[..., None] / hdiag
    r = free[..., None] * rng.standard_normal(shape + (3,))
    e = dinv * r
    zero = [np.zeros_like(W) for W in nn.init_weights(0)]
    L0, _ = nn.loss_and_grad(r, e, dinv, zero, dof, free, hvp)
    assert abs(L0) < 1e-14
    Ws = nn.init_weights(16)
    L1, _ = nn.loss_and_grad(r, e, dinv, Ws, dof, free, hvp)
    L2, _ = nn.loss_and_grad(5.0 * r, 5.0 * e, dinv, Ws, dof, free, hvp)
    assert 0.0 < L1 < 2.0 and abs(L1 - L2) < 1e-12
