"""Pins of the network oracle (periodic 3^4 convolutions, ReLU, MSE loss).

The convolution is checked against an independent formulation (numpy.roll of
the whole field per tap), the backward passes against central finite
differences of the loss, and the data/weight gradients against the adjoint
identity <dY, conv(X)> = <conv^T(dY), X>.
"""
import numpy as np
import pytest

import oracle


def roll_conv(X, W, b, dims):
    """Y(s) = b + sum_k W_k X(s + d_k) with X on the (Lt,Lz,Ly,Lx) grid."""
    Lx, Ly, Lz, Lt = dims
    Xg = X.reshape(Lt, Lz, Ly, Lx, -1)
    Y = np.zeros((Lt, Lz, Ly, Lx, W.shape[1])) + (b if b is not None else 0)
    for k in range(81):
        d = (k % 3 - 1, (k // 3) % 3 - 1, (k // 9) % 3 - 1, (k // 27) % 3 - 1)
        # value at s + d: roll by -d along each axis (x axis 3, y 2, z 1, t 0)
        Xs = np.roll(Xg, shift=(-d[3], -d[2], -d[1], -d[0]), axis=(0, 1, 2, 3))
        Y += Xs @ W[k].T
    return Y.reshape(-1, W.shape[1])


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 4, 8)])
def test_conv_matches_roll_formulation(dims):
    rng = np.random.default_rng(1)
    V = int(np.prod(dims))
    X = rng.standard_normal((V, 5))
    W = rng.standard_normal((81, 3, 5))
    b = rng.standard_normal(3)
    np.testing.assert_allclose(oracle.conv_forward(X, W, b, dims), roll_conv(X, W, b, dims), atol=1e-12)


def test_conv_adjoints():
    dims = (4, 4, 6, 4)
    rng = np.random.default_rng(2)
    V = int(np.prod(dims))
    X = rng.standard_normal((V, 4))
    W = rng.standard_normal((81, 3, 4))
    dY = rng.standard_normal((V, 3))
    Y = oracle.conv_forward(X, W, None, dims)
    dX = oracle.conv_backward_data(dY, W, dims)
    assert np.sum(dY * Y) == pytest.approx(np.sum(dX * X), rel=1e-12)
    dW, db = oracle.conv_backward_weights(dY, X, dims, 4, 3)
    assert np.sum(dY * Y) == pytest.approx(np.sum(dW * W), rel=1e-12)
    np.testing.assert_allclose(db, dY.sum(axis=0), atol=1e-12)


def test_net_gradient_matches_finite_differences():
    dims = (4, 4, 4, 4)
    ch = (5, 4, 4, 3, 2)
    rng = np.random.default_rng(3)
    V = int(np.prod(dims))
    f = rng.standard_normal((V, ch[0]))
    t = rng.standard_normal((V, ch[4]))
    n = oracle.net_param_count(ch)
    p = rng.standard_normal(n) * 0.2
    loss, grad, _ = oracle.net_loss(f, t, p, dims, ch)
    idx = rng.choice(n, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(n)
        e[i] = h
        lp, _, _ = oracle.net_loss(f, t, p + e, dims, ch, want_grad=False)
        lm, _, _ = oracle.net_loss(f, t, p - e, dims, ch, want_grad=False)
        fd = (lp - lm) / (2 * h)
        assert grad[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_expmap_matches_scipy_and_is_su3():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    from paper_1209_4008_gb300 import synth
    lam = synth.gell_mann().numpy()
    rng = np.random.default_rng(4)
    for scale in (1e-3, 0.3, 2.0):
        c = rng.standard_normal((40, 8))
        g = oracle.expmap(c, scale)
        for j in range(40):
            H = scale * np.einsum("a,aij->ij", c[j], lam) / 2
            np.testing.assert_allclose(g[j], scipy_linalg.expm(1j * H), atol=1e-14)
            # squaring doubles the rounding error once per halving (|H| up to ~4 here)
            assert np.abs(g[j] @ g[j].conj().T - np.eye(3)).max() < 1e-13
            assert abs(np.linalg.det(g[j]) - 1) < 1e-13


def test_algebra_log_inverts_expmap_to_first_order():
    rng = np.random.default_rng(5)
    c = rng.standard_normal((50, 8))
    for s in (1e-3, 1e-5):
        got = oracle.algebra_log(oracle.expmap(c, s), s)
        np.testing.assert_allclose(got, c, atol=10 * s * s * np.abs(c).max() ** 3 + 1e-9)


def test_features_contain_links_and_scaled_violation():
    from paper_1209_4008_gb300 import synth
    dims = (4, 4, 4, 4)
    U = synth.as_numpy(synth.make_field(dims, 0.6, 7, 8))
    f = oracle.features(U, 0.5)
    np.testing.assert_array_equal(f[:, :72], U.reshape(256, 4, 9).view(np.float64).reshape(256, 72))
    # sum over a of (tr lambda_a D)^2 = 2 tr D^2, and theta = sum_x tr D^2 / (3V)
    theta = np.sum((f[:, 72:] * 0.5) ** 2) / 2 / (3 * 256)
    assert theta == pytest.approx(oracle.theta(U, 0), rel=1e-12)
