"""Pins of the oracle's convolutional-surrogate layers.

  * the periodic 3x3x3 convolution equals circular cross-correlation computed with FFTs
    (numpy.fft; a different algorithm reaching the same result);
  * an identity centre tap reproduces the input, a single off-centre tap shifts it;
  * the data gradient is the adjoint of the convolution: <conv x, g> = <x, conv^T g>;
  * the weight and bias gradients satisfy <conv_{W,b} x, g> = <W, dW> + <b, db> (the
    convolution is linear in (W, b));
  * the network gradient (activations, residual jump included) matches central finite
    differences of <out, g>;
  * the activation derivatives match finite differences, and the tanh form of GELU stays
    within 1e-3 of u Phi(u).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs


def rand(shape, seed):
    return inputs.rng(seed).standard_normal(shape)


def offsets():
    return [(t % 3 - 1, (t // 3) % 3 - 1, t // 9 - 1) for t in range(27)]


def conv_fft(x, W, b):
    """y[n, co] = b[co] + sum_t sum_ci W[t, co, ci] x[n + o(t), ci] by FFT: a correlation
    with the kernel placed at -o(t)."""
    N, cin = x.shape[0], x.shape[3]
    cout = W.shape[1]
    X = np.fft.fftn(x, axes=(0, 1, 2))
    y = np.zeros((N, N, N, cout))
    for co in range(cout):
        for ci in range(cin):
            k = np.zeros((N, N, N))
            for t, (ox, oy, oz) in enumerate(offsets()):
                k[(-oz) % N, (-oy) % N, (-ox) % N] += W[t, co, ci]
            y[..., co] += np.real(np.fft.ifftn(X[..., ci] * np.fft.fftn(k)))
        y[..., co] += b[co]
    return y


@pytest.mark.parametrize("N,cin,cout", [(4, 3, 5), (6, 2, 3), (5, 4, 2)])
def test_conv_equals_fft_circular_correlation(N, cin, cout):
    x, W, b = rand((N, N, N, cin), 1), rand((27, cout, cin), 2), rand(cout, 3)
    y = O.conv3d_fwd(x, W, b)
    ref = conv_fft(x, W, b)
    assert np.abs(y - ref).max() < 1e-12 * np.abs(ref).max()


def test_identity_and_shift_kernels():
    N, C = 5, 3
    x = rand((N, N, N, C), 4)
    W = np.zeros((27, C, C))
    W[13] = np.eye(C)  # centre tap (0, 0, 0)
    b = np.arange(C, dtype=float)
    assert np.array_equal(O.conv3d_fwd(x, W, b), x + b)
    W = np.zeros((27, C, C))
    W[14] = np.eye(C)  # tap (tx, ty, tz) = (2, 1, 1): offset +1 along x
    assert np.array_equal(O.conv3d_fwd(x, W), np.roll(x, -1, axis=2))
    W = np.zeros((27, C, C))
    W[1 + 3 * 1 + 9 * 0] = np.eye(C)  # offset -1 along z
    assert np.array_equal(O.conv3d_fwd(x, W), np.roll(x, 1, axis=0))


@pytest.mark.parametrize("N,cin,cout", [(4, 3, 5), (5, 4, 4)])
def test_data_gradient_is_the_adjoint(N, cin, cout):
    x, W, g = rand((N, N, N, cin), 5), rand((27, cout, cin), 6), rand((N, N, N, cout), 7)
    lhs = np.sum(O.conv3d_fwd(x, W) * g)
    rhs = np.sum(x * O.conv3d_bwd_data(g, W))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("N,cin,cout", [(4, 3, 5), (5, 4, 2)])
def test_weight_gradient_identity(N, cin, cout):
    x, W, b, g = rand((N, N, N, cin), 8), rand((27, cout, cin), 9), rand(cout, 10), rand((N, N, N, cout), 11)
    dW, db = O.conv3d_bwd_weight(x, g)
    lhs = np.sum(O.conv3d_fwd(x, W, b) * g)
    rhs = np.sum(W * dW) + np.sum(b * db)
    assert abs(lhs - rhs) < 1e-12 * np.sum(np.abs(W * dW))
    # a second, independent check of single entries: the derivative of a linear function
    for (t, co, ci) in [(0, 0, 0), (13, cout - 1, cin - 1), (26, 1, 2 % cin)]:
        E = np.zeros_like(W)
        E[t, co, ci] = 1.0
        assert np.sum(O.conv3d_fwd(x, E) * g) == pytest.approx(dW[t, co, ci], rel=1e-12, abs=1e-12)


def small_net(seed, chans=(3, 4, 4, 2)):
    g = inputs.rng(seed)
    return [(0.3 * g.standard_normal((27, chans[i + 1], chans[i])), 0.1 * g.standard_normal(chans[i + 1]))
            for i in range(len(chans) - 1)]


@pytest.mark.parametrize("act", [O.RELU, O.GELU])
def test_network_gradient_matches_finite_differences(act):
    N = 4
    layers = small_net(12)
    x = rand((N, N, N, 3), 13)
    g = rand((N, N, N, 2), 14)

    def loss(xx, ll):
        return float(np.sum(O.surrogate_forward(xx, ll, act)[0] * g))

    out, cache = O.surrogate_forward(x, layers, act)
    dx, grads = O.surrogate_backward(cache, layers, g, act)
    eps = 1e-6
    r = inputs.rng(15)
    for _ in range(6):
        li = int(r.integers(len(layers)))
        W, b = layers[li]
        idx = tuple(int(r.integers(s)) for s in W.shape)
        Wp, Wm = W.copy(), W.copy()
        Wp[idx] += eps
        Wm[idx] -= eps
        lp = [(Wp, b) if i == li else layers[i] for i in range(len(layers))]
        lm = [(Wm, b) if i == li else layers[i] for i in range(len(layers))]
        fd = (loss(x, lp) - loss(x, lm)) / (2 * eps)
        assert grads[li][0][idx] == pytest.approx(fd, rel=1e-6, abs=1e-8)
        co = int(r.integers(b.shape[0]))
        bp, bm = b.copy(), b.copy()
        bp[co] += eps
        bm[co] -= eps
        lp = [(W, bp) if i == li else layers[i] for i in range(len(layers))]
        lm = [(W, bm) if i == li else layers[i] for i in range(len(layers))]
        fd = (loss(x, lp) - loss(x, lm)) / (2 * eps)
        assert grads[li][1][co] == pytest.approx(fd, rel=1e-6, abs=1e-8)
        xi = tuple(int(r.integers(s)) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[xi] += eps
        xm[xi] -= eps
        fd = (loss(xp, layers) - loss(xm, layers)) / (2 * eps)
        assert dx[xi] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_activations():
    u = np.linspace(-4.0, 4.0, 81) + 0.0123
    for act in (O.RELU, O.GELU):
        h = 1e-6
        fd = (O.activation(act, u + h) - O.activation(act, u - h)) / (2 * h)
        assert np.allclose(O.activation_bwd(act, u, np.ones_like(u)), fd, rtol=1e-7, atol=1e-8)
    assert np.array_equal(O.activation(O.RELU, u), np.maximum(u, 0.0))
    phi = 0.5 * (1.0 + np.array([math.erf(v / math.sqrt(2.0)) for v in u]))
    assert np.abs(O.activation(O.GELU, u) - u * phi).max() < 1e-3
