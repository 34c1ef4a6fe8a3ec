"""GPU parity of the convolutional surrogate (forward and backward) against the oracle.

FP32 reference mode (every layer on CUDA cores): 1e-5 relative L2.  BF16 mode (every
layer on the tcgen05 tensor cores, BF16 activations and input, FP32 accumulation): 1e-2
relative L2 for outputs, 2e-2 for gradients through the smooth GELU (BF16 keeps 8
significant bits; the rounding of the input and of each stored activation is ~2^-9
relative and adds up over the layers, and bias gradients are sums over all sites whose
cancellation raises their relative error: measured up to 1.2e-2 for 4 layers, 1.4e-2
for 6).  Through ReLU the gradient is discontinuous in the
pre-activation: where the BF16 pre-activation lies within its rounding noise of zero the
gate differs from the FP64 one, and those entries carry the whole gradient or none (3-10%
relative L2 measured); ReLU gradients are checked to 0.15 only, the forward to 1e-2.
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cl():
    from paper_2607_24978_gb300 import build_ext, cl as clmod
    build_ext.build()
    clmod.lib()
    return clmod


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make_net(seed, cin, cout, hidden, layers):
    g = inputs.rng(seed)
    net = []
    for l in range(layers):
        ci = cin if l == 0 else hidden
        co = cout if l == layers - 1 else hidden
        W = g.standard_normal((27, co, ci)) * np.sqrt(2.0 / (27 * ci))
        b = 0.1 * g.standard_normal(co)
        net.append((W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)))
    return net


def run(cl, N, net, act, precision, x, g, want_dx=True):
    cin, cout = net[0][0].shape[2], net[-1][0].shape[1]
    hidden = net[0][0].shape[1]
    with cl.Surrogate(N, cin, cout, hidden, len(net), act, precision) as s:
        for l, (W, b) in enumerate(net):
            s.set_weights(l, W, b)
        y = s.forward(x.astype(np.float32))
        nf = s.last_launch_count()
        dx = s.backward(g.astype(np.float32), want_dx=want_dx)
        grads = [s.grads(l) for l in range(len(net))]
    return y, dx, grads, nf


OACT = {1: O.RELU, 2: O.GELU}


@pytest.mark.parametrize("act", [1, 2])
@pytest.mark.parametrize("N,hidden,layers", [(8, 16, 4), (6, 32, 3)])
def test_fp32_mode_matches_oracle(cl, act, N, hidden, layers):
    net = make_net(1, 3, 2, hidden, layers)
    x = inputs.rng(2).standard_normal((N, N, N, 3)).astype(np.float32).astype(np.float64)
    g = inputs.rng(3).standard_normal((N, N, N, 2)).astype(np.float32).astype(np.float64)
    y, dx, grads, nf = run(cl, N, net, act, cl.CL_SG_FP32, x, g)
    yo, cache = O.surrogate_forward(x, net, OACT[act])
    dxo, go = O.surrogate_backward(cache, net, g, OACT[act])
    assert rel_l2(y, yo) < 1e-5
    assert rel_l2(dx, dxo) < 1e-5
    for l in range(layers):
        assert rel_l2(grads[l][0], go[l][0]) < 1e-5, l
        assert rel_l2(grads[l][1], go[l][1]) < 1e-5, l
    assert nf == layers


@pytest.mark.parametrize("act", [1, 2])
@pytest.mark.parametrize("hidden", [16, 32, 48])
def test_bf16_tensor_core_mode_matches_oracle(cl, act, hidden):
    N, layers = 16, 4
    net = make_net(4, 3, 2, hidden, layers)
    x = inputs.rng(5).standard_normal((N, N, N, 3)).astype(np.float32).astype(np.float64)
    g = inputs.rng(6).standard_normal((N, N, N, 2)).astype(np.float32).astype(np.float64)
    y, dx, grads, nf = run(cl, N, net, act, cl.CL_SG_BF16, x, g)
    yo, cache = O.surrogate_forward(x, net, OACT[act])
    dxo, go = O.surrogate_backward(cache, net, g, OACT[act])
    # the network part of y (the residual x is exact) carries the BF16 rounding
    assert rel_l2(y - x[..., :2], yo - x[..., :2]) < 1e-2
    tol = 2e-2 if act == 2 else 0.15
    assert rel_l2(dx, dxo) < tol
    for l in range(layers):
        assert rel_l2(grads[l][0], go[l][0]) < tol, l
        assert rel_l2(grads[l][1], go[l][1]) < tol, l


def test_bf16_matches_fp32_mode_at_production_width(cl):
    """48 channels, 6 layers (the production shape) on a 32^3 lattice: several tiles in x
    and y and several z units per block; compared with the FP32 reference mode."""
    N = 32
    net = make_net(7, 3, 2, 48, 6)
    x = inputs.rng(8).standard_normal((N, N, N, 3))
    g = inputs.rng(9).standard_normal((N, N, N, 2))
    for act in (1, 2):
        yb, dxb, gb, _ = run(cl, N, net, act, cl.CL_SG_BF16, x, g)
        yf, dxf, gf, _ = run(cl, N, net, act, cl.CL_SG_FP32, x, g)
        assert rel_l2(yb - x[..., :2], yf - x[..., :2]) < 1e-2
        if act == 2:
            assert rel_l2(dxb, dxf) < 2e-2
            for l in range(6):
                assert rel_l2(gb[l][0], gf[l][0]) < 2.5e-2, l
                assert rel_l2(gb[l][1], gf[l][1]) < 2.5e-2, l


def test_shift_network_is_exact(cl):
    """Layers that copy channels through single taps: centre (first layer), +x and +y (the
    two tensor-core layers), +z (last layer).  With inputs exactly representable in BF16 and
    positive (ReLU passes them), y[n] = x[n] + x[n + e_x + e_y + e_z] exactly: a check of the
    tap offsets, the periodic halo and the tile mapping of the tensor-core kernel."""
    N, C = 16, 16
    taps = [13, 14, 16, 22]  # (0,0,0), (+1,0,0), (0,+1,0), (0,0,+1)
    net = []
    for l in range(4):
        ci = 3 if l == 0 else C
        co = 2 if l == 3 else C
        W = np.zeros((27, co, ci))
        k = min(co, ci)
        W[taps[l], :k, :k] = np.eye(k)
        net.append((W, np.zeros(co)))
    x = (inputs.rng(10).integers(4, 16, size=(N, N, N, 3)) / 8.0).astype(np.float32)
    with cl.Surrogate(N, 3, 2, C, 4, 1, cl.CL_SG_BF16) as s:
        for l, (W, b) in enumerate(net):
            s.set_weights(l, W, b)
        y = s.forward(x)
    shifted = np.roll(np.roll(np.roll(x, -1, axis=2), -1, axis=1), -1, axis=0)
    assert np.array_equal(y, x[..., :2] + shifted[..., :2])


def test_invalid_configurations(cl):
    with pytest.raises(cl.CLError):
        cl.Surrogate(24, 3, 2, 48, 6, 1, cl.CL_SG_BF16)   # BF16 needs N % 16 == 0
    with pytest.raises(cl.CLError):
        cl.Surrogate(16, 3, 2, 40, 6, 1, cl.CL_SG_BF16)   # hidden width 16, 32 or 48
    with pytest.raises(cl.CLError):
        cl.Surrogate(16, 2, 3, 16, 6, 1, cl.CL_SG_BF16)   # out_channels <= in_channels
    with cl.Surrogate(16, 3, 2, 16, 3, 1, cl.CL_SG_BF16) as s:
        with pytest.raises(cl.CLError):
            s.backward(np.zeros((16, 16, 16, 2), np.float32))  # no forward yet
