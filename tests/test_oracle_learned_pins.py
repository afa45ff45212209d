"""Pins for the FP64 oracle of the learned initialisation (oracle/learned.py): library
special cases, adjoint identities, finite differences and closed forms."""
import numpy as np
import pytest

from oracle import learned as L

scipy_signal = pytest.importorskip("scipy.signal")


def rng(seed):
    return np.random.default_rng(seed)


def test_conv_is_a_sum_of_2d_correlations():
    """stride 1 = scipy.signal.correlate2d summed over input channels; stride 2 = its even
    samples; upsampling = the same on the nearest-neighbour x2 image."""
    x = rng(0).standard_normal((2, 3, 8, 8))
    W = rng(1).standard_normal((4, 3, 3, 3))
    b = rng(2).standard_normal(4)
    ref = np.zeros((2, 4, 8, 8))
    for n in range(2):
        for o in range(4):
            ref[n, o] = b[o] + sum(scipy_signal.correlate2d(x[n, c], W[o, c], mode="same") for c in range(3))
    assert np.allclose(L.conv3x3(x, W, b, 1), ref, atol=1e-12)
    assert np.allclose(L.conv3x3(x, W, b, 2), ref[:, :, ::2, ::2], atol=1e-12)
    xu = np.kron(x, np.ones((1, 1, 2, 2)))
    assert np.allclose(L.conv3x3(x, W, b, 1, up=True), L.conv3x3(xu, W, b, 1), atol=1e-12)


@pytest.mark.parametrize("stride,up", [(1, False), (2, False), (1, True)])
def test_conv_backward_adjoint_and_finite_differences(stride, up):
    x = rng(3).standard_normal((2, 3, 8, 8))
    W = rng(4).standard_normal((5, 3, 3, 3))
    b = rng(5).standard_normal(5)
    out = L.conv3x3(x, W, b, stride, up)
    g = rng(6).standard_normal(out.shape)
    dx, dW, db = L.conv3x3_backward(x, W, g, stride, up)
    # adjoint identity of the linear map x -> conv(x) (no bias)
    z = np.zeros_like(b)
    assert abs(np.sum(L.conv3x3(x, W, z, stride, up) * g) - np.sum(x * dx)) < 1e-10 * np.abs(np.sum(x * dx))
    # weight and bias gradients by central differences of <g, conv>
    dWd = rng(7).standard_normal(W.shape)
    h = 1e-6
    fd = (np.sum(L.conv3x3(x, W + h * dWd, b, stride, up) * g) - np.sum(L.conv3x3(x, W - h * dWd, b, stride, up) * g)) / (2 * h)
    assert abs(fd - np.sum(dW * dWd)) < 1e-6 * abs(fd)
    assert np.allclose(db, g.sum(axis=(0, 2, 3)))


def test_network_gradient_by_central_differences():
    widths = (3, 4, 5)
    params = L.init_params(widths, seed=8)
    x = rng(9).standard_normal((2, 2, 16, 16))
    t = rng(10).standard_normal((2, 2, 16, 16))
    mask = (rng(11).random((16, 16)) > 0.3).astype(float)
    loss, grads = L.net_loss_and_grads(params, x, t, mask, widths)
    h = 1e-6
    for l in (0, 2, 5):
        W, b = params[l]
        d = rng(20 + l).standard_normal(W.shape)
        plus = [(Wi + h * d, bi) if i == l else (Wi, bi) for i, (Wi, bi) in enumerate(params)]
        minus = [(Wi - h * d, bi) if i == l else (Wi, bi) for i, (Wi, bi) in enumerate(params)]
        fd = (L.net_loss_and_grads(plus, x, t, mask, widths)[0] - L.net_loss_and_grads(minus, x, t, mask, widths)[0]) / (2 * h)
        assert abs(fd - np.sum(grads[l][0] * d)) <= 1e-5 * abs(fd) + 1e-12, l
        db = rng(30 + l).standard_normal(b.shape)
        plus = [(Wi, bi + h * db) if i == l else (Wi, bi) for i, (Wi, bi) in enumerate(params)]
        minus = [(Wi, bi - h * db) if i == l else (Wi, bi) for i, (Wi, bi) in enumerate(params)]
        fd = (L.net_loss_and_grads(plus, x, t, mask, widths)[0] - L.net_loss_and_grads(minus, x, t, mask, widths)[0]) / (2 * h)
        assert abs(fd - np.sum(grads[l][1] * db)) <= 1e-5 * abs(fd) + 1e-12, l


def test_network_shapes_and_loss_at_target():
    widths = (3, 4, 5)
    params = L.init_params(widths, seed=1)
    x = rng(2).standard_normal((1, 2, 16, 16))
    acts = L.net_forward(params, x, widths)
    assert [a.shape[2] for a in acts] == [16, 8, 4, 2, 4, 8, 16]
    mask = np.ones((16, 16))
    loss, _ = L.net_loss_and_grads(params, x, acts[-1], mask, widths)
    assert loss == 0.0


def test_physics_input_of_a_constant_object_is_its_modulus():
    """For O = c the exit wave is c P, sqrt(y) = |c| |F P|, so where |F P| stays above the
    phasor floor the back-propagated estimate is |c| P conj(P) / (|P|^2 + eps max|P|^2),
    i.e. ~|c| on the probe's support."""
    m = 16
    yy, xx = np.mgrid[0:m, 0:m]
    P = np.where((yy - 7.5) ** 2 + (xx - 7.5) ** 2 <= 25, np.exp(1j * 0.1 * ((yy - 7.5) ** 2 + (xx - 7.5) ** 2)), 0)
    FP = np.abs(np.fft.fft2(P, norm="ortho"))
    below = FP < L.U_FLOOR * FP.max()
    # the closed form below holds where the floor is inactive; the frequencies under it
    # carry (numerically) nothing for this probe
    assert not below.any() or FP[below].max() < 1e-13 * FP.max()
    c = 0.8 * np.exp(0.4j)
    y = np.abs(np.fft.fft2(c * P, norm="ortho")) ** 2
    e = L.physics_input(y[None], P, eps=1e-3)[0]
    est = e[0] + 1j * e[1]
    ref = abs(c) * np.abs(P) ** 2 / (np.abs(P) ** 2 + 1e-3 * np.max(np.abs(P) ** 2))
    assert np.allclose(est, ref, atol=1e-12)


def test_stitch_reproduces_consistent_patches():
    O = np.exp(1j * rng(12).standard_normal((20, 20)))
    m = 8
    P = np.ones((m, m)) * 0.5
    pos = np.array([[0, 0], [0, 6], [5, 3], [12, 12], [10, 2]])
    patches = [O[r:r + m, c:c + m] for r, c in pos]
    out = L.stitch(patches, pos, P, O.shape)
    covered = np.zeros(O.shape, bool)
    for r, c in pos:
        covered[r:r + m, c:c + m] = True
    assert np.allclose(out[covered], O[covered])
    assert np.all(out[~covered] == 1.0)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    v = np.concatenate([rng(13).standard_normal(1000), [1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 0.0]])
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(L.to_bf16(v), ref)


def test_given_relu_masks_select_the_backward_branches():
    """relu_masks equal to the forward's own decisions change nothing; a mask that switches
    every unit of the last hidden layer off cuts the gradient of all earlier layers and
    leaves the last layer's (which the masks do not enter)."""
    widths = (3, 4, 5)
    params = L.init_params(widths, seed=8)
    params = [(W, 0.1 * rng(40 + l).standard_normal(b.shape)) for l, (W, b) in enumerate(params)]
    x = rng(9).standard_normal((1, 2, 16, 16))
    t = rng(10).standard_normal((1, 2, 16, 16))
    mask = np.ones((16, 16))
    acts = L.net_forward(params, x, widths)
    own = [a > 0.0 for a in acts[1:6]]
    _, g0 = L.net_loss_and_grads(params, x, t, mask, widths)
    _, g1 = L.net_loss_and_grads(params, x, t, mask, widths, relu_masks=own)
    for (a, b), (c, d) in zip(g0, g1):
        assert np.array_equal(a, c) and np.array_equal(b, d)
    # masking every unit of the last hidden layer off cuts the gradient of all earlier layers
    off = [m.copy() for m in own]
    off[4][:] = False
    _, g2 = L.net_loss_and_grads(params, x, t, mask, widths, relu_masks=off)
    for l in range(5):
        assert not np.any(g2[l][0]) and not np.any(g2[l][1])
    assert np.allclose(g2[5][0], g0[5][0]) and np.allclose(g2[5][1], g0[5][1])
