"""Pins of the FP64 U-Net oracle (warm-start surrogate) against things other than itself.

* the 3x3 convolution against scipy's 2-D correlation on explicitly padded images;
* the whole backward pass against central finite differences of the loss (any
  dropped term, wrong index or transposed operand in a gradient fails it);
* adjoint identities of pooling/upsampling, closed forms of max pooling with ties;
* equivariance of the network under periodic shifts along x by 2^(L-1) columns (pins
  the periodic padding and the alignment of pooling and upsampling);
* the first Adam step against its closed form; bfloat16 rounding against torch.
"""
import numpy as np
import pytest

from oracle import unet_oracle as U
from paper_2003_11069_gb300 import inputs


def _net(levels=3, base=4, in_ch=2, out_ch=3, seed=0, bias_scale=0.1):
    return inputs.unet_params(U.layer_shapes(levels, base, in_ch, out_ch), seed, bias_scale)


def test_conv3x3_matches_scipy_correlation():
    from scipy import signal
    rng = np.random.default_rng(1)
    B, H, W, Ci, Co = 2, 6, 9, 3, 4
    x = rng.normal(size=(B, H, W, Ci))
    w = rng.normal(size=(Co, 3, 3, Ci))
    b = rng.normal(size=Co)
    y = U.conv3x3(x, w, b)
    for n in range(B):
        for o in range(Co):
            ref = np.full((H, W), b[o])
            for c in range(Ci):
                img = np.pad(x[n, :, :, c], ((0, 0), (1, 1)), mode="wrap")   # periodic in x
                img = np.pad(img, ((1, 1), (0, 0)), mode="constant")         # walls in y
                ref += signal.correlate2d(img, w[o, :, :, c], mode="valid")
            assert np.allclose(y[n, :, :, o], ref, rtol=0, atol=1e-12)


def test_head_is_a_pixelwise_linear_map():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1, 2, 3, 4))
    w = rng.normal(size=(3, 4))
    b = rng.normal(size=3)
    y = U.conv1x1(x, w, b)
    for i in range(2):
        for j in range(3):
            assert np.allclose(y[0, i, j], w @ x[0, i, j] + b, atol=1e-14)


def test_maxpool_ties_and_routing():
    x = np.zeros((1, 2, 4, 1))
    x[0, :, :2, 0] = [[1.0, 3.0], [3.0, 2.0]]     # tie between (0,1) and (1,0): first wins
    x[0, :, 2:, 0] = [[-1.0, -1.0], [-1.0, -1.0]]  # all equal: (0,0) wins
    y, arg = U.maxpool2(x)
    assert y[0, 0, :, 0].tolist() == [3.0, -1.0]
    assert arg[0, 0, :, 0].tolist() == [1, 0]
    d = U.maxpool2_bwd(arg, np.array([[[[5.0], [7.0]]]]))
    assert d[0, :, :, 0].tolist() == [[0.0, 5.0, 7.0, 0.0], [0.0, 0.0, 0.0, 0.0]]


def test_upsample_adjoint_and_pool_adjoint():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 3, 5, 4))
    y = rng.normal(size=(2, 6, 10, 4))
    assert np.isclose((U.upsample2(x) * y).sum(), (x * U.upsample2_bwd(y)).sum(), rtol=1e-13)
    # max pooling is linear once its argmax is fixed: <P x, d> = <x, P^T d>
    z = rng.normal(size=(2, 6, 10, 4))
    p, arg = U.maxpool2(z)
    d = rng.normal(size=p.shape)
    assert np.isclose((p * d).sum(), (z * U.maxpool2_bwd(arg, d)).sum(), rtol=1e-13)


def test_conv_backward_is_the_adjoint():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(2, 4, 6, 3))
    w = rng.normal(size=(5, 3, 3, 3))
    d = rng.normal(size=(2, 4, 6, 5))
    dx, dw, db = U.conv3x3_bwd(x, w, d)
    assert np.isclose((U.conv3x3(x, w, np.zeros(5)) * d).sum(), (x * dx).sum(), rtol=1e-12)
    # the weight gradient is the adjoint in w
    assert np.isclose((U.conv3x3(x, w, np.zeros(5)) * d).sum(), (w * dw).sum(), rtol=1e-12)
    assert np.allclose(db, d.sum(axis=(0, 1, 2)))


@pytest.mark.parametrize("levels", [2, 3])
def test_backward_matches_central_finite_differences(levels):
    rng = np.random.default_rng(5 + levels)
    params = _net(levels=levels, seed=levels)
    x = rng.normal(size=(2, 8, 16, 2))
    t = rng.normal(size=(2, 8, 16, 3))
    lam = np.array([1.0, 0.5, 2.0])
    L, grads, _ = U.loss_and_grads(params, x, t, levels=levels, lam=lam)
    eps, worst = 1e-6, 0.0

    def loss_with(i, which, idx, delta):
        p = [(w.copy(), b.copy()) for w, b in params]
        p[i][which][idx] += delta
        return U.mse(U.forward(p, x, levels)[0], t, lam)[0]
    for i, (w, b) in enumerate(params):
        for which, arr in ((0, w), (1, b)):
            for _ in range(3):
                idx = tuple(int(rng.integers(0, n)) for n in arr.shape)
                fd = (loss_with(i, which, idx, eps) - loss_with(i, which, idx, -eps)) / (2 * eps)
                an = grads[i][which][idx]
                worst = max(worst, abs(fd - an) / (abs(fd) + abs(an) + 1e-9))
    assert worst < 1e-6, worst


def test_periodic_shift_equivariance():
    levels = 3
    params = _net(levels=levels, seed=7)
    rng = np.random.default_rng(8)
    x = rng.normal(size=(1, 8, 16, 2))
    s = 2 ** (levels - 1)
    y0 = U.forward(params, x, levels)[0]
    y1 = U.forward(params, np.roll(x, s, axis=2), levels)[0]
    assert np.allclose(np.roll(y0, s, axis=2), y1, atol=1e-12)
    # a shift by one column is not a symmetry of the pooled network (sanity of the pin)
    y2 = U.forward(params, np.roll(x, 1, axis=2), levels)[0]
    assert not np.allclose(np.roll(y0, 1, axis=2), y2, atol=1e-6)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(9)
    th, g = rng.normal(size=50), rng.normal(size=50)
    lr, eps = 1e-3, 1e-8
    th1, m, v = U.adam(th, g, np.zeros(50), np.zeros(50), 1, lr, eps=eps)
    # bias-corrected moments of the first step are g and g^2
    assert np.allclose(th1, th - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    # with a constant gradient the corrected moments stay g and g^2 at every step
    t_, m_, v_ = th1, m, v
    for t in range(2, 6):
        t_, m_, v_ = U.adam(t_, g, m_, v_, t, lr, eps=eps)
    assert np.allclose(t_, th - 5 * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-13)


def test_bf16_rounding():
    one = 1.0
    assert U.bf16(np.array([one + 2.0 ** -8]))[0] == 1.0                   # tie -> even
    assert U.bf16(np.array([one + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6     # tie -> even
    assert U.bf16(np.array([one + 2.0 ** -8 + 2.0 ** -20]))[0] == 1.0 + 2.0 ** -7
    assert U.bf16(np.array([-2.5]))[0] == -2.5
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(10).normal(size=10000) * 10.0 ** np.random.default_rng(11).uniform(-5, 5, 10000)
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.bf16(x), ref)


def test_layer_shapes_of_the_configured_network():
    sh = U.layer_shapes()  # 4 levels, base 32, 5 inputs, 3 outputs
    assert len(sh) == 2 * 4 + 3 * 3 + 1
    assert sh[0] == ("enc0a", (32, 3, 3, 5)) and sh[7] == ("enc3b", (256, 3, 3, 256))
    assert sh[8] == ("up2", (128, 3, 3, 256)) and sh[9] == ("dec2a", (128, 3, 3, 256))
    assert sh[-1] == ("head", (3, 32))
