"""The U-Net kernels (include/lbnci_unet.h) against the FP64 oracle (oracle/unet_oracle.py).

Single operators see exactly the BF16 values the oracle sees. Their bounds follow from the
arithmetic: a K-term FP32 sum s of products (exact in FP32 for BF16 operands) satisfies
|s - exact| <= K 2^-24 sum|terms| (sequential summation bound; 2^-23 is used to cover the
tensor cores' alignment truncation), and rounding s to BF16 adds at most 2^-8 |s|. The
rounded result equals the oracle's BF16 rounding of the exact value except where s falls
within the accumulation error of a rounding boundary: at least 99% of the elements must
match exactly.

A whole network chains ~2L BF16 roundings: each flipped rounding perturbs every output
of the next layer by a fraction of an ulp and so flips further roundings, and the
differences grow until they are as large as BF16 rounding itself (measured: a 3-level
network differs from the BF16-emulating oracle by 60% of the emulation's own distance to
FP64). So the network is held to "as accurate as BF16 storage permits": for the output
and every parameter gradient, the distance to the exact FP64 network is at most 1.5x the
distance of the BF16-emulating oracle plus 1e-3.
"""
import numpy as np
import pytest

from oracle import unet_oracle as U
from paper_2003_11069_gb300 import inputs, unet

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _bf16_tensor(a):
    return torch.tensor(U.bf16(a).astype(np.float32), device="cuda").to(torch.bfloat16)


def _np(t):
    return t.float().cpu().numpy().astype(np.float64)


def _op_check(got, exact, scale, K):
    """got: GPU BF16 values; exact: FP64 result; scale: sum of |terms| per element."""
    bound = 2.0 ** -8 * np.abs(exact) + K * 2.0 ** -23 * scale
    assert np.all(np.abs(got - exact) <= bound), np.max(np.abs(got - exact) / np.maximum(bound, 1e-300))
    assert np.mean(got == U.bf16(exact)) >= 0.99, np.mean(got == U.bf16(exact))


@pytest.mark.parametrize("mma", ["tcgen05", "sync"])
@pytest.mark.parametrize("B,H,W,Ci,Co,up,relu,xs_pad,ys_pad", [
    (2, 16, 32, 32, 64, 0, 1, 0, 0),
    (1, 8, 24, 64, 32, 0, 0, 32, 32),   # strided views (channel slices), 192 pixels: ragged tile
    (3, 8, 16, 64, 64, 1, 1, 0, 64),    # nearest-upsampled input
    (1, 2, 4, 256, 128, 0, 1, 0, 0),    # coarsest-level shape
    (2, 8, 32, 128, 256, 0, 1, 0, 0),   # two output-channel tiles of 128
    (1, 8, 40, 32, 96, 0, 0, 0, 32),    # three output-channel tiles of 32, 320 pixels
])
def test_conv3x3_forward(B, H, W, Ci, Co, up, relu, xs_pad, ys_pad, mma, monkeypatch):
    """mma: the convolution on the fifth-generation tensor cores (tcgen05.mma, accumulator
    in tensor memory; LBNCI_UNET_MMA=tcgen05) or on the mma.sync path (the default)."""
    monkeypatch.setenv("LBNCI_UNET_MMA", mma)
    rng = np.random.default_rng(B * 100 + Ci + Co)
    hi, wi = (H // 2, W // 2) if up else (H, W)
    xs, ys = Ci + xs_pad, Co + ys_pad
    xfull = U.bf16(rng.normal(size=(B, hi, wi, xs)))
    w = U.bf16(rng.normal(size=(Co, 3, 3, Ci)) * np.sqrt(2.0 / (9 * Ci)))
    b = rng.normal(size=Co).astype(np.float32).astype(np.float64) * 0.1
    x = xfull[..., :Ci]
    xin = U.upsample2(x) if up else x
    ref = U.conv3x3(xin, w, b)
    ref = np.maximum(ref, 0) if relu else ref
    scale = U.conv3x3(np.abs(xin), np.abs(w), np.abs(b))
    xt = _bf16_tensor(xfull)
    wt = _bf16_tensor(w.reshape(Co, 9, Ci))
    bt = torch.tensor(b.astype(np.float32), device="cuda")
    yt = torch.full((B, H, W, ys), 7.0, device="cuda", dtype=torch.bfloat16)
    unet.conv3x3(xt, xs, B, H, W, Ci, up, wt, bt, relu, yt, ys, Co)
    torch.cuda.synchronize()
    got = _np(yt)
    _op_check(got[..., :Co], ref, scale, 9 * Ci)
    assert np.all(got[..., Co:] == 7.0)   # channels outside the output slice untouched


@pytest.mark.parametrize("B,H,W,Ci,Co,up", [
    (2, 16, 32, 32, 32, 0),
    (1, 16, 64, 64, 128, 0),
    (2, 8, 16, 128, 64, 1),
])
def test_conv3x3_weight_gradient(B, H, W, Ci, Co, up):
    rng = np.random.default_rng(7 + Ci)
    hi, wi = (H // 2, W // 2) if up else (H, W)
    x = U.bf16(rng.normal(size=(B, hi, wi, Ci)))
    dy = U.bf16(rng.normal(size=(B, H, W, Co)))
    xin = U.upsample2(x) if up else x
    _, dw_ref, db_ref = U.conv3x3_bwd(xin, np.zeros((Co, 3, 3, Ci)), dy)
    _, scale, bscale = U.conv3x3_bwd(np.abs(xin), np.zeros((Co, 3, 3, Ci)), np.abs(dy))
    work = torch.empty(unet.conv3x3_wgrad_work(B, H, W, Ci, Co) // 4 + 1, device="cuda", dtype=torch.float32)
    dw = torch.zeros(Co * 9 * Ci, device="cuda", dtype=torch.float32)
    db = torch.zeros(Co, device="cuda", dtype=torch.float32)
    unet.conv3x3_wgrad(_bf16_tensor(x), Ci, B, H, W, Ci, up, _bf16_tensor(dy), Co, Co, dw, db, work)
    torch.cuda.synchronize()
    got = dw.cpu().numpy().astype(np.float64).reshape(Co, 3, 3, Ci)
    K = B * H * W
    assert np.all(np.abs(got - dw_ref) <= K * 2.0 ** -23 * scale)
    assert np.all(np.abs(db.cpu().numpy() - db_ref) <= K * 2.0 ** -23 * bscale)


def _small(levels=3, H=16, W=32, B=2, seed=0):
    cfg = unet.make_config(levels=levels, base=32, in_ch=5, out_ch=3, H=H, W=W, max_batch=B)
    shapes = U.layer_shapes(levels, 32, 5, 3)
    params = inputs.unet_params(shapes, seed, bias_scale=0.05)
    rng = np.random.default_rng(seed + 1)
    x = rng.normal(size=(B, H, W, 5)).astype(np.float32).astype(np.float64)
    t = rng.normal(size=(B, H, W, 3)).astype(np.float32).astype(np.float64)
    return cfg, params, x, t


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("levels,mma", [(2, "sync"), (3, "sync"), (4, "sync"), (3, "tcgen05")])
def test_network_forward_loss_and_gradients(levels, mma, monkeypatch):
    """mma: which kernel runs the 3x3 convolutions and their data gradients (the mma.sync
    default, or tcgen05.mma with the accumulator in tensor memory)."""
    monkeypatch.setenv("LBNCI_UNET_MMA", mma)
    cfg, params, x, t = _small(levels=levels, H=16, W=32, B=2, seed=levels)
    lam = [1.0, 0.5, 2.0]
    L_e, g_e, y_e = U.loss_and_grads(params, x, t, levels=levels, lam=lam, emulate_bf16=True)
    L_0, g_0, y_0 = U.loss_and_grads(params, x, t, levels=levels, lam=lam, emulate_bf16=False)
    with unet.Net(cfg) as net:
        net.set_params(unet.flatten(params))
        y = net.forward(x.astype(np.float32)).astype(np.float64)
        X = torch.tensor(x.astype(np.float32), device="cuda")
        T = torch.tensor(t.astype(np.float32), device="cuda")
        G = torch.zeros(net.nparams, device="cuda")
        L = net.loss_grad(X, T, lam=lam, grads=G)
        G2 = torch.zeros_like(G)
        net.loss_grad(X, T, lam=lam, grads=G2)
        g = G.cpu().numpy().astype(np.float64)
        assert torch.equal(G, G2)   # deterministic (fixed-order reductions)

    def within(got, emul, exact, what):
        assert _rel(got, exact) <= 1.5 * _rel(emul, exact) + 1e-3, (what, _rel(got, exact), _rel(emul, exact))
    within(y, y_e, y_0, "output")
    assert abs(L - L_0) <= 1.5 * abs(L_e - L_0) + 1e-3 * L_0
    got = unet.unflatten(g, unet.layer_shapes(cfg))
    for k, ((gw, gb), (ew, eb), (rw, rb)) in enumerate(zip(got, g_e, g_0)):
        within(gw, ew, rw, ("weight", k))
        within(gb, eb, rb, ("bias", k))
    if levels == 2:
        # a shallow chain: the emulation accounts for most of the GPU's rounding
        assert _rel(y, y_e) < 0.3 * _rel(y_e, y_0)


def test_forward_host_and_device_agree_and_batch_rows_independent():
    cfg, params, x, _ = _small(levels=3, B=3, seed=11)
    with unet.Net(cfg) as net:
        net.set_params(unet.flatten(params))
        y_host = net.forward(x.astype(np.float32))
        X = torch.tensor(x.astype(np.float32), device="cuda")
        Y = torch.empty((3, cfg.H, cfg.W, 3), device="cuda")
        net.forward(X, Y)
        y1 = net.forward(x[1:2].astype(np.float32))
    assert np.array_equal(y_host, Y.cpu().numpy())
    assert np.array_equal(y_host[1:2], y1)


def test_adam_steps_follow_the_oracle():
    """Three Adam steps on the GPU against the oracle's Adam (Kingma and Ba, Algorithm 1)
    driven by the oracle's gradients, with and without BF16 emulation. Adam moves every
    parameter by about lr per step whatever the size of its gradient, so the moves are
    compared with the same "as accurate as BF16 permits" rule as the gradients."""
    levels = 3
    cfg, params, x, t = _small(levels=levels, B=2, seed=21)
    lr, steps = 1e-3, 3
    flat0 = unet.flatten(params)
    with unet.Net(cfg) as net:
        net.set_params(flat0)
        X = torch.tensor(x.astype(np.float32), device="cuda")
        T = torch.tensor(t.astype(np.float32), device="cuda")
        for _ in range(steps):
            net.train_step(X, T, lr=lr)
        got = net.get_params().astype(np.float64)

    def oracle_moves(emulate):
        p = [(w.copy(), b.copy()) for w, b in params]
        m = [(np.zeros_like(w), np.zeros_like(b)) for w, b in params]
        v = [(np.zeros_like(w), np.zeros_like(b)) for w, b in params]
        for s_ in range(1, steps + 1):
            _, g, _ = U.loss_and_grads(p, x, t, levels=levels, emulate_bf16=emulate)
            for k in range(len(p)):
                nw = U.adam(p[k][0], g[k][0], m[k][0], v[k][0], s_, lr)
                nb = U.adam(p[k][1], g[k][1], m[k][1], v[k][1], s_, lr)
                p[k], m[k], v[k] = (nw[0], nb[0]), (nw[1], nb[1]), (nw[2], nb[2])
        return unet.flatten(p).astype(np.float64) - flat0
    d_got, d_emul, d_0 = got - flat0, oracle_moves(True), oracle_moves(False)
    assert _rel(d_got, d_0) <= 1.5 * _rel(d_emul, d_0) + 0.02, (_rel(d_got, d_0), _rel(d_emul, d_0))
    # Adam's step bound (Kingma and Ba, Sec. 2.1): |move| <= lr (1 - b1)/sqrt(1 - b2) per step
    assert np.max(np.abs(d_got)) <= steps * lr * 0.1 / np.sqrt(0.001) * 1.001
    assert np.mean(np.abs(d_got) > 0.5 * lr) > 0.5
