"""The warm-start U-Net: the numpy FP64 oracle against central finite
differences (CPU), and the GPU network's forward pass and gradients against
the oracle (GPU; the oracle then rounds activations to BF16 where the GPU
stores them)."""
import ctypes as C

import numpy as np
import pytest

from oracle import unet_oracle as U
from paper_2402_17337_gb300 import workloads as Wk

WIDTHS_TINY = (16, 16, 16, 16)
WIDTHS = (16, 32, 32, 48)


def rand_params(w, seed):
    rng = np.random.default_rng(seed)
    p = []
    for cin, cout, _ in U.layers(w):
        p.append(rng.standard_normal(cout * 9 * cin) * np.sqrt(2.0 / (9 * cin)))
        p.append(rng.standard_normal(cout) * 0.1)
    return np.concatenate(p)


def test_oracle_gradient_matches_finite_differences():
    w = WIDTHS_TINY
    params = rand_params(w, 1)
    feat = Wk.random_field((8, 16, 4), seed=2)
    target = Wk.random_field((8, 16), seed=3)
    loss, g = U.loss_and_grad(params, w, feat, target)
    rng = np.random.default_rng(4)
    idx = rng.choice(params.size, 40, replace=False)
    # include the first and last layers explicitly, and one weight and one
    # bias of every convolution
    per_layer, off = [], 0
    for cin, cout, _ in U.layers(w):
        per_layer += [off + (cout * 9 * cin) // 2, off + cout * 9 * cin + cout // 2]
        off += cout * 9 * cin + cout
    idx = np.concatenate([idx, [0, 5, params.size - 1, params.size - 20], per_layer])
    eps = 1e-6
    for k in idx:
        pp, pm = params.copy(), params.copy()
        pp[k] += eps
        pm[k] -= eps
        lp, _ = U.loss_and_grad(pp, w, feat, target)
        lm, _ = U.loss_and_grad(pm, w, feat, target)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (k, fd, g[k])


def test_oracle_parameter_count():
    w = (32, 64, 128, 128)
    assert U.num_params(w) == sum(co * 9 * ci + co for ci, co, _ in U.layers(w))


def _gpu_net(w, seed=7):
    import paper_2402_17337_gb300 as ibm
    from paper_2402_17337_gb300 import build
    build.build()
    return ibm.UNet(w, seed)


@pytest.mark.gpu
@pytest.mark.parametrize("H,W", [(16, 24), (32, 64)])
def test_gpu_unet_forward_and_gradients_match_oracle(H, W):
    import torch
    net = _gpu_net(WIDTHS)
    params = net.params().astype(np.float64)
    assert params.size == U.num_params(WIDTHS)
    feat = Wk.random_field((H, W, 4), seed=11).astype(np.float32)
    target = Wk.random_field((H, W), seed=12).astype(np.float32)
    fd = torch.tensor(feat, device="cuda")
    td = torch.tensor(target, device="cuda")
    out = torch.zeros(H, W, device="cuda")
    torch.cuda.synchronize()
    net.forward(fd.data_ptr(), H, W, out.data_ptr())
    torch.cuda.synchronize()
    ref, _ = U.forward(params, WIDTHS, feat.astype(np.float64), bf16=True)
    o = out.cpu().numpy()
    assert np.abs(o - ref).max() <= 2e-2 * np.abs(ref).max(), np.abs(o - ref).max() / np.abs(ref).max()
    loss = net.train_step(fd.data_ptr(), td.data_ptr(), H, W, lr=0.0, apply=False)
    g = net.grads().astype(np.float64)
    lref, gref = U.loss_and_grad(params, WIDTHS, feat.astype(np.float64), target.astype(np.float64), bf16=True)
    assert abs(loss - lref) <= 1e-2 * lref
    # per layer: relative error of the weight and bias gradients
    off = 0
    for cin, cout, _ in U.layers(WIDTHS):
        n = cout * 9 * cin + cout
        a, b = g[off:off + n], gref[off:off + n]
        err = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert err <= 5e-2, (cin, cout, err)
        off += n


@pytest.mark.gpu
def test_gpu_unet_training_reduces_loss():
    import torch
    net = _gpu_net(WIDTHS, seed=3)
    H, W = 32, 64
    yy, xx = np.meshgrid(np.linspace(0, 1, H), np.linspace(0, 1, W), indexing="ij")
    feat = np.stack([np.sin(3 * xx), np.cos(2 * yy), xx * yy, np.ones_like(xx)], axis=2).astype(np.float32)
    target = (0.5 * np.sin(3 * xx) * np.cos(2 * yy)).astype(np.float32)
    fd = torch.tensor(feat, device="cuda")
    td = torch.tensor(target, device="cuda")
    torch.cuda.synchronize()
    l0 = net.train_step(fd.data_ptr(), td.data_ptr(), H, W, lr=0.0, apply=False)
    for _ in range(200):
        l = net.train_step(fd.data_ptr(), td.data_ptr(), H, W, lr=2e-3, apply=True)
    assert l < 0.2 * l0, (l0, l)


def test_oracle_forward_matches_torch_cpu_reference():
    """The oracle's forward pass against the same network assembled from
    PyTorch CPU library operations in FP64 (cross-correlation conv2d with
    zero padding 1, 2x2 average pooling, nearest 2x upsampling, channel
    concatenation [upsampled deeper level, skip], ReLU, a head without
    ReLU whose channel 0 is the output): pins the oracle's own convolution,
    pooling and upsampling code and the wiring of the levels."""
    torch = pytest.importorskip("torch")
    import torch.nn.functional as F
    w = WIDTHS_TINY
    params = rand_params(w, 7)
    feat = Wk.random_field((16, 24, 4), seed=8)
    out, _ = U.forward(params, w, feat)
    P = U.unpack(params, w)

    def conv(x, k):
        Wk_, b, relu = P[k]
        weight = torch.tensor(Wk_.reshape(Wk_.shape[0], 3, 3, Wk_.shape[2])).permute(0, 3, 1, 2)
        y = F.conv2d(x, weight, torch.tensor(b), padding=1)
        return F.relu(y) if relu else y

    x = torch.zeros((1, 16) + feat.shape[:2], dtype=torch.float64)
    x[0, :4] = torch.tensor(feat).permute(2, 0, 1)
    e = []
    h = x
    for l in range(4):
        if l > 0:
            h = F.avg_pool2d(e[-1], 2)
        e.append(conv(conv(h, 2 * l), 2 * l + 1))
    d = e[3]
    for l, k in zip((2, 1, 0), (8, 10, 12)):
        cat = torch.cat([F.interpolate(d, scale_factor=2, mode="nearest"), e[l]], dim=1)
        d = conv(conv(cat, k), k + 1)
    ref = conv(d, 14)[0, 0].numpy()
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
