"""The proposal network's tensor-core kernels against the FP64 reference.

Two references: the plain FP64 network (inputs and weights rounded to BF16),
and the same primitives composed with BF16 rounding where the kernels store
BF16 (activations after ReLU, the loss gradient, each input gradient after
the ReLU mask). Against the second the kernels differ only by FP32 vs FP64
accumulation order and the rare BF16 rounding it flips: 1e-2 relative L2 per
parameter block, 2e-3 for the forward output. Against the first, rounding of
activations and gradients to 8-bit mantissas (relative 2^-9 each) compounds
over six layers and is amplified by cancellation in the weight-gradient sums:
forward 2e-2, gradients cosine > 0.99.
"""
import numpy as np
import pytest

from oracle import conv_net as cn

pytestmark = pytest.mark.gpu


def _bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).bfloat16().float().numpy().astype(np.float64)


def _case(T=2, H=10, W=37, seed=0):
    rng = np.random.default_rng(seed)
    params = cn.he_init(T, seed=seed)
    params = params + rng.normal(0, 0.02, size=params.shape).astype(np.float32)
    flows = rng.normal(0, 12.0, size=(T, H, W, 2)).astype(np.float32)
    target = np.stack([rng.normal(1.5, 0.5, size=(H, W)), rng.uniform(0, 1, size=(H, W))], -1).astype(np.float32)
    return params, flows, target


def _emulated(params, flows, target, T, lam_r):
    """FP64 network with BF16 rounding at the kernels' storage points."""
    layers = cn.unpack(params, T)
    acts = [_bf16(cn.net_input(flows.astype(np.float64)))]
    Wb = [(_bf16(W), b.astype(np.float32).astype(np.float64)) for W, b in layers]
    z = None
    for i, (W, b) in enumerate(Wb):
        z = cn.conv3x3(acts[-1], W, b)
        if i < len(Wb) - 1:
            acts.append(_bf16(np.maximum(z, 0.0)))
    # loss gradient at the output, as the reference computes it, stored BF16
    _, gz = _output_grad(z, target, lam_r)
    g = _bf16(gz)
    grads = []
    for i in range(len(Wb) - 1, -1, -1):
        gW, gb = cn.conv3x3_weight_grad(acts[i], g)
        grads.append((gW, gb))
        if i == 0:
            break
        g = _bf16(cn.conv3x3_input_grad(g, Wb[i][0]) * (acts[i] > 0))
    return z, cn.pack(grads[::-1])


def _output_grad(z, target, lam_r):
    """d loss / d z through the reference's loss, by its own backward pass on
    a network whose last layer is the identity."""
    t0, t1 = target[..., 0].astype(np.float64), target[..., 1].astype(np.float64)
    ok = np.isfinite(t0)
    n = z.shape[0] * z.shape[1]
    d = np.where(ok, z[..., 0] - np.where(ok, t0, 0.0), 0.0)
    g0 = np.where(np.abs(d) < 0.1, d / 0.1, np.sign(d))
    g1 = lam_r * (1.0 / (1.0 + np.exp(-z[..., 1])) - t1)
    gz = np.zeros_like(z)
    gz[..., 0] = np.where(ok, g0, 0.0) / n
    gz[..., 1] = np.where(ok, g1, 0.0) / n
    return None, gz


def _blocks(T, g):
    o = 0
    for ci, co in zip(*cn.shapes(T)):
        for n in (co * 9 * ci, co):
            yield (ci, co, n), g[o:o + n]
            o += n


def _rel(a, r):
    return np.linalg.norm(a - r) / max(np.linalg.norm(r), 1e-30)


def _cos(a, r):
    return a @ r / max(np.linalg.norm(a) * np.linalg.norm(r), 1e-30)


@pytest.fixture(scope="module")
def vd():
    from paper_2104_06789_gb300 import build, voldor
    build.build()
    return voldor


@pytest.mark.parametrize("T,H,W", [(2, 10, 37), (8, 9, 70)])
def test_forward_matches_reference(vd, T, H, W):
    import torch
    params, flows, target = _case(T, H, W, seed=T)
    net = vd.Net(T, params)
    pred = net.forward(torch.from_numpy(flows[None]).cuda()).cpu().numpy()[0]
    x = _bf16(cn.net_input(flows.astype(np.float64)))
    ref = cn.forward(_bf16(params), x, T)[-1]
    assert _rel(pred[..., :2], ref) < 2e-2
    z_emu, _ = _emulated(params, flows, target, T, 0.5)
    assert _rel(pred[..., :2], z_emu) < 2e-3
    assert np.all(pred[..., 2:] == 0)
    net.destroy()


def test_forward_into_unaligned_output(vd):
    """The last layer writes the caller's buffer directly when it is 16-byte
    aligned device memory, else the network's own buffer, which is copied:
    both give the same predictions bit for bit."""
    import ctypes

    import torch
    T, H, W = 2, 10, 37
    params, flows, _ = _case(T, H, W, seed=3)
    net = vd.Net(T, params)
    fl = torch.from_numpy(flows[None]).cuda()
    direct = net.forward(fl).cpu().numpy()
    n = H * W * 8
    buf = torch.full((n + 4,), -7.0, dtype=torch.float32, device="cuda")
    assert buf.data_ptr() % 16 == 0
    st = vd.lib().voldor_net_forward(net._h, ctypes.c_void_p(fl.data_ptr()), net._flow_dtype(fl), 1, H, W,
                                     ctypes.c_void_p(buf.data_ptr() + 4), ctypes.c_void_p(0))
    assert st == vd.OK
    got = buf.cpu().numpy()
    assert got[0] == -7.0 and np.all(got[n + 1:] == -7.0)
    assert np.array_equal(got[1:n + 1].reshape(direct.shape), direct)
    net.destroy()


@pytest.mark.parametrize("T,H,W", [(2, 10, 37), (8, 9, 70), (5, 33, 41)])
def test_gradients_match_reference(vd, T, H, W):
    import torch
    params, flows, target = _case(T, H, W, seed=T)
    target[3, 5, 0] = np.nan
    net = vd.Net(T, params)
    loss = net.train_step(torch.from_numpy(flows[None]).cuda(), torch.from_numpy(target[None]).cuda(), lr=0.0, lam_r=0.5)
    g = net.get_grads().astype(np.float64)
    x = _bf16(cn.net_input(flows.astype(np.float64)))
    loss_ref, g_ref = cn.loss_and_grads(_bf16(params), x, target.astype(np.float64), T, lam_r=0.5)
    _, g_emu = _emulated(params, flows, target, T, 0.5)
    assert loss == pytest.approx(loss_ref, rel=2e-2)
    report = []
    for (key, a), (_, r), (_, e) in zip(_blocks(T, g), _blocks(T, g_ref), _blocks(T, g_emu)):
        report.append((key, _rel(a, e), _rel(a, r), _cos(a, r)))
    bad = [r for r in report if not (r[1] < 1e-2 and r[3] > 0.99)]
    assert not bad, report
    net.destroy()


def test_training_reduces_the_loss(vd):
    import torch
    T = 2
    params, flows, target = _case(T, 24, 40, seed=5)
    net = vd.Net(T, params)
    f = torch.from_numpy(flows[None]).cuda()
    t = torch.from_numpy(target[None]).cuda()
    first = net.train_step(f, t, lr=1e-3)
    for _ in range(60):
        last = net.train_step(f, t, lr=1e-3)
    assert last < 0.7 * first, (first, last)
    w = net.get_weights()
    assert np.all(np.isfinite(w)) and not np.array_equal(w, params)
    net.destroy()


def test_learned_bootstrap_scale_alignment(vd):
    """With all weights zero the network outputs its last biases everywhere,
    so the learned bootstrap must give the depth exp(median log theta_tri)
    over the pixels strictly inside the depth range, and W = sigmoid(b_1)."""
    from paper_2104_06789_gb300 import synthetic
    w = synthetic.small_planes(seed=1000)
    p = vd.default_params(inv_depth_min=w.inv_depth_range[0], inv_depth_max=w.inv_depth_range[1],
                          hyps_per_frame=64)
    win = vd.Window(w.flows.astype(np.float32), w.K, p)
    win.bootstrap(w.poses[0])
    _, D_tri, _ = win.get_pose_depth_rigidness(poses=False, rigidness=False)
    params = np.zeros(vd.lib().voldor_net_num_params(w.T), np.float32)
    params[-2:] = (0.7, -0.4)                     # last layer's biases: log-depth, logit
    net = vd.Net(w.T, params)
    net.bootstrap(win, w.poses[0])
    _, D, Wm = win.get_pose_depth_rigidness(poses=False)
    d_min, d_max = np.float32(1 / w.inv_depth_range[1]), np.float32(1 / w.inv_depth_range[0])
    inside = (D_tri > d_min * np.float32(1.0001)) & (D_tri < d_max * np.float32(0.9999))
    v = np.sort(np.log(D_tri[inside].astype(np.float64)) - 0.7)
    expect = np.exp(v[(len(v) - 1) // 2] + 0.7)
    assert np.allclose(D, expect, rtol=2e-5), (D.min(), D.max(), expect)
    assert np.allclose(Wm, 1 / (1 + np.exp(0.4)), rtol=1e-6)
    net.destroy()
    win.destroy()


def _emulated_at(params, x0, T, ys, xs):
    """Emulated forward output at pixels (ys, xs) of the BF16 network input x0
    [H][W][2T], each from its own 13 x 13 crop (six 3x3 layers see six pixels
    to each side; the crop's zero border coincides with the image's)."""
    layers = [(_bf16(W), b.astype(np.float32).astype(np.float64)) for W, b in cn.unpack(params, T)]
    H, W = x0.shape[:2]
    out = []
    for y, x in zip(ys, xs):
        y0, y1, x0_, x1 = max(0, y - 6), min(H, y + 7), max(0, x - 6), min(W, x + 7)
        a = x0[y0:y1, x0_:x1]
        for i, (Wl, b) in enumerate(layers):
            a = cn.conv3x3(a, Wl, b)
            if i < len(layers) - 1:
                a = _bf16(np.maximum(a, 0.0))
        out.append(a[y - y0, x - x0_])
    return np.array(out)


def test_forward_full_size_sampled(vd):
    """8 images of 1242 x 375, T = 8, the launch shape of the proposal
    benchmark (1920 row strips on a persistent grid): the forward pass
    repeatable bit for bit, every image of the batch bit-identical to its own
    single-image forward, and outputs at the strip
    and row-chunk edges, image corners and interior points equal to the
    emulated BF16 network on crops."""
    import torch
    T, H, W, B = 8, 375, 1242, 8
    rng = np.random.default_rng(11)
    params = cn.he_init(T, seed=11) + rng.normal(0, 0.02, size=cn.he_init(T, seed=11).shape).astype(np.float32)
    flows = rng.normal(0, 12.0, size=(B, T, H, W, 2)).astype(np.float16)
    net = vd.Net(T, params)
    dev = torch.from_numpy(flows).cuda()
    pred = net.forward(dev).cpu().numpy()
    again = net.forward(dev).cpu().numpy()
    assert np.array_equal(again, pred), (np.sum(again != pred), np.abs(again - pred).max())
    for k in (0, 5, 7):
        one = net.forward(dev[k:k + 1].contiguous()).cpu().numpy()[0]
        assert np.array_equal(one, pred[k]), (k, np.sum(one != pred[k]), np.abs(one - pred[k]).max())
    ys = np.array([0, 1, 15, 16, 17, 200, 367, 368, 374])
    xs = np.array([0, 1, 127, 128, 129, 640, 1151, 1152, 1241])
    for k in (0, 7):
        x0 = _bf16(cn.net_input(flows[k].astype(np.float64)))
        yy, xx = np.meshgrid(ys, xs, indexing="ij")
        ref = _emulated_at(params, x0, T, yy.ravel(), xx.ravel())
        got = pred[k][yy.ravel(), xx.ravel(), :2]
        assert _rel(got, ref) < 2e-3, _rel(got, ref)
    net.destroy()


def test_gradients_batch_consistency(vd):
    """Two images of 1242 x 375 (480 row strips, more than one per CTA): the
    batch gradient equals the mean of the single-image gradients (the loss is
    a mean over pixels), up to FP32 atomic summation order."""
    import torch
    T, H, W = 2, 375, 1242
    rng = np.random.default_rng(5)
    params = cn.he_init(T, seed=5) + rng.normal(0, 0.02, size=cn.he_init(T, seed=5).shape).astype(np.float32)
    flows = rng.normal(0, 12.0, size=(2, T, H, W, 2)).astype(np.float32)
    target = np.stack([rng.normal(1.5, 0.5, size=(2, H, W)), rng.uniform(0, 1, size=(2, H, W))], -1).astype(np.float32)
    net = vd.Net(T, params)
    f, t = torch.from_numpy(flows).cuda(), torch.from_numpy(target).cuda()
    net.train_step(f, t, lr=0.0, lam_r=0.5)
    g = net.get_grads().astype(np.float64)
    gs = []
    for k in range(2):
        net.train_step(f[k:k + 1].contiguous(), t[k:k + 1].contiguous(), lr=0.0, lam_r=0.5)
        gs.append(net.get_grads().astype(np.float64))
    mean = 0.5 * (gs[0] + gs[1])
    for (key, a), (_, r) in zip(_blocks(T, g), _blocks(T, mean)):
        assert _rel(a, r) < 1e-3, (key, _rel(a, r))
    net.destroy()


def test_gradients_are_reproducible(vd):
    """The weight gradients are sums over hundreds of CTAs' partials, added in
    CTA order: two identical training steps give bit-identical gradients, and
    training from the same start gives bit-identical weights."""
    import torch
    T, H, W = 2, 375, 1242
    rng = np.random.default_rng(9)
    params = cn.he_init(T, seed=9) + rng.normal(0, 0.02, size=cn.he_init(T, seed=9).shape).astype(np.float32)
    flows = rng.normal(0, 12.0, size=(2, T, H, W, 2)).astype(np.float32)
    target = np.stack([rng.normal(1.5, 0.5, size=(2, H, W)), rng.uniform(0, 1, size=(2, H, W))], -1).astype(np.float32)
    f, t = torch.from_numpy(flows).cuda(), torch.from_numpy(target).cuda()
    grads, weights = [], []
    for _ in range(2):
        net = vd.Net(T, params)
        net.train_step(f, t, lr=0.0, lam_r=0.5)
        grads.append(net.get_grads())
        for _ in range(3):
            net.train_step(f, t, lr=1e-3, lam_r=0.5)
        weights.append(net.get_weights())
        net.destroy()
    assert np.array_equal(grads[0], grads[1])
    assert np.array_equal(weights[0], weights[1])
