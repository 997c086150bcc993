"""FP64 reference of the learned proposal network (test infrastructure).

Six 3x3 convolutions with zero padding, 2T -> 32 -> 32 -> 32 -> 32 -> 32 -> 2
channels, ReLU after the first five; input = the T flows, each divided by its
own mean flow magnitude over the image (channels 2t, 2t+1 = u_t, v_t); output channel 0 = log-depth, 1 = rigidness
logit. Loss per pixel: Huber (delta 0.1) on log-depth plus lam_r times binary
cross-entropy on the logit, averaged over pixels; a non-finite target
log-depth skips the pixel. Parameters: per layer W[Cout][3][3][Cin] then
bias[Cout], layers in order.

Plain definitions: the convolution is a sum over the nine taps of shifted
copies of the zero-padded input; the backward pass is the chain rule written
out per layer. Only tests and bench.py's CPU legs use this module.
"""
import numpy as np

WIDTH = 32


def shapes(T):
    cin = [2 * T] + [WIDTH] * 5
    cout = [WIDTH] * 5 + [2]
    return cin, cout


def num_params(T):
    cin, cout = shapes(T)
    return sum(co * 9 * ci + co for ci, co in zip(cin, cout))


def unpack(params, T):
    cin, cout = shapes(T)
    out, o = [], 0
    for ci, co in zip(cin, cout):
        W = params[o:o + co * 9 * ci].reshape(co, 3, 3, ci)
        o += co * 9 * ci
        b = params[o:o + co]
        o += co
        out.append((W, b))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def he_init(T, seed=0):
    rng = np.random.default_rng(seed)
    cin, cout = shapes(T)
    layers = []
    for ci, co in zip(cin, cout):
        std = np.sqrt(2.0 / (9 * ci))
        layers.append((rng.normal(0, std, size=(co, 3, 3, ci)), np.zeros(co)))
    return pack(layers).astype(np.float32)


def net_input(flows):
    """flows [T][H][W][2] -> x [H][W][2T], frame t scaled by 1 / mean |flow_t|."""
    T = flows.shape[0]
    out = []
    for t in range(T):
        m = np.mean(np.hypot(flows[t][..., 0], flows[t][..., 1]))
        out.append(flows[t] / m if m > 0 else np.zeros_like(flows[t]))
    return np.concatenate(out, axis=-1)


def conv3x3(x, W, b):
    """y[i, j, o] = b[o] + sum_{ky, kx, c} xpad[i + ky, j + kx, c] W[o, ky, kx, c]."""
    H, Wd, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (0, 0)))
    y = np.zeros((H, Wd, W.shape[0])) + b
    for ky in range(3):
        for kx in range(3):
            y += xp[ky:ky + H, kx:kx + Wd, :] @ W[:, ky, kx, :].T
    return y


def conv3x3_input_grad(gy, W):
    """d/dx of sum(gy * conv3x3(x, W, b))."""
    H, Wd, _ = gy.shape
    gx_p = np.zeros((H + 2, Wd + 2, W.shape[3]))
    for ky in range(3):
        for kx in range(3):
            gx_p[ky:ky + H, kx:kx + Wd, :] += gy @ W[:, ky, kx, :]
    return gx_p[1:-1, 1:-1, :]


def conv3x3_weight_grad(x, gy):
    H, Wd, C = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (0, 0)))
    gW = np.zeros((gy.shape[2], 3, 3, C))
    for ky in range(3):
        for kx in range(3):
            gW[:, ky, kx, :] = np.einsum("hwo,hwc->oc", gy, xp[ky:ky + H, kx:kx + Wd, :])
    return gW, gy.sum(axis=(0, 1))


def forward(params, x, T):
    layers = unpack(params, T)
    acts = [x]
    for i, (W, b) in enumerate(layers):
        z = conv3x3(acts[-1], W, b)
        acts.append(np.maximum(z, 0.0) if i < len(layers) - 1 else z)
    return acts


def loss_and_grads(params, x, target, T, lam_r=1.0):
    """target [H][W][2] (log-depth, rigidness). Returns (loss, grads)."""
    layers = unpack(params, T)
    acts = forward(params, x, T)
    z = acts[-1]
    t0, t1 = target[..., 0], target[..., 1]
    ok = np.isfinite(t0)
    n = z.shape[0] * z.shape[1]
    d = np.where(ok, z[..., 0] - np.where(ok, t0, 0.0), 0.0)
    delta = 0.1
    ad = np.abs(d)
    huber = np.where(ad < delta, 0.5 * d * d / delta, ad - 0.5 * delta)
    g0 = np.where(ad < delta, d / delta, np.sign(d))
    z1 = z[..., 1]
    bce = np.logaddexp(0.0, z1) - t1 * z1
    g1 = lam_r * (1.0 / (1.0 + np.exp(-z1)) - t1)
    loss = float(np.sum(np.where(ok, huber + lam_r * bce, 0.0)) / n)
    gz = np.zeros_like(z)
    gz[..., 0] = np.where(ok, g0, 0.0) / n
    gz[..., 1] = np.where(ok, g1, 0.0) / n
    grads = []
    g = gz
    for i in range(len(layers) - 1, -1, -1):
        W, b = layers[i]
        gW, gb = conv3x3_weight_grad(acts[i], g)
        grads.append((gW, gb))
        if i == 0:
            break
        g = conv3x3_input_grad(g, W) * (acts[i] > 0)
    return loss, pack(grads[::-1])
