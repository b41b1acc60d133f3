"""FP64 NumPy reference of the warm-start U-Net (test infrastructure).

Only ``tests/`` may import this module.  It defines, in plain NumPy, the
network the library trains and runs on the GPU for the learned warm start of
the Poisson solve (not part of the paper): a U-Net on NHWC tensors with
3x3 "same" convolutions, ReLU, 2x2 average pooling, nearest 2x upsampling,
channel concatenation of the skip connections and a final 1x1 convolution,
with its forward pass, its backward pass and the MSE loss.  Gradients are
pinned in the tests by central finite differences; the convolution by an
independent scipy.signal correlation.

Parameter order (flat vector): for each convolution in network order,
weights W[ky, kx, cin, cout] then bias[cout].
"""
import numpy as np


def conv_specs(base=16, levels=4, cin=3, cout=1):
    """[(cin, cout, ksize)] of all convolutions in network order."""
    ch = [base * (2 ** l) for l in range(levels)]
    specs = []
    c = cin
    for l in range(levels):                       # encoder (last level = bottleneck)
        specs += [(c, ch[l], 3), (ch[l], ch[l], 3)]
        c = ch[l]
    for l in range(levels - 2, -1, -1):           # decoder
        specs += [(c + ch[l], ch[l], 3), (ch[l], ch[l], 3)]
        c = ch[l]
    specs.append((c, cout, 1))
    return specs


def n_params(specs):
    return sum(k * k * ci * co + co for ci, co, k in specs)


def unpack(theta, specs):
    out, o = [], 0
    for ci, co, k in specs:
        nw = k * k * ci * co
        W = theta[o:o + nw].reshape(k, k, ci, co)
        o += nw
        b = theta[o:o + co]
        o += co
        out.append((W, b))
    return out


# Rounding applied to convolution operands (inputs, weights, output
# gradients): None for plain FP64, or a function such as `bf16_round` to
# reproduce the storage precision of a BF16 implementation.
ROUND = None


def bf16_round(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def _r(a):
    return a if ROUND is None else ROUND(a)


def conv(x, W, b):
    """x (B, H, W, Ci), W (k, k, Ci, Co): zero-padded 'same' correlation."""
    x, W = _r(x), _r(W)
    k = W.shape[0]
    p = k // 2
    B, H, Wd, Ci = x.shape
    xp = np.pad(x, ((0, 0), (p, p), (p, p), (0, 0)))
    y = np.zeros((B, H, Wd, W.shape[3]))
    for ky in range(k):
        for kx in range(k):
            y += np.einsum("bhwc,cd->bhwd", xp[:, ky:ky + H, kx:kx + Wd, :], W[ky, kx])
    return y + b


def conv_backward(x, W, gy):
    """Gradients of conv w.r.t. its input, weights and bias."""
    x, W, gy = _r(x), _r(W), _r(gy)
    k = W.shape[0]
    p = k // 2
    B, H, Wd, Ci = x.shape
    xp = np.pad(x, ((0, 0), (p, p), (p, p), (0, 0)))
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for ky in range(k):
        for kx in range(k):
            gW[ky, kx] = np.einsum("bhwc,bhwd->cd", xp[:, ky:ky + H, kx:kx + Wd, :], gy)
            gxp[:, ky:ky + H, kx:kx + Wd, :] += np.einsum("bhwd,cd->bhwc", gy, W[ky, kx])
    gx = gxp[:, p:p + H, p:p + Wd, :]
    return gx, gW, gy.sum(axis=(0, 1, 2))


def pool(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool_backward(gy):
    return np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2) * 0.25


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_backward(gy):
    B, H, W, C = gy.shape
    return gy.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def forward(theta, x, specs, levels=4, cache=None):
    """Network output (B, H, W, cout); fills `cache` for the backward pass."""
    P = unpack(theta, specs)
    c = cache if cache is not None else {}
    c["x"] = x
    acts = []            # (input, pre-activation) per conv
    skips = []
    h = x
    li = 0
    for l in range(levels):
        for _ in range(2):
            W, b = P[li]
            z = conv(h, W, b)
            acts.append((h, z))
            h = np.maximum(z, 0.0)
            li += 1
        if l < levels - 1:
            skips.append(h)
            h = pool(h)
    for l in range(levels - 2, -1, -1):
        h = np.concatenate([up(h), skips[l]], axis=3)
        for _ in range(2):
            W, b = P[li]
            z = conv(h, W, b)
            acts.append((h, z))
            h = np.maximum(z, 0.0)
            li += 1
    W, b = P[li]
    out = conv(h, W, b)
    acts.append((h, out))
    c["acts"] = acts
    return out


def loss_and_grad(theta, x, target, specs, levels=4):
    """MSE loss mean((out - target)^2) and its gradient w.r.t. theta."""
    cache = {}
    out = forward(theta, x, specs, levels, cache)
    n = out.size
    loss = float(np.sum((out - target) ** 2) / n)
    g = 2.0 * (out - target) / n
    P = unpack(theta, specs)
    grads = [None] * len(P)
    acts = cache["acts"]
    li = len(P) - 1
    h_in, _ = acts[li]
    gh, gW, gb = conv_backward(h_in, P[li][0], g)
    grads[li] = (gW, gb)
    li -= 1
    skip_grads = {}
    # decoder stages in reverse: the first one undone joined skip level 0
    for l in range(0, levels - 1):
        for _ in range(2):
            h_in, z = acts[li]
            gz = gh * (z > 0)
            gh, gW, gb = conv_backward(h_in, P[li][0], gz)
            grads[li] = (gW, gb)
            li -= 1
        # split the concatenation [up(h), skip]
        c_up = gh.shape[3] - specs[2 * l + 1][1]
        skip_grads[l] = gh[..., c_up:]
        gh = up_backward(gh[..., :c_up])
    # encoder (reverse), bottleneck first
    for l in range(levels - 1, -1, -1):
        if l < levels - 1:
            gh = pool_backward(gh) + skip_grads[l]
        for _ in range(2):
            h_in, z = acts[li]
            gz = gh * (z > 0)
            gh, gW, gb = conv_backward(h_in, P[li][0], gz)
            grads[li] = (gW, gb)
            li -= 1
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat
