"""FP64 reference of the warm-start network: forward pass, MSE loss, backward pass, Adam.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the benchmark's CPU
baseline, never by the library.

The network maps the point-spread functions of a science/template pair, sampled as 32 x 32
stamps at the nine centres of a 3 x 3 grid over the frame (18 input channels: science then
template for each grid cell, cells row-major), to the delta-basis kernel coefficients of
the fit (L^2 nP(DK) values, in the fit's unknown order).  Layers:

    4 x [conv 3x3, stride 2, zero padding 1, 32 output channels, ReLU]   32 -> 16 -> 8 -> 4 -> 2
    flatten (channel, row, column)  ->  linear 128 -> n_out

Parameters are one flat float vector in the order conv1 W [32][18][3][3], conv1 b [32],
conv2 W, b, conv3 W, b, conv4 W, b, linear W [n_out][128], linear b [n_out].

Loss: mean squared error over the batch and the outputs.  Adam (Kingma & Ba, 2015,
Algorithm 1): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2, p <- p - lr mhat / (sqrt(vhat) + eps)
with mhat = m / (1 - b1^t), vhat = v / (1 - b2^t).

Each layer is written from its definition with numpy array slicing; nothing is fused.
"""
import numpy as np

IN_CH, HW, CH, N_CONV = 18, 32, 32, 4


def param_shapes(n_out: int):
    shapes = []
    cin = IN_CH
    for _ in range(N_CONV):
        shapes += [(CH, cin, 3, 3), (CH,)]
        cin = CH
    side = HW >> N_CONV
    shapes += [(n_out, CH * side * side), (n_out,)]
    return shapes


def param_count(n_out: int) -> int:
    return int(sum(np.prod(s) for s in param_shapes(n_out)))


def unflatten(params, n_out: int):
    out, k = [], 0
    for s in param_shapes(n_out):
        m = int(np.prod(s))
        out.append(np.asarray(params[k:k + m], dtype=np.float64).reshape(s))
        k += m
    return out


def flatten(arrays):
    return np.concatenate([np.asarray(a, dtype=np.float64).ravel() for a in arrays])


def conv_forward(x, W, b):
    """z[n, o, i, j] = b[o] + sum_{c, u, v} W[o, c, u, v] x[n, c, 2i + u - 1, 2j + v - 1]
    (zero outside the input)."""
    n, c, h, w = x.shape
    ho, wo = (h + 1) // 2, (w + 1) // 2
    xp = np.zeros((n, c, h + 2, w + 2))
    xp[:, :, 1:h + 1, 1:w + 1] = x
    z = np.zeros((n, W.shape[0], ho, wo)) + b[None, :, None, None]
    for u in range(3):
        for v in range(3):
            patch = xp[:, :, u:u + 2 * ho:2, v:v + 2 * wo:2]          # [n, c, ho, wo]
            z += np.einsum('oc,ncij->noij', W[:, :, u, v], patch)
    return z


def conv_backward(x, W, gz):
    """Gradients of the convolution above: (dL/dx, dL/dW, dL/db) given gz = dL/dz."""
    n, c, h, w = x.shape
    ho, wo = gz.shape[2], gz.shape[3]
    xp = np.zeros((n, c, h + 2, w + 2))
    xp[:, :, 1:h + 1, 1:w + 1] = x
    gW = np.zeros_like(W)
    gxp = np.zeros_like(xp)
    for u in range(3):
        for v in range(3):
            patch = xp[:, :, u:u + 2 * ho:2, v:v + 2 * wo:2]
            gW[:, :, u, v] = np.einsum('noij,ncij->oc', gz, patch)
            gxp[:, :, u:u + 2 * ho:2, v:v + 2 * wo:2] += np.einsum('oc,noij->ncij', W[:, :, u, v], gz)
    gb = gz.sum(axis=(0, 2, 3))
    return gxp[:, :, 1:h + 1, 1:w + 1], gW, gb


def forward(params, stamps, n_out: int):
    """Returns (output [n, n_out], cache of layer inputs and activations)."""
    P = unflatten(params, n_out)
    a = np.asarray(stamps, dtype=np.float64)
    cache = []
    for layer in range(N_CONV):
        W, b = P[2 * layer], P[2 * layer + 1]
        z = conv_forward(a, W, b)
        cache.append((a, z))
        a = np.maximum(z, 0.0)
    flat = a.reshape(a.shape[0], -1)
    Wl, bl = P[2 * N_CONV], P[2 * N_CONV + 1]
    y = flat @ Wl.T + bl
    cache.append((flat, None))
    return y, cache


def mse(y, target):
    d = y - np.asarray(target, dtype=np.float64)
    return float(np.mean(d * d)), 2.0 * d / d.size


def gradients(params, stamps, target, n_out: int):
    """(loss, flat gradient of the loss with respect to params, gradient w.r.t. stamps)."""
    P = unflatten(params, n_out)
    y, cache = forward(params, stamps, n_out)
    loss, gy = mse(y, target)
    flat, _ = cache[N_CONV]
    Wl = P[2 * N_CONV]
    grads = [None] * len(P)
    grads[2 * N_CONV] = gy.T @ flat
    grads[2 * N_CONV + 1] = gy.sum(axis=0)
    ga = (gy @ Wl).reshape(cache[N_CONV - 1][1].shape)
    for layer in reversed(range(N_CONV)):
        x, z = cache[layer]
        gz = ga * (z > 0)
        ga, grads[2 * layer], grads[2 * layer + 1] = conv_backward(x, P[2 * layer], gz)
    return loss, flatten(grads), ga


def adam_step(params, grad, m, v, t: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns (params, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v
