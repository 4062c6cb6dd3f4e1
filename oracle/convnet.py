"""Convolutional network of the learned mesh warm start (oracle; test infrastructure only).

The network maps per-node features of the mesh problem of Sec. 4 to the node
displacement that starts the Jacobi iteration.  It is a stack of 3x3
cross-correlations with zero padding,

    a^0 = input,   z^l[co](y, x) = b^l[co] + sum_{ci, dy, dx} w^l[co, ci, dy+1, dx+1] a^l[ci](y+dy, x+dx),
    a^{l+1} = tanh(z^l) for hidden layers,  output = z^{L-1},

trained on the mean squared error with Adam (Kingma & Ba, "Adam: a method for
stochastic optimization", 2015, Algorithm 1).  Weights are stored in bfloat16
(round to nearest even from the float32 master copy); everything here is
float64 arithmetic on those values.

Written out from the definitions: the forward pass is the sum above, the
backward pass is its chain rule written element-wise (no im2col, no FFT).
"""
import numpy as np


def bf16_round(a):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64.

    bfloat16 keeps the top 16 bits of the IEEE binary32 pattern; rounding adds
    0x7FFF plus the lowest kept bit before truncating (round half to even).
    """
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    keep_lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + keep_lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isnan(f), np.nan, out)


def conv3x3(a, w, b=None):
    """z[n, co, y, x] = b[co] + sum_{ci, dy, dx} w[co, ci, dy, dx] a_pad[n, ci, y + dy, x + dx].

    a: [N][Cin][H][W]; w: [Cout][Cin][3][3]; zero padding of one pixel."""
    N, Cin, H, W = a.shape
    Cout = w.shape[0]
    ap = np.zeros((N, Cin, H + 2, W + 2))
    ap[:, :, 1:-1, 1:-1] = a
    z = np.zeros((N, Cout, H, W))
    for dy in range(3):
        for dx in range(3):
            win = ap[:, :, dy:dy + H, dx:dx + W]                 # [N][Cin][H][W]
            z += np.einsum("oc,nchw->nohw", w[:, :, dy, dx], win)
    if b is not None:
        z += np.asarray(b, dtype=np.float64)[None, :, None, None]
    return z


def conv3x3_backward(a, w, g):
    """Gradients of L through z = conv3x3(a, w, b), given g = dL/dz:

    dL/dw[co, ci, dy, dx] = sum_{n, y, x} g[n, co, y, x] a_pad[n, ci, y + dy, x + dx]
    dL/db[co]             = sum_{n, y, x} g[n, co, y, x]
    dL/da[n, ci, y, x]    = sum_{co, dy, dx} w[co, ci, dy, dx] g_pad[n, co, y + 1 - dy, x + 1 - dx]
    """
    N, Cin, H, W = a.shape
    ap = np.zeros((N, Cin, H + 2, W + 2))
    ap[:, :, 1:-1, 1:-1] = a
    Cout = w.shape[0]
    gw = np.zeros((Cout, Cin, 3, 3))
    for dy in range(3):
        for dx in range(3):
            gw[:, :, dy, dx] = np.einsum("nohw,nchw->oc", g, ap[:, :, dy:dy + H, dx:dx + W])
    gb = g.sum(axis=(0, 2, 3))
    gp = np.zeros((N, Cout, H + 2, W + 2))
    gp[:, :, 1:-1, 1:-1] = g
    ga = np.zeros_like(a, dtype=np.float64)
    for dy in range(3):
        for dx in range(3):
            win = gp[:, :, 2 - dy:2 - dy + H, 2 - dx:2 - dx + W]  # g at (y + 1 - dy, x + 1 - dx)
            ga += np.einsum("oc,nohw->nchw", w[:, :, dy, dx], win)
    return gw, gb, ga


def forward(ws, bs, a0, bf16_inputs=False):
    """Activations [a^0, a^1, ..., output] of the network with layers (ws[l], bs[l]); with
    bf16_inputs each layer's input is first rounded to bf16 (a tensor-core layer's operand)."""
    acts = [np.asarray(a0, dtype=np.float64)]
    L = len(ws)
    for l in range(L):
        a = bf16_round(acts[-1]) if bf16_inputs else acts[-1]
        z = conv3x3(a, ws[l], bs[l])
        acts.append(np.tanh(z) if l < L - 1 else z)
    return acts


def mse(pred, target):
    """L = mean((pred - target)^2) and dL/dpred = 2 (pred - target) / n."""
    d = np.asarray(pred, dtype=np.float64) - np.asarray(target, dtype=np.float64)
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(ws, acts, g_out):
    """(dL/dw^l, dL/db^l) for every layer, given the activations of `forward` and g_out = dL/d(output)."""
    L = len(ws)
    gws, gbs = [None] * L, [None] * L
    g = g_out
    for l in range(L - 1, -1, -1):
        if l < L - 1:
            g = g * (1.0 - acts[l + 1] ** 2)           # through tanh: d tanh(z)/dz = 1 - tanh(z)^2
        gws[l], gbs[l], ga = conv3x3_backward(acts[l], ws[l], g)
        g = ga
    return gws, gbs


def adam(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015, Algorithm 1); returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
