"""FP64 numpy reference of the surrogate network (test infrastructure only).

A stack of 3x3x3 convolutions with zero padding ("same" size), ReLU after
every layer but the last, on channels-last volumes x[D, H, W, C].  Weights
are W[27, Cout, Cin] with tap t = (kz*3 + ky)*3 + kx reading the input at
offset (kz-1, ky-1, kx-1); biases b[Cout].  The loss is the mean squared
error over the voxels of a mask and all output channels.

``round_bf16`` emulates the CUDA path's storage precision (round to nearest
even to 8 mantissa bits) so that the reference can see the same rounded
operands; the arithmetic itself stays FP64.  Only the tests import this
module; it shares no code with the CUDA kernels.
"""
import numpy as np

TAPS = [(kz, ky, kx) for kz in range(3) for ky in range(3) for kx in range(3)]


def round_bf16(a):
    """Round an array to bfloat16 (nearest even) and return it as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3d(x, W, b):
    """y[z,y,x,o] = b[o] + sum_{t,i} W[t,o,i] x[z+kz-1, y+ky-1, x+kx-1, i] (zero outside)."""
    D, H, Wd, _ = x.shape
    xp = np.zeros((D + 2, H + 2, Wd + 2, x.shape[3]))
    xp[1:-1, 1:-1, 1:-1] = x
    y = np.broadcast_to(b, (D, H, Wd, W.shape[1])).astype(np.float64).copy()
    for t, (kz, ky, kx) in enumerate(TAPS):
        y += np.einsum("zyxi,oi->zyxo", xp[kz:kz + D, ky:ky + H, kx:kx + Wd], W[t])
    return y


def conv3d_backward(x, W, dy):
    """Gradients of conv3d with respect to x, W and b for upstream dy."""
    D, H, Wd, _ = x.shape
    xp = np.zeros((D + 2, H + 2, Wd + 2, x.shape[3]))
    xp[1:-1, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W, dtype=np.float64)
    for t, (kz, ky, kx) in enumerate(TAPS):
        dW[t] = np.einsum("zyxo,zyxi->oi", dy, xp[kz:kz + D, ky:ky + H, kx:kx + Wd])
        dxp[kz:kz + D, ky:ky + H, kx:kx + Wd] += np.einsum("zyxo,oi->zyxi", dy, W[t])
    db = dy.sum(axis=(0, 1, 2))
    return dxp[1:-1, 1:-1, 1:-1], dW, db


def forward(x, params, bf16=False):
    """Returns the list of layer outputs (post-ReLU, last layer linear).
    With bf16=True every stored activation (input and hidden layers) and
    weight is rounded to bfloat16 as the CUDA path stores them."""
    acts = [round_bf16(x) if bf16 else np.asarray(x, np.float64)]
    n = len(params)
    for l, (W, b) in enumerate(params):
        Wl = round_bf16(W) if bf16 else W
        y = conv3d(acts[-1], Wl, b)
        if l < n - 1:
            y = np.maximum(y, 0.0)
            if bf16:
                y = round_bf16(y)
        acts.append(y)
    return acts


def mse(y, target, mask):
    """Mean over masked voxels and channels of (y - target)^2, and d/dy."""
    m = np.asarray(mask, np.float64)[..., None]
    cnt = m.sum() * y.shape[-1]
    d = (y - target) * m
    return float((d * d).sum() / cnt), 2.0 * d / cnt


def backward(acts, params, dy, bf16=False):
    """Parameter gradients for upstream gradient dy of the last output."""
    grads = [None] * len(params)
    g = dy
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        Wl = round_bf16(W) if bf16 else W
        dx, dW, db = conv3d_backward(acts[l], Wl, g)
        grads[l] = (dW, db)
        if l > 0:
            g = dx * (acts[l] > 0.0)  # ReLU of layer l-1
    return grads
