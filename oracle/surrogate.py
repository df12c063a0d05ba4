"""FP64 CPU oracle of the convolutional surrogate (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this module.  It restates, in plain numpy, what the library's BF16
kernels compute: a 3x3 cross-correlation with circular padding, its data and
weight gradients, the 4-layer residual network F + Net(F, eta) on normalised
fields, the mean squared error and the Adam update.  The paper has no learned
component; these are the definitions of the library's own surrogate.

Layouts: activations NHWC (b, y, x, c); weights w[co, tap, ci] with
tap = 3 dy + dx, dy, dx in {0, 1, 2}; output[y, x] reads input[y + dy - 1, x + dx - 1].
Pinned by tests/test_surrogate_oracle.py against scipy.signal.correlate2d
(boundary="wrap") and against central finite differences.
"""
from __future__ import annotations

import numpy as np

LAYERS = ((16, 32), (32, 32), (32, 32), (32, 8))   # (cin, cout), channel-padded
CIN_REAL = (4, 32, 32, 32)
COUT_REAL = (32, 32, 32, 3)


def _shift(a, dy, dx):
    """a[:, y + dy - 1, x + dx - 1, :] at (y, x) (circular)."""
    return np.roll(a, shift=(-(dy - 1), -(dx - 1)), axis=(1, 2))


def conv_forward(x, w, b):
    """y[b, y, x, co] = b[co] + sum_{tap, ci} w[co, tap, ci] x[b, y+dy-1, x+dx-1, ci]."""
    y = np.zeros(x.shape[:3] + (w.shape[0],))
    for tap in range(9):
        dy, dx = divmod(tap, 3)
        y += _shift(x, dy, dx) @ w[:, tap, :].T
    return y + b


def conv_backward_data(dy, w):
    """dL/dx for y = conv_forward(x, w, b) given dL/dy."""
    dx = np.zeros(dy.shape[:3] + (w.shape[2],))
    for tap in range(9):
        ty, tx = divmod(tap, 3)
        # x[q] enters y[q - d]: shift dy by +d
        dx += np.roll(dy, shift=(ty - 1, tx - 1), axis=(1, 2)) @ w[:, tap, :]
    return dx


def conv_backward_weight(x, dy):
    """dL/dw[co, tap, ci] and dL/db[co] for y = conv_forward(x, w, b)."""
    co, ci = dy.shape[3], x.shape[3]
    dw = np.zeros((co, 9, ci))
    for tap in range(9):
        ty, tx = divmod(tap, 3)
        xs = _shift(x, ty, tx).reshape(-1, ci)
        dw[:, tap, :] = dy.reshape(-1, co).T @ xs
    return dw, dy.reshape(-1, co).sum(axis=0)


def unpack(params):
    """Flat parameter vector (library layout) -> [(w, b)] per layer."""
    out, off = [], 0
    for cin, cout in LAYERS:
        w = params[off: off + cout * 9 * cin].reshape(cout, 9, cin)
        off += cout * 9 * cin
        b = params[off: off + cout]
        off += cout
        out.append((w, b))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in layers])


def normalise(fields, eta, rho0, eta_c, eta_s):
    """Planes [B, 3, H, W] -> state [B, H, W, 8] and network input [B, H, W, 16]."""
    f = np.asarray(fields, np.float64)
    B, _, H, W = f.shape
    state = np.zeros((B, H, W, 8))
    state[..., 0] = f[:, 0] / rho0 - 1.0
    state[..., 1] = f[:, 1] / rho0
    state[..., 2] = f[:, 2] / rho0
    x0 = np.zeros((B, H, W, 16))
    x0[..., :3] = state[..., :3]
    x0[..., 3] = ((np.asarray(eta, np.float64) - eta_c) / eta_s)[:, None, None]
    return state, x0


def denormalise(state, rho0):
    f = np.zeros((state.shape[0], 3) + state.shape[1:3])
    f[:, 0] = rho0 * (state[..., 0] + 1.0)
    f[:, 1] = rho0 * state[..., 1]
    f[:, 2] = rho0 * state[..., 2]
    return f


def conserved_channels(conserve):
    """Field channels whose sample mean one application keeps: bit 0 the
    density (the particle number is fixed), bit 1 both polarisation channels."""
    return [c for c, bit in ((0, 1), (1, 2), (2, 2)) if conserve & bit]


def project(r, conserve):
    """P r: the per-sample mean over the grid removed from the conserved channels."""
    r = np.array(r, np.float64)
    for c in conserved_channels(conserve):
        r[..., c] -= r[..., c].mean(axis=(1, 2), keepdims=True)
    return r


def forward(params, state, x0, round_act=None, conserve=0):
    """One application F + P Net(F, eta): returns (new state, activations)."""
    L = unpack(params)
    acts = [x0]
    a = x0
    for k in range(3):
        a = np.maximum(conv_forward(a, *L[k]), 0.0)
        if round_act is not None:
            a = round_act(a)
        acts.append(a)
    out = project(conv_forward(a, *L[3]), conserve)
    return state + out, acts


def loss_and_grad(params, state, x0, target, round_act=None, conserve=0):
    """MSE over the 3 field channels and its gradient (library layout); the
    projection P is symmetric, so the gradient reaching the last layer is P g."""
    L = unpack(params)
    pred, acts = forward(params, state, x0, round_act, conserve)
    d = pred[..., :3] - target[..., :3]
    npx = d.shape[0] * d.shape[1] * d.shape[2]
    loss = float((d * d).sum() / (3 * npx))
    g = np.zeros_like(pred)
    g[..., :3] = 2.0 * d / (3 * npx)
    g = project(g, conserve)
    grads = [None] * 4
    for k in (3, 2, 1, 0):
        dw, db = conv_backward_weight(acts[k], g)
        grads[k] = (dw, db)
        if k > 0:
            g = conv_backward_data(g, L[k][0]) * (acts[k] > 0)
    return loss, pack(grads)


def adam(params, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba); returns updated (params, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_bits(a):
    """BF16 bit patterns (uint16) of the BF16-rounded values of a."""
    return (bf16_round(a).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


def from_bf16_bits(u):
    return (np.asarray(u, np.uint32) << 16).view(np.float32).astype(np.float64)
