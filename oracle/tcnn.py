"""Plain float64 restatement of the tile-proposal network, for gradient checks.

TEST INFRASTRUCTURE ONLY (tests and bench CPU legs).  The network: a 64 x 64
uint8 patch normalised to (v - 128) / 64; three 3 x 3 convolutions with
stride 2, padding 1 and ReLU (1 -> 8 -> 16 -> 16 channels, 64 -> 32 -> 16 ->
8 pixels); global average pool; linear 16 -> 1 logit.  Loss: weighted binary
cross-entropy with logits, averaged over the batch.  Written from those
definitions with numpy slicing; shares nothing with the CUDA kernels.
Pinned by tests/test_oracle_tcnn.py (scipy correlation, finite differences).
"""

from __future__ import annotations

import numpy as np

SHAPES = [("W1", (8, 1, 3, 3)), ("b1", (8,)), ("W2", (16, 8, 3, 3)), ("b2", (16,)),
          ("W3", (16, 16, 3, 3)), ("b3", (16,)), ("wf", (16,)), ("bf", (1,))]
NP = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p: np.ndarray) -> dict:
    p = np.asarray(p, dtype=np.float64)
    out, off = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = p[off:off + n].reshape(shape)
        off += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SHAPES])


def normalise(tiles_u8: np.ndarray) -> np.ndarray:
    return (np.asarray(tiles_u8, np.float64) - 128.0) / 64.0


def conv_s2(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x (N, C, S, S) -> (N, O, S/2, S/2): b[o] + sum_{c,ky,kx} W[o,c,ky,kx] x[c, 2y+ky-1, 2x+kx-1]."""
    n, c, s, _ = x.shape
    so = s // 2
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    out = np.zeros((n, W.shape[0], so, so))
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, :, ky:ky + 2 * so:2, kx:kx + 2 * so:2]  # (n, c, so, so)
            out += np.einsum("ncyx,oc->noyx", patch, W[:, :, ky, kx])
    return out + b[None, :, None, None]


def conv_s2_back(x: np.ndarray, W: np.ndarray, dout: np.ndarray):
    """Gradients of conv_s2 w.r.t. W, b and x, given dL/dout."""
    n, c, s, _ = x.shape
    so = s // 2
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    dW = np.zeros_like(W)
    dxp = np.zeros_like(xp)
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, :, ky:ky + 2 * so:2, kx:kx + 2 * so:2]
            dW[:, :, ky, kx] = np.einsum("noyx,ncyx->oc", dout, patch)
            dxp[:, :, ky:ky + 2 * so:2, kx:kx + 2 * so:2] += np.einsum("noyx,oc->ncyx", dout, W[:, :, ky, kx])
    db = dout.sum(axis=(0, 2, 3))
    return dW, db, dxp[:, :, 1:-1, 1:-1]


def forward(tiles_u8: np.ndarray, params: np.ndarray):
    """Logits (N,) and the intermediate activations."""
    P = unpack(params)
    x0 = normalise(tiles_u8)[:, None]
    a1 = np.maximum(conv_s2(x0, P["W1"], P["b1"]), 0.0)
    a2 = np.maximum(conv_s2(a1, P["W2"], P["b2"]), 0.0)
    a3 = np.maximum(conv_s2(a2, P["W3"], P["b3"]), 0.0)
    g = a3.mean(axis=(2, 3))
    z = g @ P["wf"] + P["bf"][0]
    return z, (x0, a1, a2, a3, g)


def loss(tiles_u8, labels, params, pos_weight: float = 1.0) -> float:
    z, _ = forward(tiles_u8, params)
    y = np.asarray(labels, np.float64)
    w = np.where(y > 0.5, pos_weight, 1.0)
    softplus = np.logaddexp(0.0, z)
    return float(np.mean(w * (softplus - y * z)))


def loss_grad(tiles_u8, labels, params, pos_weight: float = 1.0):
    """Loss and its gradient w.r.t. the flat parameters (float64)."""
    P = unpack(params)
    z, (x0, a1, a2, a3, g) = forward(tiles_u8, params)
    y = np.asarray(labels, np.float64)
    n = len(y)
    w = np.where(y > 0.5, pos_weight, 1.0)
    L = float(np.mean(w * (np.logaddexp(0.0, z) - y * z)))
    dz = w * (1.0 / (1.0 + np.exp(-z)) - y) / n
    grads = {"wf": g.T @ dz, "bf": np.array([dz.sum()])}
    dg = np.outer(dz, P["wf"])
    da3 = (dg / 64.0)[:, :, None, None] * np.ones_like(a3) * (a3 > 0)
    grads["W3"], grads["b3"], da2 = conv_s2_back(a2, P["W3"], da3)
    da2 = da2 * (a2 > 0)
    grads["W2"], grads["b2"], da1 = conv_s2_back(a1, P["W2"], da2)
    da1 = da1 * (a1 > 0)
    grads["W1"], grads["b1"], _ = conv_s2_back(x0, P["W1"], da1)
    return L, pack(grads)


def adam(params, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
    """One bias-corrected Adam step with decoupled weight decay (float64)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * (mh / (np.sqrt(vh) + eps) + wd * params), m, v
