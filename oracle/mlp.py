"""Float64 reference of the learned Voigt-profile surrogate (test infrastructure).

Only the tests, the smoke entry point and the benchmark's CPU baseline use this
module; the library never does.

The network (a stand-in for the on-the-fly profile evaluation of Section 3.2's
Core-and-Voigt treatment; the paper itself has no network):
    f  = (x / 16, log10(a) + 2, u / 16)
    h1 = GELU(W1 f + b1),  h2 = GELU(W2 h1 + b2),  y = w3 . h2 + b3  ~ ln H(a, x - u)
    GELU(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))
Loss: L = (1/n) sum_s (y_s - t_s)^2.  Gradients by the chain rule, written out
layer by layer below (dy = dL/dy per sample without the 1/n):
    dy = 2 (y - t)
    dw3 = sum dy h2,          db3 = sum dy
    delta2 = dy w3 GELU'(z2), dW2 = sum delta2 h1^T,  db2 = sum delta2
    delta1 = (W2^T delta2) GELU'(z1),  dW1 = sum delta1 f^T,  db1 = sum delta1
each sum over the samples and divided by n.

``emulate=True`` reproduces where the library rounds to bfloat16 (round to
nearest even of the float32 value): W1, W2, w3; h1; delta2; dy h2 (for dw3);
delta1 and f (for dW1, db1).  ``emulate=False`` is the exact float64 network,
whose gradient is pinned by finite differences in the tests.
"""

from __future__ import annotations

import numpy as np

H = 64
OFF = {"W1": 0, "b1": 192, "W2": 256, "b2": 4352, "w3": 4416, "b3": 4480}
N_PARAMS = 4481
C_GELU = np.sqrt(2.0 / np.pi)
K_GELU = 0.044715


def bf16(x):
    """Round to bfloat16 (through float32, round to nearest even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64).reshape(np.shape(x))


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return dict(W1=p[0:192].reshape(H, 3), b1=p[192:256], W2=p[256:4352].reshape(H, H), b2=p[4352:4416],
                w3=p[4416:4480], b3=p[4480])


def pack(d):
    return np.concatenate([d["W1"].reshape(-1), d["b1"], d["W2"].reshape(-1), d["b2"], d["w3"], [d["b3"]]])


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(C_GELU * (z + K_GELU * z ** 3)))


def gelu_prime(z):
    t = np.tanh(C_GELU * (z + K_GELU * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * C_GELU * (1.0 + 3.0 * K_GELU * z * z)


def features(xau):
    xau = np.asarray(xau, dtype=np.float64).reshape(-1, 3)
    return np.stack([xau[:, 0] / 16.0, np.log10(xau[:, 1]) + 2.0, xau[:, 2] / 16.0], axis=1)


def _forward(p, xau, emulate):
    w = unpack(p)
    r = bf16 if emulate else (lambda v: np.asarray(v, dtype=np.float64))
    W1, W2, w3 = r(w["W1"]), r(w["W2"]), r(w["w3"])
    f = features(xau)
    z1 = f @ W1.T + w["b1"]
    h1 = r(gelu(z1))
    z2 = h1 @ W2.T + w["b2"]
    h2 = gelu(z2)
    y = h2 @ w3 + w["b3"]
    return dict(f=f, z1=z1, h1=h1, z2=z2, h2=h2, y=y, W1=W1, W2=W2, w3=w3)


def forward(p, xau, emulate: bool = True):
    """Predicted ln H for every sample."""
    return _forward(p, xau, emulate)["y"]


def loss_and_grad(p, xau, target, emulate: bool = True):
    """(L, dL/dp) in the library's parameter layout."""
    c = _forward(p, xau, emulate)
    r = bf16 if emulate else (lambda v: np.asarray(v, dtype=np.float64))
    t = np.asarray(target, dtype=np.float64).reshape(-1)
    n = t.size
    e = c["y"] - t
    loss = float(np.sum(e * e) / n)
    dy = 2.0 * e
    d2 = r(dy[:, None] * c["w3"][None, :] * gelu_prime(c["z2"]))
    g = {}
    g["b3"] = np.sum(dy) / n
    g["w3"] = np.sum(r(dy[:, None] * c["h2"]), axis=0) / n
    g["W2"] = d2.T @ c["h1"] / n
    g["b2"] = np.sum(d2, axis=0) / n
    d1 = r((d2 @ c["W2"]) * gelu_prime(c["z1"]))
    g["W1"] = d1.T @ r(c["f"]) / n
    g["b1"] = np.sum(d1, axis=0) / n
    return loss, pack(g)


def adam_step(p, g, m, v, step: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma & Ba 2015) in float64; returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# training domain of the surrogate; outside it the exact evaluation is used
X_MAX, U_MAX, A_MIN, A_MAX = 16.0, 10.0, 1e-3, 1e-1


def weights_bf16(p):
    """Parameters with W1, W2, w3 rounded to bfloat16 (biases untouched)."""
    q = np.asarray(p, dtype=np.float64).copy()
    for a, b in ((0, 192), (256, 4352), (4416, 4480)):
        q[a:b] = bf16(q[a:b])
    return q


def profile_with_fallback(p, method="hum1wei24"):
    """H(a, x, u) of the Core-and-Voigt solve with the surrogate: exp(network) inside
    the training domain (decided on float32 values, as the kernel does), the Voigt
    function of ``method`` at x - u outside it.  The network runs in float64 with
    bfloat16-rounded weights and unrounded activations (the in-solve evaluation)."""
    from .voigt import voigt_h
    q = weights_bf16(p)

    def H(a, x, u):
        a, x, u = (np.asarray(v, dtype=np.float64) for v in (a, x, u))
        shape = np.broadcast(a, x, u).shape
        a, x, u = (np.broadcast_to(v, shape).reshape(-1) for v in (a, x, u))
        a32, x32, u32 = a.astype(np.float32), x.astype(np.float32), u.astype(np.float32)
        inside = (a32 >= np.float32(A_MIN)) & (a32 <= np.float32(A_MAX)) & (np.abs(x32) <= X_MAX) & (np.abs(u32) <= U_MAX)
        out = np.empty(a.size)
        if inside.any():
            xau = np.stack([x[inside], a[inside], u[inside]], axis=1)
            out[inside] = np.exp(forward(q, xau, emulate=False))
        if (~inside).any():
            out[~inside] = voigt_h(a[~inside], x[~inside] - u[~inside], method=method)
        return out.reshape(shape)
    return H
