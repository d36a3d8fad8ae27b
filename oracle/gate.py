"""FP64 CPU oracle of the learned candidate gate (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module; the product path never does.  It shares no code with the
CUDA library.

The gate is not part of the paper.  It predicts, from a candidate's geometry,
whether the 1-bounce solve of that candidate (Sec. 3.5, Sec. 4) returns any
admissible path, so that candidates predicted empty can be skipped.  This
module states, in plain FP64 numpy:

* ``features``: the 24 inputs per candidate.  They restate the specular
  constraint h x n = 0 (Eq. eq_ch) at the triangle's three vertices: the
  tangential mismatch d_i between the shading normal and the generalised half
  vector h = eta_0 w_0 + eta_1 w_2 (unit directions from the vertex to the two
  endpoints) in a frame perpendicular to the half vector at the centroid.
  Where d(u, v) is close to affine over the triangle, the path exists when the
  origin lies in the triangle (d_0, d_1, d_2), and its barycentric coordinates
  there approximate (1 - u - v, u, v).
* the network: 32 (24 used) -> 64 -> 64 -> 64 -> 1, ReLU hidden layers and a
  sigmoid output.  Its arithmetic is defined with BF16 operands: the inputs,
  every hidden activation fed to a matrix product and the three weight
  matrices are rounded to BF16 (round to nearest even); the biases, the
  output weights w4 and b4 stay FP32 values; products are accumulated
  exactly (here in FP64).
* the weighted binary cross-entropy loss, its gradient (backpropagation with
  the BF16 rounding passed straight through) and one Adam step.
"""
from __future__ import annotations

import numpy as np

N_FEAT = 24
N_IN = 32
N_HID = 64

# Flat FP32 parameter vector layout (row-major W[in][out]).
OFF_W1 = 0
OFF_B1 = OFF_W1 + N_IN * N_HID
OFF_W2 = OFF_B1 + N_HID
OFF_B2 = OFF_W2 + N_HID * N_HID
OFF_W3 = OFF_B2 + N_HID
OFF_B3 = OFF_W3 + N_HID * N_HID
OFF_W4 = OFF_B3 + N_HID
OFF_B4 = OFF_W4 + N_HID
N_PARAMS = OFF_B4 + 1


# ------------------------------------------------------------------ BF16
def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64.

    BF16 keeps the upper 16 bits of the FP32 encoding; rounding adds half an
    ulp of the kept part (0x7fff) plus the lowest kept bit, then truncates.
    """
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


# -------------------------------------------------------------- features
def _unit(v):
    n = np.sqrt(np.sum(v * v, axis=-1, keepdims=True))
    return v / np.maximum(n, 1e-30)


def _half(x0, x2, p, e0, e1):
    """Generalised half vector at p, normalised: eta_0 w_0 + eta_1 w_2."""
    return _unit(e0[:, None] * _unit(x0 - p) + e1[:, None] * _unit(x2 - p))


def features(x0, x2, eta0, eta1, types, P, N):
    """Features of n candidates.

    x0, x2: [n, 3] endpoints; eta0, eta1: [n]; types: [n] (0 = R, 1 = T);
    P, N: [n, 3, 3] triangle vertices and vertex normals.  Reflection uses
    eta_0 = eta_1 = 1.  Returns [n, 24] float64:

      0-5   d_i / S: tangential mismatch at vertex i (2D), S = max_i |d_i|
      6-8   (d_0 x d_1, d_1 x d_2, d_2 x d_0) / S^2   (2D cross products)
      9-11  barycentric coordinates of the origin in (d_0, d_1, d_2),
            clamped to [-4, 4]; 0 when the d triangle is degenerate
            (|sum of the crosses| <= 1e-6)
      12    the smallest of 9-11
      13    log2(S) / 8
      14    s (n_c . h_c) with n_c the mean unit normal and s its sign
      15-20 vertex positions minus the centroid in the tangent frame / L,
            L = longest edge
      21    log2(L / |x0 - c|) / 8
      22    h_c . unit(x0 - c)
      23    the type (0 reflection, 1 refraction)
    """
    x0 = np.asarray(x0, np.float64)
    x2 = np.asarray(x2, np.float64)
    P = np.asarray(P, np.float64)
    N = np.asarray(N, np.float64)
    types = np.asarray(types)
    refr = types == 1
    e0 = np.where(refr, np.asarray(eta0, np.float64), 1.0)
    e1 = np.where(refr, np.asarray(eta1, np.float64), 1.0)
    n = x0.shape[0]
    c = P.mean(axis=1)
    hc = _half(x0, x2, c, e0, e1)
    edge = P[:, 1] - P[:, 0]
    e1v = _unit(edge - np.sum(edge * hc, -1, keepdims=True) * hc)
    e2v = np.cross(hc, e1v)
    nh = _unit(N)
    nc = _unit(nh.sum(axis=1))
    s = np.where(np.sum(nc * hc, -1) >= 0.0, 1.0, -1.0)
    d = np.empty((n, 3, 2))
    for i in range(3):
        di = s[:, None] * nh[:, i] - _half(x0, x2, P[:, i], e0, e1)
        d[:, i, 0] = np.sum(di * e1v, -1)
        d[:, i, 1] = np.sum(di * e2v, -1)
    S = np.maximum(np.sqrt((d * d).sum(-1)).max(-1), 1e-30)
    dn = d / S[:, None, None]
    f = np.zeros((n, N_FEAT))
    f[:, 0:6] = dn.reshape(n, 6)

    def cr(i, j):
        return dn[:, i, 0] * dn[:, j, 1] - dn[:, i, 1] * dn[:, j, 0]

    c01, c12, c20 = cr(0, 1), cr(1, 2), cr(2, 0)
    f[:, 6], f[:, 7], f[:, 8] = c01, c12, c20
    D = c01 + c12 + c20
    ok = np.abs(D) > 1e-6
    Ds = np.where(ok, D, 1.0)
    lam = np.stack([c12 / Ds, c20 / Ds, c01 / Ds], -1)
    lam = np.where(ok[:, None], np.clip(lam, -4.0, 4.0), 0.0)
    f[:, 9:12] = lam
    f[:, 12] = lam.min(-1)
    f[:, 13] = np.log2(S) / 8.0
    f[:, 14] = s * np.sum(nc * hc, -1)
    L = np.maximum(np.max(np.stack([np.linalg.norm(P[:, 1] - P[:, 0], axis=-1),
                                    np.linalg.norm(P[:, 2] - P[:, 1], axis=-1),
                                    np.linalg.norm(P[:, 0] - P[:, 2], axis=-1)], -1), -1), 1e-30)
    for i in range(3):
        r = P[:, i] - c
        f[:, 15 + 2 * i] = np.sum(r * e1v, -1) / L
        f[:, 16 + 2 * i] = np.sum(r * e2v, -1) / L
    w0 = x0 - c
    f[:, 21] = np.log2(L / np.maximum(np.linalg.norm(w0, axis=-1), 1e-30)) / 8.0
    f[:, 22] = np.sum(hc * _unit(w0), -1)
    f[:, 23] = refr.astype(np.float64)
    return f


def chain_features(tri_soa, x_first, x_last, eta, types, chains):
    """Features of the 1-bounce chains (query, tri0, -1) of a problem in the
    library's layout (tri_soa [18][T], per-query arrays)."""
    ch = np.asarray(chains)
    q, t = ch[:, 0], ch[:, 1]
    T = np.asarray(tri_soa, np.float64)
    P = np.stack([T[0:3, t].T, T[3:6, t].T, T[6:9, t].T], 1)
    N = np.stack([T[9:12, t].T, T[12:15, t].T, T[15:18, t].T], 1)
    eta = np.asarray(eta, np.float64).reshape(-1, 3)
    ty = np.asarray(types).reshape(-1, 2)[q, 0]
    return features(np.asarray(x_first).reshape(-1, 3)[q], np.asarray(x_last).reshape(-1, 3)[q],
                    eta[q, 0], eta[q, 1], ty, P, N)


# ---------------------------------------------------------------- network
def unpack(theta):
    t = np.asarray(theta, np.float64)
    return (t[OFF_W1:OFF_B1].reshape(N_IN, N_HID), t[OFF_B1:OFF_W2],
            t[OFF_W2:OFF_B2].reshape(N_HID, N_HID), t[OFF_B2:OFF_W3],
            t[OFF_W3:OFF_B3].reshape(N_HID, N_HID), t[OFF_B3:OFF_W4],
            t[OFF_W4:OFF_B4], t[OFF_B4])


def pad_inputs(f):
    x = np.zeros((f.shape[0], N_IN))
    x[:, :N_FEAT] = f
    return x


def forward(theta, f, quantize=True):
    """Logits z4 of n feature rows, and the intermediates of the pass.

    quantize=False drops every BF16 rounding (the plain FP64 network the
    gradient pins use)."""
    q = bf16 if quantize else (lambda a: np.asarray(a, np.float64))
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(theta)
    x = q(pad_inputs(f))
    z1 = x @ q(W1) + b1
    h1 = np.maximum(z1, 0.0)
    z2 = q(h1) @ q(W2) + b2
    h2 = np.maximum(z2, 0.0)
    z3 = q(h2) @ q(W3) + b3
    h3 = np.maximum(z3, 0.0)
    z4 = h3 @ w4 + b4
    return z4, (x, z1, z2, z3, q)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def softplus(z):
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def loss(z4, y, pos_weight):
    """Mean weighted binary cross-entropy of logits: label 1 weighs
    pos_weight, label 0 weighs 1; -log sigmoid(z) = softplus(z) - z and
    -log(1 - sigmoid(z)) = softplus(z)."""
    y = np.asarray(y, np.float64)
    w = np.where(y > 0.5, pos_weight, 1.0)
    return float(np.mean(w * (softplus(z4) - y * z4)))


def grad(theta, f, y, pos_weight, quantize=True):
    """Loss and its gradient with respect to the flat parameter vector."""
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(theta)
    z4, (x, z1, z2, z3, q) = forward(theta, f, quantize)
    y = np.asarray(y, np.float64)
    n = z4.shape[0]
    w = np.where(y > 0.5, pos_weight, 1.0)
    L = float(np.mean(w * (softplus(z4) - y * z4)))
    dz4 = w * (sigmoid(z4) - y) / n
    h1, h2, h3 = np.maximum(z1, 0), np.maximum(z2, 0), np.maximum(z3, 0)
    g = np.zeros(N_PARAMS)
    g[OFF_W4:OFF_B4] = h3.T @ dz4
    g[OFF_B4] = dz4.sum()
    dz3 = np.outer(dz4, w4) * (z3 > 0)
    g[OFF_W3:OFF_B3] = (q(h2).T @ dz3).ravel()
    g[OFF_B3:OFF_W4] = dz3.sum(0)
    dz2 = (dz3 @ q(W3).T) * (z2 > 0)
    g[OFF_W2:OFF_B2] = (q(h1).T @ dz2).ravel()
    g[OFF_B2:OFF_W3] = dz2.sum(0)
    dz1 = (dz2 @ q(W2).T) * (z1 > 0)
    g[OFF_W1:OFF_B1] = (x.T @ dz1).ravel()
    g[OFF_B1:OFF_W2] = dz1.sum(0)
    return L, g


def adam_step(theta, m, v, g, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1) at 1-based step `step`."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
