"""FP64 reference of the moment-fit warm-start network (test infrastructure).

The network proposes the Newton start of the discrete ten-moment fit
(Sec. 2.2, Algorithm 1 "moment fitting"): from 12 inputs of a fit's targets
it predicts t = eta* - eta_0, the Newton solution minus the cold start in
the fit's scaled coordinates. Plain numpy in float64, written from the
definitions: inputs, a 12 -> 128 -> 128 -> 10 perceptron with GELU
(0.5 z (1 + erf(z / sqrt 2))) on the hidden layers, standardised inputs,
outputs y = asinh(t / ysc) standardised by (ym, ys), and the mean-square
loss on those with its gradient by the chain rule.

Parameter blob (float32 on the device, float64 here), in order:
  xm[12] xs[12] ym[10] ys[10] ysc[10] | W1[128][12] b1[128] | W2[128][128]
  b2[128] | W3[10][128] b3[10]
Training sample (24 floats): x[12], t[10], flag, pad.
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_HID, N_OUT = 12, 128, 10
SAMPLE = 24
_SIZES = [("xm", (N_IN,)), ("xs", (N_IN,)), ("ym", (N_OUT,)), ("ys", (N_OUT,)), ("ysc", (N_OUT,)),
          ("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in _SIZES)
TRAINED = ("W1", "b1", "W2", "b2", "W3", "b3")


def unpack(w):
    """Views of the parameter blob by name."""
    w = np.asarray(w, dtype=np.float64)
    out, off = {}, 0
    for name, shape in _SIZES:
        k = int(np.prod(shape))
        out[name] = w[off:off + k].reshape(shape)
        off += k
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1) for name, _ in _SIZES])


def inputs(targets, vmin, dv, vmax):
    """The 12 inputs of one fit from its targets (n, nu_a, E2_ab with
    E2 = int v v f in the order xx, xy, xz, yy, yz, zz) and the velocity box:
    Theta_ab / (dv_a dv_b), the offset of u from the nearest cell centre in
    cells, and the position of u in the box. None if the targets are not a
    valid fit target (n <= 0, or a non-positive diagonal temperature)."""
    t = np.asarray(targets, dtype=np.float64)
    n = t[0]
    if not (n > 0.0):
        return None
    u = t[1:4] / n
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    x = np.zeros(N_IN)
    for q, (a, b) in enumerate(pairs):
        x[q] = (t[4 + q] / n - u[a] * u[b]) / (dv[a] * dv[b])
    if not (x[0] > 0 and x[3] > 0 and x[5] > 0):
        return None
    for a in range(3):
        k = math.floor((u[a] - vmin[a]) / dv[a])  # the cell containing u
        centre = vmin[a] + (k + 0.5) * dv[a]
        x[6 + a] = (u[a] - centre) / dv[a]
        x[9 + a] = (u[a] - vmin[a]) / (vmax[a] - vmin[a])
    return x


def _erf(z):
    return np.vectorize(math.erf)(z)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def _layers(p, x):
    xs = (np.asarray(x, dtype=np.float64) - p["xm"]) / p["xs"]
    z1 = xs @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    y = h2 @ p["W3"].T + p["b3"]
    return xs, z1, h1, z2, h2, y


def forward(w, x):
    """eta* - eta_0 predicted for inputs x[n][12]."""
    p = unpack(w)
    y = _layers(p, x)[-1]
    return p["ysc"] * np.sinh(y * p["ys"] + p["ym"])


def loss_and_grad(w, samples):
    """Mean over samples and outputs of the squared standardised error, and
    its gradient with respect to the blob (zero for the normalisation)."""
    p = unpack(w)
    s = np.asarray(samples, dtype=np.float64)
    x, t = s[:, :N_IN], s[:, N_IN:N_IN + N_OUT]
    xs, z1, h1, z2, h2, y = _layers(p, x)
    ts = (np.arcsinh(t / p["ysc"]) - p["ym"]) / p["ys"]
    d = y - ts
    count = d.size
    loss = float(np.sum(d * d) / count)
    dy = 2.0 * d / count
    g = {name: np.zeros(shape) for name, shape in _SIZES}
    g["W3"] = dy.T @ h2
    g["b3"] = dy.sum(axis=0)
    dz2 = (dy @ p["W3"]) * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * gelu_grad(z1)
    g["W1"] = dz1.T @ xs
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)
