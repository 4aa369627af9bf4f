"""Pins of the FP64 reference network (oracle/mlp.py) of the moment-fit warm
start (Sec. 2.2): closed forms of its inputs and of single-path networks
(which catch transposed or misrouted weights), GELU values, and its loss
gradient against central differences (which catches any backward error)."""
import math

import numpy as np

from oracle import mlp as M


def _blob(rng, scale=0.3):
    p = {"xm": rng.normal(size=12) * 0.1, "xs": 0.5 + rng.uniform(size=12),
         "ym": rng.normal(size=10) * 0.1, "ys": 0.5 + rng.uniform(size=10), "ysc": 10.0 ** rng.uniform(-6, -1, size=10),
         "W1": rng.normal(size=(128, 12)) * scale, "b1": rng.normal(size=128) * 0.1,
         "W2": rng.normal(size=(128, 128)) * scale / 4, "b2": rng.normal(size=128) * 0.1,
         "W3": rng.normal(size=(10, 128)) * scale / 4, "b3": rng.normal(size=10) * 0.1}
    return M.pack(p)


def test_blob_size_and_layout():
    assert M.NPARAM == 19520
    w = np.arange(M.NPARAM, dtype=np.float64)
    p = M.unpack(w)
    assert p["xm"][0] == 0 and p["ysc"][0] == 44 and p["W1"][0, 0] == 54 and p["W1"][1, 0] == 54 + 12
    assert p["W2"][0, 0] == 54 + 1536 + 128 and p["b3"][-1] == M.NPARAM - 1


def test_gelu_values():
    assert M.gelu(np.array([0.0]))[0] == 0.0
    assert abs(M.gelu(np.array([8.0]))[0] - 8.0) < 1e-12
    assert abs(M.gelu(np.array([-8.0]))[0]) < 1e-12
    # gelu(1) = Phi(1), the standard normal CDF at 1
    assert abs(M.gelu(np.array([1.0]))[0] - 0.5 * (1 + math.erf(1 / math.sqrt(2)))) < 1e-15
    z = np.linspace(-3, 3, 13)
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.allclose(M.gelu_grad(z), fd, atol=1e-8)


def test_inputs_closed_form():
    vmin, dv = np.array([-4.0, -2.0, -1.0]), np.array([0.5, 0.25, 0.125])
    vmax = vmin + 16 * dv
    n = 2.0
    u = np.array([vmin[0] + 5.5 * dv[0], vmin[1] + 8.25 * dv[1], vmin[2] + 3.5 * dv[2]])
    th = np.array([[4 * dv[0] ** 2, 0.1 * dv[0] * dv[1], 0.0],
                   [0.1 * dv[0] * dv[1], 9 * dv[1] ** 2, -0.2 * dv[1] * dv[2]],
                   [0.0, -0.2 * dv[1] * dv[2], 2.25 * dv[2] ** 2]])
    E2 = n * (th + np.outer(u, u))
    t = np.array([n, *(n * u), E2[0, 0], E2[0, 1], E2[0, 2], E2[1, 1], E2[1, 2], E2[2, 2]])
    x = M.inputs(t, vmin, dv, vmax)
    assert np.allclose(x[:6], [4, 0.1, 0, 9, -0.2, 2.25], atol=1e-12)
    assert np.allclose(x[6:9], [0.0, -0.25, 0.0], atol=1e-12)  # 5.5 and 3.5 are centres; 8.25 is 1/4 below 8.5
    assert np.allclose(x[9:], (u - vmin) / (vmax - vmin), atol=1e-15)
    assert M.inputs(np.r_[0.0, t[1:]], vmin, dv, vmax) is None


def test_single_path_network_closed_form():
    """One non-zero weight per layer: y_o = W3[o,j] gelu(W2[j,k] gelu(W1[k,i] xs_i + b1[k]) + b2[j]) + b3[o],
    t_o = ysc sinh(y_o ys + ym)."""
    p = {name: np.zeros(shape) for name, shape in M._SIZES}
    p["xm"][:] = 0.5
    p["xs"][:] = 2.0
    p["ym"][:] = 0.25
    p["ys"][:] = 3.0
    p["ysc"][:] = 1e-3
    i, k, j, o = 7, 100, 3, 9
    p["W1"][k, i] = 1.5
    p["b1"][k] = -0.2
    p["W2"][j, k] = -0.7
    p["b2"][j] = 0.3
    p["W3"][o, j] = 2.0
    p["b3"][2] = 0.4
    x = np.zeros((1, 12))
    x[0, i] = 1.3
    xs = (1.3 - 0.5) / 2.0
    h1 = M.gelu(np.array([1.5 * xs - 0.2]))[0]
    h2 = M.gelu(np.array([-0.7 * h1 + 0.3]))[0]
    want = np.full(10, 0.25)
    want[2] = 0.4 * 3.0 + 0.25
    want[o] = 2.0 * h2 * 3.0 + 0.25
    want = 1e-3 * np.sinh(want)
    # the zero-input units still pass gelu(0) = 0
    assert np.allclose(M.forward(M.pack(p), x)[0], want, atol=1e-14)


def test_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    w = _blob(rng)
    s = np.zeros((6, M.SAMPLE))
    s[:, :12] = rng.normal(size=(6, 12))
    s[:, 12:22] = rng.normal(size=(6, 10)) * 10.0 ** rng.uniform(-6, -1, size=(6, 10))
    s[:, 22] = 1.0
    loss, g = M.loss_and_grad(w, s)
    p = M.unpack(g)
    assert np.all(p["xm"] == 0) and np.all(p["ys"] == 0) and np.all(p["ysc"] == 0)
    first = 54  # the trained parameters start after the normalisation constants
    idx = list(rng.choice(np.arange(first, M.NPARAM), size=80, replace=False))
    idx += [first, first + 1536, first + 1536 + 128 + 5, M.NPARAM - 1, M.NPARAM - 11]  # block edges
    h = 1e-6
    for q in idx:
        wp, wm = w.copy(), w.copy()
        wp[q] += h
        wm[q] -= h
        fd = (M.loss_and_grad(wp, s)[0] - M.loss_and_grad(wm, s)[0]) / (2 * h)
        assert abs(fd - g[q]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (q, fd, g[q])
    assert loss > 0
