"""ORACLE -- test infrastructure only.  fp64 numpy statement of the per-query
parameter MLP (not part of the paper; it predicts the query-processing knobs
cut and heap_factor that Section 5.3 sweeps globally).

Architecture: 64 -> 128 -> 64 -> 2, ReLU hidden layers; parameters packed as
W1[128][64], b1[128], W2[64][128], b2[64], W3[2][64], b3[2].  Outputs o map to
cut = clamp(round(3 + 27 sigmoid(o0)), 3, 30), heap_factor = 0.5 + 0.5
sigmoid(o1).  Loss = mean over rows of sum_j (sigmoid(o_j) - t_j)^2.
"""
from __future__ import annotations

import numpy as np

IN, H1, H2, OUT = 64, 128, 64, 2
SHAPES = [("W1", (H1, IN)), ("b1", (H1,)), ("W2", (H2, H1)), ("b2", (H2,)), ("W3", (OUT, H2)), ("b3", (OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = w[o:o + n].reshape(shp)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def init(seed=0):
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in SHAPES:
        if name.startswith("W"):
            p[name] = rng.standard_normal(shp) * np.sqrt(2.0 / shp[1])
        else:
            p[name] = np.zeros(shp)
    return pack(p)


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def forward(w, x):
    """Returns (o, cache)."""
    p = unpack(w)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ p["W1"].T + p["b1"]
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ p["W2"].T + p["b2"]
    a2 = np.maximum(z2, 0.0)
    o = a2 @ p["W3"].T + p["b3"]
    return o, (x, z1, a1, z2, a2, o)


def params_from_output(o):
    o = np.asarray(o, dtype=np.float64)
    cut = np.clip(np.rint(3.0 + 27.0 * sigmoid(o[:, 0])), 3, 30).astype(np.int64)
    hf = 0.5 + 0.5 * sigmoid(o[:, 1])
    return cut, hf


def loss(w, x, t):
    o, _ = forward(w, x)
    e = sigmoid(o) - np.asarray(t, dtype=np.float64)
    return float((e * e).sum(axis=1).mean())


def grad(w, x, t):
    """Analytic gradient of loss(w, x, t), packed like w."""
    p = unpack(w)
    o, (x, z1, a1, z2, a2, _) = forward(w, x)
    n = x.shape[0]
    s = sigmoid(o)
    do = 2.0 * (s - t) * s * (1.0 - s) / n
    g = {"W3": do.T @ a2, "b3": do.sum(0)}
    dz2 = (do @ p["W3"]) * (z2 > 0)
    g["W2"] = dz2.T @ a1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * (z1 > 0)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(0)
    return pack(g)
