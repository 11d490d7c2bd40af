"""FP64 CPU oracle of the learned surrogate's network (test infrastructure only).

Only tests, the smoke check and the benchmark's baseline arm may import this
module; it shares no code with the CUDA path.

Network: x (2) -> GELU(W1 x + b1) (256) -> GELU(W2 . + b2) (256) ->
GELU(W3 . + b3) (256) -> W4 . + b4 (n_out); GELU(z) = z Phi(z) with the exact
error function; loss = (1/rows) sum_r ||y_r - t_r||^2.  With the Fourier
input layer (``fourier=(tau_lo, tau_hi)``) a row x is (q, m) and the first
layer is the fixed encoding h1 = (cos(omega tau_f), sin(omega tau_f)),
f < 128, tau_f = tau_lo + f (tau_hi - tau_lo) / 127, omega = 200 eta^(-3/8)
m^(-5/8), eta = q / (1 + q)^2; W1 and b1 are then unused.  Parameters are one flat
vector W1 (256x2), b1, W2 (256x256), b2, W3 (256x256), b3, W4 (n_out x 256), b4,
row-major -- the same order the C ABI uses.  Backward is the chain rule
written out by hand; it is pinned by central finite differences.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

W = 256


def layout(n_out: int):
    sizes = [("W1", (W, 2)), ("b1", (W,)), ("W2", (W, W)), ("b2", (W,)), ("W3", (W, W)), ("b3", (W,)),
             ("W4", (n_out, W)), ("b4", (n_out,))]
    out, off = {}, 0
    for name, shp in sizes:
        n = int(np.prod(shp))
        out[name] = (off, shp)
        off += n
    return out, off


def unpack(p, n_out):
    lay, n = layout(n_out)
    p = np.asarray(p, np.float64)
    assert p.size == n
    return {k: p[o:o + int(np.prod(s))].reshape(s) for k, (o, s) in lay.items()}


def pack(d, n_out):
    lay, n = layout(n_out)
    p = np.zeros(n)
    for k, (o, s) in lay.items():
        p[o:o + int(np.prod(s))] = np.asarray(d[k], np.float64).ravel()
    return p


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def fourier_features(X, tau_lo, tau_hi):
    """(rows, 256): cos then sin of omega(q, m) tau_f for 128 frequencies."""
    X = np.asarray(X, np.float64)
    q, m = X[:, 0], X[:, 1]
    eta = q / (1.0 + q) ** 2
    omega = 200.0 * eta ** (-3.0 / 8.0) * m ** (-5.0 / 8.0)
    tau = tau_lo + (tau_hi - tau_lo) * np.arange(W // 2) / (W // 2 - 1)
    ph = omega[:, None] * tau[None, :]
    return np.concatenate([np.cos(ph), np.sin(ph)], axis=1)


def forward(p, X, n_out, keep=False, fourier=None):
    P = unpack(p, n_out)
    X = np.asarray(X, np.float64)
    if fourier is not None:
        z1 = None
        h1 = fourier_features(X, *fourier)
    else:
        z1 = X @ P["W1"].T + P["b1"]
        h1 = gelu(z1)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = gelu(z2)
    z3 = h2 @ P["W3"].T + P["b3"]
    h3 = gelu(z3)
    y = h3 @ P["W4"].T + P["b4"]
    if keep:
        return y, (X, z1, h1, z2, h2, z3, h3)
    return y


def loss(p, X, T, n_out, fourier=None):
    y = forward(p, X, n_out, fourier=fourier)
    return float(np.sum((y - np.asarray(T, np.float64)) ** 2) / len(X))


def grad(p, X, T, n_out, fourier=None):
    """(gradient vector, loss) of the loss above."""
    P = unpack(p, n_out)
    y, (X, z1, h1, z2, h2, z3, h3) = forward(p, X, n_out, keep=True, fourier=fourier)
    B = len(X)
    dy = 2.0 * (y - np.asarray(T, np.float64)) / B
    g = {"W4": dy.T @ h3, "b4": dy.sum(0)}
    dz3 = (dy @ P["W4"]) * gelu_grad(z3)
    g["W3"], g["b3"] = dz3.T @ h2, dz3.sum(0)
    dz2 = (dz3 @ P["W3"]) * gelu_grad(z2)
    g["W2"], g["b2"] = dz2.T @ h1, dz2.sum(0)
    if fourier is not None:  # the fixed input layer has no parameters
        g["W1"], g["b1"] = np.zeros_like(P["W1"]), np.zeros_like(P["b1"])
    else:
        dz1 = (dz2 @ P["W2"]) * gelu_grad(z1)
        g["W1"], g["b1"] = dz1.T @ X, dz1.sum(0)
    return pack(g, n_out), float(np.sum((y - T) ** 2) / B)


def to_bf16(a):
    """Round FP32/FP64 values to the nearest BF16 (ties to even), as FP64."""
    f = np.asarray(a, np.float32).copy()
    u = f.view(np.uint32)
    r = ((u >> 16) & 1) + np.uint32(0x7FFF)
    u = ((u + r) & np.uint32(0xFFFF0000)).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def round_weights(p, n_out):
    """Weights rounded to BF16 (what the GPU multiplies with); biases as given."""
    d = unpack(p, n_out)
    for k in ("W1", "W2", "W3", "W4"):
        d[k] = to_bf16(d[k])
    return pack(d, n_out)
