"""Surrogate workflow around the C ABI: coefficient targets from the greedy's
C matrix, input scaling, training and evaluation against exact projection.

All compute runs in the CUDA library (rb_mlp_*, rb_generate, rb_project);
this module only reshapes tensors and computes summary statistics.
"""
from __future__ import annotations

import time

from . import rb


def targets_from_C(C):
    """(k, M) complex128 -> (M, 2k) float32 with Re/Im interleaved per coefficient."""
    import torch
    return torch.view_as_real(C.t().contiguous()).reshape(C.shape[1], -1).to(torch.float32).contiguous()


# The coefficients c_l(q, m) oscillate: each changes sign 46-103 times across
# the family's omega band.  With inputs on [-1, 1] the Glorot-initialised first
# layer spans only a few GELU transitions and training stalls at the
# zero-prediction loss; spreading the inputs over [-SPAN, SPAN] gives the first
# layer enough transitions to follow them.
SPAN = 16.0


def scale_inputs(q, m, q_range=(1.0, 10.0), m_range=(0.8, 1.2), span=SPAN):
    """Affine map of the (q, m) box onto [-span, span]^2, float32 (rows, 2)."""
    import torch
    q = torch.as_tensor(q, dtype=torch.float64)
    m = torch.as_tensor(m, dtype=torch.float64)
    x0 = span * (2 * (q - q_range[0]) / (q_range[1] - q_range[0]) - 1)
    x1 = span * (2 * (m - m_range[0]) / (m_range[1] - m_range[0]) - 1)
    return torch.stack([x0, x1], 1).to(torch.float32).contiguous()


def relative_errors(Y, Tref):
    """Per-row ||y - t|| / ||t||, plus the absolute ||y - t|| (the waveform-space
    error of the reconstruction, Q being orthonormal)."""
    import torch
    d = torch.linalg.norm((Y.double() - Tref.double()), dim=1)
    n = torch.linalg.norm(Tref.double(), dim=1).clamp_min(1e-300)
    return d / n, d


def summarize(e):
    import torch
    e = e.double()
    return {"median": float(e.median()), "p95": float(torch.quantile(e, 0.95)), "max": float(e.max())}


def chirp_tau_band(N: int, t_c: float = 1.05):
    """[tau_lo, tau_hi] of the chirp family's phase variable tau_i =
    (t_c - t_i)^(5/8), t_i = i / N: a snapshot is sum_i a_i exp(-i omega tau_i),
    so each basis coefficient is a sum of exp(-i omega tau_i) over this band."""
    return (t_c - (N - 1) / N) ** 0.625, t_c ** 0.625


def inputs(net: "rb.MLP", q, m):
    """The network's input rows: (q, m) themselves for the Fourier input
    layer, else their affine scaling."""
    import torch
    if net.fourier is not None:
        return torch.stack([torch.as_tensor(q, dtype=torch.float64), torch.as_tensor(m, dtype=torch.float64)],
                           1).to(torch.float32).contiguous()
    return scale_inputs(q, m)


def nearest_in_omega(q, m, qt, mt, device="cuda"):
    """The non-learned baseline: for each held-out (qt, mt), the index of the
    training snapshot nearest in omega (the family depends on (q, m) only
    through omega)."""
    import torch
    from . import synth
    om = torch.as_tensor(synth.chirp_omega(q, m), device=device)
    omt = torch.as_tensor(synth.chirp_omega(qt, mt), device=device)
    order = torch.argsort(om)
    pos = torch.searchsorted(om[order], omt).clamp(1, om.numel() - 1)
    left, right = order[pos - 1], order[pos]
    return torch.where((omt - om[left]).abs() <= (om[right] - omt).abs(), left, right)


def train(ctx: rb.RB, q, m, C, epochs=200, batch=1024, lr=1e-3, seed=4, fourier=None, split=False):
    """fourier: (tau_lo, tau_hi) for the Fourier input layer (chirp_tau_band(N))."""
    T = targets_from_C(C).cuda(ctx.device)
    net = rb.MLP(ctx, T.shape[1], batch_cap=max(batch, 4096), seed=seed, fourier=fourier, split=split)
    X = inputs(net, q, m).cuda(ctx.device)
    t0 = time.perf_counter()
    curve = net.train(X, T, epochs, batch, lr, seed)
    ctx.stream.synchronize()
    return net, curve, time.perf_counter() - t0
