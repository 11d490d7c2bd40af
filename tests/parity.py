"""Parity protocol between the CUDA path and the FP64 oracle.

The CUDA path runs first; its pivots are then replayed in the oracle.  At
every step the oracle's own argmax must equal the GPU pivot whenever the
top-two gap exceeds max(1e-12 * err_max, delta_l); otherwise the GPU pivot's
exact error must lie within that margin of the max.  delta_l is the FP64
bookkeeping noise of Eq. (Residual): c0 * (l + sqrt(N)) * u * max ||s||^2.
The sqrt(N) term is the oracle's own: its norms and coefficients are
sequential FP64 sums over the N samples, whose rounding grows like sqrt(N) u
(measured against direct residual norms in tests/test_oracle_pins.py: about
1.3 sqrt(N) u at N = 8192 and 16384); the l term covers the l rounded updates
of the running sum.
"""
import math

import numpy as np

U = 2.0 ** -53


def delta(l, N, scale, c0=4.0):
    return c0 * (l + math.sqrt(max(N, 1))) * U * scale


def replay_and_check(orc, S, gpu, tol, kmax, rel_gap=1e-12, omp=False):
    """Returns the replayed oracle result; asserts the pivot protocol.
    omp: the oracle's OpenMP build (column loops on all host cores, results
    bit-identical to the single-threaded build) for full-size replays."""
    M, N = S.shape
    piv = np.asarray(gpu["pivots"])
    k = len(piv)
    rep = orc.rb_greedy(S, tol, kmax, forced=piv, omp=omp)
    assert rep["k"] == k, (rep["k"], k)
    assert list(rep["pivots"]) == list(piv)
    scale = rep["err_curve"][0]
    for l in range(k):
        emax = rep["own_max"][l]
        margin = max(rel_gap * emax, delta(l, N, scale))
        assert emax - rep["forced_err"][l] <= margin, (l, emax, rep["forced_err"][l], margin)
        if emax - rep["second_max"][l] > margin:
            assert rep["own_argmax"][l] == piv[l], l
    return rep


def basis_tol(err_curve, k):
    """Per-vector tolerance: cancellation amplifies rounding by 1/||v||."""
    d = np.sqrt(np.maximum(np.asarray(err_curve[:k]), 1e-300))
    return np.maximum(1e-12, 64 * U * math.sqrt(max(k, 1)) / d)


def column_norms(S, block=4096):
    """||s_j|| for every row of S, in blocks (S may be tens of GB)."""
    out = np.empty(S.shape[0])
    for a in range(0, S.shape[0], block):
        x = S[a:a + block].view(np.float64)
        out[a:a + block] = np.sqrt(np.einsum("ij,ij->i", x, x))
    return out


def compare(gpu, rep, S, err_atol=1e-12, c_rel=0.0, norms=None):
    """c_rel: extra C tolerance relative to ||s_j|| (the split form's sweep
    rounding, a stated bound of that form); norms: ||s_j|| if already known.
    Returns the measured deviations from the oracle."""
    k = rep["k"]
    ec_g, ec_r = np.asarray(gpu["err_curve"]), rep["err_curve"]
    assert np.max(np.abs(ec_g - ec_r)) <= err_atol, np.max(np.abs(ec_g - ec_r))
    bt = basis_tol(ec_r, k)
    dq = np.max(np.abs(np.asarray(gpu["Q"]) - rep["Q"]), axis=1) if k else np.zeros(0)
    assert np.all(dq <= bt), (np.max(dq / bt), int(np.argmax(dq / bt)))
    info = dict(k=int(k), max_err_curve_diff=float(np.max(np.abs(ec_g - ec_r))),
                max_dq=float(np.max(dq)) if k else 0.0,
                max_dq_over_tol=float(np.max(dq / bt)) if k else 0.0)
    if "C" in gpu and k:
        Cg = np.asarray(gpu["C"])[:k]
        if c_rel > 0.0 and norms is None:
            norms = column_norms(S)
        ctol = bt[:, None] + 1e-13 + (c_rel * norms[None, :] if c_rel > 0.0 else 0.0)
        dC = np.abs(Cg - rep["C"])
        r = dC / ctol
        assert np.all(r <= 1.0), np.max(r)
        info.update(max_dC=float(np.max(dC)), max_dC_over_tol=float(np.max(r)))
    if "final_err" in gpu:
        df = np.max(np.abs(np.asarray(gpu["final_err"]) - rep["final_err"]))
        assert df <= err_atol, df
        info.update(max_final_err_diff=float(df))
    return info


def first_divergence(a, b):
    n = min(len(a), len(b))
    for i in range(n):
        if a[i] != b[i]:
            return i
    return n
