"""FP64 CPU oracle of the empirical-interpolation step (test infrastructure only).

Only tests, the smoke check and the benchmark's baseline arm may import this
module; it shares no code with the CUDA path.

The paper's software ("QR+DEIM", Sec. 6 and its overview, Sec. 6.1) selects
empirical interpolation (EI) nodes for the greedy basis with the greedy EIM /
DEIM algorithm it cites (the algorithm itself is not printed in the paper).
This oracle writes that published algorithm out from its definition:

  * p_1 = argmax_x |e_1(x)|;
  * for i = 2..k: interpolate e_i on the nodes p_1..p_{i-1} with e_1..e_{i-1}
    (solve V_{i-1} c = e_i(P), V_{i-1}[m, l] = e_l(p_m)), take the residual
    r_i = e_i - sum_l c_l e_l and p_i = argmax_x |r_i(x)| over the grid points
    not yet chosen (lowest index among equal maxima);
  * the interpolant I[f](x) = sum_m B[x, m] f(p_m) with B = E^T V^{-1}, so that
    I[e_l] = e_l for every basis function (B V = E^T).

Out-of-sample validation (Sec. 6.1): for a snapshot t, the projection
error ||t - Q Q^H t||^2 and the interpolation error ||t - I[t]||^2, both
computed directly from their definitions.

Pins (tests/test_eim_oracle_pins.py): the nodes equal the row pivots of
LAPACK's LU with partial pivoting on real bases and a hand-worked example;
the interpolant meets its defining identities; the validation errors meet
closed forms (snapshots in and orthogonal to the basis span) and the
interpolation bound ||t - I[t]|| <= (1 + ||B||_2) ||t - Q Q^H t||.

Layout as in oracle.py: E (k, N) with row l = basis function e_l on the grid.
"""
from __future__ import annotations

import numpy as np


def _argmax_free(a: np.ndarray, taken) -> int:
    a = a.copy()
    if len(taken):
        a[np.asarray(taken, dtype=np.int64)] = -1.0
    return int(np.flatnonzero(a == a.max())[0])


def eim(E, forced=None) -> dict:
    """Greedy EIM nodes of the basis rows of E (k, N).

    With ``forced`` (a node sequence from another implementation) step i uses
    forced[i] as p_i; the oracle still reports its own argmax ``own[i]`` and
    the squared residuals at both (``r2_own[i]``, ``r2_forced[i]``) and the
    runner-up (``r2_second[i]``) so that a caller can judge near ties.  Returns nodes, V (k, k), B (N, k), and the
    squared residual maxima."""
    E = np.asarray(E, dtype=np.complex128)
    k, N = E.shape
    P: list[int] = []
    own, r2_own, r2_second, r2_forced = [], [], [], []
    for i in range(k):
        e = E[i]
        if i == 0:
            r = e.copy()
        else:
            A = E[:i][:, P].T                       # A[m, l] = e_l(p_m)
            c = np.linalg.solve(A, e[P])
            r = e - c @ E[:i]
        a = np.abs(r) ** 2
        p_own = _argmax_free(a, P)
        own.append(p_own)
        r2_own.append(float(a[p_own]))
        r2_second.append(float(a[_argmax_free(a, P + [p_own])]) if N - len(P) > 1 else -1.0)
        p = p_own if forced is None else int(forced[i])
        r2_forced.append(float(a[p]))
        P.append(p)
    V = E[:, P].T if k else np.zeros((0, 0), np.complex128)  # V[m, l] = e_l(p_m)
    B = np.linalg.solve(V.T, E).T if k else np.zeros((N, 0), np.complex128)
    return dict(nodes=np.asarray(P, dtype=np.int64), V=V, B=B, own=np.asarray(own, dtype=np.int64),
                r2_own=np.asarray(r2_own), r2_second=np.asarray(r2_second), r2_forced=np.asarray(r2_forced))


def interpolate(B, nodes, F) -> np.ndarray:
    """I[f] for every row f of F (M', N): rows of the result are
    sum_m B[:, m] f(p_m)."""
    F = np.asarray(F, dtype=np.complex128)
    return F[:, np.asarray(nodes)] @ np.asarray(B).T


def validate(Q, B, nodes, T) -> dict:
    """Out-of-sample errors of the basis Q (k, N) and its interpolant (B,
    nodes) on the snapshots T (M', N): squared projection and interpolation
    errors per snapshot, from the definitions."""
    Q = np.asarray(Q, dtype=np.complex128)
    T = np.asarray(T, dtype=np.complex128)
    C = T @ Q.conj().T                              # C[j, l] = q_l^H t_j
    R = T - C @ Q
    err_proj = np.sum(np.abs(R) ** 2, axis=1)
    err_eim = np.sum(np.abs(T - interpolate(B, nodes, T)) ** 2, axis=1)
    return dict(err_proj=err_proj, err_eim=err_eim)
