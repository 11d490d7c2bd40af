"""FP64 CPU oracle of the reconstruction step (test infrastructure only).

Only tests, the smoke check and the benchmark's baseline arm may import this
module; it shares no code with the CUDA path.

Reconstruction algorithm (Alg. 4, Sec. 5.2.2 "A reconstruction approach to QR"):
after a j-term MGS with pivoting (here: the greedy, Alg. 3 = Alg. 2 by Prop.
5.3), S ~= Q_j R(1:j, 1:M) with R(1:j, 1:M) = Q_j^H S -- the greedy's
coefficient matrix C up to the column order, which changes no singular value
or left singular vector.  Then

  * SVD  R(1:j, 1:M) = V Sigma W^H              (Alg. 4, step 5)
  * k = number of singular values above tau2    (step 6: sigma_{k+1} < tau2 < sigma_k)
  * X_k = Q_j V(:, 1:k)                         (step 7; read as all j basis vectors
                                                 times the first k columns of V, the
                                                 only reading with matching shapes,
                                                 Theorem 5.6: X_j = Q_k V_j)

Error statements used as pins: Theorem 5.6 (exact rank: ||S - X_i X_i^H S||_2
= sigma_{i+1}(S)) and Theorem 5.8 (sigma_{i+1}(S) <= ||S - X_i X_i^H S||_2 <=
sigma_{i+1}(C) + ||S - Q_j C||_2).

The SVD is LAPACK's (numpy.linalg.svd), a library primitive used as one step.
Each left singular vector is fixed up to a unit complex factor; the oracle
makes the largest-magnitude entry of each column of V real and positive
(lowest row index among equal magnitudes), the same convention the CUDA path
uses.

Python layout as in oracle.py: Q (j, N) with row l = q_l, C (j, M) with
C[l, m] = q_l^H s_m; X is returned as (k, N), row c = x_c.
"""
from __future__ import annotations

import numpy as np


def normalize_phases(V: np.ndarray) -> np.ndarray:
    """Scale each column of V by a unit complex number so that its entry of
    largest magnitude (lowest index among equals) is real and positive."""
    V = np.array(V, dtype=np.complex128, copy=True)
    for c in range(V.shape[1]):
        a = np.abs(V[:, c])
        p = int(np.flatnonzero(a == a.max())[0])
        if a[p] > 0:
            V[:, c] *= np.conj(V[p, c]) / a[p]
    return V


def reconstruct(Q, C, tau2: float) -> dict:
    """Alg. 4 steps 5-7 on the greedy's output.  Returns sigma (j,), V (j, j)
    with normalised phases, k, and X (k, N)."""
    Q = np.asarray(Q, dtype=np.complex128)
    C = np.asarray(C, dtype=np.complex128)
    j = C.shape[0]
    if j == 0:
        return dict(sigma=np.zeros(0), V=np.zeros((0, 0), np.complex128), k=0, X=np.zeros((0, Q.shape[1]), np.complex128))
    U, s, _ = np.linalg.svd(C, full_matrices=False)   # C = U diag(s) W^H, U is j x j
    V = normalize_phases(U)
    k = int(np.sum(s > tau2))
    X = V[:, :k].T @ Q                                 # x_c = sum_l V[l, c] q_l
    return dict(sigma=s, V=V, k=k, X=X)


def residual_norm2(S, X) -> float:
    """||A - X X^H A||_2 for A = S^T (the paper's N x M snapshot matrix) and an
    orthonormal basis given as rows of X."""
    S = np.asarray(S, dtype=np.complex128)
    X = np.asarray(X, dtype=np.complex128)
    A = S.T
    if X.shape[0] == 0:
        return float(np.linalg.norm(A, 2))
    B = X.T                                            # N x k, columns x_c
    R = A - B @ (B.conj().T @ A)
    return float(np.linalg.norm(R, 2))
