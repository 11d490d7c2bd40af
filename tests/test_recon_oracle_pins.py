"""Pins of the reconstruction oracle (Alg. 4) against what the paper's
theorems and plain linear algebra fix (CPU)."""
import numpy as np
import pytest

from paper_1805_06124_gb300 import synth

recon = pytest.importorskip("oracle.recon_oracle")


def _greedy(orc, S, tol, kmax):
    r = orc.rb_greedy(S, tol, kmax)
    return r["Q"], r["C"], r


def test_exact_rank_reaches_svd(orc):
    """Theorem 5.6: for S of exact rank r and the full greedy basis (j = r),
    ||S - X_i X_i^H S||_2 = sigma_{i+1}(S) for every i <= r, and the
    singular values of C equal those of S."""
    S = synth.low_rank(60, 40, 6, seed=11)               # 60 snapshots of length 40, rank 6
    scale = float(np.max(np.sum(np.abs(S) ** 2, axis=1)))
    Q, C, r = _greedy(orc, S, 1e-12 * scale, 40)
    assert r["k"] == 6
    sv = np.linalg.svd(S.T, compute_uv=False)
    out = recon.reconstruct(Q, C, 0.0)
    np.testing.assert_allclose(out["sigma"], sv[:6], rtol=1e-12)
    for i in range(1, 6):
        Xi = out["V"][:, :i].T @ Q
        np.testing.assert_allclose(recon.residual_norm2(S, Xi), sv[i], rtol=1e-9, atol=1e-12 * sv[0])


def test_bounds_of_theorem_5_8(orc):
    """Chirps truncated at j < rank: POD optimality below, sigma(C) plus the
    greedy's own residual above (Theorem 5.8), for every k <= j."""
    S = synth.chirps(256, 400, seed=3)
    Q, C, r = _greedy(orc, S, 1e-6, 200)
    j = r["k"]
    A = S.T
    sv = np.linalg.svd(A, compute_uv=False)
    resid = np.linalg.norm(A - Q.T @ C, 2)                # ||S - Q_j C||_2 = ||R_22||_2
    out = recon.reconstruct(Q, C, 0.0)
    for k in range(1, j + 1):
        Xk = out["V"][:, :k].T @ Q
        e = recon.residual_norm2(S, Xk)
        assert e >= sv[k] * (1 - 1e-10)
        assert e <= (out["sigma"][k] if k < j else 0.0) + resid * (1 + 1e-10) + 1e-13
    # the reconstructed basis beats the greedy basis of the same size wherever
    # the singular values decay (the point of Alg. 4)
    k = j // 2
    e_rec = recon.residual_norm2(S, out["V"][:, :k].T @ Q)
    e_qr = recon.residual_norm2(S, Q[:k])
    assert e_rec <= e_qr * (1 + 1e-12)


def test_orthonormal_basis_and_phase_convention(orc):
    S = synth.chirps(128, 300, seed=2)
    Q, C, r = _greedy(orc, S, 1e-8, 100)
    out = recon.reconstruct(Q, C, 1e-3)
    X = out["X"]
    np.testing.assert_allclose(X.conj() @ X.T, np.eye(out["k"]), atol=1e-13)
    V = out["V"]
    for c in range(V.shape[1]):
        p = int(np.argmax(np.abs(V[:, c])))
        assert abs(V[p, c].imag) < 1e-15 and V[p, c].real > 0
    # k counts the singular values above tau2
    assert out["k"] == int(np.sum(out["sigma"] > 1e-3))
    assert np.all(np.diff(out["sigma"]) <= 0)
