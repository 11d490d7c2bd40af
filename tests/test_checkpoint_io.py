"""Checkpoint files round-trip on the host (no GPU)."""
import numpy as np
import pytest

from paper_1805_06124_gb300 import checkpoint


def test_round_trip(tmp_path):
    rng = np.random.default_rng(0)
    k, N, M, kmax = 4, 6, 9, 7
    res = dict(k=k, Q=rng.standard_normal((kmax, N)) + 1j * rng.standard_normal((kmax, N)),
               pivots=np.arange(kmax)[::-1].copy(), C=rng.standard_normal((kmax, M)) + 0j,
               err_curve=np.linspace(1, 0, kmax + 1), rdiag=np.ones(kmax))
    p = str(tmp_path / "a.npz")
    checkpoint.save(p, res, 1e-10)
    ck = checkpoint.load(p)
    assert (ck["k"], ck["N"], ck["M"], ck["tol"]) == (k, N, M, 1e-10)
    np.testing.assert_array_equal(ck["Q"], res["Q"][:k])
    np.testing.assert_array_equal(ck["pivots"], res["pivots"][:k])
    np.testing.assert_array_equal(ck["C"], res["C"][:k])
    np.testing.assert_array_equal(ck["err_curve"], res["err_curve"][:k + 1])


def test_inconsistent_file_rejected(tmp_path):
    p = str(tmp_path / "b.npz")
    np.savez(p, k=2, N=3, M=4, tol=0.0, Q=np.zeros((2, 3)), pivots=np.zeros(2), C=np.zeros((2, 5)),
             err_curve=np.zeros(3), rdiag=np.zeros(2))
    with pytest.raises(ValueError):
        checkpoint.load(p)
