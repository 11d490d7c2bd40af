"""Pins of the empirical-interpolation oracle (CPU): what LAPACK, a worked
example and the interpolant's defining identities fix."""
import numpy as np
import pytest
import scipy.linalg

from paper_1805_06124_gb300 import synth

eim = pytest.importorskip("oracle.eim_oracle")


def lu_row_pivots(A, k):
    """Rows chosen by LAPACK's getrf (partial pivoting) in its first k steps."""
    _, piv = scipy.linalg.lu_factor(A)
    perm = np.arange(A.shape[0])
    for i in range(k):
        perm[i], perm[piv[i]] = perm[piv[i]], perm[i]
    return perm[:k]


def test_hand_worked_example():
    """e_1 = (1, 3, 2), e_2 = (1, 1, 0): p_1 = 1 (|3| largest); c = e_2(1) / e_1(1)
    = 1/3, r_2 = e_2 - e_1/3 = (2/3, 0, -2/3) -> first maximum at x = 0."""
    E = np.array([[1.0, 3.0, 2.0], [1.0, 1.0, 0.0]])
    out = eim.eim(E)
    assert list(out["nodes"]) == [1, 0]
    np.testing.assert_allclose(out["r2_own"], [9.0, 4.0 / 9.0])
    np.testing.assert_allclose(out["V"], [[3.0, 1.0], [1.0, 1.0]])


@pytest.mark.parametrize("k,N,seed", [(5, 40, 0), (30, 400, 1), (60, 1000, 2)])
def test_nodes_equal_lu_partial_pivoting(k, N, seed):
    """On a real basis the EIM residual of e_i is column i of the Schur
    complement of LU with partial pivoting on E^T, so the nodes are getrf's
    row pivots (both take the first maximum)."""
    rng = np.random.default_rng(seed)
    E = np.linalg.qr(rng.standard_normal((N, k)))[0].T
    out = eim.eim(E)
    np.testing.assert_array_equal(out["nodes"], lu_row_pivots(E.T, k))


def test_interpolant_identities():
    S = synth.chirps(300, 500, seed=4)
    Q = np.linalg.qr(S[:40].T)[0].T           # 40 orthonormal chirp-space functions
    out = eim.eim(Q)
    P, V, B = out["nodes"], out["V"], out["B"]
    assert len(set(P.tolist())) == len(P)
    np.testing.assert_allclose(B @ V, Q.T, atol=1e-10)           # I[e_l] = e_l
    F = np.random.default_rng(0).standard_normal((7, 300)) + 0j
    IF = eim.interpolate(B, P, F)
    np.testing.assert_allclose(IF[:, P], F[:, P], atol=1e-10)   # I[f](p_m) = f(p_m)
    np.testing.assert_allclose(B[P], np.eye(len(P)), atol=1e-10)


def test_forced_replay_reports_own_choice():
    rng = np.random.default_rng(5)
    E = np.linalg.qr(rng.standard_normal((50, 6)))[0].T
    free = eim.eim(E)
    forced = free["nodes"].copy()
    forced[3] = [x for x in range(50) if x not in forced[:4]][0]
    rep = eim.eim(E, forced=forced[:4].tolist() + [0, 0])
    assert rep["own"][3] == free["nodes"][3] and rep["nodes"][3] == forced[3]
    assert rep["r2_forced"][3] <= rep["r2_own"][3]


def test_validation_closed_forms():
    S = synth.chirps(256, 400, seed=6)
    Q = np.linalg.qr(S[:30].T)[0].T
    out = eim.eim(Q)
    rng = np.random.default_rng(1)
    inside = (rng.standard_normal((5, 30)) + 1j * rng.standard_normal((5, 30))) @ Q
    v = eim.validate(Q, out["B"], out["nodes"], inside)
    assert np.all(v["err_proj"] < 1e-20 * 30) and np.all(v["err_eim"] < 1e-18 * 30)
    # orthogonal to the span: the projection error is ||t||^2
    T = rng.standard_normal((5, 256)) + 1j * rng.standard_normal((5, 256))
    T = T - (T @ Q.conj().T) @ Q
    v = eim.validate(Q, out["B"], out["nodes"], T)
    np.testing.assert_allclose(v["err_proj"], np.sum(np.abs(T) ** 2, axis=1), rtol=1e-12)
    # interpolation error >= projection error, and <= (1 + ||B||_2)^2 times it
    W = S[30:60]
    v = eim.validate(Q, out["B"], out["nodes"], W)
    lam = 1.0 + np.linalg.norm(out["B"], 2)
    assert np.all(v["err_eim"] >= v["err_proj"] * (1 - 1e-10))
    assert np.all(v["err_eim"] <= lam ** 2 * v["err_proj"] * (1 + 1e-10))
