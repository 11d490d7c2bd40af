"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code path: closed forms,
brute-force least squares, LAPACK's pivoted QR, the second oracle (Alg. 2),
and invariants stated in the paper (Thm. 3.2, Thm. 4.1/4.2, Cor. 4.3,
Prop. 5.3, Cor. 5.4).  None needs a GPU.
"""
import numpy as np
import pytest
import scipy.linalg

from paper_1805_06124_gb300 import synth

U = 2.0 ** -53


def _greedy(orc, S, tol=1e-30, kmax=None, **kw):
    M, N = S.shape
    if kmax is None:
        kmax = min(M, N)
    return orc.rb_greedy(S, tol, kmax, **kw)


# ---------------------------------------------------------------- closed forms

def _cplx(a):
    a = np.asarray(a, np.float64)
    return a[..., 0] + 1j * a[..., 1]


def test_hand_worked_2x2(orc):
    """Alg. 3 by hand (tests/golden/alg3_hand_worked_2x2.json, with its
    derivation): s_0 = (1, 0), s_1 = (1, 1) -> pivots (1, 0), errors
    (2, 1/2, 0), and the stopping rule on squared errors."""
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "alg3_hand_worked_2x2.json")) as f:
        fx = json.load(f)
    S = _cplx(fx["S_columns"])
    r = _greedy(orc, S, tol=fx["tol"], kmax=fx["kmax"])
    assert r["status"] == orc.OK and r["k"] == len(fx["pivots"])
    assert list(r["pivots"]) == fx["pivots"]
    np.testing.assert_allclose(r["err_curve"], fx["err_curve"], atol=1e-15)
    np.testing.assert_allclose(r["Q"], _cplx(fx["Q_rows"]), atol=1e-15)
    np.testing.assert_allclose(r["C"], _cplx(fx["C"]), atol=1e-15)
    np.testing.assert_allclose(r["rdiag"], fx["rdiag"], atol=1e-15)
    r1 = _greedy(orc, S, tol=fx["tol_loose"], kmax=fx["kmax"])
    assert r1["k"] == 1 and list(r1["pivots"]) == fx["pivots_loose"]
    np.testing.assert_allclose(r1["err_curve"], fx["err_curve_loose"], atol=1e-15)


def test_exact_ties_lowest_index(orc):
    """Columns of the identity all have norm 1 and stay tied: ties go to the
    lowest index at every step."""
    S = np.eye(5, dtype=np.complex128)
    r = _greedy(orc, S)
    assert list(r["pivots"]) == [0, 1, 2, 3, 4]
    np.testing.assert_array_equal(r["err_curve"], [1, 1, 1, 1, 1, 0])


def test_orthogonal_columns_distinct_norms(orc):
    """Mutually orthogonal columns: pivots in descending norm, q = s/||s||,
    err_curve = sorted squared norms."""
    rng = np.random.default_rng(11)
    N, M = 20, 9
    A = rng.standard_normal((N, M)) + 1j * rng.standard_normal((N, M))
    Uo, _ = np.linalg.qr(A)
    d = rng.uniform(0.5, 3.0, M)
    S = np.ascontiguousarray((Uo * d[None, :]).T)
    r = _greedy(orc, S)
    order = np.argsort(-d, kind="stable")
    assert list(r["pivots"]) == list(order)
    np.testing.assert_allclose(r["err_curve"][:-1], d[order] ** 2, rtol=1e-14)
    assert abs(r["err_curve"][-1]) < 1e-14
    np.testing.assert_allclose(r["Q"], S[order] / d[order][:, None], atol=1e-14)


def test_exact_rank(orc):
    """S = A B with rank r: the greedy stops after exactly r vectors.  The
    residual after r steps is zero in exact arithmetic; the bookkeeping
    ||s||^2 - sum |c|^2 resolves it only to a few u * ||s||^2."""
    S = synth.low_rank(40, 30, 7, seed=5)
    scale = np.max(np.sum(np.abs(S) ** 2, axis=1))
    r = _greedy(orc, S, tol=1e-11 * scale)
    assert r["k"] == 7 and r["status"] == orc.OK
    assert r["err_curve"][7] < 64 * U * scale
    assert r["err_curve"][6] > 1e-6 * scale


def test_duplicates_never_picked_twice(orc):
    S = synth.random_complex(12, 16, seed=3, scales=np.linspace(1, 2, 12))
    S[7] = S[2]
    S[9] = 1j * S[4]
    r = _greedy(orc, S, tol=1e-10)
    piv = list(r["pivots"])
    assert len(set(piv)) == len(piv)
    assert not (2 in piv and 7 in piv)
    assert not (4 in piv and 9 in piv)
    assert r["k"] == 10


def test_real_input_gives_real_basis(orc):
    rng = np.random.default_rng(4)
    S = rng.standard_normal((15, 11)).astype(np.complex128)
    r = _greedy(orc, S)
    assert np.all(r["Q"].imag == 0) and np.all(r["C"].imag == 0)


def test_degenerate_inputs(orc):
    Z = np.zeros((6, 5), np.complex128)
    r = _greedy(orc, Z, tol=1e-30)
    assert r["k"] == 0 and r["status"] == orc.OK and r["err_curve"][0] == 0.0
    S = synth.random_complex(6, 5, seed=1)
    r = _greedy(orc, S, tol=1e9)
    assert r["k"] == 0 and r["status"] == orc.OK
    r = _greedy(orc, S, tol=1e-30, kmax=2)
    assert r["k"] == 2 and r["status"] == orc.KMAX_REACHED
    S[3, 2] = np.nan
    assert _greedy(orc, S)["status"] == orc.ENONFINITE
    S = synth.random_complex(3, 8, seed=2)  # M < N: stops at M vectors
    r = _greedy(orc, S, tol=0.0)
    assert r["k"] == 3


# -------------------------------------------------------------- brute force

def _bruteforce_greedy(S, kmax):
    """At each step the squared residual of every unpicked column is
    obtained by least squares on the ORIGINAL pivot columns (no basis)."""
    M, N = S.shape
    picked, curve = [], []
    for _ in range(kmax + 1):
        best, bval = -1, -1.0
        for j in range(M):
            if j in picked:
                continue
            if picked:
                A = S[picked].T
                x, *_ = np.linalg.lstsq(A, S[j], rcond=None)
                res = S[j] - A @ x
            else:
                res = S[j]
            e = float(np.vdot(res, res).real)
            if e > bval:
                best, bval = j, e
        curve.append(bval if best >= 0 else 0.0)
        if best < 0 or len(picked) == kmax:
            break
        picked.append(best)
    return picked, np.array(curve)


@pytest.mark.parametrize("case", ["random", "chirp_scaled"])
def test_bruteforce_least_squares(orc, case):
    if case == "random":
        S = synth.random_complex(10, 12, seed=7, scales=np.linspace(1.0, 1.5, 10))
        kmax = 9
    else:
        S = synth.chirps(16, 12, seed=0) * np.linspace(1.0, 1.3, 12)[:, None]
        kmax = 8
    r = _greedy(orc, S, tol=0.0, kmax=kmax)
    piv, curve = _bruteforce_greedy(S, kmax)
    assert list(r["pivots"]) == piv
    scale = curve[0]
    np.testing.assert_allclose(r["err_curve"], curve[:len(r["err_curve"])], rtol=0, atol=1e-13 * scale)


# ------------------------------------------------- equivalence and LAPACK

@pytest.mark.parametrize("case", ["chirp", "random"])
def test_rb_greedy_equals_mgs_pivot(orc, case):
    """Prop. 5.3: Alg. 2 and Alg. 3 pick the same pivots and build the same
    basis (same column, same normalisation, hence same phase)."""
    if case == "chirp":
        S = synth.chirps(128, 200, seed=0) * np.linspace(1.0, 1.01, 200)[:, None]
        tol = 1e-10
    else:
        S = synth.random_complex(60, 80, seed=9, scales=np.linspace(1, 3, 60))
        tol = 1e-3
    a = orc.rb_greedy(S, tol, 200)
    b = orc.mgs_pivot(S, tol, 200)
    assert a["k"] == b["k"] and a["k"] > 5
    assert list(a["pivots"]) == list(b["pivots"])
    np.testing.assert_allclose(a["rdiag"], b["rdiag"], rtol=1e-6, atol=1e-12)
    for l in range(a["k"]):
        tol_l = 1e-14 / max(a["rdiag"][l], 1e-300) + 1e-13
        assert np.max(np.abs(a["Q"][l] - b["Q"][l])) < max(tol_l, 1e-10)
    # R of Alg. 2 equals C = Q^H S of Alg. 3 on and above the pivot diagonal
    for l in range(a["k"]):
        live = [j for j in range(S.shape[0]) if j not in list(a["pivots"][:l])]
        np.testing.assert_allclose(a["C"][l, live], b["R"][l, live], atol=1e-8)


def test_lapack_pivoted_qr(orc):
    """scipy / LAPACK zgeqp3: same pivots while gaps are clear, and
    |R(l,l)|^2 equals the greedy error curve (Cor. 5.4)."""
    S = synth.chirps(256, 300, seed=2) * np.linspace(1.0, 1.02, 300)[:, None]
    r = orc.rb_greedy(S, 1e-10, 300)
    k = r["k"]
    Qr, R, P = scipy.linalg.qr(S.T, pivoting=True, mode="economic")
    d2 = np.abs(np.diag(R)[:k]) ** 2
    np.testing.assert_allclose(d2, r["err_curve"][:k], rtol=1e-6, atol=1e-13)
    # pivots agree up to the first step whose top-two gap is not clear
    same = 0
    for l in range(k):
        if P[l] != r["pivots"][l]:
            break
        same += 1
    assert same >= min(k, 20)


# ---------------------------------------------------------------- invariants

@pytest.fixture(scope="module")
def chirp_run(orc):
    S = synth.chirps(256, 400, seed=0)
    r = orc.rb_greedy(S, 1e-10, 300)
    return S, r


def test_triangular_identity(chirp_run):
    """Thm. 4.2 with Cor. 5.4: C[:, pivots] is upper triangular with real
    positive diagonal R(l,l) and R(l,l)^2 = err_curve[l]."""
    S, r = chirp_run
    k = r["k"]
    T = r["C"][:, r["pivots"]]
    assert np.max(np.abs(np.tril(T, -1))) < 1e-13
    d = np.diag(T)
    assert np.all(np.abs(d.imag) < 1e-13) and np.all(d.real > 0)
    np.testing.assert_allclose(d.real, r["rdiag"], rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(r["rdiag"] ** 2, r["err_curve"][:k], rtol=1e-6, atol=1e-14)


def test_monotone_error_curve(chirp_run):
    """Prop. 5.3: the diagonal of R (hence the error curve) is non-increasing."""
    _, r = chirp_run
    e = r["err_curve"]
    assert np.all(np.diff(e) <= 4 * (r["k"] + 10) * U * e[0])
    assert r["status"] == 0 and e[-1] < 1e-10 <= e[-2]


def test_consistency_and_orthonormality(chirp_run):
    """Bookkeeping err_j equals the directly computed ||s - Q Q^H s||^2 and
    the IMGS basis is orthonormal to 1e-13 (Sec. 6.1.2)."""
    S, r = chirp_run
    Q = r["Q"]
    P = S - (S @ Q.conj().T) @ Q
    direct = np.sum(np.abs(P) ** 2, axis=1)
    assert np.max(np.abs(direct - r["final_err"])) < 1e-14
    G = Q.conj() @ Q.T
    assert np.linalg.norm(G - np.eye(r["k"]), 2) < 1e-13
    np.testing.assert_allclose(r["C"], Q.conj() @ S.T, atol=1e-14)
    assert set(r["passes"][1:]) <= {1, 2, 3}


def test_pod_bounds(chirp_run):
    """Thm. 3.2 and Thm. 4.1 / Cor. 4.3: the POD (SVD) error is a lower bound
    in both norms, and the max-norm error is at most the 2-norm error."""
    S, r = chirp_run
    k = r["k"]
    sv = np.linalg.svd(S.T, compute_uv=False)
    Q = r["Q"]
    E = (S - (S @ Q.conj().T) @ Q).T
    fro2 = np.sum(np.abs(E) ** 2)
    two = np.linalg.norm(E, 2)
    assert fro2 >= np.sum(sv[k:] ** 2) * (1 - 1e-9) - 1e-26
    assert two >= sv[k] * (1 - 1e-9)
    assert np.max(r["final_err"]) <= two ** 2 * (1 + 1e-9) + 1e-26
    assert np.isclose(np.max(np.delete(r["final_err"], r["pivots"])), r["err_curve"][-1], rtol=1e-12)


def test_forced_replay_of_own_pivots(orc):
    S = synth.chirps(64, 90, seed=1)
    a = orc.rb_greedy(S, 1e-10, 90)
    b = orc.rb_greedy(S, 1e-10, 90, forced=a["pivots"])
    assert list(b["pivots"]) == list(a["pivots"])
    np.testing.assert_array_equal(b["err_curve"], a["err_curve"])
    np.testing.assert_array_equal(b["own_argmax"][:a["k"]], a["pivots"])
    np.testing.assert_array_equal(b["forced_err"][:a["k"]], b["own_max"][:a["k"]])


def test_project_matches_library_matmul(orc):
    rng = np.random.default_rng(0)
    Q = rng.standard_normal((5, 33)) + 1j * rng.standard_normal((5, 33))
    X = rng.standard_normal((17, 33)) + 1j * rng.standard_normal((17, 33))
    np.testing.assert_allclose(orc.project(Q, X), Q.conj() @ X.T, atol=1e-13)


def test_split_definition(orc):
    S = synth.chirps(64, 10, seed=4) * 3.7
    hi, lo = orc.split(S)
    np.testing.assert_array_equal(hi, S.astype(np.complex64))
    rem = S - hi.astype(np.complex128)
    np.testing.assert_array_equal(lo, rem.astype(np.complex64))
    assert np.max(np.abs(S - hi - lo.astype(np.complex128)) / np.abs(S)) <= 2.0 ** -47


def test_openmp_build_gives_identical_results(orc):
    """The -fopenmp build of the oracle (column loops over all host cores)
    returns bit-identical results: each column is still summed sequentially."""
    from paper_1805_06124_gb300 import synth
    S = synth.chirps(256, 700, seed=8)
    a = orc.rb_greedy(S, 1e-10, 200)
    try:
        b = orc.rb_greedy(S, 1e-10, 200, omp=True)
    except Exception as e:  # no OpenMP runtime on this host
        pytest.skip(f"no -fopenmp build: {e}")
    assert a["k"] == b["k"]
    np.testing.assert_array_equal(a["pivots"], b["pivots"])
    np.testing.assert_array_equal(a["err_curve"], b["err_curve"])
    np.testing.assert_array_equal(a["Q"], b["Q"])
    np.testing.assert_array_equal(a["C"], b["C"])


@pytest.mark.parametrize("N,M", [(16384, 1024), (1024, 2048)])
def test_bookkeeping_noise_within_parity_margin(orc, N, M):
    """The noise model of the parity protocol: the oracle's final errors from
    the Eq. (Residual) bookkeeping (sequential FP64 norms and coefficients)
    deviate from the direct residual norms ||s_j - Q Q^H s_j||^2 (no
    cancellation: accurate to about 1e-20 here) by less than half of the
    margin delta(k, N) = 4 (k + sqrt(N)) u max||s||^2 that the GPU replays
    allow each side.  A bookkeeping mistake (a dropped term, a wrong index)
    would show here as a deviation of order the errors themselves."""
    import sys
    import os
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import parity
    S = synth.chirps(N, M, seed=2)
    r = orc.rb_greedy(S, 1e-10, 300)
    Q, k = r["Q"], r["k"]
    R = S - (Q.conj() @ S.T).T @ Q
    direct = np.sum(R.real ** 2 + R.imag ** 2, axis=1)
    dev = np.max(np.abs(r["final_err"] - direct))
    assert dev <= 0.5 * parity.delta(k, N, r["err_curve"][0]), (dev, parity.delta(k, N, r["err_curve"][0]))
    assert dev > 0.0  # rounding is there, so the check is not vacuous
