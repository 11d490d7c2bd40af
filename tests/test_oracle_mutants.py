"""The oracle's pins must catch plausible mistakes.

Each planted variant of ``oracle/rb_oracle.c`` (compiled with -DORC_PLANT=n,
CPU only) carries one mistake: a missing conjugate in c = q^H s, a dropped
imaginary term in |c|^2, ties going to the highest index, no
re-orthogonalisation, and an off-by-one in the stopping test.  For every
variant at least one of the independent pins below must fail.
"""
import numpy as np
import pytest

from paper_1805_06124_gb300 import synth


def _bruteforce(S, kmax):
    M = S.shape[0]
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
        curve.append(bval)
        if len(picked) == kmax:
            break
        picked.append(best)
    return picked, np.array(curve)


def _pins_pass(orc, plant):
    """True when every pin passes for the given build."""
    # hand-worked 2x2 with the stopping rule
    S = np.array([[1, 0], [1, 1]], np.complex128)
    r = orc.rb_greedy(S, 1.0, 2, plant=plant)
    if r["k"] != 1 or list(r["pivots"]) != [1]:
        return False
    # ties go to the lowest index
    r = orc.rb_greedy(np.eye(4, dtype=np.complex128), 1e-30, 4, plant=plant)
    if list(r["pivots"]) != [0, 1, 2, 3]:
        return False
    # brute-force least squares on complex data
    S = synth.random_complex(8, 10, seed=7, scales=np.linspace(1.0, 1.5, 8))
    r = orc.rb_greedy(S, 0.0, 6, plant=plant)
    piv, curve = _bruteforce(S, 6)
    if list(r["pivots"]) != piv or not np.allclose(r["err_curve"], curve[:7], rtol=0, atol=1e-12 * curve[0]):
        return False
    # orthonormality of the basis on a hard chirp case (tail far below 1e-10)
    S = synth.chirps(128, 160, seed=0)
    r = orc.rb_greedy(S, 1e-26, 160, plant=plant)
    G = r["Q"].conj() @ r["Q"].T
    if np.linalg.norm(G - np.eye(r["k"]), 2) > 1e-13:
        return False
    return True


def test_unplanted_oracle_passes(orc):
    assert _pins_pass(orc, 0)


@pytest.mark.parametrize("plant", [1, 2, 3, 4, 5])
def test_planted_mistake_is_caught(orc, plant):
    orc.build(plant)
    assert not _pins_pass(orc, plant)
