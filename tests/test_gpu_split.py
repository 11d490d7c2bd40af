"""Split-precision form (complex64 hi + lo storage) against the FP64 oracle.

The oracle runs on the complex128 S; the CUDA path gets the oracle's own
hi/lo split of the same S.  hi + lo equals S to 2^-48 relative, so the
split form is held to the FP64 form's protocol and tolerances.
"""
import numpy as np
import pytest

import parity
from paper_1805_06124_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbm():
    from paper_1805_06124_gb300 import rb
    return rb


def npy(d):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in d.items()}


def c_rel(N):
    """The split form's stated C tolerance relative to ||s_j||: a quarter of
    the sweep bound eta = 2^-46 sqrt(N) (measured errors stay below 2^-42.4
    at N = 16384, i.e. about eta / 10), plus 2^-42 for the FP16 pieces of the
    projection onto lo (at most 2^-18.4 relative per product of |q| |lo|,
    |lo| <= 2^-24 |s|)."""
    return 2.0 ** -48 * np.sqrt(N) + 2.0 ** -42


def split_upload(orc, S, ld=None):
    hi, lo = orc.split(S)
    M, N = S.shape
    ld = ld or (N + (N & 1))
    H = torch.zeros((M, ld), dtype=torch.complex64, device="cuda")
    L = torch.zeros((M, ld), dtype=torch.complex64, device="cuda")
    H[:, :N] = torch.from_numpy(hi).cuda()
    L[:, :N] = torch.from_numpy(lo).cuda()
    return H[:, :N], L[:, :N]


def test_split_config1_parity(orc, rbm):
    S = synth.chirps(1024, 2048, seed=0)
    c = rbm.RB(device=0)
    H, L = split_upload(orc, S)
    g = npy(c.greedy_split(H, L, 1e-10, 300))
    assert g["status"] == 0
    rep = parity.replay_and_check(orc, S, g, 1e-10, 300)
    info = parity.compare(g, rep, S, c_rel=c_rel(S.shape[1]))
    print("split k", g["k"], "switch at", g["switch_iter"], info)
    # the candidates stay few: no switch, C is completed on lo once, when the loop ends
    assert g["switch_iter"] == -1
    assert np.max(g["final_err"]) < 1e-10 + 1e-12
    c.close()


def test_split_sweep_accuracy_n16384(orc, rbm):
    """At the bench's row count the hi-only sweep's rounding stays far inside
    the bound eta = 2^-46 sqrt(N) that the candidate test assumes: C (whose
    error is dominated by it) is compared with the oracle's replay."""
    N, M = 16384, 1536
    S = synth.chirps(N, M, seed=4)
    c = rbm.RB(device=0)
    H, L = split_upload(orc, S)
    g = npy(c.greedy_split(H, L, 1e-10, 200))
    rep = parity.replay_and_check(orc, S, g, 1e-10, 200)
    parity.compare(g, rep, S, c_rel=c_rel(S.shape[1]))
    k = rep["k"]
    nrm = np.linalg.norm(S, axis=1)
    rel = np.max(np.abs(g["C"][:k] - rep["C"]) / nrm[None, :])
    eta = 2.0 ** -46 * np.sqrt(N)
    print("k", k, "max |dC| / ||s||", rel, "eta", eta)
    assert rel < eta / 4
    c.close()


@pytest.mark.parametrize("shape", [(777, 1031, 778), (33, 65, 40), (2, 9, 2), (64, 1, 64)])
def test_split_ragged_parity(orc, rbm, shape):
    N, M, ld = shape
    S = synth.chirps(N, M, seed=5) * np.linspace(1.0, 1.2, M)[:, None]
    c = rbm.RB(device=0)
    H, L = split_upload(orc, S, ld)
    kmax = min(N, M)
    g = npy(c.greedy_split(H, L, 1e-10, kmax))
    rep = parity.replay_and_check(orc, S, g, 1e-10, kmax)
    parity.compare(g, rep, S, c_rel=c_rel(S.shape[1]))
    c.close()


def test_split_large_tol(orc, rbm):
    """A loose tol ends the loop on the certified bounds alone; the final
    projection onto lo still makes C and the errors exact."""
    S = synth.chirps(512, 700, seed=2)
    c = rbm.RB(device=0)
    H, L = split_upload(orc, S)
    g = npy(c.greedy_split(H, L, 1e-4, 700))
    rep = parity.replay_and_check(orc, S, g, 1e-4, 700)
    parity.compare(g, rep, S, c_rel=c_rel(S.shape[1]))
    c.close()


def test_split_exact_rank(orc, rbm):
    """Rank-7 input: the bounds certify the stop after exactly 7 vectors."""
    S = synth.low_rank(400, 300, 7, seed=6)
    scale = float(np.max(np.sum(np.abs(S) ** 2, axis=1)))
    c = rbm.RB(device=0)
    H, L = split_upload(orc, S)
    g = npy(c.greedy_split(H, L, 1e-11 * scale, 50))
    assert g["k"] == 7 and g["status"] == 0
    rep = parity.replay_and_check(orc, S, g, 1e-11 * scale, 50)
    parity.compare(g, rep, S, err_atol=1e-12 * scale, c_rel=c_rel(S.shape[1]))
    c.close()


def test_split_many_candidates(orc, rbm):
    """tol below the bound widths: in the last iterations every column is a
    candidate and the exact re-check alone decides the pivots."""
    S = synth.chirps(1024, 2048, seed=0)
    c = rbm.RB(device=0)
    H, L = split_upload(orc, S)
    g = npy(c.greedy_split(H, L, 1e-13, 300))
    assert g["status"] == 0
    rep = parity.replay_and_check(orc, S, g, 1e-13, 300)
    info = parity.compare(g, rep, S, c_rel=c_rel(S.shape[1]))
    print("k", g["k"], info)
    c.close()


def test_split_kmax_and_random(orc, rbm):
    S = synth.random_complex(300, 200, seed=8, scales=np.linspace(0.5, 2.0, 300))
    c = rbm.RB(device=0)
    H, L = split_upload(orc, S)
    g = npy(c.greedy_split(H, L, 0.0, 37))
    assert g["k"] == 37 and g["status"] == rbm.KMAX_REACHED
    rep = parity.replay_and_check(orc, S, g, 0.0, 37)
    parity.compare(g, rep, S, err_atol=1e-12 * rep["err_curve"][0], c_rel=c_rel(S.shape[1]))
    c.close()


def test_split_matches_fp64_form_on_gpu_split(orc, rbm):
    """rb_split on the GPU then rb_greedy_split equals rb_greedy (FP64 form)."""
    S = synth.chirps(1000, 1500, seed=7)
    c = rbm.RB(device=0)
    St = torch.from_numpy(S).cuda()
    hi, lo = c.split(St, ldh=1000)
    a = npy(c.greedy_split(hi, lo, 1e-10, 300))
    b = npy(c.greedy(St, 1e-10, 300))
    # the two forms take their norms with different double-float code, so the
    # first step's bitwise ties among unit columns may resolve differently;
    # the curves must agree and the replay protocol must hold for both
    assert abs(a["k"] - b["k"]) <= 2
    for g, cr in ((a, c_rel(S.shape[1])), (b, 0.0)):
        rep = parity.replay_and_check(orc, S, g, 1e-10, 300)
        parity.compare(g, rep, S, c_rel=cr)
    c.close()


@pytest.mark.parametrize("kmax", [64, 65, 130])
def test_split_several_row_tiles(orc, rbm, kmax):
    """Bases of 64, 65 and 130 vectors: the projection onto lo runs over one,
    two (the second holding two rows) and three 128-row tiles of the basis."""
    S = synth.random_complex(520, 333, seed=kmax, scales=np.exp(-np.linspace(0.0, 8.0, 520)))
    c = rbm.RB(device=0)
    H, L = split_upload(orc, S)
    g = npy(c.greedy_split(H, L, 0.0, kmax))
    assert g["k"] == kmax and g["status"] == rbm.KMAX_REACHED
    rep = parity.replay_and_check(orc, S, g, 0.0, kmax)
    parity.compare(g, rep, S, err_atol=1e-12 * rep["err_curve"][0], c_rel=c_rel(S.shape[1]))
    c.close()


def _rows_after_switch_fp64_tol(g, rep, ks):
    """Rows of C from the switch on come from the hi + lo (double-float)
    sweep: the FP64 form's C tolerance, without the split form's c_rel."""
    k = rep["k"]
    bt = parity.basis_tol(rep["err_curve"], k)
    dC = np.abs(np.asarray(g["C"])[ks:k] - rep["C"][ks:k])
    r = dC / (bt[ks:k, None] + 1e-13)
    assert np.all(r <= 1.0), np.max(r)
    return float(np.max(dC)) if k > ks else 0.0


def test_split_switch_on_error_threshold(orc, rbm):
    """opt.switch_err: once every error is certified below
    switch_err * max ||s_j||^2 the basis so far is projected onto lo and the
    later sweeps read hi + lo.  The pivots, curve, basis and errors meet the
    FP64 protocol; the rows of C before the switch the split form's C
    tolerance, the later rows the FP64 form's."""
    S = synth.chirps(1024, 2048, seed=0)
    tol, kmax = 1e-10, 300
    c = rbm.RB(device=0, switch_err=1e-6)
    H, L = split_upload(orc, S)
    g = npy(c.greedy_split(H, L, tol, kmax))
    assert g["status"] == 0
    ks = g["switch_iter"]
    assert 0 < ks < g["k"], (ks, g["k"])
    ec = np.asarray(g["err_curve"])
    assert ec[ks] < 1e-6 * ec[0]           # the rule that fired
    rep = parity.replay_and_check(orc, S, g, tol, kmax)
    info = parity.compare(g, rep, S, c_rel=c_rel(S.shape[1]))
    info["max_dC_after_switch"] = _rows_after_switch_fp64_tol(g, rep, ks)
    # the same pivots as the run without the switch
    c2 = rbm.RB(device=0)
    g2 = npy(c2.greedy_split(H, L, tol, kmax))
    assert list(g2["pivots"]) == list(g["pivots"]) and g2["switch_iter"] == -1
    print("switch at", ks, "of", g["k"], info)
    c.close()
    c2.close()


def test_split_switch_on_candidate_count_large_m(orc, rbm):
    """tol far below the hi-only bound widths on a large M: in the last
    iterations the bounds admit most columns as candidates, the count passes
    M/8 and the form switches to hi + lo sweeps.  The same run with the
    switch disabled (RB_FLAG_SPLIT_NO_SWITCH) re-checks every candidate.
    Both meet the protocol against the oracle."""
    N, M = 2048, 65536
    S = synth.chirps(N, M, seed=7)
    # below the bound widths (about 2 eta sum_l |c~_lj| ~ 3e-12 here), well above
    # the bookkeeping noise, so the stop is not a near-tie with tol
    tol, kmax = 3e-12, 400
    H, L = split_upload(orc, S)
    res = {}
    for sw in (True, False):
        c = rbm.RB(device=0, split_switch=sw)
        g = npy(c.greedy_split(H, L, tol, kmax))
        c.close()
        assert g["status"] == 0
        rep = parity.replay_and_check(orc, S, g, tol, kmax, omp=True)
        info = parity.compare(g, rep, S, c_rel=c_rel(N))
        if sw:
            assert 0 < g["switch_iter"] <= g["k"]
            info["max_dC_after_switch"] = _rows_after_switch_fp64_tol(g, rep, g["switch_iter"])
        else:
            assert g["switch_iter"] == -1
        info.update(switch_iter=int(g["switch_iter"]), ms=round(float(g["ms_total"]), 3))
        res[sw] = info
    print("switch", res[True], "no switch", res[False])


def test_split_switch_then_exact_rank_and_kmax(orc, rbm):
    """A switch at the first iterations (switch_err = 1: every error is below
    the largest norm), then the loop ends in the hi + lo phase: on exact rank
    (IMGS finds the pivot in the span) and on kmax."""
    S = synth.low_rank(400, 300, 7, seed=6)
    scale = float(np.max(np.sum(np.abs(S) ** 2, axis=1)))
    c = rbm.RB(device=0, switch_err=1.0)
    H, L = split_upload(orc, S)
    g = npy(c.greedy_split(H, L, 1e-11 * scale, 50))
    assert g["k"] == 7 and g["status"] == 0 and 0 < g["switch_iter"] <= 2, (g["k"], g["status"], g["switch_iter"])
    rep = parity.replay_and_check(orc, S, g, 1e-11 * scale, 50)
    parity.compare(g, rep, S, err_atol=1e-12 * scale, c_rel=c_rel(S.shape[1]))
    S2 = synth.chirps(512, 700, seed=2)
    H2, L2 = split_upload(orc, S2)
    g2 = npy(c.greedy_split(H2, L2, 1e-12, 10))
    assert g2["k"] == 10 and g2["status"] == rbm.KMAX_REACHED and 0 < g2["switch_iter"] < 10, g2["switch_iter"]
    rep2 = parity.replay_and_check(orc, S2, g2, 1e-12, 10)
    parity.compare(g2, rep2, S2, c_rel=c_rel(S2.shape[1]))
    c.close()
