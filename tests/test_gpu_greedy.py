"""Parity of the CUDA path against the FP64 oracle (needs a GB300).

All calls go through the C ABI (``paper_1805_06124_gb300.rb``).  The oracle
and the CUDA path get the identical bytes of S (generated on the host by
``synth`` and uploaded), except in the generator test itself.
"""
import math

import numpy as np
import pytest

from paper_1805_06124_gb300 import synth
import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def rbm():
    from paper_1805_06124_gb300 import rb
    return rb


@pytest.fixture(scope="module", params=["df32", "fp64"])
def ctx(request, rbm):
    c = rbm.RB(device=0, sweep=request.param)
    yield c
    c.close()


def npy(d):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in d.items()}


def upload(S, ld=None):
    M, N = S.shape
    if ld is None or ld == N:
        return torch.from_numpy(S).cuda()
    buf = torch.zeros((M, ld), dtype=torch.complex128, device="cuda")
    buf[:, :N] = torch.from_numpy(S).cuda()
    return buf[:, :N]


# ------------------------------------------------------------ greedy parity

def test_config1_parity(orc, ctx):
    """1024 x 2048 chirps, seed 0, tol 1e-10, kmax 300 (the small config)."""
    S = synth.chirps(1024, 2048, seed=0)
    g = npy(ctx.greedy(upload(S), 1e-10, 300))
    assert g["status"] == 0 and 40 <= g["k"] <= 70
    rep = parity.replay_and_check(orc, S, g, 1e-10, 300)
    info = parity.compare(g, rep, S)
    print("config1", ctx.stream, g["k"], info, "passes", g["imgs_passes"])
    G = g["Q"].conj() @ g["Q"].T
    assert np.linalg.norm(G - np.eye(g["k"]), 2) < 1e-13
    # unforced oracle: identical pivots up to the first step whose gap is not clear
    own = orc.rb_greedy(S, 1e-10, 300)
    d = parity.first_divergence(list(own["pivots"]), list(g["pivots"]))
    if d < min(own["k"], g["k"]):
        e = rep["own_max"][d]
        assert e - rep["second_max"][d] <= max(1e-12 * e, parity.delta(d, S.shape[1], rep["err_curve"][0]))


@pytest.mark.parametrize("period", [0, 3])
def test_recompute_period_parity(orc, rbm, period):
    """The periodic exact recompute of acc_j (every `period` iterations; 0 =
    off) keeps the replay protocol and the tolerances; C is not requested, so
    the recompute reads the workspace copy of the coefficients."""
    S = synth.chirps(1024, 2048, seed=0)
    c = rbm.RB(device=0, recompute_period=period)
    g = npy(c.greedy(upload(S), 1e-10, 300, want_C=(period == 0)))
    rep = parity.replay_and_check(orc, S, g, 1e-10, 300)
    parity.compare(g, rep, S)
    c.close()


@pytest.mark.parametrize("shape", [(777, 1031, 800), (33, 65, 33), (1, 7, 1), (64, 1, 64), (257, 300, 263)])
def test_ragged_shapes_parity(orc, ctx, shape):
    """Odd N (ragged 128-bit tail), padded leading dimension, M not a
    multiple of the CTA width, single-row and single-column problems."""
    N, M, ld = shape
    S = synth.chirps(N, M, seed=5) * np.linspace(1.0, 1.2, M)[:, None]
    kmax = min(N, M)
    g = npy(ctx.greedy(upload(S, ld), 1e-10, kmax))
    rep = parity.replay_and_check(orc, S, g, 1e-10, kmax)
    parity.compare(g, rep, S)


def test_random_complex_parity(orc, ctx):
    S = synth.random_complex(300, 200, seed=8, scales=np.linspace(0.5, 2.0, 300))
    g = npy(ctx.greedy(upload(S), 1e-6, 200))
    rep = parity.replay_and_check(orc, S, g, 1e-6, 200)
    parity.compare(g, rep, S, err_atol=1e-12 * rep["err_curve"][0])


def test_edge_cases(orc, ctx, rbm):
    S = synth.random_complex(6, 5, seed=1)
    g = npy(ctx.greedy(upload(S), 1e9, 5))                 # tol above every norm
    assert g["k"] == 0 and g["status"] == 0
    np.testing.assert_allclose(g["err_curve"], [np.max(np.sum(np.abs(S) ** 2, 1))], rtol=1e-14)
    g = npy(ctx.greedy(upload(S), 0.0, 2))                 # kmax reached
    assert g["k"] == 2 and g["status"] == rbm.KMAX_REACHED
    g = npy(ctx.greedy(upload(S), 0.0, 0))                 # kmax = 0
    assert g["k"] == 0 and g["status"] == rbm.KMAX_REACHED
    Z = np.zeros((4, 9), np.complex128)                    # all-zero matrix
    g = npy(ctx.greedy(upload(Z), 0.0, 4))
    assert g["k"] == 0 and g["status"] == 0
    S2 = S.copy()
    S2[2] = 0                                              # a zero column is never picked
    g = npy(ctx.greedy(upload(S2), 1e-20, 5))
    assert 2 not in list(g["pivots"])
    S3 = S.copy()
    S3[4, 1] = np.nan
    with pytest.raises(rbm.RBError) as e:
        ctx.greedy(upload(S3), 1e-10, 5)
    assert e.value.status == rbm.ENONFINITE
    I = np.eye(6, dtype=np.complex128)                     # exact ties -> lowest index
    g = npy(ctx.greedy(upload(I), 0.5, 6))
    assert list(g["pivots"]) == [0, 1, 2, 3, 4, 5]


def test_bad_arguments(ctx, rbm):
    S = upload(synth.random_complex(6, 5, seed=1))
    with pytest.raises(rbm.RBError) as e:
        ctx.greedy(S, -1.0, 3)
    assert e.value.status == rbm.EINVAL
    with pytest.raises(rbm.RBError) as e:
        ctx.greedy(S, float("nan"), 3)
    assert e.value.status == rbm.EINVAL


def test_host_entry_point_matches_device(ctx):
    S = synth.chirps(300, 500, seed=3)
    d = npy(ctx.greedy(upload(S), 1e-10, 100))
    h = npy(ctx.greedy_host(torch.from_numpy(S).pin_memory(), 1e-10, 100))
    assert d["k"] == h["k"]
    for key in ("pivots", "err_curve", "Q", "C", "final_err", "rdiag"):
        np.testing.assert_array_equal(d[key], h[key])
    # padded host rows (ld > N) take the strided copy; pageable memory works too
    P = torch.zeros((500, 307), dtype=torch.complex128)
    P[:, :300] = torch.from_numpy(S)
    h2 = npy(ctx.greedy_host(P[:, :300], 1e-10, 100))
    for key in ("pivots", "err_curve", "Q", "C", "final_err", "rdiag"):
        np.testing.assert_array_equal(d[key], h2[key])
    # caller-owned output buffers, reused by two calls in a row
    out = ctx.host_outputs(300, 500, 100)
    Sp = torch.from_numpy(S).pin_memory()
    for _ in range(2):
        h3 = npy(ctx.greedy_host(Sp, 1e-10, 100, out=out))
        for key in ("pivots", "err_curve", "Q", "C", "final_err", "rdiag"):
            np.testing.assert_array_equal(d[key], h3[key])


# ------------------------------------------------------- generator / split

def test_generator_matches_host(rbm):
    c = rbm.RB(device=0)
    q, m = synth.chirp_params(257, seed=0)
    Sg = c.generate(q, m, 1000).cpu().numpy()
    Sh = synth.chirp_matrix(1000, q, m)
    rel = np.max(np.abs(Sg - Sh)) / np.max(np.abs(Sh))
    assert rel < 1e-12, rel
    c.close()


def test_split_bit_exact(orc, rbm):
    c = rbm.RB(device=0)
    S = synth.chirps(333, 77, seed=2) * 3.3
    hi, lo = c.split(upload(S), ldh=340)
    h0, l0 = orc.split(S)
    np.testing.assert_array_equal(hi.cpu().numpy(), h0)
    np.testing.assert_array_equal(lo.cpu().numpy(), l0)
    c.close()


def _tc_bound(Q, X):
    """Stated accuracy of the tensor-core projection: a few 2^-48 of
    max|q_l| max|x_j| (2N) per coefficient (16 taken here)."""
    return 16 * 2.0 ** -48 * np.max(np.abs(Q)) * np.max(np.abs(X)) * 2 * Q.shape[1]


@pytest.mark.parametrize("path", ["tensor_cores", "fp64"])
def test_project_parity(orc, rbm, path):
    """37 x 517 basis onto 333 columns: on the tensor cores 6 tiles of 3
    exact chunks, one chunk per block, so every tile is the sum of three
    blocks' parts (the stream-K fix-up)."""
    c = rbm.RB(device=0, project_fp64=(path == "fp64"))
    rng = np.random.default_rng(0)
    Q = rng.standard_normal((37, 517)) + 1j * rng.standard_normal((37, 517))
    X = rng.standard_normal((333, 517)) + 1j * rng.standard_normal((333, 517))
    Cg = c.project(upload(Q), upload(X)).cpu().numpy()
    Cr = orc.project(Q, X)
    tol = _tc_bound(Q, X) if path == "tensor_cores" else 1e-12
    assert np.max(np.abs(Cg - Cr)) < tol, (np.max(np.abs(Cg - Cr)), tol)
    c.close()


def test_trace_per_iteration(orc, rbm):
    """rb_trace: one entry per vector built; the pass counts add up to the
    call's total and stay below the cap (the paper reports fewer than three
    passes, Sec. 6.1.2); with timing, the sweep times add up to ms_sweep."""
    c = rbm.RB(device=0, timing=True)
    S = synth.chirps(1024, 2048, seed=0)
    g = c.greedy(upload(S), 1e-10, 300)
    t = c.trace()
    k = g["k"]
    assert len(t["imgs_passes"]) == k
    assert sum(t["imgs_passes"]) == g["imgs_passes"]
    # the first vector has no basis to be orthogonalised against
    ps = t["imgs_passes"]
    assert ps[0] in (0, 1) and all(1 <= p_ <= 4 for p_ in ps[1:]) and np.mean(ps[1:]) < 3, ps
    assert all(x > 0 for x in t["sweep_ms"]) and all(x > 0 for x in t["imgs_ms"])
    assert abs(sum(t["sweep_ms"]) - g["ms_sweep"]) < 1e-3 * max(g["ms_sweep"], 1.0)
    # a resumed call traces only the vectors it built
    part = c.greedy(upload(S), 1e-10, 10)
    r = c.greedy_resume(upload(S), 1e-10, 300, part)
    assert len(c.trace()["imgs_passes"]) == r["k"] - 10
    c.close()


@pytest.mark.parametrize("k", [64, 65, 130])
def test_project_tc_row_tiles(orc, rbm, k):
    """k = 64, 65, 130: one, two (the second almost empty) and three 128-row
    tiles of the tensor-core projection; odd N (K padding to whole chunks),
    ragged columns; every tile shared by four blocks."""
    c = rbm.RB(device=0)
    rng = np.random.default_rng(k)
    Q = rng.standard_normal((k, 777)) + 1j * rng.standard_normal((k, 777))
    X = rng.standard_normal((301, 777)) + 1j * rng.standard_normal((301, 777))
    Cg = c.project(upload(Q), upload(X)).cpu().numpy()
    Cr = orc.project(Q, X)
    assert np.max(np.abs(Cg - Cr)) < _tc_bound(Q, X), (np.max(np.abs(Cg - Cr)), _tc_bound(Q, X))
    c.close()


@pytest.mark.parametrize("k,N,M", [(1, 1, 1), (2, 3, 5), (1, 700, 1), (64, 2000, 64), (5, 4096, 130)])
def test_project_tc_small_shapes(orc, rbm, k, N, M):
    """Edge shapes of the stream-K projection: one sample (K padded to one
    exact chunk), one column, k = 1 (two rows), one tile of several chunks
    shared by as many blocks, a tile count equal to the chunk count."""
    c = rbm.RB(device=0)
    rng = np.random.default_rng(k * 1000 + N + M)
    Q = rng.standard_normal((k, N)) + 1j * rng.standard_normal((k, N))
    X = rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))
    Cg = c.project(upload(Q), upload(X)).cpu().numpy()
    Cr = orc.project(Q, X)
    assert np.max(np.abs(Cg - Cr)) < _tc_bound(Q, X), (np.max(np.abs(Cg - Cr)), _tc_bound(Q, X))
    c.close()


def test_project_tc_column_batches(orc, rbm):
    """N = 8192 and 20,000 columns: 313 column tiles of 32 chunks over the
    persistent blocks (about 66 chunks each, so most blocks start or end
    inside a tile and the fix-up adds the parts), each slicing its columns
    inside the GEMM; checked against the oracle on columns at both ends, in
    the middle and near the end."""
    c = rbm.RB(device=0)
    N, M = 8192, 20000
    rng = np.random.default_rng(11)
    Q = rng.standard_normal((53, N)) + 1j * rng.standard_normal((53, N))
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    X = c.generate(*synth.chirp_params(M, seed=12), N)
    Cg = c.project(upload(Q), X)
    cols = np.r_[0:40, 9900:10100, 18550:18650, M - 40:M]
    Xs = X[torch.from_numpy(cols).cuda()].cpu().numpy()
    Cr = orc.project(Q, Xs)
    Cs = Cg[:, torch.from_numpy(cols).cuda()].cpu().numpy()
    assert np.max(np.abs(Cs - Cr)) < _tc_bound(Q, Xs), np.max(np.abs(Cs - Cr))
    c.close()
    del X, Cg
    torch.cuda.empty_cache()


def test_project_tc_chirps_ragged(orc, rbm):
    """Basis of a chirp greedy projected onto held-out chirps: odd N, k not a
    multiple of the tile, Mx not a multiple of 64; within 1e-12 of the oracle."""
    c = rbm.RB(device=0)
    S = synth.chirps(1999, 700, seed=3)
    g = c.greedy(upload(S), 1e-10, 300)
    Q = g["Q"].cpu().numpy()
    X = synth.chirps(1999, 1111, seed=9)
    Cg = c.project(g["Q"], upload(X)).cpu().numpy()
    Cr = orc.project(Q, X)
    assert np.max(np.abs(Cg - Cr)) < 1e-12, np.max(np.abs(Cg - Cr))
    c.close()


# ------------------------------------------------- full size, sampled checks

@pytest.mark.parametrize("sweep", ["df32"])
def test_config2_full_size_sampled(orc, rbm, sweep):
    """8192 x 262,144 chirps (seed 1), tol 1e-12, kmax 800 -- the benchmark's
    launch configuration -- checked on 48 sampled columns against the
    oracle's projection, plus the identities of Cor. 5.4 on all pivots."""
    N, M, tol, kmax = 8192, 262144, 1e-12, 800
    c = rbm.RB(device=0, sweep=sweep)
    q, m = synth.chirp_params(M, seed=1)
    S = c.generate(q, m, N)
    g = c.greedy(S, tol, kmax)
    k = g["k"]
    assert g["status"] == 0 and 40 <= k <= 90
    ec = g["err_curve"].cpu().numpy()
    assert ec[k] < tol <= ec[k - 1]
    assert np.all(np.diff(ec) <= parity.delta(k, N, ec[0]))
    rd = g["rdiag"].cpu().numpy()
    # R(l,l)^2 (a direct norm) equals the bookkeeping max error up to the
    # FP64 noise of Eq. (Residual) at N = 8192 (a few 1e-14 here)
    np.testing.assert_allclose(rd ** 2, ec[:k], rtol=1e-9, atol=1e-13)
    piv = g["pivots"].cpu().numpy()
    Q = g["Q"].cpu().numpy()
    Gm = orc.project(Q, Q)
    assert np.linalg.norm(Gm - np.eye(k), 2) < 1e-13
    T = g["C"][:, torch.from_numpy(piv).cuda()].cpu().numpy()
    assert np.max(np.abs(np.tril(T, -1))) < 1e-12
    np.testing.assert_allclose(np.diag(T).real, rd, rtol=1e-9, atol=1e-13)
    rng = np.random.default_rng(123)
    cols = np.unique(np.concatenate([rng.integers(0, M, 40), piv[:8]]))
    Ss = S[torch.from_numpy(cols).cuda()].cpu().numpy()
    Cs = g["C"][:, torch.from_numpy(cols).cuda()].cpu().numpy()
    fe = g["final_err"][torch.from_numpy(cols).cuda()].cpu().numpy()
    Cr = orc.project(Q, Ss)
    bt = parity.basis_tol(ec, k)
    assert np.all(np.max(np.abs(Cs - Cr), axis=1) <= bt + 1e-13)
    direct = np.sum(np.abs(Ss - Cr.T @ Q) ** 2, axis=1)
    assert np.max(np.abs(direct - fe)) < 1e-12
    c.close()
    del S, g
    torch.cuda.empty_cache()


# ------------------------------------------------------- failure detection

def test_allocation_failure_is_reported_and_recoverable(rbm, monkeypatch):
    c = rbm.RB(device=0)
    S = upload(synth.chirps(64, 80, seed=1))
    monkeypatch.setenv("RB_TEST_FAIL_ALLOC", "1")
    with pytest.raises(rbm.RBError) as e:
        c.greedy(S, 1e-10, 50)
    assert e.value.status == rbm.ENOMEM
    monkeypatch.delenv("RB_TEST_FAIL_ALLOC")
    g = c.greedy(S, 1e-10, 50)
    assert g["k"] > 5
    c.close()


def test_bounded_wait_times_out_and_context_survives(rbm):
    import ctypes
    c = rbm.RB(device=0)
    f = c.lib.rb_debug_wait_selftest
    f.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int]
    f.restype = ctypes.c_int
    assert f(c._h, 1000, 0) == rbm.ETIMEOUT       # nothing arrives: the wait runs out and returns
    assert f(c._h, 1000, 1) == rbm.OK             # positive control
    g = c.greedy(upload(synth.chirps(64, 80, seed=1)), 1e-10, 50)
    assert g["k"] > 5                             # the context is still usable
    c.close()
