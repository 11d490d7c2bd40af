"""Parity of the empirical-interpolation step and the out-of-sample
validation on the GPU against the FP64 oracle (needs a GB300).

Node parity follows the greedy's replay protocol: the oracle replays the
GPU's nodes, each must be a maximum of the oracle's residual up to rounding,
and must equal the oracle's own choice wherever the runner-up is clearly
smaller.  The basis comes from the GPU greedy; the oracle gets its bytes."""
import numpy as np
import pytest
import scipy.linalg

from paper_1805_06124_gb300 import synth

torch = pytest.importorskip("torch")
eim_o = pytest.importorskip("oracle.eim_oracle")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def ctx():
    from paper_1805_06124_gb300 import rb
    c = rb.RB(device=0)
    yield c
    c.close()


def greedy_basis(ctx, S, tol, kmax):
    g = ctx.greedy(torch.from_numpy(np.ascontiguousarray(S)).cuda(), tol, kmax)
    assert g["status"] in (0, 1)
    return g["Q"]


def check_eim(ctx, Q):
    out = ctx.eim(Q)
    Qh = Q.cpu().numpy()
    k, N = Qh.shape
    nodes = out["nodes"].cpu().numpy()
    rep = eim_o.eim(Qh, forced=nodes)
    assert len(set(nodes.tolist())) == k and nodes.min() >= 0 and nodes.max() < N
    scale = np.max(np.abs(Qh)) ** 2
    for i in range(k):
        # the GPU's node is a maximum of the oracle's residual up to rounding
        assert rep["r2_forced"][i] >= rep["r2_own"][i] * (1 - 1e-9) - 1e-24 * scale, i
        if rep["r2_own"][i] - rep["r2_second"][i] > 1e-8 * rep["r2_own"][i]:
            assert nodes[i] == rep["own"][i], i
    V = out["V"].cpu().numpy()
    np.testing.assert_array_equal(V, Qh[:, nodes].T)                 # a gather: bit-exact
    cond = np.linalg.cond(V)
    B = out["B"].cpu().numpy().T                                      # (N, k)
    tol = 64 * k * U * cond * max(1.0, np.max(np.abs(rep["B"])))
    assert np.max(np.abs(B - rep["B"])) <= tol, (np.max(np.abs(B - rep["B"])), tol)
    assert np.max(np.abs(B @ V - Qh.T)) <= tol
    Vi = out["Vinv"].cpu().numpy()
    assert np.max(np.abs(Vi @ V - np.eye(k))) <= 64 * k * U * cond + 1e-12
    return out


def test_chirp_basis(ctx):
    Q = greedy_basis(ctx, synth.chirps(1024, 2048, seed=0), 1e-10, 300)
    assert 40 <= Q.shape[0] <= 70
    check_eim(ctx, Q)


@pytest.mark.parametrize("k,N,seed", [(1, 50, 0), (7, 37, 1), (40, 40, 2), (60, 3000, 3)])
def test_real_basis_equals_lu_pivots(ctx, k, N, seed):
    """Real orthonormal bases: the nodes are LAPACK getrf's row pivots
    (k = 1, a ragged N, k = N, and many rows)."""
    rng = np.random.default_rng(seed)
    Qr = np.linalg.qr(rng.standard_normal((N, k)))[0].T
    out = check_eim(ctx, torch.from_numpy(np.ascontiguousarray(Qr, dtype=np.complex128)).cuda())
    _, piv = scipy.linalg.lu_factor(Qr.T)
    perm = np.arange(N)
    for i in range(k):
        perm[i], perm[piv[i]] = perm[piv[i]], perm[i]
    np.testing.assert_array_equal(out["nodes"].cpu().numpy(), perm[:k])


def test_empty_and_dependent(ctx):
    from paper_1805_06124_gb300 import rb
    out = ctx.eim(torch.zeros((0, 16), dtype=torch.complex128, device="cuda"))
    assert out["nodes"].numel() == 0
    Q = torch.zeros((2, 8), dtype=torch.complex128, device="cuda")
    Q[0, 3] = 1.0
    Q[1, 3] = 1.0                      # q_2 = q_1: the second residual vanishes
    with pytest.raises(rb.RBError) as ei:
        ctx.eim(Q)
    assert ei.value.status == rb.ESTATE
    with pytest.raises(rb.RBError):
        ctx.eim(torch.zeros((9, 8), dtype=torch.complex128, device="cuda"))   # k > N
    check_eim(ctx, greedy_basis(ctx, synth.chirps(128, 256, seed=9), 1e-8, 60))  # context still usable


def test_validation_out_of_sample(ctx):
    """Basis and interpolant from chirps of seed 0; errors on 3000 chirps of
    another seed against the oracle's direct definitions."""
    Q = greedy_basis(ctx, synth.chirps(1024, 2048, seed=0), 1e-10, 300)
    e = ctx.eim(Q)
    T = synth.chirps(1024, 3000, seed=11)
    v = ctx.validate(Q, torch.from_numpy(T).cuda(), e["nodes"], e["Vinv"])
    ref = eim_o.validate(Q.cpu().numpy(), e["B"].cpu().numpy().T, e["nodes"].cpu().numpy(), T)
    tnorm = np.sum(np.abs(T) ** 2, axis=1)
    ep, ee = v["err_proj"].cpu().numpy(), v["err_eim"].cpu().numpy()
    assert np.max(np.abs(ep - ref["err_proj"]) / tnorm) < 1e-12
    assert np.max(np.abs(ee - ref["err_eim"]) / tnorm) < 1e-11
    assert np.all(ee >= ep * (1 - 1e-9) - 1e-14)
    # projection errors only, and the empty basis
    v2 = ctx.validate(Q, torch.from_numpy(T).cuda())
    assert "err_eim" not in v2 and torch.equal(v2["err_proj"], v["err_proj"])
    v0 = ctx.validate(None, torch.from_numpy(T[:5]).cuda(), torch.zeros(0, dtype=torch.int64, device="cuda"))
    np.testing.assert_allclose(v0["err_proj"].cpu().numpy(), tnorm[:5], rtol=1e-14)
    np.testing.assert_allclose(v0["err_eim"].cpu().numpy(), tnorm[:5], rtol=1e-14)


def test_full_size_sampled(ctx):
    """The 8192 x 262,144 greedy basis (seed 1, tol 1e-12): nodes by replay,
    and validation on 16,384 chirps of seed 7 checked on 64 sampled ones."""
    from paper_1805_06124_gb300 import rb
    c = rb.RB(device=0)
    N, M = 8192, 262144
    S = c.generate(*synth.chirp_params(M, seed=1), N)
    Q = c.greedy(S, 1e-12, 800)["Q"]
    del S
    torch.cuda.empty_cache()
    e = check_eim(c, Q)
    q7, m7 = synth.chirp_params(16384, seed=7)
    T = c.generate(q7, m7, N)
    v = c.validate(Q, T, e["nodes"], e["Vinv"])
    cols = np.random.default_rng(3).choice(16384, 64, replace=False)
    Th = T[torch.from_numpy(cols).cuda()].cpu().numpy()
    ref = eim_o.validate(Q.cpu().numpy(), e["B"].cpu().numpy().T, e["nodes"].cpu().numpy(), Th)
    tnorm = np.sum(np.abs(Th) ** 2, axis=1)
    assert np.max(np.abs(v["err_proj"].cpu().numpy()[cols] - ref["err_proj"]) / tnorm) < 1e-12
    assert np.max(np.abs(v["err_eim"].cpu().numpy()[cols] - ref["err_eim"]) / tnorm) < 1e-11
    c.close()
