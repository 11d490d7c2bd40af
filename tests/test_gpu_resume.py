"""Resume of the greedy from a checkpoint and iterative enrichment (new
snapshots appended to S), against the uninterrupted GPU run and the FP64
oracle (needs a GB300)."""
import numpy as np
import pytest

from paper_1805_06124_gb300 import checkpoint, synth
import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1805_06124_gb300 import rb
    c = rb.RB(device=0, recompute_period=16)
    yield c
    c.close()


def npy(d):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in d.items()}


def test_resume_matches_uninterrupted(orc, ctx, tmp_path):
    """Stop at k0 = 16 (kmax), save, load, resume to tol: the same pivots and
    basis as one uninterrupted call (with the bookkeeping rebuilt at k0 = 16
    in both), and the oracle's replay protocol holds for the whole run."""
    S = synth.chirps(1024, 2048, seed=0)
    Sd = torch.from_numpy(S).cuda()
    full = npy(ctx.greedy(Sd, 1e-10, 300))
    part = ctx.greedy(Sd, 1e-10, 16)
    assert part["status"] == 1 and part["k"] == 16
    path = str(tmp_path / "ck.npz")
    checkpoint.save(path, part, 1e-10)
    ck = checkpoint.load(path)
    assert ck["k"] == 16 and ck["M"] == 2048
    res = npy(ctx.greedy_resume(Sd, 1e-10, 300, ck))
    assert res["status"] == 0 and res["k"] == full["k"]
    np.testing.assert_array_equal(res["pivots"], full["pivots"])
    scale = full["err_curve"][0]
    assert np.max(np.abs(res["err_curve"] - full["err_curve"])) <= 1e-14 * scale
    assert np.max(np.abs(res["Q"] - full["Q"])) <= 1e-13
    assert np.max(np.abs(res["C"] - full["C"])) <= 1e-13
    rep = parity.replay_and_check(orc, S, res, 1e-10, 300)
    parity.compare(res, rep, S)


def test_enrichment_with_new_snapshots(orc, ctx):
    """Basis of 2048 chirps (seed 0), then 1024 new chirps (seed 5) appended:
    the resumed run projects the new columns, keeps the old basis, and every
    snapshot ends below tol; the new pivots satisfy the replay protocol."""
    S1 = synth.chirps(1024, 2048, seed=0)
    S2 = synth.chirps(1024, 1024, seed=5)
    g1 = ctx.greedy(torch.from_numpy(S1).cuda(), 1e-10, 300)
    k0 = g1["k"]
    S = np.concatenate([S1, S2])
    res = npy(ctx.greedy_resume(torch.from_numpy(S).cuda(), 1e-10, 400, g1, Mc=2048))
    assert res["status"] == 0 and res["k"] >= k0
    np.testing.assert_array_equal(res["pivots"][:k0], g1["pivots"].cpu().numpy())
    Q = res["Q"]
    assert np.linalg.norm(Q.conj() @ Q.T - np.eye(res["k"]), 2) < 1e-13
    # the projected coefficients of the new snapshots
    Cn = S2.conj() @ Q[:k0].T                         # (1024, k0): conj(s) . q = conj(q^H s)
    assert np.max(np.abs(res["C"][:k0, 2048:] - Cn.conj().T)) < 1e-12
    direct = np.sum(np.abs(S - (S @ Q.conj().T) @ Q) ** 2, axis=1)
    assert np.all(direct < 1e-10 + 1e-12)
    assert np.max(np.abs(direct - res["final_err"])) < 1e-12
    rep = orc.rb_greedy(S, 1e-10, 400, forced=res["pivots"])
    margin_scale = rep["err_curve"][0]
    for l in range(k0, res["k"]):
        emax = rep["own_max"][l]
        margin = max(1e-12 * emax, parity.delta(l, 1024, margin_scale))
        assert emax - rep["forced_err"][l] <= margin, l
        if emax - rep["second_max"][l] > margin:
            assert rep["own_argmax"][l] == res["pivots"][l], l


def test_resume_edge_cases(ctx):
    from paper_1805_06124_gb300 import rb
    S = synth.chirps(256, 512, seed=3)
    Sd = torch.from_numpy(S).cuda()
    g = ctx.greedy(Sd, 1e-8, 200)
    # a finished run resumed with the same tol stops at once
    r = ctx.greedy_resume(Sd, 1e-8, 200, g)
    assert r["status"] == 0 and r["k"] == g["k"]
    np.testing.assert_array_equal(r["pivots"].cpu().numpy(), g["pivots"].cpu().numpy())
    # k0 = kmax: nothing to add
    part = ctx.greedy(Sd, 1e-8, 5)
    r = ctx.greedy_resume(Sd, 1e-8, 5, part)
    assert r["status"] == 1 and r["k"] == 5
    # an empty checkpoint is a plain run
    empty = dict(Q=np.zeros((0, 256), np.complex128), pivots=np.zeros(0, np.int64),
                 C=np.zeros((0, 512), np.complex128), err_curve=np.zeros(0), rdiag=np.zeros(0))
    r = ctx.greedy_resume(Sd, 1e-8, 200, empty)
    np.testing.assert_array_equal(r["pivots"].cpu().numpy(), g["pivots"].cpu().numpy())
    # repeated pivots are rejected, and the context stays usable
    bad = dict(part)
    bad["pivots"] = part["pivots"].clone()
    bad["pivots"][1] = bad["pivots"][0]
    with pytest.raises(rb.RBError) as ei:
        ctx.greedy_resume(Sd, 1e-8, 200, bad)
    assert ei.value.status == rb.EINVAL
    r = ctx.greedy_resume(Sd, 1e-8, 200, part)
    assert r["status"] == 0 and r["k"] == g["k"]
