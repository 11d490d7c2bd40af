"""The column-sharded greedy's CUDA engine (rb_shard_*, rb.Shard) on one GPU.

Several shards of one snapshot matrix live in one process and exchange through
sharded.LocalComm (the broadcast buffer is shared): the arithmetic of every
column is the in-core sweep's and the pivot column and its norm are the
owner's bytes, so the sharded run must equal rb_greedy bit for bit -- pivots,
error curve, basis, R diagonal, and each shard's coefficients and final
errors.  The pivots are also replayed through the oracle (Alg. 3).
"""
import numpy as np
import pytest

import parity
from paper_1805_06124_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bits_equal(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return a.shape == b.shape and np.array_equal(a.view(np.uint8), b.view(np.uint8))


@pytest.mark.parametrize("bounds,period", [((0, 700, 701, 2048), 16), ((0, 1024, 2048), 3)])
def test_shards_on_one_gpu_equal_rb_greedy(orc, bounds, period):
    from paper_1805_06124_gb300 import rb, sharded
    S_h = synth.chirps(1024, 2048, seed=0)
    S = torch.from_numpy(S_h).cuda()
    tol, kmax = 1e-10, 300
    ctx = rb.RB(device=0, recompute_period=period)
    ref = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in ctx.greedy(S, tol, kmax).items()}
    shards = [rb.Shard(ctx, S[a:b], a, kmax) for a, b in zip(bounds[:-1], bounds[1:])]
    r = sharded.greedy_sharded(shards, sharded.LocalComm(), tol, kmax)
    assert r["status"] == ref["status"] and r["k"] == ref["k"]
    assert list(r["pivots"]) == list(ref["pivots"])
    assert _bits_equal(np.array(r["err_curve"]), ref["err_curve"])
    for sh, out, (a, b) in zip(shards, r["shards"], zip(bounds[:-1], bounds[1:])):
        assert out["k"] == ref["k"]
        assert _bits_equal(out["Q"].cpu().numpy(), ref["Q"])
        assert _bits_equal(out["rdiag"].cpu().numpy(), ref["rdiag"])
        assert _bits_equal(out["C"].cpu().numpy(), ref["C"][:, a:b])
        assert _bits_equal(out["final_err"].cpu().numpy(), ref["final_err"][a:b])
    g = dict(pivots=np.array(r["pivots"]), err_curve=np.array(r["err_curve"]), Q=r["shards"][0]["Q"].cpu().numpy())
    rep = parity.replay_and_check(orc, S_h, g, tol, kmax)
    parity.compare(g, rep, S_h)
    for sh in shards:
        sh.close()
    ctx.close()


def test_shard_stopping_rules_and_errors():
    from paper_1805_06124_gb300 import rb, sharded
    ctx = rb.RB(device=0)
    S = torch.from_numpy(synth.chirps(64, 90, seed=4)).cuda()
    shards = [rb.Shard(ctx, S[0:40], 0, 5), rb.Shard(ctx, S[40:90], 40, 5)]
    r = sharded.greedy_sharded(shards, sharded.LocalComm(), 0.0, 5)
    assert r["status"] == sharded.KMAX_REACHED and r["k"] == 5 and len(r["err_curve"]) == 6
    # a NaN in one shard fails the whole run
    S2 = S.clone()
    S2[50, 3] = float("nan")
    shards2 = [rb.Shard(ctx, S2[0:40], 0, 5), rb.Shard(ctx, S2[40:90], 40, 5)]
    r2 = sharded.greedy_sharded(shards2, sharded.LocalComm(), 1e-10, 5)
    assert r2["status"] == rb.ENONFINITE and r2["k"] == 0
    # kmax vectors already built: a further append is refused
    with pytest.raises(rb.RBError):
        shards[0].append(shards[0].new_buffer(), 0)
    for sh in shards + shards2:
        sh.close()
    ctx.close()
