"""Batched greedy (one persistent sweep launch over uneven problems) against
the FP64 oracle, problem by problem, with the single-problem parity protocol."""
import numpy as np
import pytest

import parity
from paper_1805_06124_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def npy(d):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in d.items()}


def test_batched_parity_uneven(orc):
    from paper_1805_06124_gb300 import rb
    c = rb.RB(device=0)
    shapes = [(700, 1500, 5), (1024, 333, 6), (65, 900, 7), (3, 10, 8), (512, 2047, 9), (2000, 64, 10)]
    Ss, hosts = [], []
    for N, M, seed in shapes:
        q, m = synth.chirp_params(M, seed, q_range=(1.0 + seed / 10, 9.0), m_range=(0.85, 1.15))
        S = synth.chirp_matrix(N, q, m)
        hosts.append(S)
        Ss.append(torch.from_numpy(S).cuda())
    outs = c.greedy_batched(Ss, 1e-10, 300)
    for S, o in zip(hosts, outs):
        g = npy(o)
        kmax = 300
        rep = parity.replay_and_check(orc, S, g, 1e-10, kmax)
        parity.compare(g, rep, S)
    # a second call reuses the cached autotune choice and must give the same results
    outs2 = c.greedy_batched(Ss, 1e-10, 300)
    for a, b in zip(outs, outs2):
        np.testing.assert_array_equal(a["pivots"].cpu().numpy(), b["pivots"].cpu().numpy())
        np.testing.assert_array_equal(a["err_curve"].cpu().numpy(), b["err_curve"].cpu().numpy())
    c.close()


def test_batched_statuses_and_kmax(orc):
    from paper_1805_06124_gb300 import rb
    c = rb.RB(device=0)
    S1 = torch.from_numpy(synth.random_complex(40, 30, seed=1)).cuda()
    S2 = torch.from_numpy(synth.chirps(128, 200, seed=2)).cuda()
    outs = c.greedy_batched([S1, S2], 0.0, 12)
    assert [o["k"] for o in outs] == [12, 12]
    assert all(o["status"] == rb.KMAX_REACHED for o in outs)
    for S, o in ((S1, outs[0]), (S2, outs[1])):
        g = npy(o)
        rep = parity.replay_and_check(orc, S.cpu().numpy(), g, 0.0, 12)
        parity.compare(g, rep, S.cpu().numpy(), err_atol=1e-12 * max(1.0, rep["err_curve"][0]))
    c.close()


def _uneven_batch():
    shapes = [(700, 1500, 5), (1024, 333, 6), (65, 900, 7), (3, 10, 8), (512, 2047, 9), (2000, 64, 10)]
    hosts = []
    for N, M, seed in shapes:
        q, m = synth.chirp_params(M, seed, q_range=(1.0 + seed / 10, 9.0), m_range=(0.85, 1.15))
        hosts.append(synth.chirp_matrix(N, q, m))
    return hosts


@pytest.fixture(scope="module")
def uneven_batch():
    return _uneven_batch()


@pytest.mark.parametrize("variant", list(range(24)))
def test_batched_every_sweep_variant(orc, uneven_batch, variant):
    """Every sweep variant the autotuner can pick (rb_options.batched_variant =
    2 v + c: v = 0..5 read complex128 and split in registers, v = 6..11 read
    the pre-split copy; c = 32 or 128 columns per chunk), each held to the
    single-problem parity protocol on every problem of the uneven batch."""
    from paper_1805_06124_gb300 import rb
    c = rb.RB(device=0, batched_variant=variant)
    Ss = [torch.from_numpy(S).cuda() for S in uneven_batch]
    outs = c.greedy_batched(Ss, 1e-10, 300)
    for S, o in zip(uneven_batch, outs):
        g = npy(o)
        rep = parity.replay_and_check(orc, S, g, 1e-10, 300)
        parity.compare(g, rep, S)
    c.close()


def test_batched_96_problems_sampled_replay(orc):
    """The benchmark's 96-problem batch (seed 3, 127 GB complex128) in the
    autotuned launch configuration; four of its problems (the smallest, the
    largest N, the largest M and the median size) are replayed through the
    oracle with the parity protocol, and every problem's error curve must
    end below tol with a non-increasing curve."""
    from paper_1805_06124_gb300 import rb
    if torch.cuda.mem_get_info(0)[0] < 150e9:
        pytest.skip("needs about 140 GB of free device memory")
    probs, used = synth.batched_problems(96, 3)
    c = rb.RB(device=0)
    Ss = []
    for p in probs:
        q, m = synth.chirp_params(p["M"], p["seed"], q_range=p["q_range"], m_range=p["m_range"])
        Ss.append(c.generate(q, m, p["N"]))
    # the benchmark's call (no C, so the same pre-split decision), plus final errors
    outs = c.greedy_batched(Ss, 1e-10, 300, want_C=False)
    for o in outs:
        ec = o["err_curve"].cpu().numpy()
        k = o["k"]
        assert o["status"] == 0 and ec[k] < 1e-10 <= ec[k - 1]
        assert np.all(np.diff(ec) <= parity.delta(k, 8192, ec[0]))
    sizes = [p["N"] * p["M"] for p in probs]
    pick = {int(np.argmin(sizes)), int(np.argmax([p["N"] for p in probs])),
            int(np.argmax([p["M"] for p in probs])), int(np.argsort(sizes)[len(sizes) // 2])}
    for b in sorted(pick):
        S = Ss[b].cpu().numpy()
        g = npy(outs[b])
        rep = parity.replay_and_check(orc, S, g, 1e-10, 300, omp=True)
        info = parity.compare(g, rep, S)
        print("batched problem", b, probs[b]["N"], probs[b]["M"], info)
    c.close()
    del Ss
    torch.cuda.empty_cache()
