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
