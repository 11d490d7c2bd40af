"""The exchange of the column-sharded greedy (paper_1805_06124_gb300.sharded,
the paper's parallel scheme of Sec. 6.1.3) on two gloo ranks on the CPU.

Each rank's arithmetic is a small numpy engine written here (test code: norms,
CGS-form IMGS passes with Hoffmann's kappa test, the Eq. (Residual)
bookkeeping), standing in for one GPU's rb.Shard.  What is under test is the
exchange: the max-loc reduction with ties to the lowest global index, the
broadcast of the pivot column from its owner, the stopping rule and the
partition bookkeeping.  The pivots and the error curve must satisfy the
parity protocol against the single-process FP64 oracle on the whole matrix
(Alg. 3), and equal those of the same engines run in one process.
"""
import math
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


class NumpyShard:
    """One rank's columns in numpy (FP64)."""

    def __init__(self, S_local, col0, kmax, kappa=2.0, max_passes=4):
        self.S = np.ascontiguousarray(S_local)
        self.M, self.N = self.S.shape
        self.col0, self.kmax = col0, kmax
        self.kappa2, self.max_passes = kappa * kappa, max_passes
        self.Q = np.zeros((0, self.N), np.complex128)

    def new_buffer(self):
        return np.zeros(self.N + 1, np.complex128)

    def _best(self):
        err = self.norm2 - self.acc
        err = np.where(self.picked, -np.inf, err)
        if self.M == 0 or not np.any(np.isfinite(err)):
            return -math.inf, -1
        j = int(np.argmax(err))  # first maximum: lowest index among equal errors
        return float(err[j]), self.col0 + j

    def init(self):
        self.norm2 = np.sum(self.S.real ** 2 + self.S.imag ** 2, axis=1)
        self.acc = np.zeros(self.M)
        self.picked = np.zeros(self.M, bool)
        return self._best()

    def column(self, j, buf):
        jl = j - self.col0
        buf[:self.N] = self.S[jl]
        buf[self.N] = self.norm2[jl]

    def append(self, buf, j):
        v = buf[:self.N].copy()
        before = float(buf[self.N].real)
        if self.Q.shape[0] > 0:
            for _ in range(self.max_passes):
                v = v - self.Q.T @ (self.Q.conj() @ v)
                after = float(np.vdot(v, v).real)
                if after >= before / self.kappa2:
                    break
                before = after
            else:
                raise RuntimeError("IMGS did not pass the kappa test")
        nv2 = float(np.vdot(v, v).real)
        if not nv2 > 0.0:
            return -math.inf, -1, False
        q = v / math.sqrt(nv2)
        self.Q = np.vstack([self.Q, q[None, :]])
        jl = j - self.col0
        if 0 <= jl < self.M:
            self.picked[jl] = True
        c = self.S @ q.conj()
        self.acc += c.real ** 2 + c.imag ** 2
        e, i = self._best()
        return e, i, True

    def finish(self):
        return dict(k=self.Q.shape[0], Q=self.Q, final_err=self.norm2 - self.acc)


def _split(S, bounds):
    return [(S[a:b], a) for a, b in zip(bounds[:-1], bounds[1:])]


def _worker(rank, world, port, S, blocks_per_rank, tol, kmax, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1805_06124_gb300 import sharded
    engines = [NumpyShard(Sl, c0, kmax) for Sl, c0 in blocks_per_rank[rank]]
    r = sharded.greedy_sharded(engines, sharded.TorchComm(dist), tol, kmax)
    out[rank] = dict(status=r["status"], k=r["k"], pivots=list(r["pivots"]), err_curve=list(r["err_curve"]),
                     Q=r["shards"][0]["Q"])
    dist.barrier()
    dist.destroy_process_group()


def _run(S, blocks_per_rank, tol, kmax):
    port = 29700 + os.getpid() % 1000
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(len(blocks_per_rank), port, S, blocks_per_rank, tol, kmax, out),
             nprocs=len(blocks_per_rank), join=True)
    return [out[r] for r in range(len(blocks_per_rank))]


def test_two_ranks_match_the_oracle_and_one_process(orc):
    sys.path.insert(0, HERE)
    import parity
    from paper_1805_06124_gb300 import sharded, synth
    S = synth.chirps(96, 150, seed=3) * np.linspace(1.0, 1.3, 150)[:, None]
    tol, kmax = 1e-10, 96
    # rank 0 holds columns 0..69, rank 1 holds 70..149 as two blocks
    blocks = [[(S[0:70], 0)], [(S[70:110], 70), (S[110:150], 110)]]
    res = _run(S, blocks, tol, kmax)
    a, b = res
    assert a["pivots"] == b["pivots"] and a["err_curve"] == b["err_curve"] and a["status"] == b["status"] == 0
    assert np.array_equal(a["Q"], b["Q"])  # every rank built the same basis
    # the same engines in one process
    local = sharded.greedy_sharded([NumpyShard(Sl, c0, kmax) for Sl, c0 in _split(S, [0, 70, 110, 150])],
                                   sharded.LocalComm(), tol, kmax)
    assert local["pivots"] == a["pivots"] and local["err_curve"] == a["err_curve"]
    # parity protocol against the single-process oracle on the whole matrix
    g = dict(pivots=np.array(a["pivots"]), err_curve=np.array(a["err_curve"]), Q=a["Q"])
    rep = parity.replay_and_check(orc, S, g, tol, kmax)
    parity.compare(g, rep, S)


def test_ties_across_ranks_go_to_the_lowest_global_index():
    """Mutually orthogonal columns of equal norm: every step is an exact tie;
    the pivots must come in increasing global index whatever rank holds them."""
    from paper_1805_06124_gb300 import sharded
    N = 12
    S = np.eye(N, dtype=np.complex128)[::-1].copy()  # column j = e_{N-1-j}, all norms 1
    blocks = [[(S[6:12], 6)], [(S[0:6], 0)]]          # rank 0 holds the higher indices
    res = _run(S, blocks, 0.5, N)
    assert res[0]["pivots"] == list(range(N)) == res[1]["pivots"]
    assert res[0]["status"] == 0 and res[0]["err_curve"][:N] == [1.0] * N


def test_stopping_rules_kmax_and_rank():
    from paper_1805_06124_gb300 import sharded, synth
    S = synth.low_rank(40, 30, 5, seed=2)
    blocks = [[(S[0:25], 0)], [(S[25:40], 25)]]
    res = _run(S, blocks, 0.0, 3)                # kmax reached
    assert res[0]["status"] == sharded.KMAX_REACHED and res[0]["k"] == 3
    # exact rank 5: the errors fall to rounding level after five vectors
    scale = float(np.max(np.sum(np.abs(S) ** 2, axis=1)))
    local = sharded.greedy_sharded([NumpyShard(Sl, c0, 40) for Sl, c0 in _split(S, [0, 25, 40])],
                                   sharded.LocalComm(), 1e-10 * scale, 40)
    assert local["status"] == 0 and local["k"] == 5
    assert local["err_curve"][5] < 1e-12 * scale
