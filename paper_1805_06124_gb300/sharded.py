"""Column-sharded RB-greedy: the exchange of the paper's parallel scheme.

The paper's parallel code (Sec. 6.1.3) distributes the snapshot columns over
MPI processes: each process updates its columns' errors and finds its local
maximum, the processes agree on the global pivot with a max-loc all-reduce,
and the owner sends that column to a master process, which orthogonalises it
and broadcasts the new basis vector.  Here the owner broadcasts the pivot
column instead and every process orthogonalises it against its own copy of
the basis (the same deterministic kernels on identical inputs give identical
vectors), so one collective carries the column and no process waits for a
master.  This module is that exchange, around per-rank engines that do the
arithmetic:

  * ``rb.Shard`` -- one GPU's columns through the C ABI (``rb_shard_*``); the
    exchanged buffers are CUDA tensors (NCCL, or one process holding several
    shards on one GPU through ``LocalComm``);
  * any object with the same methods (``col0``, ``M``, ``N``, ``new_buffer``,
    ``init``, ``column``, ``append``, ``finish``), e.g. a CPU stand-in in the
    tests of the exchange logic over gloo.

Every process calls ``greedy_sharded`` with the engines it owns.  Per
iteration there is one all-gather of 24 bytes per process (local candidate
error, global index, status) and one broadcast of the pivot column
(16 (N + 1) bytes) from its owner.  Ties between processes go to the lowest
global column index, as in the single-GPU argmax, so the pivot sequence does
not depend on the partition.  Stopping rule (Alg. 3, reading of the tolerance
on squared errors): stop when the largest error is below tol, when kmax
vectors are built, or when min(N, M_total) are.

The column partition is the caller's: contiguous blocks, any sizes; each
process may hold any number of blocks.
"""
from __future__ import annotations

import math

OK, KMAX_REACHED = 0, 1


class LocalComm:
    """One process holding every shard (no exchange)."""
    rank, size = 0, 1

    def allgather(self, triple):
        return [triple]

    def gather_ranges(self, ranges):
        return [ranges]

    def broadcast(self, buf, src):
        return buf


class TorchComm:
    """torch.distributed (NCCL for CUDA buffers, gloo for CPU buffers).

    ``device``: where the small all-gather tensor lives (``"cuda:i"`` for NCCL,
    ``"cpu"`` for gloo)."""

    def __init__(self, dist, device="cpu", group=None):
        self.dist, self.group, self.device = dist, group, device
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def allgather(self, triple):
        import torch
        t = torch.tensor(list(triple), dtype=torch.float64, device=self.device)
        out = torch.empty(3 * self.size, dtype=torch.float64, device=self.device)
        self.dist.all_gather_into_tensor(out, t, group=self.group)
        v = out.tolist()  # one read of all ranks' triples
        return [tuple(v[3 * r:3 * r + 3]) for r in range(self.size)]

    def gather_ranges(self, ranges):
        out = [None] * self.size
        self.dist.all_gather_object(out, ranges, group=self.group)
        return out

    def broadcast(self, buf, src):
        import torch
        t = buf if isinstance(buf, torch.Tensor) else torch.from_numpy(buf)
        self.dist.broadcast(t, src=src, group=self.group)
        return buf


def _better(e1, i1, e2, i2):
    """(e1, i1) beats (e2, i2): larger error, ties to the lower index; i < 0 = none."""
    if i1 < 0:
        return False
    if i2 < 0:
        return True
    return e1 > e2 or (e1 == e2 and i1 < i2)


def _best(cands):
    be, bi = -math.inf, -1
    for e, i in cands:
        if _better(e, i, be, bi):
            be, bi = e, i
    return be, bi


def greedy_sharded(engines, comm, tol: float, kmax: int):
    """Runs the greedy over all processes' engines; returns this process's
    view: the global pivots and error curve (identical on every process), the
    status, and each local engine's ``finish()`` result (its basis copy, its
    columns' coefficients and final errors)."""
    if not engines:
        raise ValueError("every process needs at least one shard")
    N = engines[0].N
    ranges = comm.gather_ranges([(int(e.col0), int(e.M)) for e in engines])
    owners = []
    for p, rs in enumerate(ranges):
        for (c0, m) in rs:
            owners.append((c0, c0 + m, p))
    owners.sort()
    for (a0, a1, _), (b0, _b1, _) in zip(owners, owners[1:]):
        if a1 > b0:
            raise ValueError("column blocks overlap")
    m_total = sum(b - a for a, b, _ in owners)
    min_nm = min(N, m_total)

    def owner_of(j):
        for a, b, p in owners:
            if a <= j < b:
                return p
        raise ValueError(f"column {j} is owned by no process")

    def reduce(cands, status):
        e, i = _best(cands)
        got = comm.allgather((e, float(i), float(status)))
        ge, gi = _best([(t[0], int(t[1])) for t in got])
        gs = int(min(t[2] for t in got))
        return ge, gi, gs

    status_local = OK
    cands = []
    for e in engines:
        try:
            cands.append(e.init())
        except Exception as exc:  # a NaN or Inf in one shard fails the whole run, on every process
            status_local = getattr(exc, "status", -4)
            cands.append((-math.inf, -1))
    buf = engines[0].new_buffer()
    pivots, err_curve = [], []
    k, status = 0, OK
    while True:
        ge, gi, gs = reduce(cands, status_local)
        if gs < 0:
            status = gs
            break
        err_curve.append(ge if gi >= 0 else 0.0)
        if gi < 0 or ge < tol:
            status = OK
            break
        if k >= kmax:
            status = KMAX_REACHED
            break
        if k >= min_nm:
            status = OK
            break
        src = owner_of(gi)
        if comm.rank == src:
            for e in engines:
                if e.col0 <= gi < e.col0 + e.M:
                    e.column(gi, buf)
                    break
        comm.broadcast(buf, src)
        cands = []
        appended = True
        for e in engines:
            be, bi, app = e.append(buf, gi)
            appended = appended and app
            cands.append((be, bi))
        if not appended:  # the pivot lay in the span: exact rank reached
            status = OK
            break
        pivots.append(gi)
        k += 1
    results = [e.finish() for e in engines]
    return dict(status=status, k=k, pivots=pivots, err_curve=err_curve, shards=results)
