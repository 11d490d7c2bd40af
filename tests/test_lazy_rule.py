"""The lazy chunk rule of the host-resident greedy, checked on the CPU against
the oracle's coefficients.

The FP64-form bookkeeping (Eq. (Residual), Sec. 6.1.2) gives err_j =
||s_j||^2 - acc_j with acc_j a running sum of |c_lj|^2 and a compensated
recompute every `period` iterations.  The streamed greedy skips a chunk of
columns while its stale error bound plus (k + 16) 2^-51 max ||s_j||^2 stays
below the best error of the iteration, and applies the skipped rows in order
when it next reads the chunk.  Here that rule runs in numpy on the C rows of
the FP64 oracle's greedy; the argmax of every iteration must equal the one
that updating every column every iteration gives (same rows, same
arithmetic), every skipped chunk's current errors must lie under its bound
plus margin and strictly under the best error, the sums after the final
flush must equal the eager ones bit for bit, and the eager argmaxes must be
the oracle's own pivots.
"""
import math

import numpy as np
import pytest

from paper_1805_06124_gb300 import synth

oracle = pytest.importorskip("oracle.oracle")

PERIOD = 16


def recompute(c):
    """acc from the stored coefficients of one column, correctly rounded
    (math.fsum), as a different rounding of the running sum."""
    return math.fsum(np.concatenate([c.real * c.real, c.imag * c.imag]).tolist())


def apply_rows(C, acc, cols, l0, l1):
    """Rows l0..l1 (inclusive) of C into acc for columns `cols`: the running
    sum, with the recompute before every row that is a positive multiple of
    the period."""
    for l in range(l0, l1 + 1):
        if l > 0 and l % PERIOD == 0:
            acc[cols] = [recompute(C[:l, j]) for j in cols]
        c = C[l, cols]
        acc[cols] = acc[cols] + (c.real * c.real + c.imag * c.imag)


def best_of(err, cols, picked):
    """(err, idx) maximum over unpicked columns, ties to the lowest index."""
    cols = np.asarray(cols)
    cols = cols[~picked[cols]]
    if cols.size == 0:
        return (-np.inf, -1)
    e = err[cols]
    m = e.max()
    return (float(m), int(cols[np.flatnonzero(e == m)[0]]))


def lazy_vs_eager(C, norm2, first, Mr, cols, gamma=0.99):
    K, M = C.shape
    acc_e = np.zeros(M)
    acc_l = np.zeros(M)
    picked = np.zeros(M, bool)
    picked[first] = True
    starts = list(range(Mr, M, cols))
    chunks = [np.arange(s, min(s + cols, M)) for s in starts]
    last = np.zeros(len(chunks), int)
    bound = np.array([norm2[c].max() for c in chunks])
    nmax = bound.copy()
    reads = 0
    pivots = []
    resident = np.arange(Mr)
    for k in range(K - 1):
        # eager: every column takes row k
        apply_rows(C, acc_e, np.arange(M), k, k)
        pe = best_of(norm2 - acc_e, np.arange(M), picked)
        # lazy: resident columns eagerly, chunks by the two rounds
        apply_rows(C, acc_l, resident, k, k)
        R = best_of(norm2 - acc_l, resident, picked)
        margin = (k + 16) * 2.0 ** -51 * nmax
        ub = np.where(np.isfinite(bound), bound + margin, -np.inf)
        stale = last <= k
        mx = ub[stale].max() if stale.any() else -np.inf
        best = R
        for rnd in (0, 1):
            th = max(R[0], gamma * mx) if rnd == 0 and mx > 0 else best[0]
            sel = [i for i in range(len(chunks)) if last[i] <= k and np.isfinite(bound[i]) and ub[i] >= th]
            for i in sel:
                apply_rows(C, acc_l, chunks[i], last[i], k)
                b = best_of(norm2 - acc_l, chunks[i], picked)
                bound[i] = b[0] if b[1] >= 0 else -np.inf
                last[i] = k + 1
                reads += 1
                if b[1] >= 0 and (b[0] > best[0] or (b[0] == best[0] and (best[1] < 0 or b[1] < best[1]))):
                    best = b
        assert best == pe, (k, best, pe)
        # the certificate: every chunk left stale has its current errors (the
        # eager ones) at most its bound plus margin, and strictly below the best
        err_e = norm2 - acc_e
        for i in range(len(chunks)):
            if last[i] <= k:
                cur = best_of(err_e, chunks[i], picked)[0]
                assert cur <= ub[i] and cur < best[0], (k, i, cur, ub[i], best)
        pivots.append(pe[1])
        picked[pe[1]] = True
    # the flush: every chunk takes its pending rows; the sums equal the eager ones bit for bit
    for i in range(len(chunks)):
        apply_rows(C, acc_l, chunks[i], last[i], K - 2)
    assert np.array_equal(acc_l[:M], acc_e[:M])
    return pivots, reads / max(1, len(chunks) * (K - 1))


@pytest.mark.parametrize("Mr,cols", [(0, 1), (1000, 1), (1000, 7), (0, 64)])
def test_lazy_rule_matches_eager_argmax(Mr, cols):
    """Chirps 256 x 3000 (seed 4), tol 1e-10: the lazy rule's argmax equals
    the eager one at every iteration (recompute at 16, 32, ...), for resident
    parts 0 and 1000 and chunks of 1, 7 (ragged) and 64 columns, and the
    eager argmaxes are the oracle's pivots."""
    S = synth.chirps(256, 3000, seed=4)
    g = oracle.rb_greedy(S, 1e-10, 300)
    assert g["k"] > 2 * PERIOD
    C = g["C"]
    norm2 = np.array([np.vdot(s, s).real for s in S])
    pivots, frac = lazy_vs_eager(C, norm2, int(g["pivots"][0]), Mr, cols)
    assert pivots == [int(p) for p in g["pivots"][1:]]
    if cols == 1:
        assert frac < 0.8


def test_margin_covers_recompute_drift():
    """The margin itself: across a recompute the error can rise (the running
    sum may have rounded above the correctly rounded one), but never by more
    than (k + 16) 2^-51 ||s||^2.  Random sequences of squared coefficients
    that exhaust a unit norm to 1e-12 (where the rounding of acc dominates
    err), half of them with negligible terms after k0: the error at a stale
    read k0 against the error after the recompute at the next multiple of the
    period and further terms up to k."""
    rng = np.random.default_rng(11)
    rises, worst = 0, 0.0
    for _ in range(3000):
        K = int(rng.integers(PERIOD + 2, 6 * PERIOD))
        t = rng.random(K) ** 8
        t *= (1.0 - 1e-12) / t.sum()
        k0 = int(rng.integers(1, K - 1))
        if rng.random() < 0.5:
            # a column nearly orthogonal to the later vectors: its later terms
            # are below the rounding of acc, so only the recompute moves it
            t[k0:] *= 1e-20
        l = (k0 // PERIOD + 1) * PERIOD
        if l >= K:
            continue
        k = int(rng.integers(l, K))
        acc = 0.0
        for x in t[:k0]:
            acc = acc + x
        stale = 1.0 - acc
        acc = math.fsum(t[:l].tolist())
        for x in t[l:k + 1]:
            acc = acc + x
        new = 1.0 - acc
        if new > stale:
            rises += 1
            worst = max(worst, (new - stale) / 2.0 ** -52)
        # the sum only grows: the newer error is the smaller in exact arithmetic
        assert new <= stale + (k + 16) * 2.0 ** -51, (k0, l, k, new - stale)
    assert rises > 0, "the test never saw a rise: it does not exercise the margin"
    print("rises", rises, "worst rise in ulps of 1:", worst)
