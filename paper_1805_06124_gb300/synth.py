"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle's
checks.  This module holds input generation only: none of the method's
arithmetic (no projections, no pivoting, no Gram-Schmidt).

The snapshot family stands in for the paper's IMRPhenomPv2 gravitational-wave
snapshots (Sec. 6.1.1), which need LALSuite:

    s_j(t_i) = (t_c - t_i)^(-1/4) * exp(-i * omega_j * (t_c - t_i)^(5/8)),
    t_i = i / N (i = 0..N-1), t_c = 1.05,
    omega_j = 200 * eta_j^(-3/8) * m_j^(-5/8),  eta_j = q_j / (1 + q_j)^2,

with q ~ U[1, 10] and m ~ U[0.8, 1.2] drawn from ``numpy.random.default_rng``
(PCG64): first q for all M columns, then m for all M columns.  Every column is
normalised to unit 2-norm in FP64.

Layout: a snapshot matrix is returned as a C-contiguous complex128 array of
shape (M, N), row j being the snapshot s_j (the paper's column j).
"""
from __future__ import annotations

import math

import numpy as np

T_C = 1.05


def chirp_params(M: int, seed: int, q_range=(1.0, 10.0), m_range=(0.8, 1.2)):
    """Draw (q, m) for M snapshots: q for all columns first, then m."""
    rng = np.random.default_rng(seed)
    q = rng.uniform(q_range[0], q_range[1], M)
    m = rng.uniform(m_range[0], m_range[1], M)
    return q, m


def chirp_omega(q, m):
    """omega = 200 eta^(-3/8) m^(-5/8) with eta = q / (1+q)^2."""
    q = np.asarray(q, np.float64)
    m = np.asarray(m, np.float64)
    eta = q / (1.0 + q) ** 2
    return 200.0 * eta ** (-3.0 / 8.0) * m ** (-5.0 / 8.0)


def chirp_matrix(N: int, q, m, t_c: float = T_C, normalise: bool = True) -> np.ndarray:
    """(M, N) complex128 chirp snapshots, unit-norm rows when ``normalise``."""
    omega = chirp_omega(q, m)
    tau = t_c - np.arange(N, dtype=np.float64) / N
    amp = tau ** -0.25
    ph = tau ** 0.625
    S = amp[None, :] * np.exp(-1j * omega[:, None] * ph[None, :])
    if normalise:
        S /= np.sqrt(np.sum(S.real ** 2 + S.imag ** 2, axis=1))[:, None]
    return np.ascontiguousarray(S)


def chirps(N: int, M: int, seed: int, **kw) -> np.ndarray:
    """The benchmark chirp family: chirp_params then chirp_matrix."""
    q, m = chirp_params(M, seed, **{k: v for k, v in kw.items() if k in ("q_range", "m_range")})
    return chirp_matrix(N, q, m)


def chirps_blocked(N: int, M: int, seed: int, block: int = 4096, threads: int | None = None) -> np.ndarray:
    """The same snapshots as ``chirps`` for large M: the (q, m) draws are made
    once for all columns, then the rows are filled in blocks on a thread pool
    (numpy's elementwise loops release the GIL), so the peak memory is the
    output plus one block of temporaries per thread."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    q, m = chirp_params(M, seed)
    S = np.empty((M, N), np.complex128)

    def fill(a):
        S[a:a + block] = chirp_matrix(N, q[a:a + block], m[a:a + block])

    with ThreadPoolExecutor(max_workers=threads or min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(fill, range(0, M, block)))
    return S


def random_complex(M: int, N: int, seed: int, scales=None) -> np.ndarray:
    """Gaussian complex (M, N) matrix; optional per-snapshot scales."""
    rng = np.random.default_rng(seed)
    S = rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))
    if scales is not None:
        S *= np.asarray(scales, np.float64)[:, None]
    return np.ascontiguousarray(S)


def low_rank(M: int, N: int, r: int, seed: int) -> np.ndarray:
    """Exact rank-r complex (M, N) matrix A @ B with Gaussian factors."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((M, r)) + 1j * rng.standard_normal((M, r))
    B = rng.standard_normal((r, N)) + 1j * rng.standard_normal((r, N))
    return np.ascontiguousarray(A @ B)


def batched_problems(nprob: int = 96, seed: int = 3, budget_bytes: float = 200e9):
    """Problem sizes and parameter boxes for the batched workload.

    Per problem, in this order: N = round(exp(U[ln 512, ln 8192])),
    M = round(exp(U[ln 4096, ln 131072])), a q interval from two sorted
    U[1, 10] draws and an m interval from two sorted U[0.8, 1.2] draws, each
    widened to at least 5% of its full range.  If the complex128 total
    exceeds ``budget_bytes`` the draw is repeated with seed+1 (the seed used
    is returned).
    """
    s = seed
    while True:
        rng = np.random.default_rng(s)
        probs = []
        total = 0.0
        for _ in range(nprob):
            N = int(round(math.exp(rng.uniform(math.log(512), math.log(8192)))))
            M = int(round(math.exp(rng.uniform(math.log(4096), math.log(131072)))))
            qa, qb = np.sort(rng.uniform(1.0, 10.0, 2))
            ma, mb = np.sort(rng.uniform(0.8, 1.2, 2))
            qa, qb = _widen(qa, qb, 1.0, 10.0)
            ma, mb = _widen(ma, mb, 0.8, 1.2)
            probs.append(dict(N=N, M=M, q_range=(float(qa), float(qb)), m_range=(float(ma), float(mb)),
                              seed=int(rng.integers(0, 2**31 - 1))))
            total += 16.0 * N * M
        if total <= budget_bytes:
            return probs, s
        s += 1


def _widen(a, b, lo, hi, frac=0.05):
    w = frac * (hi - lo)
    if b - a >= w:
        return a, b
    c = 0.5 * (a + b)
    a, b = c - 0.5 * w, c + 0.5 * w
    if a < lo:
        a, b = lo, lo + w
    if b > hi:
        a, b = hi - w, hi
    return a, b
