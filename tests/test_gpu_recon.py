"""Parity of the reconstruction step (Alg. 4, Sec. 5.2.2) on the GPU against
the FP64 oracle: the singular values of C, the left singular vectors (unique
up to a unit factor where the singular value is separated; the factor is then
fixed by the phase convention), k, and the enriched basis X_k = Q_j V(:, 1:k),
plus the error statements of Theorems 5.6 and 5.8 on the GPU's basis.

Q and C come from the GPU greedy; the oracle receives the identical bytes."""
import numpy as np
import pytest

from paper_1805_06124_gb300 import synth

torch = pytest.importorskip("torch")
recon = pytest.importorskip("oracle.recon_oracle")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53
MAX_J = 112


@pytest.fixture(scope="module")
def ctx():
    from paper_1805_06124_gb300 import rb
    c = rb.RB(device=0)
    yield c
    c.close()


def greedy_on_gpu(ctx, S, tol, kmax):
    g = ctx.greedy(torch.from_numpy(np.ascontiguousarray(S)).cuda(), tol, kmax)
    assert g["status"] in (0, 1)
    return g["Q"], g["C"], g


def tau_between(s, k):
    """A threshold with exactly k singular values above it."""
    if k <= 0:
        return 2.0 * s[0]
    if k >= len(s):
        return 0.0
    return float(np.sqrt(s[k - 1] * s[k])) if s[k] > 0 else 0.5 * s[k - 1]


def check_against_oracle(ctx, Q, C, kpick):
    """Runs the GPU reconstruction with a threshold between the oracle's
    sigma_kpick and sigma_{kpick+1} and compares everything with the oracle."""
    Qh, Ch = Q.cpu().numpy(), C.cpu().numpy()
    j = Qh.shape[0]
    s_lapack = np.linalg.svd(Ch, compute_uv=False) if j else np.zeros(0)
    tau2 = tau_between(s_lapack, kpick) if j else 1.0
    out = ctx.reconstruct(Q, C, tau2)
    ref = recon.reconstruct(Qh, Ch, tau2)
    assert out["k"] == ref["k"] == min(kpick, j)
    if j == 0:
        assert out["X"].shape[0] == 0
        return out
    sig = out["sigma"].cpu().numpy()
    s_ref = ref["sigma"]
    s1 = s_ref[0]
    # singular values: both sides are backward stable, |d sigma| <= O(u) ||C||_2
    np.testing.assert_allclose(sig, s_ref, rtol=1e-11, atol=64 * j * U * s1)
    assert np.all(np.diff(sig) <= 0)
    V = out["V"].cpu().numpy()
    assert np.linalg.norm(V.conj().T @ V - np.eye(j), 2) < 64 * j * U
    # phase convention: the largest-magnitude entry (lowest row among equals)
    # is real and positive
    for c in range(j):
        a = np.abs(V[:, c])
        p = int(np.flatnonzero(a >= a.max() * (1 - 1e-13))[0])
        assert V[p, c].imag == 0.0 and V[p, c].real > 0, c
    # vectors, column by column where the singular value is separated:
    # angle <= O(u) ||C|| / gap on each side
    Vr = ref["V"]
    checked = 0
    for c in range(j):
        others = np.delete(s_ref, c)
        gap = np.min(np.abs(others - s_ref[c])) if j > 1 else s1
        bound = 256 * j * U * s1 / max(gap, 1e-300) + 1e-13
        if bound > 1e-3:
            continue
        ph = np.vdot(Vr[:, c], V[:, c])
        ph /= abs(ph)
        assert np.linalg.norm(V[:, c] - ph * Vr[:, c]) <= bound, (c, gap)
        # where the maximal entry is clear, the two conventions pick the same factor
        a = np.sort(np.abs(Vr[:, c]))
        if j == 1 or a[-1] - a[-2] > 1e3 * bound:
            assert abs(ph - 1.0) <= 4 * bound, c
        checked += 1
    assert checked >= min(j, 3)
    # X_k = Q_j V(:, 1:k): the kernel's sums of j products
    k = out["k"]
    X = out["X"].cpu().numpy()
    assert X.shape == (k, Qh.shape[1])
    if k:
        Xe = V[:, :k].T @ Qh
        assert np.max(np.abs(X - Xe)) <= 4 * j * U * np.max(np.abs(Qh)) * np.sqrt(j)
        assert np.linalg.norm(X.conj() @ X.T - np.eye(k), 2) < 1e-12
    return out


def test_chirps_small_config(ctx):
    """1024 x 2048 chirps, seed 0, tol 1e-10 (the small greedy case)."""
    S = synth.chirps(1024, 2048, seed=0)
    Q, C, g = greedy_on_gpu(ctx, S, 1e-10, 300)
    assert 40 <= g["k"] <= 70
    check_against_oracle(ctx, Q, C, 12)


def test_exact_rank_theorem_5_6(ctx):
    """Exact rank r: sigma(C) = sigma(S) and ||S - X_i X_i^H S||_2 = sigma_{i+1}(S)."""
    S = synth.low_rank(600, 400, 12, seed=5)
    scale = float(np.max(np.sum(np.abs(S) ** 2, axis=1)))
    Q, C, g = greedy_on_gpu(ctx, S, 1e-12 * scale, 400)
    assert g["k"] == 12
    out = check_against_oracle(ctx, Q, C, 12)
    sv = np.linalg.svd(S.T, compute_uv=False)
    np.testing.assert_allclose(out["sigma"].cpu().numpy(), sv[:12], rtol=1e-11, atol=1e-13 * sv[0])
    V = out["V"].cpu().numpy()
    Qh = Q.cpu().numpy()
    for i in range(1, 12):
        e = recon.residual_norm2(S, V[:, :i].T @ Qh)
        assert abs(e - sv[i]) <= 1e-10 * sv[i] + 1e-12 * sv[0], i


def test_bounds_theorem_5_8(ctx):
    """Chirps truncated at j below the numerical rank: for every k <= j,
    sigma_{k+1}(S) <= ||S - X_k X_k^H S||_2 <= sigma_{k+1}(C) + ||S - Q_j C||_2."""
    S = synth.chirps(512, 1024, seed=3)
    Q, C, g = greedy_on_gpu(ctx, S, 1e-6, 300)
    j = g["k"]
    out = ctx.reconstruct(Q, C, 0.0)
    assert out["k"] == j
    A = S.T
    sv = np.linalg.svd(A, compute_uv=False)
    Qh, Ch = Q.cpu().numpy(), C.cpu().numpy()
    resid = np.linalg.norm(A - Qh.T @ Ch, 2)
    sig = out["sigma"].cpu().numpy()
    V = out["V"].cpu().numpy()
    for k in range(1, j + 1):
        e = recon.residual_norm2(S, V[:, :k].T @ Qh)
        assert e >= sv[k] * (1 - 1e-10), k
        assert e <= (sig[k] if k < j else 0.0) + resid * (1 + 1e-10) + 1e-13, k
    # the reconstructed basis is no worse than the greedy basis of the same size
    k = j // 2
    assert recon.residual_norm2(S, V[:, :k].T @ Qh) <= recon.residual_norm2(S, Qh[:k]) * (1 + 1e-12)


@pytest.mark.parametrize("N,M,kmax,kpick", [
    (64, 5, 1, 1),           # j = 1
    (300, 4096 + 37, 33, 7),  # two Gram chunks, a ragged tile of rows (33 = 32 + 1)
    (256, 70, 70, 70),        # k = j, tau2 = 0
    (200, 300, 20, 0),        # k = 0 (tau2 above sigma_1)
    (512, 9000, MAX_J, 40),   # j at its maximum, three Gram chunks, four row tiles
])
def test_edge_shapes(ctx, N, M, kmax, kpick):
    scales = np.exp(-np.linspace(0.0, 12.0, M)) * (1.0 + 0.5 * np.sin(np.arange(M)))
    S = synth.random_complex(M, N, seed=N + M, scales=scales)
    Q, C, g = greedy_on_gpu(ctx, S, 0.0, kmax)
    assert g["k"] == kmax
    check_against_oracle(ctx, Q, C, kpick)


def test_empty_and_too_large(ctx):
    Q = torch.zeros((0, 16), dtype=torch.complex128, device="cuda")
    C = torch.zeros((0, 8), dtype=torch.complex128, device="cuda")
    out = ctx.reconstruct(Q, C, 0.0)
    assert out["k"] == 0 and out["X"].shape == (0, 16) and out["sigma"].numel() == 0
    Q = torch.zeros((MAX_J + 1, 256), dtype=torch.complex128, device="cuda")
    C = torch.zeros((MAX_J + 1, 256), dtype=torch.complex128, device="cuda")
    with pytest.raises(Exception):
        ctx.reconstruct(Q, C, 0.0)
    # the context stays usable
    S = synth.chirps(128, 256, seed=9)
    Qg, Cg, g = greedy_on_gpu(ctx, S, 1e-8, 60)
    check_against_oracle(ctx, Qg, Cg, 5)


def test_full_size_sampled(ctx):
    """8192 x 262,144 chirps (seed 1), tol 1e-12: the benchmark's greedy
    workload followed by the reconstruction, checked against the oracle on
    the full C (j x 262,144) and X on sampled rows."""
    from paper_1805_06124_gb300 import rb
    c = rb.RB(device=0)
    N, M = 8192, 262144
    q, m = synth.chirp_params(M, seed=1)
    S = c.generate(q, m, N)
    g = c.greedy(S, 1e-12, 800)
    del S
    torch.cuda.empty_cache()
    Q, C = g["Q"], g["C"]
    j = g["k"]
    assert 40 <= j <= 90
    out = check_against_oracle(c, Q, C, 20)
    assert out["k"] == 20
    c.close()


def test_phase_timing_and_counts():
    """With timing on, every phase of the last call has a CUDA-event time and
    the Jacobi counts are consistent (pass 2 starts from the pass-1 basis and
    needs few sweeps)."""
    from paper_1805_06124_gb300 import rb
    c = rb.RB(device=0, timing=True)
    S = synth.chirps(1024, 2048, seed=0)
    Q, C, g = greedy_on_gpu(c, S, 1e-10, 300)
    j = g["k"]
    c.reconstruct(Q, C, 0.0)
    st = c.reconstruct_stats()
    assert all(v > 0.0 for v in st["ms"].values()), st
    assert 1 <= st["sweeps"][0] <= 60 and 1 <= st["sweeps"][1] <= 8, st
    assert st["rotations"][0] >= j * (j - 1) // 2 and st["rotations"][1] > 0, st
    c.close()
