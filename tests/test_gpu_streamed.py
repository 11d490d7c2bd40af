"""The greedy on snapshots held in host memory (rb_greedy_streamed, needs a
GB300): parity with the FP64 oracle through the replay protocol, and bit
identity with the in-core rb_greedy on the same bytes (same pivots, Q, C,
errors) for every split between resident and streamed columns, chunk widths
that leave ragged chunks, odd N, the periodic recompute across lazily
skipped iterations, pinned and pageable host memory, and the exact-rank and
kmax stops."""
import ctypes

import numpy as np
import pytest

from paper_1805_06124_gb300 import synth
import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("Q", "pivots", "err_curve", "rdiag", "C", "final_err")


@pytest.fixture(scope="module")
def rbm():
    from paper_1805_06124_gb300 import rb
    return rb


@pytest.fixture(scope="module")
def ctx(rbm):
    c = rbm.RB(device=0)
    yield c
    c.close()


def npy(d):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in d.items()}


def host(S, pin=True):
    t = torch.from_numpy(np.ascontiguousarray(S))
    return t.pin_memory() if pin else t


def assert_identical(a, b):
    assert a["status"] == b["status"] and a["k"] == b["k"]
    for key in KEYS:
        x, y = a[key], b[key]
        assert x.shape == y.shape, key
        assert np.array_equal(x.view(np.uint8) if x.dtype.kind in "fc" else x,
                              y.view(np.uint8) if y.dtype.kind in "fc" else y), key


def in_core(ctx, S, tol, kmax):
    return npy(ctx.greedy(torch.from_numpy(np.ascontiguousarray(S)).cuda(), tol, kmax))


@pytest.mark.parametrize("resident,cols", [(0, 64), (1000, 64), (1000, 37), (1000, 1), (2999, 64), (3000, 64), (-1, 0)])
def test_identical_to_in_core(ctx, resident, cols):
    """1024 x 3000 chirps (seed 4, tol 1e-10): every output bit-identical to
    rb_greedy for resident parts from none to all; 3000 - 1000 = 2000
    streamed columns in chunks of 64 (last chunk 16) or 37 (last chunk 2)."""
    S = synth.chirps(1024, 3000, seed=4)
    ref = in_core(ctx, S, 1e-10, 300)
    assert 40 <= ref["k"] <= 80
    g = npy(ctx.greedy_streamed(host(S), 1e-10, 300, resident=resident, chunk_cols=cols))
    assert_identical(g, ref)
    st = ctx.streamed_stats()
    if resident < 0:
        assert st["resident"] == 3000 and st["chunks"] == 0
    else:
        assert st["resident"] == resident and st["chunk_cols"] == (cols or 1)
        assert st["chunks"] == -(-(3000 - resident) // cols)
        # every chunk is read at least once (iteration 0) and at most once per
        # iteration plus the flush
        assert st["chunks"] <= st["chunk_reads"] <= st["chunks"] * (g["k"] + 1)


def test_lazy_reads_skip_chunks(ctx):
    """With half of the columns resident, chunks whose errors cannot reach the
    iteration's best error are not read: far fewer chunk reads than chunks x
    iterations, with the same result."""
    S = synth.chirps(1024, 8192, seed=6)
    ref = in_core(ctx, S, 1e-10, 300)
    fr = {}
    for cols in (32, 1):
        g = npy(ctx.greedy_streamed(host(S), 1e-10, 300, resident=4096, chunk_cols=cols))
        assert_identical(g, ref)
        st = ctx.streamed_stats()
        fr[cols] = st["chunk_reads"] / (st["chunks"] * g["k"])
        print("chunk read fraction", cols, fr[cols], st)
    assert fr[32] < 0.8 and fr[1] < fr[32]


def test_oracle_parity_and_odd_n(ctx, orc):
    """Odd N (the last element on lane 0), pageable host memory (registered
    for the call), the recompute every 16 iterations across skipped ones:
    parity with the FP64 oracle by the replay protocol, and identity with
    rb_greedy."""
    S = synth.chirps(515, 1500, seed=8)
    g = npy(ctx.greedy_streamed(host(S, pin=False), 1e-10, 300, resident=300, chunk_cols=50))
    assert g["k"] > 32
    rep = parity.replay_and_check(orc, S, g, 1e-10, 300)
    parity.compare(g, rep, S)
    assert_identical(g, in_core(ctx, S, 1e-10, 300))


@pytest.mark.parametrize("case", ["low_rank", "kmax", "tiny", "kmax0"])
def test_stops(ctx, case):
    """Exact rank (IMGS finds nothing new or the error drops below tol), the
    kmax stop with skipped chunks pending (the flush completes C), and tiny
    shapes (one column; fewer columns than one chunk)."""
    if case == "low_rank":
        S = synth.low_rank(700, 400, 12, seed=5)
        tol, kmax, res, cols = 1e-24, 400, 100, 64
    elif case == "kmax":
        S = synth.chirps(512, 2000, seed=2)
        tol, kmax, res, cols = 1e-12, 7, 500, 16
    elif case == "tiny":
        S = synth.chirps(64, 5, seed=1)
        tol, kmax, res, cols = 1e-10, 5, 1, 64
    else:
        S = synth.chirps(128, 300, seed=1)
        tol, kmax, res, cols = 1e-10, 0, 100, 8
    ref = in_core(ctx, S, tol, kmax)
    g = npy(ctx.greedy_streamed(host(S), tol, kmax, resident=res, chunk_cols=cols))
    assert_identical(g, ref)
    if case == "kmax":
        assert g["status"] == 1 and g["k"] == 7


def test_nonfinite_input(ctx, rbm):
    """A NaN in a streamed column: the same RB_ENONFINITE as the in-core call."""
    S = synth.chirps(128, 300, seed=1)
    S[250, 17] = np.nan
    for run in (lambda: ctx.greedy(torch.from_numpy(S).cuda(), 1e-10, 50),
                lambda: ctx.greedy_streamed(host(S), 1e-10, 50, resident=100)):
        with pytest.raises(rbm.RBError) as e:
            run()
        assert e.value.status == rbm.ENONFINITE


def test_rejects_device_memory(ctx, rbm):
    S = torch.zeros((16, 32), dtype=torch.complex128, device="cuda")
    with pytest.raises(TypeError):
        ctx.greedy_streamed(S, 0.0, 4)
    r = rbm.Result()
    Q = torch.zeros((4, 32), dtype=torch.complex128, device="cuda")
    piv = torch.zeros(4, dtype=torch.int64, device="cuda")
    ec = torch.zeros(5, dtype=torch.float64, device="cuda")
    r.Q, r.ldQ = Q.data_ptr(), 32
    r.pivots = ctypes.cast(piv.data_ptr(), ctypes.POINTER(ctypes.c_longlong))
    r.err_curve = ctypes.cast(ec.data_ptr(), ctypes.POINTER(ctypes.c_double))
    st = ctx.lib.rb_greedy_streamed(ctx._h, S.data_ptr(), 32, 16, 32, 0.0, 4, -1, 0, ctypes.byref(r))
    assert st == rbm.EINVAL
    # bad chunk widths and the plain-FP64 sweep option are refused
    Sh = host(synth.chirps(64, 40, seed=2))
    with pytest.raises(rbm.RBError) as e:
        ctx.greedy_streamed(Sh, 0.0, 4, chunk_cols=-1)
    assert e.value.status == rbm.EINVAL
    c64 = rbm.RB(device=0, sweep="fp64")
    with pytest.raises(rbm.RBError) as e:
        c64.greedy_streamed(Sh, 0.0, 4)
    assert e.value.status == rbm.EINVAL
    c64.close()
    # the context stays usable
    S2 = synth.chirps(128, 300, seed=3)
    assert_identical(npy(ctx.greedy_streamed(host(S2), 1e-8, 50, resident=100)), in_core(ctx, S2, 1e-8, 50))


def test_full_size_half_resident(rbm):
    """8192 x 262,144 chirps (seed 1), tol 1e-12: half of the columns
    resident, the other 17 GB read from pinned host memory; pivots, the error
    curve, R's diagonal and sampled columns of C and Q identical to the
    in-core greedy."""
    c = rbm.RB(device=0)
    N, M = 8192, 262144
    q, m = synth.chirp_params(M, seed=1)
    Sd = c.generate(q, m, N)
    ref = c.greedy(Sd, 1e-12, 800)
    Sh = torch.empty((M, N), dtype=torch.complex128).pin_memory()
    Sh.copy_(Sd)
    del Sd
    keep = {k: ref[k].cpu().numpy() for k in ("pivots", "err_curve", "rdiag")}
    cols = np.random.default_rng(0).choice(M, 512, replace=False)
    keep["C"] = ref["C"][:, cols].cpu().numpy()
    keep["Q"] = ref["Q"][:, ::97].cpu().numpy()
    k = ref["k"]
    del ref
    torch.cuda.empty_cache()
    g = c.greedy_streamed(Sh, 1e-12, 800, resident=M // 2)
    assert g["k"] == k
    for key in ("pivots", "err_curve", "rdiag"):
        assert np.array_equal(g[key].cpu().numpy(), keep[key]), key
    assert np.array_equal(g["C"][:, cols].cpu().numpy(), keep["C"])
    assert np.array_equal(g["Q"][:, ::97].cpu().numpy(), keep["Q"])
    st = c.streamed_stats()
    print("full size", g["ms_total"], st)
    c.close()
