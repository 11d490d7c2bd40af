"""The allocation-free greedy entry point (rb_greedy_noalloc).

Some callers cannot call cudaMalloc (their device memory belongs to a
framework's pool, or they must not grow their footprint after start-up).
rb_greedy_noalloc serves them with a fixed scratch array inside the library.
This test calls it through the C ABI, twice in a row (the second call sees
the first call's leftovers in the shared scratch), and checks both results
against the existing rb_greedy entry point with the same plain-FP64 sweep and
the same options (bit for bit: the same kernels run in the same order), and
replays the pivots through the oracle.  It also checks that sizes
beyond the scratch limits are refused with a message.

The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

import parity
from paper_1805_06124_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc_fn(rb):
    lib = rb.load()
    f = lib.rb_greedy_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_double,
                  ctypes.c_int, ctypes.POINTER(rb.Options), ctypes.POINTER(rb.Result), ctypes.c_char_p,
                  ctypes.c_size_t]
    f.restype = ctypes.c_int
    return f


def _call_noalloc(rb, f, S, tol, kmax, recompute_period=None, want_C=True):
    M, N = S.shape
    dev = S.device
    Q = torch.zeros((kmax, N), dtype=torch.complex128, device=dev)
    piv = torch.full((kmax,), -1, dtype=torch.int64, device=dev)
    ec = torch.zeros((kmax + 1,), dtype=torch.float64, device=dev)
    C = torch.zeros((kmax, M), dtype=torch.complex128, device=dev)
    fe = torch.zeros((M,), dtype=torch.float64, device=dev)
    rd = torch.zeros((kmax,), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    r = rb.Result()
    r.Q, r.ldQ = Q.data_ptr(), N
    r.pivots = ctypes.cast(piv.data_ptr(), rb.c_ll_p)
    r.err_curve = ctypes.cast(ec.data_ptr(), rb.c_double_p)
    r.C, r.ldC = (C.data_ptr() if want_C else None), M
    r.final_err = ctypes.cast(fe.data_ptr(), rb.c_double_p)
    r.rdiag = ctypes.cast(rd.data_ptr(), rb.c_double_p)
    r.status = 99  # must be overwritten by the call
    opt = rb.Options()
    rb.load().rb_default_options(ctypes.byref(opt))
    opt.stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream or 1)
    if recompute_period is not None:
        opt.recompute_period = recompute_period
    err = ctypes.create_string_buffer(256)
    st = f(S.data_ptr(), N, M, S.stride(0), tol, kmax, ctypes.byref(opt), ctypes.byref(r), err, 256)
    k = r.k
    got = dict(k=k, status=r.status, pivots=piv[:k].cpu().numpy(), err_curve=ec[:k + 1].cpu().numpy(),
               Q=Q[:k].cpu().numpy(), final_err=fe.cpu().numpy(), rdiag=rd[:k].cpu().numpy())
    if want_C:
        got["C"] = C[:k].cpu().numpy()
    return st, err.value.decode(), got


def _npy(d):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in d.items()}


def _assert_same_bits(got, ref):
    """The allocation-free call runs the same kernels in the same order as
    rb_greedy with the plain-FP64 sweep, so every output is bit-identical."""
    assert got["k"] == ref["k"]
    for key in ("pivots", "err_curve", "Q", "final_err", "rdiag", "C"):
        if key in got and key in ref:
            a, b = np.asarray(got[key]), np.asarray(ref[key])
            assert a.shape == b.shape, key
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), key


@pytest.mark.parametrize("period", [16, 3])
def test_noalloc_matches_rb_greedy_twice(orc, period):
    """Two calls in a row (the second sees the first call's leftovers in the
    shared scratch array) against rb_greedy with the same options, bit for
    bit, and against the oracle's replay of the pivots."""
    from paper_1805_06124_gb300 import rb
    f = _noalloc_fn(rb)
    S1h = synth.chirps(1024, 2048, seed=0)
    S2h = synth.chirps(777, 1031, seed=5) * np.linspace(1.0, 1.2, 1031)[:, None]
    ctx = rb.RB(device=0, sweep="fp64", recompute_period=period)
    for Sh, tol, kmax in ((S1h, 1e-10, 300), (S2h, 1e-10, 777)):
        S = torch.from_numpy(Sh).cuda()
        ref = _npy(ctx.greedy(S, tol, kmax))
        for call in range(2):
            st, msg, got = _call_noalloc(rb, f, S, tol, kmax, recompute_period=period)
            assert st == ref["status"] and got["status"] == st, (call, st, got["status"], msg)
            _assert_same_bits(got, ref)
            assert torch.cuda.current_device() == 0
        rep = parity.replay_and_check(orc, Sh, got, tol, kmax)
        parity.compare(got, rep, Sh)
    ctx.close()


def test_noalloc_without_C_runs_without_recompute():
    """Without out->C the fixed array has no room for the coefficients, so the
    periodic recompute is off: the result equals rb_greedy with the recompute
    switched off."""
    from paper_1805_06124_gb300 import rb
    f = _noalloc_fn(rb)
    S = torch.from_numpy(synth.chirps(1024, 2048, seed=0)).cuda()
    ctx = rb.RB(device=0, sweep="fp64", recompute_period=0)
    ref = _npy(ctx.greedy(S, 1e-10, 300, want_C=False))
    ctx.close()
    st, msg, got = _call_noalloc(rb, f, S, 1e-10, 300, recompute_period=16, want_C=False)
    assert st == ref["status"], msg
    _assert_same_bits(got, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1805_06124_gb300 import rb
    f = _noalloc_fn(rb)
    S = torch.zeros((4, 16385), dtype=torch.complex128, device="cuda")
    st, msg, _ = _call_noalloc(rb, f, S, 1e-10, 4)
    assert st == rb.EINVAL and "exceed" in msg, msg
