"""The allocation-free greedy entry point (rb_greedy_noalloc).

Some callers cannot call cudaMalloc (their device memory belongs to a
framework's pool, or they must not grow their footprint after start-up).
rb_greedy_noalloc serves them with a fixed scratch array inside the library.
This test calls it through the C ABI, twice in a row (the second call sees
the first call's leftovers in the shared scratch), and checks both results
against the existing rb_greedy entry point with the same plain-FP64 sweep,
within the tolerances of the other parity tests.  It also checks that sizes
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


def _call_noalloc(rb, f, S, tol, kmax):
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
    r.C, r.ldC = C.data_ptr(), M
    r.final_err = ctypes.cast(fe.data_ptr(), rb.c_double_p)
    r.rdiag = ctypes.cast(rd.data_ptr(), rb.c_double_p)
    opt = rb.Options()
    rb.load().rb_default_options(ctypes.byref(opt))
    opt.stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream or 1)
    err = ctypes.create_string_buffer(256)
    st = f(S.data_ptr(), N, M, S.stride(0), tol, kmax, ctypes.byref(opt), ctypes.byref(r), err, 256)
    k = r.k
    return st, err.value.decode(), dict(k=k, pivots=piv[:k].cpu().numpy(), err_curve=ec[:k + 1].cpu().numpy(),
                                        Q=Q[:k].cpu().numpy(), C=C[:k].cpu().numpy(),
                                        final_err=fe.cpu().numpy(), rdiag=rd[:k].cpu().numpy())


def test_noalloc_matches_rb_greedy_twice():
    from paper_1805_06124_gb300 import rb
    f = _noalloc_fn(rb)
    S1 = torch.from_numpy(synth.chirps(1024, 2048, seed=0)).cuda()
    S2 = torch.from_numpy(synth.chirps(777, 1031, seed=5) * np.linspace(1.0, 1.2, 1031)[:, None]).cuda()
    ctx = rb.RB(device=0, sweep="fp64")
    for S, tol, kmax in ((S1, 1e-10, 300), (S2, 1e-10, 777)):
        ref = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in ctx.greedy(S, tol, kmax).items()}
        for call in range(2):
            st, msg, got = _call_noalloc(rb, f, S, tol, kmax)
            assert st == ref["status"], (call, st, msg)
            assert got["k"] == ref["k"]
            assert list(got["pivots"]) == list(ref["pivots"])
            np.testing.assert_allclose(got["err_curve"], ref["err_curve"], rtol=0, atol=1e-12)
            np.testing.assert_allclose(got["final_err"], ref["final_err"], rtol=0, atol=1e-12)
            bt = parity.basis_tol(ref["err_curve"], ref["k"])
            assert np.all(np.max(np.abs(got["Q"] - ref["Q"]), axis=1) <= bt)
            assert np.all(np.max(np.abs(got["C"] - ref["C"]), axis=1) <= bt + 1e-13)
            np.testing.assert_allclose(got["rdiag"], ref["rdiag"], rtol=1e-12, atol=1e-15)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1805_06124_gb300 import rb
    f = _noalloc_fn(rb)
    S = torch.zeros((4, 16385), dtype=torch.complex128, device="cuda")
    st, msg, _ = _call_noalloc(rb, f, S, 1e-10, 4)
    assert st == rb.EINVAL and "exceed" in msg, msg
