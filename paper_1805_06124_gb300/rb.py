"""Thin ctypes binding of the C ABI in ``include/rb.h``.

Argument marshalling only: every step of the method runs in the CUDA
library ``_build/librb_gb300.so``.  PyTorch supplies device memory and the
stream.  There is no CPU fallback: if the library is missing or no GPU is
present, the calls raise.

Python-side layouts (all C-contiguous torch tensors on the GPU):
  S      complex128 (M, N)    row j = snapshot s_j (the paper's column j)
  Q      complex128 (kmax, N) row l = basis vector q_l
  C      complex128 (kmax, M) C[l, j] = q_l^H s_j
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int, c_double, c_ll, c_void_p, c_uint = ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_uint
c_double_p = ctypes.POINTER(ctypes.c_double)
c_ll_p = ctypes.POINTER(ctypes.c_longlong)

OK, KMAX_REACHED = 0, 1
EINVAL, ENOMEM, ECUDA, ENONFINITE, EORTHO, ETIMEOUT, ESTATE = -1, -2, -3, -4, -5, -6, -7
SWEEP = {"df32": 0, "fp64": 1}
FLAG_TIMING = 1
FLAG_PROJECT_FP64 = 2
FLAG_SPLIT_NO_SWITCH = 4
MLP_FOURIER, MLP_SPLIT = 1, 2


class Options(ctypes.Structure):
    _fields_ = [("device", c_int), ("sweep", c_int), ("imgs_kappa", c_double), ("imgs_max_passes", c_int),
                ("switch_err", c_double), ("iters_per_sync", c_int), ("stream", c_void_p), ("flags", c_uint),
                ("recompute_period", c_int), ("batched_variant", c_int), ("timeout_cycles", ctypes.c_ulonglong)]


class Result(ctypes.Structure):
    _fields_ = [("Q", c_void_p), ("ldQ", c_ll), ("pivots", c_ll_p), ("err_curve", c_double_p),
                ("C", c_void_p), ("ldC", c_ll), ("final_err", c_double_p), ("rdiag", c_double_p),
                ("k", c_int), ("imgs_passes", c_int), ("switch_iter", c_int), ("n_launches", c_int),
                ("n_sweeps", c_int), ("ms_total", c_double), ("ms_sweep", c_double), ("sweep_bytes", c_double),
                ("status", c_int)]


class Problem(ctypes.Structure):
    _fields_ = [("S", c_void_p), ("N", c_ll), ("M", c_ll), ("ldS", c_ll)]


class RBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"rb status {status}: {msg}")
        self.status = status


_LIB = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load the CUDA library (building it first when asked)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    lib.rb_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.rb_default_options.restype = None
    lib.rb_create.argtypes = [ctypes.POINTER(Options), ctypes.POINTER(c_void_p)]
    lib.rb_create.restype = c_int
    lib.rb_destroy.argtypes = [c_void_p]
    lib.rb_destroy.restype = None
    lib.rb_last_error.argtypes = [c_void_p]
    lib.rb_last_error.restype = ctypes.c_char_p
    lib.rb_generate.argtypes = [c_void_p, c_void_p, c_void_p, c_ll, c_ll, c_void_p, c_ll]
    lib.rb_split.argtypes = [c_void_p, c_void_p, c_ll, c_ll, c_ll, c_void_p, c_void_p, c_ll]
    lib.rb_greedy.argtypes = [c_void_p, c_void_p, c_ll, c_ll, c_ll, c_double, c_int, ctypes.POINTER(Result)]
    lib.rb_greedy_host.argtypes = [c_void_p, c_void_p, c_ll, c_ll, c_ll, c_double, c_int, ctypes.POINTER(Result)]
    lib.rb_greedy_streamed.argtypes = [c_void_p, c_void_p, c_ll, c_ll, c_ll, c_double, c_int, c_ll, c_ll,
                                       ctypes.POINTER(Result)]
    lib.rb_streamed_stats.argtypes = [c_void_p, ctypes.POINTER(c_ll), ctypes.POINTER(c_double),
                                      ctypes.POINTER(c_double)]
    lib.rb_greedy_split.argtypes = [c_void_p, c_void_p, c_void_p, c_ll, c_ll, c_ll, c_double, c_int,
                                    ctypes.POINTER(Result)]
    lib.rb_project.argtypes = [c_void_p, c_void_p, c_ll, c_int, c_ll, c_void_p, c_ll, c_ll, c_void_p, c_ll]
    lib.rb_reconstruct.argtypes = [c_void_p, c_void_p, c_ll, c_int, c_ll, c_void_p, c_ll, c_ll, c_double, c_void_p,
                                   c_ll, c_void_p, c_void_p, ctypes.POINTER(c_int)]
    lib.rb_reconstruct_stats.argtypes = [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_int)]
    lib.rb_trace.argtypes = [c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_double), ctypes.POINTER(c_double),
                             c_int, ctypes.POINTER(c_int)]
    lib.rb_greedy_resume.argtypes = [c_void_p, c_void_p, c_ll, c_ll, c_ll, c_double, c_int, c_int, c_ll,
                                     ctypes.POINTER(Result)]
    lib.rb_eim.argtypes = [c_void_p, c_void_p, c_ll, c_int, c_ll, c_void_p, c_void_p, c_void_p, c_ll, c_void_p]
    lib.rb_validate.argtypes = [c_void_p, c_void_p, c_ll, c_int, c_ll, c_void_p, c_void_p, c_void_p, c_ll, c_ll,
                                c_void_p, c_void_p]
    lib.rb_greedy_batched.argtypes = [c_void_p, c_int, ctypes.POINTER(Problem), c_double, c_int,
                                      ctypes.POINTER(Result)]
    lib.rb_greedy_batched.restype = c_int
    lib.rb_shard_create.argtypes = [c_void_p, c_void_p, c_ll, c_ll, c_ll, c_ll, c_int, ctypes.POINTER(Result),
                                    ctypes.POINTER(c_void_p)]
    lib.rb_shard_destroy.argtypes = [c_void_p]
    lib.rb_shard_destroy.restype = None
    lib.rb_shard_init.argtypes = [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_ll)]
    lib.rb_shard_column.argtypes = [c_void_p, c_ll, c_void_p, ctypes.POINTER(c_double)]
    lib.rb_shard_append.argtypes = [c_void_p, c_void_p, c_double, c_ll, ctypes.POINTER(c_double),
                                    ctypes.POINTER(c_ll), ctypes.POINTER(c_int)]
    lib.rb_shard_finish.argtypes = [c_void_p, c_void_p, ctypes.POINTER(c_int)]
    for f in ("rb_generate", "rb_split", "rb_greedy", "rb_greedy_host", "rb_greedy_split", "rb_project",
              "rb_reconstruct", "rb_reconstruct_stats", "rb_eim", "rb_validate", "rb_greedy_resume", "rb_trace",
              "rb_shard_create", "rb_shard_init", "rb_shard_column", "rb_shard_append", "rb_shard_finish"):
        getattr(lib, f).restype = c_int
    _LIB = lib
    return lib


def _torch():
    import torch
    return torch


def _ld(t) -> int:
    """Leading dimension (in elements) of a 2-D row-major tensor."""
    return int(t.stride(0)) if t.shape[0] > 1 else int(t.shape[1])


def _check2d(t, dtype, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.dim() != 2 or t.dtype != dtype or t.stride(1) != 1:
        raise TypeError(f"{name} must be a 2-D {dtype} tensor with unit column stride")
    if not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")


class RB:
    """One rb_ctx.  ``stream`` defaults to torch's current stream on ``device``."""

    def __init__(self, device: int = 0, sweep: str = "df32", kappa: float = 2.0, max_passes: int = 4,
                 switch_err: float = 0.0, iters_per_sync: int = 8, stream=None, timing: bool = False,
                 project_fp64: bool = False, recompute_period: int = 16, batched_variant: int = -1,
                 timeout_cycles: int = 0, split_switch: bool = True):
        torch = _torch()
        self.lib = load()
        self.device = device
        opt = Options()
        self.lib.rb_default_options(ctypes.byref(opt))
        opt.device = device
        opt.sweep = SWEEP[sweep]
        opt.imgs_kappa = kappa
        opt.imgs_max_passes = max_passes
        opt.switch_err = switch_err
        opt.iters_per_sync = iters_per_sync
        opt.recompute_period = recompute_period
        opt.batched_variant = batched_variant
        opt.timeout_cycles = timeout_cycles
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        # torch's legacy default stream has handle 0; pass cudaStreamLegacy
        # (0x1) so the library orders its work with torch instead of
        # creating a private stream.
        opt.stream = c_void_p(stream.cuda_stream or 1)
        opt.flags = ((FLAG_TIMING if timing else 0) | (FLAG_PROJECT_FP64 if project_fp64 else 0) |
                     (0 if split_switch else FLAG_SPLIT_NO_SWITCH))
        h = c_void_p()
        st = self.lib.rb_create(ctypes.byref(opt), ctypes.byref(h))
        if st != OK:
            raise RBError(st, "rb_create failed")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self.lib.rb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st < 0:
            raise RBError(st, self.lib.rb_last_error(self._h).decode())
        return st

    # ---------------------------------------------------------------- calls
    def generate(self, q, m, N: int, ld: int | None = None):
        """Chirp snapshots on the GPU from per-column parameters (q, m)."""
        torch = _torch()
        q = torch.as_tensor(q, dtype=torch.float64, device=f"cuda:{self.device}").contiguous()
        m = torch.as_tensor(m, dtype=torch.float64, device=f"cuda:{self.device}").contiguous()
        M = q.numel()
        ld = N if ld is None else ld
        with torch.cuda.stream(self.stream):
            S = torch.empty((M, ld), dtype=torch.complex128, device=q.device)[:, :N]
        self._check(self.lib.rb_generate(self._h, q.data_ptr(), m.data_ptr(), N, M, S.data_ptr(), ld))
        return S

    def split(self, S, ldh: int | None = None, out=None):
        """hi/lo complex64 split of S (rb_split).  out: optional (hi, lo) views
        of shape (M, N) with a common row stride, written in place."""
        torch = _torch()
        _check2d(S, torch.complex128, "S")
        M, N = S.shape
        if out is not None:
            hi, lo = out
            if (hi.dtype != torch.complex64 or lo.dtype != torch.complex64 or tuple(hi.shape) != (M, N)
                    or tuple(lo.shape) != (M, N) or hi.stride(1) != 1 or lo.stride(1) != 1
                    or _ld(hi) != _ld(lo)):
                raise ValueError("split: out must be two complex64 (M, N) views with one row stride")
            self._check(self.lib.rb_split(self._h, S.data_ptr(), N, M, _ld(S), hi.data_ptr(), lo.data_ptr(),
                                          _ld(hi)))
            return hi, lo
        ldh = N if ldh is None else ldh
        with torch.cuda.stream(self.stream):
            hi = torch.empty((M, ldh), dtype=torch.complex64, device=S.device)
            lo = torch.empty((M, ldh), dtype=torch.complex64, device=S.device)
        self._check(self.lib.rb_split(self._h, S.data_ptr(), N, M, _ld(S), hi.data_ptr(), lo.data_ptr(), ldh))
        return hi[:, :N], lo[:, :N]

    def _alloc_result(self, N, M, kmax, dev, want_C, want_final):
        torch = _torch()
        kc = max(kmax, 1)
        bufs = dict(Q=torch.zeros((kc, N), dtype=torch.complex128, device=dev),
                    pivots=torch.full((kc,), -1, dtype=torch.int64, device=dev),
                    err_curve=torch.zeros((kc + 1,), dtype=torch.float64, device=dev),
                    rdiag=torch.zeros((kc,), dtype=torch.float64, device=dev))
        if want_C:
            bufs["C"] = torch.zeros((kc, M), dtype=torch.complex128, device=dev)
        if want_final:
            bufs["final_err"] = torch.zeros((M,), dtype=torch.float64, device=dev)
        r = Result()
        r.Q = bufs["Q"].data_ptr()
        r.ldQ = N
        r.pivots = ctypes.cast(bufs["pivots"].data_ptr(), c_ll_p)
        r.err_curve = ctypes.cast(bufs["err_curve"].data_ptr(), c_double_p)
        r.rdiag = ctypes.cast(bufs["rdiag"].data_ptr(), c_double_p)
        r.C = bufs["C"].data_ptr() if want_C else None
        r.ldC = M
        r.final_err = ctypes.cast(bufs["final_err"].data_ptr(), c_double_p) if want_final else None
        return r, bufs

    @staticmethod
    def _pack(st, r, bufs):
        k = r.k
        out = dict(status=st, k=k, imgs_passes=r.imgs_passes, switch_iter=r.switch_iter, n_launches=r.n_launches,
                   n_sweeps=r.n_sweeps, ms_total=r.ms_total, ms_sweep=r.ms_sweep, sweep_bytes=r.sweep_bytes)
        out["Q"] = bufs["Q"][:k]
        out["pivots"] = bufs["pivots"][:k]
        out["err_curve"] = bufs["err_curve"][:k + 1]
        out["rdiag"] = bufs["rdiag"][:k]
        if "C" in bufs:
            out["C"] = bufs["C"][:k]
        if "final_err" in bufs:
            out["final_err"] = bufs["final_err"]
        return out

    def greedy(self, S, tol: float, kmax: int, want_C: bool = True, want_final_err: bool = True):
        """RB-greedy (Alg. 3) on device snapshots S (M, N) complex128."""
        torch = _torch()
        _check2d(S, torch.complex128, "S")
        M, N = S.shape
        with torch.cuda.stream(self.stream):
            r, bufs = self._alloc_result(N, M, kmax, S.device, want_C, want_final_err)
        st = self._check(self.lib.rb_greedy(self._h, S.data_ptr(), N, M, _ld(S), float(tol), int(kmax),
                                            ctypes.byref(r)))
        return self._pack(st, r, bufs)

    def greedy_resume(self, S, tol: float, kmax: int, checkpoint: dict, Mc: int | None = None,
                      want_final_err: bool = True):
        """RB-greedy on device snapshots S (M, N) continued from ``checkpoint``
        (a result dict or a loaded checkpoint: Q (k0, N), pivots (k0,), C (k0,
        Mc), err_curve (k0 + 1,), rdiag (k0,); arrays or tensors).  Columns
        Mc..M-1 of S are new snapshots (default Mc = C's column count)."""
        torch = _torch()
        _check2d(S, torch.complex128, "S")
        M, N = S.shape
        dev = S.device
        as_t = lambda x, dt: torch.as_tensor(x, dtype=dt).to(dev)
        Q0 = as_t(checkpoint["Q"], torch.complex128)
        k0 = int(Q0.shape[0])
        piv0 = as_t(checkpoint["pivots"], torch.int64)[:k0]
        C0 = as_t(checkpoint["C"], torch.complex128)[:k0]
        ec0 = as_t(checkpoint["err_curve"], torch.float64)[:k0]
        rd0 = as_t(checkpoint["rdiag"], torch.float64)[:k0]
        Mc = int(C0.shape[1]) if Mc is None else int(Mc)
        if k0 > kmax or Q0.shape[1] != N or C0.shape[1] < Mc or Mc > M or piv0.numel() != k0:
            raise ValueError("checkpoint does not match S / kmax")
        with torch.cuda.stream(self.stream):
            r, bufs = self._alloc_result(N, M, kmax, dev, True, want_final_err)
            if k0:
                bufs["Q"][:k0] = Q0
                bufs["pivots"][:k0] = piv0
                bufs["C"][:k0, :Mc] = C0[:, :Mc]
                bufs["err_curve"][:k0] = ec0
                bufs["rdiag"][:k0] = rd0
        st = self._check(self.lib.rb_greedy_resume(self._h, S.data_ptr(), N, M, _ld(S), float(tol), int(kmax), k0, Mc,
                                                   ctypes.byref(r)))
        return self._pack(st, r, bufs)

    def greedy_split(self, hi, lo, tol: float, kmax: int, want_C: bool = True, want_final_err: bool = True):
        """Split-precision RB-greedy on hi/lo complex64 tensors of shape (M, N)
        sharing one even leading dimension."""
        torch = _torch()
        _check2d(hi, torch.complex64, "hi")
        _check2d(lo, torch.complex64, "lo")
        if hi.shape != lo.shape or _ld(hi) != _ld(lo):
            raise ValueError("hi and lo must have the same shape and leading dimension")
        M, N = hi.shape
        with torch.cuda.stream(self.stream):
            r, bufs = self._alloc_result(N, M, kmax, hi.device, want_C, want_final_err)
        st = self._check(self.lib.rb_greedy_split(self._h, hi.data_ptr(), lo.data_ptr(), N, M, _ld(hi), float(tol),
                                                  int(kmax), ctypes.byref(r)))
        return self._pack(st, r, bufs)

    def greedy_batched(self, Ss, tol: float, kmax: int, want_C: bool = True, want_final_err: bool = True):
        """Independent RB-greedy problems (a list of (M_b, N_b) complex128 CUDA
        tensors) in one batched call; returns one result dict per problem."""
        torch = _torch()
        n = len(Ss)
        probs = (Problem * n)()
        results = (Result * n)()
        keep = []
        for b, S in enumerate(Ss):
            _check2d(S, torch.complex128, f"S[{b}]")
            M, N = S.shape
            probs[b].S, probs[b].N, probs[b].M, probs[b].ldS = S.data_ptr(), N, M, _ld(S)
            with torch.cuda.stream(self.stream):
                r, bufs = self._alloc_result(N, M, kmax, S.device, want_C, want_final_err)
            results[b] = r
            keep.append(bufs)
        st = self._check(self.lib.rb_greedy_batched(self._h, n, probs, float(tol), int(kmax), results))
        return [self._pack(results[b].status, results[b], keep[b]) for b in range(n)]

    @staticmethod
    def host_outputs(N: int, M: int, kmax: int, want_C: bool = True, want_final_err: bool = True, pin: bool = True):
        """Host output buffers for greedy_host, to be reused across calls
        (pinned by default; allocating pinned memory is slow)."""
        torch = _torch()
        kc = max(kmax, 1)
        # the library fills every entry that is returned (the first k rows, all
        # M final errors), so the large buffers are not zeroed
        bufs = dict(Q=torch.empty((kc, N), dtype=torch.complex128, pin_memory=pin),
                    pivots=torch.empty((kc,), dtype=torch.int64, pin_memory=pin),
                    err_curve=torch.empty((kc + 1,), dtype=torch.float64, pin_memory=pin),
                    rdiag=torch.empty((kc,), dtype=torch.float64, pin_memory=pin))
        if want_C:
            bufs["C"] = torch.empty((kc, M), dtype=torch.complex128, pin_memory=pin)
        if want_final_err:
            bufs["final_err"] = torch.empty((M,), dtype=torch.float64, pin_memory=pin)
        return bufs

    def greedy_streamed(self, S, tol: float, kmax: int, resident: int = -1, chunk_cols: int = 0,
                        want_C: bool = True, want_final_err: bool = True):
        """RB-greedy on snapshots S (M, N) complex128 that stay in HOST memory
        (a CPU tensor; pinned memory is used in place, pageable memory is
        mapped for the call).  Columns 0..resident-1 keep a split copy on the
        device (-1: as many as fit); the rest are read in chunks of
        ``chunk_cols`` (0: 1).  Outputs are device tensors, bit-identical to
        ``greedy``'s."""
        torch = _torch()
        if (not isinstance(S, torch.Tensor) or S.dim() != 2 or S.dtype != torch.complex128 or S.is_cuda
                or S.stride(1) != 1):
            raise TypeError("S must be a 2-D complex128 CPU tensor with unit column stride")
        M, N = S.shape
        dev = torch.device("cuda", self.device)
        with torch.cuda.stream(self.stream):
            r, bufs = self._alloc_result(N, M, kmax, dev, want_C, want_final_err)
        st = self._check(self.lib.rb_greedy_streamed(self._h, S.data_ptr(), N, M, _ld(S), float(tol), int(kmax),
                                                     int(resident), int(chunk_cols), ctypes.byref(r)))
        return self._pack(st, r, bufs)

    def streamed_stats(self) -> dict:
        """Counters of the last greedy_streamed call."""
        cnt = (c_ll * 4)()
        hb, mi = c_double(), c_double()
        self._check(self.lib.rb_streamed_stats(self._h, cnt, ctypes.byref(hb), ctypes.byref(mi)))
        return dict(resident=cnt[0], chunks=cnt[1], chunk_cols=cnt[2], chunk_reads=cnt[3],
                    host_bytes=hb.value, ms_init=mi.value)

    def greedy_host(self, S, tol: float, kmax: int, want_C: bool = True, want_final_err: bool = True, out=None):
        """Same as greedy, with S and all outputs in host memory (CPU tensors;
        pinned memory gives the fastest copies).  ``out``: buffers from
        host_outputs (reused; the returned tensors are views of them)."""
        torch = _torch()
        if S.dim() != 2 or S.dtype != torch.complex128 or S.is_cuda or S.stride(1) != 1:
            raise TypeError("S must be a 2-D complex128 CPU tensor with unit column stride")
        M, N = S.shape
        kc = max(kmax, 1)
        if out is None:
            bufs = self.host_outputs(N, M, kmax, want_C, want_final_err, pin=S.is_pinned())
        else:
            bufs = out
            want_C, want_final_err = "C" in bufs, "final_err" in bufs
            if (tuple(bufs["Q"].shape) != (kc, N) or bufs["pivots"].numel() < kc or bufs["err_curve"].numel() < kc + 1
                    or bufs["rdiag"].numel() < kc or (want_C and tuple(bufs["C"].shape) != (kc, M))
                    or (want_final_err and bufs["final_err"].numel() < M)):
                raise ValueError("out buffers do not match (N, M, kmax); build them with host_outputs")
        r = Result()
        r.Q = bufs["Q"].data_ptr()
        r.ldQ = N
        r.pivots = ctypes.cast(bufs["pivots"].data_ptr(), c_ll_p)
        r.err_curve = ctypes.cast(bufs["err_curve"].data_ptr(), c_double_p)
        r.rdiag = ctypes.cast(bufs["rdiag"].data_ptr(), c_double_p)
        r.C = bufs["C"].data_ptr() if want_C else None
        r.ldC = M
        r.final_err = ctypes.cast(bufs["final_err"].data_ptr(), c_double_p) if want_final_err else None
        st = self._check(self.lib.rb_greedy_host(self._h, S.data_ptr(), N, M, _ld(S), float(tol), int(kmax),
                                                 ctypes.byref(r)))
        return self._pack(st, r, bufs)

    def project(self, Q, X, k: int | None = None):
        """C[l, j] = q_l^H x_j for l < k (Q: (k, N), X: (Mx, N), both complex128)."""
        torch = _torch()
        _check2d(Q, torch.complex128, "Q")
        _check2d(X, torch.complex128, "X")
        k = Q.shape[0] if k is None else k
        N = Q.shape[1]
        if X.shape[1] != N:
            raise ValueError("Q and X disagree on N")
        Mx = X.shape[0]
        with torch.cuda.stream(self.stream):
            C = torch.empty((max(k, 1), Mx), dtype=torch.complex128, device=X.device)
        self._check(self.lib.rb_project(self._h, Q.data_ptr(), N, k, _ld(Q), X.data_ptr(), Mx, _ld(X),
                                        C.data_ptr(), Mx))
        return C[:k]

    def reconstruct(self, Q, C, tau2: float):
        """Reconstruction (Alg. 4): SVD of C (j, M) = V Sigma W^H and the enriched
        basis X = rows x_c = sum_l V[l, c] q_l for the k singular values above
        tau2.  Q (j, N) and C as returned by greedy.  Returns a dict with sigma
        (j,) float64, V (j, j) complex128 (column c = left singular vector c, its
        largest-magnitude entry real positive), k, and X (k, N)."""
        torch = _torch()
        _check2d(Q, torch.complex128, "Q")
        _check2d(C, torch.complex128, "C")
        j, N = Q.shape
        if C.shape[0] != j:
            raise ValueError("Q and C disagree on j")
        M = C.shape[1]
        dev = Q.device
        with torch.cuda.stream(self.stream):
            X = torch.empty((max(j, 1), N), dtype=torch.complex128, device=dev)
            sigma = torch.empty(max(j, 1), dtype=torch.float64, device=dev)
            V = torch.empty((max(j, 1), max(j, 1)), dtype=torch.complex128, device=dev)
        k = c_int(0)
        self._check(self.lib.rb_reconstruct(self._h, Q.data_ptr(), N, j, _ld(Q) if j else N, C.data_ptr(), M,
                                            _ld(C) if j else M, float(tau2), X.data_ptr(), N, sigma.data_ptr(),
                                            V.data_ptr(), ctypes.byref(k)))
        return dict(sigma=sigma[:j], V=V[:j, :j], k=int(k.value), X=X[:k.value])

    def eim(self, Q, want_V: bool = True, want_B: bool = True, want_Vinv: bool = True):
        """Empirical interpolation nodes of the basis rows of Q (k, N): nodes
        (k,) int64, V (k, k) with V[m, l] = q_l(p_m), B (k, N) with row m =
        the interpolant's m-th cardinal function (I[f] = sum_m f(p_m) B[m]),
        Vinv (k, k) = V^{-1}."""
        torch = _torch()
        _check2d(Q, torch.complex128, "Q")
        k, N = Q.shape
        dev = Q.device
        kk = max(k, 1)
        with torch.cuda.stream(self.stream):
            nodes = torch.empty(kk, dtype=torch.int64, device=dev)
            V = torch.empty((kk, kk), dtype=torch.complex128, device=dev) if want_V else None
            B = torch.empty((kk, N), dtype=torch.complex128, device=dev) if want_B else None
            Vi = torch.empty((kk, kk), dtype=torch.complex128, device=dev) if want_Vinv else None
        ptr = lambda t: t.data_ptr() if t is not None else None
        self._check(self.lib.rb_eim(self._h, Q.data_ptr(), N, k, _ld(Q) if k else N, nodes.data_ptr(), ptr(V),
                                    ptr(B), N, ptr(Vi)))
        out = dict(nodes=nodes[:k])
        if want_V:
            out["V"] = V[:k, :k]
        if want_B:
            out["B"] = B[:k]
        if want_Vinv:
            out["Vinv"] = Vi[:k, :k]
        return out

    def validate(self, Q, T, nodes=None, Vinv=None):
        """Out-of-sample errors of the basis rows of Q (k, N) on the snapshot
        rows of T (Mt, N): err_proj and, given rb_eim's nodes and Vinv,
        err_eim (squared 2-norms, float64 (Mt,))."""
        torch = _torch()
        _check2d(T, torch.complex128, "T")
        Mt, N = T.shape
        k = 0 if Q is None else Q.shape[0]
        if k:
            _check2d(Q, torch.complex128, "Q")
            if Q.shape[1] != N:
                raise ValueError("Q and T disagree on N")
        want_eim = nodes is not None
        if want_eim and k and (Vinv is None or nodes.numel() != k):
            raise ValueError("err_eim needs the k nodes and Vinv of rb_eim")
        with torch.cuda.stream(self.stream):
            ep = torch.empty(max(Mt, 1), dtype=torch.float64, device=T.device)
            ee = torch.empty(max(Mt, 1), dtype=torch.float64, device=T.device) if want_eim else None
        self._check(self.lib.rb_validate(self._h, Q.data_ptr() if k else None, N, k, _ld(Q) if k else N,
                                         nodes.data_ptr() if (want_eim and k) else None,
                                         Vinv.data_ptr() if (want_eim and k) else None, T.data_ptr(), Mt,
                                         _ld(T) if Mt else N, ep.data_ptr(), ee.data_ptr() if want_eim else None))
        out = dict(err_proj=ep[:Mt])
        if want_eim:
            out["err_eim"] = ee[:Mt]
        return out

    def trace(self):
        """Per-iteration trace of the last FP64-form greedy call: IMGS passes,
        and sweep / IMGS times in ms (with timing=True)."""
        n = c_int(0)
        self._check(self.lib.rb_trace(self._h, None, None, None, 0, ctypes.byref(n)))
        cap = n.value
        ps, sw, im = (c_int * max(cap, 1))(), (c_double * max(cap, 1))(), (c_double * max(cap, 1))()
        self._check(self.lib.rb_trace(self._h, ps, sw, im, cap, ctypes.byref(n)))
        return dict(imgs_passes=list(ps[:cap]), sweep_ms=list(sw[:cap]), imgs_ms=list(im[:cap]))

    RECON_PHASES = ("gram1_fp32", "jacobi1_fp32", "newton_schulz", "transform_df32", "gram2_df32",
                    "jacobi2_fp64", "basis")

    def reconstruct_stats(self):
        """Phase times (ms; needs timing=True) and Jacobi sweeps/rotations of
        the last reconstruct call."""
        ms = (c_double * 7)()
        cnt = (c_int * 4)()
        self._check(self.lib.rb_reconstruct_stats(self._h, ms, cnt))
        return dict(ms=dict(zip(self.RECON_PHASES, list(ms))), sweeps=(cnt[0], cnt[2]), rotations=(cnt[1], cnt[3]))


class Shard:
    """One rank's columns of the column-sharded greedy (rb_shard_*): the
    engine that paper_1805_06124_gb300.sharded drives.  S: this rank's
    snapshots, a CUDA complex128 (M, N) tensor; col0: the global index of its
    first column.  The buffers exchanged between ranks are (N + 1,) complex128
    CUDA tensors: the pivot column, then its stored norm in the real part of
    the last entry."""

    def __init__(self, ctx: "RB", S, col0: int, kmax: int, want_C: bool = True):
        torch = _torch()
        _check2d(S, torch.complex128, "S")
        self.ctx, self.lib, self.S = ctx, ctx.lib, S
        self.M, self.N = S.shape
        self.col0, self.kmax = int(col0), int(kmax)
        with torch.cuda.stream(ctx.stream):
            self._r, self._bufs = ctx._alloc_result(self.N, self.M, kmax, S.device, want_C, True)
        h = c_void_p()
        ctx._check(self.lib.rb_shard_create(ctx._h, S.data_ptr(), self.N, self.M, _ld(S), self.col0, self.kmax,
                                            ctypes.byref(self._r), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self.lib.rb_shard_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def new_buffer(self):
        torch = _torch()
        return torch.zeros((self.N + 1,), dtype=torch.complex128, device=self.S.device)

    def init(self):
        e, j = c_double(), c_ll()
        self.ctx._check(self.lib.rb_shard_init(self._h, ctypes.byref(e), ctypes.byref(j)))
        return e.value, j.value

    def column(self, j: int, buf):
        """Column j (owned here) into buf[:N], its norm into buf[N], on the
        device (asynchronous on the context's stream)."""
        self.ctx._check(self.lib.rb_shard_column(self._h, int(j), buf.data_ptr(), None))

    def append(self, buf, j: int):
        """IMGS of the received pivot column (buf from the owner, its norm in
        buf[N], read on the device) and the sweep of this rank's columns;
        returns (best_err, best_idx, appended)."""
        e, jj, app = c_double(), c_ll(), c_int()
        self.ctx._check(self.lib.rb_shard_append(self._h, buf.data_ptr(), -1.0, int(j), ctypes.byref(e),
                                                 ctypes.byref(jj), ctypes.byref(app)))
        return e.value, jj.value, bool(app.value)

    def finish(self):
        k = c_int()
        st = self.lib.rb_shard_finish(self._h, self._bufs["final_err"].data_ptr(), ctypes.byref(k))
        k = k.value
        out = dict(status=st, k=k, Q=self._bufs["Q"][:k], pivots=self._bufs["pivots"][:k], rdiag=self._bufs["rdiag"][:k],
                   final_err=self._bufs["final_err"])
        if "C" in self._bufs:
            out["C"] = self._bufs["C"][:k]
        return out


class MLP:
    """Learned surrogate (q, m) -> 2k coefficients on one RB context's stream.

    Inputs X are (rows, 2) float32, targets T (rows, n_out) float32, all CUDA
    tensors; the caller scales the inputs (e.g. to [-1, 1])."""

    def __init__(self, ctx: "RB", n_out: int, batch_cap: int = 4096, seed: int = 0, fourier=None,
                 split: bool = False):
        """fourier: (tau_lo, tau_hi) for the fixed Fourier input layer of
        RB_MLP_FOURIER (inputs are then the physical (q, m)); split: the
        RB_MLP_SPLIT forward (BF16 hi + lo pieces)."""
        lib = ctx.lib
        if not hasattr(lib.rb_mlp_create, "_rb_typed"):
            lib.rb_mlp_create.argtypes = [c_void_p, c_int, c_int, ctypes.c_ulonglong, ctypes.POINTER(c_void_p)]
            lib.rb_mlp_create.restype = c_int
            lib.rb_mlp_create_ex.argtypes = [c_void_p, c_int, c_int, ctypes.c_ulonglong, c_uint, c_double, c_double,
                                             ctypes.POINTER(c_void_p)]
            lib.rb_mlp_create_ex.restype = c_int
            lib.rb_mlp_destroy.argtypes = [c_void_p]
            lib.rb_mlp_destroy.restype = None
            lib.rb_mlp_num_params.argtypes = [c_void_p]
            lib.rb_mlp_num_params.restype = c_ll
            for f in ("rb_mlp_get_params", "rb_mlp_set_params"):
                getattr(lib, f).argtypes = [c_void_p, c_void_p]
                getattr(lib, f).restype = c_int
            lib.rb_mlp_infer.argtypes = [c_void_p, c_void_p, c_ll, c_void_p]
            lib.rb_mlp_infer.restype = c_int
            lib.rb_mlp_grad.argtypes = [c_void_p, c_void_p, c_void_p, c_ll, c_void_p, c_void_p]
            lib.rb_mlp_grad.restype = c_int
            lib.rb_mlp_train.argtypes = [c_void_p, c_void_p, c_void_p, c_ll, c_int, c_int, c_double,
                                         ctypes.c_ulonglong, c_void_p]
            lib.rb_mlp_train.restype = c_int
            lib.rb_mlp_create._rb_typed = True
        self.ctx, self.lib, self.n_out = ctx, lib, n_out
        self.fourier, self.split = fourier, split
        flags = (MLP_FOURIER if fourier is not None else 0) | (MLP_SPLIT if split else 0)
        tl, th = (float(fourier[0]), float(fourier[1])) if fourier is not None else (0.0, 0.0)
        h = c_void_p()
        st = lib.rb_mlp_create_ex(ctx._h, n_out, batch_cap, seed, flags, tl, th, ctypes.byref(h))
        if st != OK:
            raise RBError(st, "rb_mlp_create failed")
        self._h = h
        self.n_params = int(lib.rb_mlp_num_params(h))

    def close(self):
        if getattr(self, "_h", None):
            self.lib.rb_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st, what):
        if st < 0:
            raise RBError(st, what)
        return st

    def _dev(self):
        return f"cuda:{self.ctx.device}"

    def get_params(self):
        torch = _torch()
        with torch.cuda.stream(self.ctx.stream):
            p = torch.empty(self.n_params, dtype=torch.float32, device=self._dev())
        self._chk(self.lib.rb_mlp_get_params(self._h, p.data_ptr()), "rb_mlp_get_params")
        self.ctx.stream.synchronize()
        return p

    def set_params(self, p):
        torch = _torch()
        p = p.to(device=self._dev(), dtype=torch.float32).contiguous()
        self.ctx.stream.wait_stream(torch.cuda.current_stream())
        self._chk(self.lib.rb_mlp_set_params(self._h, p.data_ptr()), "rb_mlp_set_params")
        self.ctx.stream.synchronize()

    def _inputs(self, X, T=None):
        torch = _torch()
        X = X.to(device=self._dev(), dtype=torch.float32).contiguous()
        T = None if T is None else T.to(device=self._dev(), dtype=torch.float32).contiguous()
        self.ctx.stream.wait_stream(torch.cuda.current_stream())
        return X, T

    def infer(self, X):
        torch = _torch()
        X, _ = self._inputs(X)
        with torch.cuda.stream(self.ctx.stream):
            Y = torch.empty((X.shape[0], self.n_out), dtype=torch.float32, device=self._dev())
        self._chk(self.lib.rb_mlp_infer(self._h, X.data_ptr(), X.shape[0], Y.data_ptr()), "rb_mlp_infer")
        self.ctx.stream.synchronize()
        return Y

    def grad(self, X, T):
        torch = _torch()
        X, T = self._inputs(X, T)
        with torch.cuda.stream(self.ctx.stream):
            g = torch.empty(self.n_params, dtype=torch.float32, device=self._dev())
            loss = torch.empty(1, dtype=torch.float32, device=self._dev())
        self._chk(self.lib.rb_mlp_grad(self._h, X.data_ptr(), T.data_ptr(), X.shape[0], g.data_ptr(),
                                       loss.data_ptr()), "rb_mlp_grad")
        self.ctx.stream.synchronize()
        return g, float(loss.item())

    def train(self, X, T, epochs: int, batch: int = 1024, lr: float = 1e-3, seed: int = 0):
        torch = _torch()
        X, T = self._inputs(X, T)
        with torch.cuda.stream(self.ctx.stream):
            curve = torch.zeros(max(epochs, 1), dtype=torch.float32, device=self._dev())
        self._chk(self.lib.rb_mlp_train(self._h, X.data_ptr(), T.data_ptr(), X.shape[0], epochs, batch, float(lr),
                                        seed, curve.data_ptr()), "rb_mlp_train")
        return curve[:epochs]
