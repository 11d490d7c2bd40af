"""FP64 CPU oracle for the greedy reduced-basis method (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this module.  It
shares no code with the CUDA path (``paper_1805_06124_gb300``) and the CUDA
path never imports it.

The arithmetic lives in ``rb_oracle.c`` (plain sequential FP64 C, compiled
with ``-ffp-contract=off`` so that x86 and Arm hosts give identical bits).

Paper: Antil, Chen, Field, arXiv 1805.06124.
  * ``rb_greedy``  -- Alg. 3 (RB-greedy) with the Eq. (Residual) bookkeeping of
    Sec. 6.1.2 and Hoffmann's MGSCI re-orthogonalisation (Sec. 6.1.2, kappa=2).
  * ``mgs_pivot``  -- Alg. 2 (MGS with column pivoting), an independent second
    oracle used for the equivalence of Prop. 5.3.
  * ``project``    -- orthogonal projection coefficients q_l^H x_j (Sec. 2).
  * ``split``      -- the hi/lo complex64 storage of a complex128 matrix.

Layout used throughout the Python side: a snapshot matrix S (N x M in the
paper) is a C-contiguous complex128 array of shape (M, N): row j is the
snapshot s_j.  Q has shape (k, N) (row l = basis vector q_l), C has shape
(k, M) with C[l, j] = q_l^H s_j.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict[int, ctypes.CDLL] = {}

OK, KMAX_REACHED, EINVAL, ENOMEM, ENONFINITE, EORTHO = 0, 1, -1, -2, -4, -5

_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_i64_p = ctypes.POINTER(ctypes.c_longlong)
_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_float_p = ctypes.POINTER(ctypes.c_float)


def lib_path(plant: int = 0, omp: bool = False) -> str:
    name = "liborc.so" if plant == 0 else f"liborc_plant{plant}.so"
    if omp:
        name = "liborc_omp.so"
    return os.path.join(_BUILD, name)


def build(plant: int = 0, force: bool = False, omp: bool = False) -> str:
    """Compile the oracle (or a planted-mistake variant used by the oracle's
    own mutation tests) with gcc into ``oracle/_build``.  ``omp``: the same
    source with -fopenmp (column loops over all host cores; identical
    results), used only to time the paper's shared-memory scheme."""
    out = lib_path(plant, omp)
    with _LOCK:
        if (not force and os.path.exists(out)
                and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
            return out
        os.makedirs(_BUILD, exist_ok=True)
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               f"-DORC_PLANT={plant}"] + (["-fopenmp"] if omp else []) + [_SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def _lib(plant: int = 0, omp: bool = False) -> ctypes.CDLL:
    key = "omp" if omp else plant
    if key not in _LIBS:
        lib = ctypes.CDLL(build(plant, omp=omp))
        lib.orc_rb_greedy.restype = ctypes.c_int
        lib.orc_rb_greedy.argtypes = [
            _c_double_p, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong,
            ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int,
            _c_i64_p, ctypes.c_int,
            _c_double_p, _c_i64_p, _c_double_p, _c_double_p,
            _c_double_p, _c_double_p, _c_int_p,
            _c_i64_p, _c_double_p, _c_double_p, _c_double_p,
            _c_int_p]
        lib.orc_mgs_pivot.restype = ctypes.c_int
        lib.orc_mgs_pivot.argtypes = [
            _c_double_p, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong,
            ctypes.c_double, ctypes.c_int,
            _c_double_p, _c_i64_p, _c_double_p, _c_double_p, _c_double_p, _c_int_p]
        lib.orc_project.restype = ctypes.c_int
        lib.orc_project.argtypes = [
            _c_double_p, ctypes.c_longlong, ctypes.c_int, ctypes.c_longlong,
            _c_double_p, ctypes.c_longlong, ctypes.c_longlong,
            _c_double_p, ctypes.c_longlong]
        lib.orc_split.restype = ctypes.c_int
        lib.orc_split.argtypes = [
            _c_double_p, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong,
            _c_float_p, _c_float_p, ctypes.c_longlong]
        _LIBS[key] = lib
    return _LIBS[key]


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_c_double_p)


def _snapshots(S: np.ndarray) -> tuple[np.ndarray, int, int, int]:
    """Return (buffer, N, M, ld) for an (M, N) or (M, ld)[:, :N] complex128 view."""
    S = np.asarray(S)
    if S.dtype != np.complex128 or S.ndim != 2:
        raise TypeError("S must be a 2-D complex128 array of shape (M, N)")
    M, N = S.shape
    if S.strides[1] != 16:
        S = np.ascontiguousarray(S)
    ld = S.strides[0] // 16 if M > 1 else N
    if ld < N:
        S = np.ascontiguousarray(S)
        ld = N
    return S, N, M, ld


def rb_greedy(S, tol: float, kmax: int, kappa: float = 2.0, max_passes: int = 4,
              forced=None, plant: int = 0, omp: bool = False) -> dict:
    """RB-greedy (Alg. 3) in FP64.  See the module docstring for layouts.

    ``forced``: optional sequence of pivots to replay (forced-replay mode);
    the result then also carries, per replayed step, the oracle's own argmax,
    its max error, the forced column's error and the runner-up error.
    ``omp``: run the column loops on all host cores (identical results).
    """
    S, N, M, ld = _snapshots(S)
    kcap = max(int(kmax), 0)
    Q = np.zeros((max(kcap, 1), N), np.complex128)
    piv = np.full(max(kcap, 1), -1, np.int64)
    errc = np.zeros(kcap + 1, np.float64)
    C = np.zeros((max(kcap, 1), M), np.complex128)
    ferr = np.zeros(M, np.float64)
    rdiag = np.zeros(max(kcap, 1), np.float64)
    passes = np.zeros(max(kcap, 1), np.int32)
    nf = 0
    fptr = None
    if forced is not None:
        forced = np.ascontiguousarray(np.asarray(forced, np.int64))
        nf = int(forced.size)
        fptr = forced.ctypes.data_as(_c_i64_p)
    ndiag = max(nf, 1)
    own_arg = np.full(ndiag, -1, np.int64)
    own_max = np.zeros(ndiag)
    f_err = np.zeros(ndiag)
    second = np.zeros(ndiag)
    k = ctypes.c_int(0)
    st = _lib(plant, omp).orc_rb_greedy(
        _dp(S.view(np.float64)), N, M, ld, float(tol), kcap, float(kappa), int(max_passes),
        fptr, nf,
        _dp(Q.view(np.float64)), piv.ctypes.data_as(_c_i64_p), _dp(errc), _dp(C.view(np.float64)),
        _dp(ferr), _dp(rdiag), passes.ctypes.data_as(_c_int_p),
        own_arg.ctypes.data_as(_c_i64_p), _dp(own_max), _dp(f_err), _dp(second),
        ctypes.byref(k))
    k = k.value
    out = dict(status=st, k=k, Q=Q[:k].copy(), pivots=piv[:k].copy(), err_curve=errc[:k + 1].copy(),
               C=C[:k].copy(), final_err=ferr, rdiag=rdiag[:k].copy(), passes=passes[:k].copy())
    if forced is not None:
        n = min(nf, k + 1)
        out.update(own_argmax=own_arg[:n].copy(), own_max=own_max[:n].copy(),
                   forced_err=f_err[:n].copy(), second_max=second[:n].copy())
    return out


def mgs_pivot(S, tol: float, kmax: int, plant: int = 0) -> dict:
    """MGS with column pivoting (Alg. 2) on a private copy of S, FP64."""
    S, N, M, ld = _snapshots(S)
    kcap = max(int(kmax), 0)
    Q = np.zeros((max(kcap, 1), N), np.complex128)
    piv = np.full(max(kcap, 1), -1, np.int64)
    rdiag = np.zeros(max(kcap, 1))
    R = np.zeros((max(kcap, 1), M), np.complex128)
    errc = np.zeros(kcap + 1)
    k = ctypes.c_int(0)
    st = _lib(plant).orc_mgs_pivot(
        _dp(S.view(np.float64)), N, M, ld, float(tol), kcap,
        _dp(Q.view(np.float64)), piv.ctypes.data_as(_c_i64_p), _dp(rdiag), _dp(R.view(np.float64)),
        _dp(errc), ctypes.byref(k))
    k = k.value
    return dict(status=st, k=k, Q=Q[:k].copy(), pivots=piv[:k].copy(), rdiag=rdiag[:k].copy(),
                R=R[:k].copy(), err_curve=errc[:k + 1].copy())


def project(Q, X, plant: int = 0) -> np.ndarray:
    """C[l, j] = q_l^H x_j for Q of shape (k, N) and X of shape (Mx, N)."""
    Q = np.ascontiguousarray(np.asarray(Q, np.complex128))
    X, N, Mx, ldx = _snapshots(X)
    k = Q.shape[0]
    if Q.shape[1] != N:
        raise ValueError("Q and X disagree on N")
    C = np.zeros((k, Mx), np.complex128)
    st = _lib(plant).orc_project(_dp(Q.view(np.float64)), N, k, N, _dp(X.view(np.float64)), Mx, ldx,
                                 _dp(C.view(np.float64)), Mx)
    if st != OK:
        raise ValueError(f"orc_project failed: {st}")
    return C


def split(S, plant: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """hi = fl32(s), lo = fl32(s - hi), both round-to-nearest, per component."""
    S, N, M, ld = _snapshots(S)
    hi = np.zeros((M, N), np.complex64)
    lo = np.zeros((M, N), np.complex64)
    st = _lib(plant).orc_split(_dp(S.view(np.float64)), N, M, ld,
                               hi.view(np.float32).ctypes.data_as(_c_float_p),
                               lo.view(np.float32).ctypes.data_as(_c_float_p), N)
    if st != OK:
        raise ValueError(f"orc_split failed: {st}")
    return hi, lo
