"""Checkpoints of a greedy run on disk (host I/O only).

A checkpoint is what rb_greedy_resume needs to continue a run: the basis Q
(k, N), pivots (k,), coefficients C (k, M), err_curve (k + 1,) and rdiag
(k,), plus the run's N, M and tol.  The file is a NumPy ``.npz`` archive
(the software of the paper exports the basis and pivots in text, GSL-binary
and NumPy formats, Sec. 6.1).
"""
from __future__ import annotations

import numpy as np

KEYS = ("Q", "pivots", "C", "err_curve", "rdiag")


def _host(x):
    return x.detach().cpu().numpy() if hasattr(x, "detach") else np.asarray(x)


def save(path: str, result: dict, tol: float) -> None:
    """Write the first k entries of a greedy result dict."""
    k = int(result["k"])
    arrs = {key: _host(result[key]) for key in KEYS}
    arrs["Q"], arrs["pivots"], arrs["C"], arrs["rdiag"] = (arrs["Q"][:k], arrs["pivots"][:k], arrs["C"][:k],
                                                           arrs["rdiag"][:k])
    arrs["err_curve"] = arrs["err_curve"][:k + 1]
    N, M = arrs["Q"].shape[1], arrs["C"].shape[1]
    np.savez(path, k=k, N=N, M=M, tol=tol, **arrs)


def load(path: str) -> dict:
    """Read a checkpoint: a dict with k, N, M, tol and the arrays of KEYS."""
    with np.load(path) as z:
        out = {key: z[key] for key in KEYS}
        out.update(k=int(z["k"]), N=int(z["N"]), M=int(z["M"]), tol=float(z["tol"]))
    if out["Q"].shape != (out["k"], out["N"]) or out["C"].shape != (out["k"], out["M"]):
        raise ValueError(f"inconsistent checkpoint {path}")
    return out
