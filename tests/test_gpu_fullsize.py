"""Full-size parity: the benchmark workloads replayed through the FP64 oracle.

Every column of the GPU result is checked, not a sample:
  * 8192 x 262,144 chirps (seed 1), tol 1e-12, kmax 800 -- the FP64 form in
    the benchmark's launch configuration (double-float sweep);
  * 16384 x 196,608 chirps (seed 2), tol 1e-10 -- the FP64 form and the
    split-precision form on the same snapshots.
The GPU generates S; the oracle gets the identical bytes (downloaded).  The
GPU runs first, then the oracle (its OpenMP build: the same arithmetic, each
column summed sequentially, bit-identical to the single-threaded build)
replays the GPU's pivots (Alg. 3 with forced pivots) and the parity protocol
of Alg. 3 / Prop. 5.3 is applied to every step: the oracle's own argmax must
be the GPU pivot wherever the top-two gap is clear, otherwise the GPU pivot's
exact error lies within the FP64 bookkeeping margin of the max.  Error curve,
final errors (all M), basis and coefficients (all k x M) are then compared
with the tolerances of the other parity tests; the split form adds its
stated C bound (2^-48 sqrt(N) + 2^-42) ||s_j||.  The measured deviations are printed
(run pytest with -s to see them).

Host memory: S is held once on the host (34 GB and 51.5 GB).
"""
import json
import os

import numpy as np
import pytest

import parity
from paper_1805_06124_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbm():
    from paper_1805_06124_gb300 import rb
    return rb


def _free_gb():
    try:
        return torch.cuda.mem_get_info(0)[0] / 1e9
    except Exception:
        return 0.0


def _host_gb():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 1e6
    except Exception:
        pass
    return 0.0


def _download(t):
    """Device tensor -> host numpy array, in 1 GiB pieces (no second full copy)."""
    out = np.empty(tuple(t.shape), dtype=np.complex128 if t.dtype == torch.complex128 else np.float64)
    flat_out = out.reshape(out.shape[0], -1)
    rows = max(1, (1 << 30) // max(1, out[0:1].nbytes))
    for a in range(0, out.shape[0], rows):
        flat_out[a:a + rows] = t[a:a + rows].reshape(min(rows, out.shape[0] - a), -1).cpu().numpy()
    return out


def _npy(g):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in g.items()}


def _report(name, info):
    print(f"[full-size parity] {name}: " + json.dumps(info, sort_keys=True), flush=True)
    path = os.environ.get("RB_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"case": name, **info}, sort_keys=True) + "\n")


def _unforced_prefix_check(rep, own, gpu_piv, N):
    """Identical pivots up to the first step whose top-two gap is not clear."""
    d = parity.first_divergence(list(own["pivots"]), list(gpu_piv))
    if d < min(own["k"], len(gpu_piv)):
        e = rep["own_max"][d]
        assert e - rep["second_max"][d] <= max(1e-12 * e, parity.delta(d, N, rep["err_curve"][0])), d
    return d


def test_config2_full_size_oracle_replay(orc, rbm):
    N, M, tol, kmax = 8192, 262144, 1e-12, 800
    if _free_gb() < 80 or _host_gb() < 60:
        pytest.skip("needs about 70 GB of device and 40 GB of host memory")
    c = rbm.RB(device=0)
    q, m = synth.chirp_params(M, seed=1)
    S = c.generate(q, m, N)
    g = _npy(c.greedy(S, tol, kmax))
    c.close()
    Sh = _download(S)
    del S
    torch.cuda.empty_cache()
    assert g["status"] == 0 and 40 <= g["k"] <= 90
    rep = parity.replay_and_check(orc, Sh, g, tol, kmax, omp=True)
    info = parity.compare(g, rep, Sh)
    own = orc.rb_greedy(Sh, tol, kmax, omp=True)
    info["unforced_common_prefix"] = _unforced_prefix_check(rep, own, g["pivots"], N)
    info["unforced_k"] = int(own["k"])
    _report("fp64 form 8192x262144 tol 1e-12", info)


@pytest.fixture(scope="module")
def cfg3(rbm):
    """16384 x 196,608 chirps, seed 2, generated on the GPU, one host copy."""
    N, M = 16384, 196608
    if _free_gb() < 120 or _host_gb() < 80:
        pytest.skip("needs about 110 GB of device and 60 GB of host memory")
    q, m = synth.chirp_params(M, seed=2)
    c = rbm.RB(device=0)
    S = c.generate(q, m, N)
    Sh = _download(S)
    c.close()
    del S
    torch.cuda.empty_cache()
    d = dict(N=N, M=M, q=q, m=m, S=Sh, norms=parity.column_norms(Sh))
    yield d
    d.clear()


def _regen(c, cfg):
    """The generator is deterministic: the device copy equals the host copy."""
    S = c.generate(cfg["q"], cfg["m"], cfg["N"])
    for j in (0, cfg["M"] // 2, cfg["M"] - 1):
        assert np.array_equal(S[j].cpu().numpy(), cfg["S"][j])
    return S


def _cfg3_unforced(orc, cfg):
    if "own" not in cfg:
        cfg["own"] = orc.rb_greedy(cfg["S"], 1e-10, 800, omp=True)
    return cfg["own"]


def test_config3_fp64_form_full_size_oracle_replay(orc, rbm, cfg3):
    tol, kmax = 1e-10, 800
    c = rbm.RB(device=0)
    S = _regen(c, cfg3)
    g = _npy(c.greedy(S, tol, kmax))
    c.close()
    del S
    torch.cuda.empty_cache()
    assert g["status"] == 0
    rep = parity.replay_and_check(orc, cfg3["S"], g, tol, kmax, omp=True)
    info = parity.compare(g, rep, cfg3["S"], norms=cfg3["norms"])
    own = _cfg3_unforced(orc, cfg3)
    info["unforced_common_prefix"] = _unforced_prefix_check(rep, own, g["pivots"], cfg3["N"])
    info["unforced_k"] = int(own["k"])
    _report("fp64 form 16384x196608 tol 1e-10", info)


def test_config3_split_form_full_size_oracle_replay(orc, rbm, cfg3):
    """The split form (hi/lo made by rb_split on the GPU, bit-exact with the
    oracle's split) against the oracle on complex128 S: its error against
    the FP64 oracle for the error curve, the basis, C and the final errors."""
    tol, kmax = 1e-10, 800
    N = cfg3["N"]
    c = rbm.RB(device=0)
    S = _regen(c, cfg3)
    hi, lo = c.split(S)
    del S
    torch.cuda.empty_cache()
    g = _npy(c.greedy_split(hi, lo, tol, kmax))
    c.close()
    del hi, lo
    torch.cuda.empty_cache()
    assert g["status"] == 0 and g["switch_iter"] == -1  # few candidates: no switch
    rep = parity.replay_and_check(orc, cfg3["S"], g, tol, kmax, omp=True)
    info = parity.compare(g, rep, cfg3["S"], c_rel=2.0 ** -48 * np.sqrt(N) + 2.0 ** -42, norms=cfg3["norms"])
    k = rep["k"]
    info["max_dC_over_norm"] = float(np.max(np.abs(g["C"][:k] - rep["C"]) / cfg3["norms"][None, :]))
    own = _cfg3_unforced(orc, cfg3)
    info["unforced_common_prefix"] = _unforced_prefix_check(rep, own, g["pivots"], N)
    info["unforced_k"] = int(own["k"])
    assert np.max(g["final_err"]) < tol + 1e-12
    _report("split form 16384x196608 tol 1e-10", info)
