"""The MLP surrogate's CUDA kernels against the FP64 oracle network.

Gradients and outputs are compared on identical BF16-rounded weights; the GPU
also rounds its activations to BF16 for the tensor cores, hence the 2e-2
per-tensor relative L2 tolerance."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo
from paper_1805_06124_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbm():
    from paper_1805_06124_gb300 import rb
    return rb


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("n_out,rows", [(106, 512), (40, 200), (128, 1024)])
def test_grad_and_forward_parity(rbm, n_out, rows):
    ctx = rbm.RB(device=0)
    net = rbm.MLP(ctx, n_out, batch_cap=1024, seed=7)
    rng = np.random.default_rng(n_out)
    p = net.get_params().cpu().numpy().astype(np.float64)
    p += rng.standard_normal(p.size) * 0.01      # non-zero biases too
    net.set_params(torch.from_numpy(p))
    X = rng.uniform(-1, 1, (rows, 2))
    T = rng.standard_normal((rows, n_out)) * 0.5
    g, L = net.grad(torch.from_numpy(X), torch.from_numpy(T))
    pr = mo.round_weights(p.astype(np.float32).astype(np.float64), n_out)
    gr, Lr = mo.grad(pr, X, T, n_out)
    assert abs(L - Lr) <= 1e-2 * Lr, (L, Lr)
    gg = g.cpu().numpy().astype(np.float64)
    lay, _ = mo.layout(n_out)
    for name, (o, s) in lay.items():
        n = int(np.prod(s))
        r = rel(gg[o:o + n], gr[o:o + n])
        assert r <= 2e-2, (name, r)
    Y = net.infer(torch.from_numpy(X)).cpu().numpy()
    assert rel(Y, mo.forward(pr, X, n_out)) <= 2e-2
    net.close()
    ctx.close()


def test_training_reduces_loss(rbm):
    ctx = rbm.RB(device=0)
    rng = np.random.default_rng(0)
    X = rng.uniform(-1, 1, (8192, 2))
    T = np.stack([np.sin(3 * X[:, 0]) * np.cos(2 * X[:, 1]), X[:, 0] * X[:, 1], np.exp(X[:, 0]) / 3] * 8, 1)
    net = rbm.MLP(ctx, T.shape[1], batch_cap=1024, seed=1)
    curve = net.train(torch.from_numpy(X), torch.from_numpy(T), epochs=40, batch=512, lr=2e-3, seed=3).cpu().numpy()
    assert np.all(np.isfinite(curve))
    assert curve[-1] < curve[0] / 20, curve[[0, -1]]
    net.close()
    ctx.close()


def test_surrogate_small_end_to_end(rbm):
    """Greedy on 512 x 8192 chirps -> C -> MLP; held-out coefficients against
    exact projection Q^H s.  Without a surrogate the only prediction available
    without generating and projecting the snapshot is zero (relative error 1);
    the trained network must beat it clearly."""
    from paper_1805_06124_gb300 import surrogate
    ctx = rbm.RB(device=0)
    N, M = 512, 8192
    q, m = synth.chirp_params(M, seed=4)
    S = ctx.generate(q, m, N)
    g = ctx.greedy(S, 1e-8, 200)
    net, curve, _ = surrogate.train(ctx, q, m, g["C"], epochs=300, batch=512, lr=2e-3, seed=4)
    qt, mt = synth.chirp_params(1024, seed=5)
    St = ctx.generate(qt, mt, N)
    Ct = ctx.project(g["Q"], St)
    Tt = surrogate.targets_from_C(Ct)
    Y = net.infer(surrogate.scale_inputs(qt, mt))
    rel_e, _ = surrogate.relative_errors(Y, Tt)
    s = surrogate.summarize(rel_e)
    print("surrogate small", g["k"], s, float(curve[-1]))
    assert curve[-1] < 0.8 * curve[0]
    assert s["median"] < 0.9
    net.close()
    ctx.close()


@pytest.mark.parametrize("split", [False, True])
def test_fourier_input_grad_and_forward_parity(rbm, split):
    """Fourier input layer (RB_MLP_FOURIER) against the FP64 oracle: gradients
    within the BF16 backward's tolerance; the forward within 2e-2 on BF16
    weights, and within 1e-3 of the unrounded network with the split forward
    (RB_MLP_SPLIT: BF16 hi + lo pieces)."""
    from paper_1805_06124_gb300 import surrogate
    n_out, rows = 106, 512
    band = surrogate.chirp_tau_band(8192)
    ctx = rbm.RB(device=0)
    net = rbm.MLP(ctx, n_out, batch_cap=1024, seed=7, fourier=band, split=split)
    rng = np.random.default_rng(11)
    p = net.get_params().cpu().numpy().astype(np.float64)
    p += rng.standard_normal(p.size) * 0.01
    net.set_params(torch.from_numpy(p))
    q, m = synth.chirp_params(rows, seed=12)
    X = np.stack([q, m], 1)
    T = rng.standard_normal((rows, n_out)) * 0.5
    g, L = net.grad(torch.from_numpy(X), torch.from_numpy(T))
    p32 = p.astype(np.float32).astype(np.float64)
    pr = mo.round_weights(p32, n_out)
    gr, Lr = mo.grad(pr, X, T, n_out, fourier=band)
    assert abs(L - Lr) <= 1e-2 * Lr, (L, Lr)
    gg = g.cpu().numpy().astype(np.float64)
    lay, _ = mo.layout(n_out)
    for name, (o, s) in lay.items():
        n = int(np.prod(s))
        if name in ("W1", "b1"):
            assert not np.any(gg[o:o + n]), name
            continue
        r = rel(gg[o:o + n], gr[o:o + n])
        assert r <= 2e-2, (name, r)
    Y = net.infer(torch.from_numpy(X)).cpu().numpy()
    if split:
        r = rel(Y, mo.forward(p32, X, n_out, fourier=band))
        assert r <= 1e-3, r
    else:
        assert rel(Y, mo.forward(pr, X, n_out, fourier=band)) <= 2e-2
    net.close()
    ctx.close()


def test_surrogate_beats_nearest_training_snapshot(rbm):
    """What the trained network gains over the method without it: on held-out
    parameters, the network's coefficients against exact projection Q^H s are
    closer than those of the training snapshot nearest in omega (the
    non-learned baseline), at the median and the 95th percentile.  Greedy on
    2048 x 16384 chirps (seed 4, tol 1e-10), Fourier input layer, split
    forward, 400 epochs; 2048 held-out parameters (seed 5)."""
    from paper_1805_06124_gb300 import surrogate
    ctx = rbm.RB(device=0)
    N, M, Mt = 2048, 16384, 2048
    q, m = synth.chirp_params(M, seed=4)
    S = ctx.generate(q, m, N)
    g = ctx.greedy(S, 1e-10, 300)
    del S
    net, curve, _ = surrogate.train(ctx, q, m, g["C"], epochs=400, batch=1024, lr=3e-3, seed=4,
                                    fourier=surrogate.chirp_tau_band(N), split=True)
    qt, mt = synth.chirp_params(Mt, seed=5)
    Ct = ctx.project(g["Q"], ctx.generate(qt, mt, N))
    Tt = surrogate.targets_from_C(Ct)
    Y = net.infer(surrogate.inputs(net, qt, mt).cuda())
    e_mlp = surrogate.summarize(surrogate.relative_errors(Y, Tt)[0])
    nn = surrogate.nearest_in_omega(q, m, qt, mt)
    e_nn = surrogate.summarize(surrogate.relative_errors(surrogate.targets_from_C(g["C"])[nn], Tt)[0])
    print("surrogate vs nearest training snapshot", g["k"], e_mlp, e_nn)
    assert e_mlp["median"] < e_nn["median"], (e_mlp, e_nn)
    assert e_mlp["p95"] < e_nn["p95"], (e_mlp, e_nn)
    net.close()
    ctx.close()
