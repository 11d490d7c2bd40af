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
