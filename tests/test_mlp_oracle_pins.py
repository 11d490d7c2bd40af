"""Pins of the MLP oracle: central finite differences of its loss, GELU closed
forms, and BF16 rounding against PyTorch's conversion (a library routine)."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo


def _problem(n_out=6, rows=5, seed=0):
    rng = np.random.default_rng(seed)
    _, n = mo.layout(n_out)
    p = rng.standard_normal(n) * 0.2
    X = rng.uniform(-1, 1, (rows, 2))
    T = rng.standard_normal((rows, n_out))
    return p, X, T


def test_gradient_matches_central_differences():
    n_out = 6
    p, X, T = _problem(n_out)
    g, L = mo.grad(p, X, T, n_out)
    assert np.isclose(L, mo.loss(p, X, T, n_out), rtol=1e-14)
    rng = np.random.default_rng(1)
    lay, n = mo.layout(n_out)
    idx = np.concatenate([rng.choice(np.arange(o, o + int(np.prod(s))), 4, replace=False) for o, s in lay.values()])
    h = 1e-6
    for i in idx:
        e = np.zeros(n)
        e[i] = h
        fd = (mo.loss(p + e, X, T, n_out) - mo.loss(p - e, X, T, n_out)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_gelu_closed_forms():
    assert mo.gelu(0.0) == 0.0 and mo.gelu_grad(0.0) == 0.5
    assert np.isclose(mo.gelu(10.0), 10.0, rtol=1e-15) and abs(mo.gelu(-10.0)) < 1e-20
    # GELU(1) = Phi(1) = 0.8413447460685429...
    assert np.isclose(mo.gelu(1.0), 0.8413447460685429, rtol=1e-15)
    z = np.linspace(-4, 4, 17)
    fd = (mo.gelu(z + 1e-6) - mo.gelu(z - 1e-6)) / 2e-6
    np.testing.assert_allclose(mo.gelu_grad(z), fd, rtol=1e-8, atol=1e-9)


def test_bf16_rounding_matches_library():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(3).standard_normal(10000).astype(np.float32) * 10
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mo.to_bf16(x), ref)


def test_pack_unpack_roundtrip():
    p, _, _ = _problem(9)
    np.testing.assert_array_equal(mo.pack(mo.unpack(p, 9), 9), p)
