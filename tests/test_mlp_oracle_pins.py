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


def test_fourier_gradient_matches_central_differences():
    """The Fourier-input network's backward against finite differences of its
    loss; W1 and b1 do not enter the loss (zero gradient)."""
    n_out = 6
    p, _, T = _problem(n_out)
    rng = np.random.default_rng(3)
    X = np.stack([rng.uniform(1.0, 10.0, 5), rng.uniform(0.8, 1.2, 5)], 1)
    four = (0.154, 1.031)
    g, L = mo.grad(p, X, T, n_out, fourier=four)
    assert np.isclose(L, mo.loss(p, X, T, n_out, fourier=four), rtol=1e-14)
    lay, n = mo.layout(n_out)
    o1, s1 = lay["W1"]
    ob, sb = lay["b1"]
    assert not np.any(g[o1:o1 + int(np.prod(s1))]) and not np.any(g[ob:ob + int(np.prod(sb))])
    idx = np.concatenate([rng.choice(np.arange(o, o + int(np.prod(s))), 4, replace=False)
                          for k, (o, s) in lay.items() if k not in ("W1", "b1")])
    h = 1e-6
    for i in idx:
        e = np.zeros(n)
        e[i] = h
        fd = (mo.loss(p + e, X, T, n_out, fourier=four) - mo.loss(p - e, X, T, n_out, fourier=four)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_fourier_features_use_the_generators_omega():
    """The encoding's omega is the snapshot generator's (synth.chirp_omega,
    an independent implementation of the family's definition): a chirp
    sample s(t_i) carries the phase omega tau_i, so at tau_f = tau_i the
    feature pair is the sample's normalised phasor (conjugated)."""
    from paper_1805_06124_gb300 import synth
    q, m = np.array([1.7, 6.2]), np.array([0.85, 1.13])
    N = 64
    S = synth.chirp_matrix(N, q, m, normalise=False)
    tau = (1.05 - np.arange(N) / N) ** 0.625
    i = 5
    F = mo.fourier_features(np.stack([q, m], 1), tau[i], tau[i] + 1.0)  # tau_0 = tau_i
    phasor = S[:, i] / np.abs(S[:, i])
    np.testing.assert_allclose(F[:, 0], phasor.real, rtol=0, atol=1e-12)
    np.testing.assert_allclose(F[:, 128], -phasor.imag, rtol=0, atol=1e-12)
