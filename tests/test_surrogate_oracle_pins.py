"""Pins of the surrogate oracle (oracle/surrogate.py) against what mathematics fixes: finite
differences, closed forms, a library bfloat16 cast and planted low-rank structure."""
import numpy as np
import pytest

from oracle import surrogate as SO


def _small_net(rng, shapes):
    return [(rng.normal(0, 1 / np.sqrt(i), (o, i)), rng.normal(0, 0.1, o)) for (o, i) in shapes]


def test_gelu_closed_forms():
    z = np.linspace(-6, 6, 241)
    assert SO.gelu(0.0) == 0.0 and SO.gelu_grad(0.0) == 0.5
    np.testing.assert_allclose(SO.gelu(z) - SO.gelu(-z), z, atol=1e-15)     # Phi(z) + Phi(-z) = 1
    np.testing.assert_allclose(SO.gelu(np.array([8.0, -8.0])), [8.0, 0.0], atol=1e-13)
    h = 1e-6
    fd = (SO.gelu(z + h) - SO.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(SO.gelu_grad(z), fd, atol=1e-9)


def test_bf16_rounding_matches_a_library_cast():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-3, 1000), [0.0, -0.0, 1.0, 3.0]])
    # exact ties: float32 values halfway between two bfloat16 numbers
    ties = (np.arange(1, 200, dtype=np.uint32) << 16 | 0x8000).view(np.float32).astype(np.float64)
    x = np.concatenate([x, ties, -ties])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(SO.bf16(x), ref)


@pytest.mark.parametrize("quantize", [False])
def test_gradients_match_central_differences(quantize):
    rng = np.random.default_rng(1)
    shapes = SO.layer_shapes(n_in=5, hidden=7, n_hidden=3, n_out=4)
    layers = _small_net(rng, shapes)
    X = rng.uniform(-1, 1, (6, 5))
    T = rng.normal(0, 1, (6, 4))
    w = np.array([0.25, 0.25, 0.25, 1.0])
    _, grads = SO.loss_and_grad(layers, X, T, w, quantize=quantize)
    flat = SO.flatten(layers)
    g_flat = SO.flatten(grads)
    h = 1e-6
    fd = np.empty_like(flat)
    for i in range(flat.size):
        e = np.zeros_like(flat); e[i] = h
        lp, _ = SO.loss_and_grad(SO.unflatten(flat + e, shapes), X, T, w, quantize=False)
        lm, _ = SO.loss_and_grad(SO.unflatten(flat - e, shapes), X, T, w, quantize=False)
        fd[i] = (lp - lm) / (2 * h)
    np.testing.assert_allclose(g_flat, fd, rtol=1e-6, atol=1e-9)


def test_quantized_forward_is_the_bf16_operand_product():
    rng = np.random.default_rng(2)
    shapes = SO.layer_shapes(n_in=3, hidden=5, n_hidden=1, n_out=2)
    layers = _small_net(rng, shapes)
    X = rng.uniform(-1, 1, (4, 3))
    y, _ = SO.forward(layers, X, quantize=True)
    (W1, b1), (W2, b2) = layers
    # written out element by element
    for n in range(4):
        h = [SO.gelu(sum(SO.bf16(X[n, i]) * SO.bf16(W1[j, i]) for i in range(3)) + b1[j]) for j in range(5)]
        for o in range(2):
            ref = sum(SO.bf16(h[j]) * SO.bf16(W2[o, j]) for j in range(5)) + b2[o]
            assert abs(y[n, o] - ref) <= 1e-14 * (1 + abs(ref))


def test_adam_first_step_closed_form_and_mask():
    rng = np.random.default_rng(3)
    w = rng.normal(0, 1, 50)
    g = rng.normal(0, 1, 50)
    new, m, v = SO.adam(w, g, np.zeros(50), np.zeros(50), t=1, lr=1e-2, eps=0.0)
    # m_hat = g and v_hat = g^2 at t = 1, so every weight moves by exactly lr against sign(g)
    np.testing.assert_allclose(new, w - 1e-2 * np.sign(g), rtol=0, atol=1e-15)
    mask = np.arange(50) % 2 == 0
    new2, m2, v2 = SO.adam(w, g, np.zeros(50), np.zeros(50), t=1, lr=1e-2, mask=mask)
    assert np.array_equal(new2[~mask], w[~mask]) and np.all(m2[~mask] == 0) and np.all(v2[~mask] == 0)


def test_pca_recovers_planted_structure():
    rng = np.random.default_rng(4)
    n, p, r = 400, 60, 5
    U, _ = np.linalg.qr(rng.normal(size=(n, r)))
    U -= U.mean(axis=0)                           # centred scores
    U, _ = np.linalg.qr(U)
    V, _ = np.linalg.qr(rng.normal(size=(p, r)))
    s = np.array([50.0, 20.0, 8.0, 3.0, 1.0])
    mu = rng.normal(size=p)
    X = mu + (U * s) @ V.T
    m, basis, sv = SO.pca(X, 5)
    np.testing.assert_allclose(m, mu + ((U * s) @ V.T).mean(axis=0), atol=1e-12)
    np.testing.assert_allclose(sv, s, rtol=1e-10)
    np.testing.assert_allclose(basis @ basis.T, np.eye(5), atol=1e-12)
    # same subspace: projecting V onto the basis loses nothing
    np.testing.assert_allclose(np.linalg.norm(basis @ V, axis=0), 1.0, atol=1e-10)
