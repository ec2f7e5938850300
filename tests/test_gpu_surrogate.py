"""GPU parity of the surrogate's building blocks through the C-ABI: network gradients and the
Adam step against the FP64 oracle (oracle/surrogate.py), PCA against an exact SVD, the
split-BF16 reconstruction against an FP64 product, and the query path."""
import numpy as np
import pytest

from oracle import surrogate as SO
from paper_2301_04259_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
LO, HI = synth.SURROGATE_LO, synth.SURROGATE_HI


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2301_04259_gb300 import soap
    return soap


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _scaled(x):
    return 2.0 * (np.asarray(x, np.float64) - LO) / (HI - LO) - 1.0


def _batch(seed, B):
    rng = np.random.default_rng(seed)
    x = synth.surrogate_params(seed, B)
    t = rng.normal(0, 1, (B, 129)).astype(np.float32)
    w = np.full(129, 1.0 / 128, np.float32)
    w[128] = 0.5
    return x, t, w


def test_gradients_match_oracle(S):
    B = 256
    s = S.soap_surrogate_create(LO, HI, B)
    try:
        flat = synth.surrogate_init(0)
        S.soap_surrogate_set_params(s, flat)
        x, t, w = _batch(1, B)
        loss_g, g_gpu = S.soap_surrogate_gradients(s, _t(x), _t(t), w)
    finally:
        S.soap_surrogate_free(s)
    layers = SO.unflatten(flat.astype(np.float64), SO.layer_shapes())
    loss_o, grads_o = SO.loss_and_grad(layers, _scaled(x), t.astype(np.float64), w.astype(np.float64))
    assert abs(loss_g - loss_o) <= 1e-4 * abs(loss_o)
    g_o = SO.flatten(grads_o)
    off = 0
    for (o, i), (gW, gb) in zip(SO.layer_shapes(), grads_o):
        for ref in (gW.ravel(), gb):
            got = g_gpu[off:off + ref.size]
            off += ref.size
            # FP32 accumulation and BF16 rounding-boundary flips of single operands
            assert np.abs(got - ref).max() <= 1e-2 * np.abs(ref).max() + 1e-7
            assert np.median(np.abs(got - ref)) <= 1e-3 * np.abs(ref).max() + 1e-8
    assert off == g_o.size


@pytest.mark.parametrize("stage", [0, 1])
def test_adam_step_matches_oracle(S, stage):
    B = 256
    s = S.soap_surrogate_create(LO, HI, B)
    try:
        flat = synth.surrogate_init(2)
        S.soap_surrogate_set_params(s, flat)
        x, t, w = _batch(3, B)
        _, g = S.soap_surrogate_gradients(s, _t(x), _t(t), w)
        S.soap_surrogate_set_params(s, flat)
        S.soap_surrogate_train(s, _t(x), _t(t), epochs=1, lr=1e-3, w_out=w, stage=stage)
        after = S.soap_surrogate_get_params(s)
    finally:
        S.soap_surrogate_free(s)
    n = flat.size
    head = np.zeros(n, bool)
    w5 = n - 129 * 256 - 129
    head[w5 + 128 * 256: w5 + 129 * 256] = True
    head[n - 1] = True
    mask = head if stage == 1 else ~head
    ref, _, _ = SO.adam(flat.astype(np.float64), g.astype(np.float64), np.zeros(n), np.zeros(n), t=1, lr=1e-3,
                        mask=mask)
    # The step sums the batch in shuffled order, so a gradient near zero differs from the one
    # computed above by FP32 rounding; the first Adam step -lr g / (|g| + eps) depends on such a
    # gradient's exact value only when |g| is not far above eps.  Where |g| >> eps the step is
    # exact; elsewhere it is bounded by lr.
    big = np.abs(g) > 1e-5
    np.testing.assert_allclose(after[big], ref[big], rtol=0, atol=2e-7 + 1e-6 * np.abs(ref).max())
    assert np.all(np.abs(after.astype(np.float64) - flat) <= 1e-3 * (1 + 1e-5) + 1e-7)
    assert np.array_equal(after[~mask], flat[~mask])
    assert big[mask].mean() > 0.9


def test_training_reduces_the_loss(S):
    B, n = 1024, 16384
    x = synth.surrogate_params(5, n)
    xs = _scaled(x)
    rng = np.random.default_rng(6)
    P = rng.normal(0, 1, (8, 129))
    t = np.sin(xs @ P).astype(np.float32)                 # a smooth target
    w = np.full(129, 1.0 / 129, np.float32)
    s = S.soap_surrogate_create(LO, HI, B)
    try:
        S.soap_surrogate_set_params(s, synth.surrogate_init(7))
        losses = S.soap_surrogate_train(s, _t(x), _t(t), epochs=20, lr=2e-3, w_out=w, stage=0)
    finally:
        S.soap_surrogate_free(s)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.15 * losses[0], losses


def test_pca_matches_exact_svd(S):
    rng = np.random.default_rng(8)
    n, p, k = 3000, 2000, 16
    s_true = np.concatenate([np.linspace(100, 20, 16), np.linspace(2, 1, 8)])
    U, _ = np.linalg.qr(rng.normal(size=(n, 24)))
    V, _ = np.linalg.qr(rng.normal(size=(p, 24)))
    X = (rng.normal(size=p) + (U * s_true) @ V.T + 0.01 * rng.normal(size=(n, p))).astype(np.float32)
    omega = synth.gaussian_test_matrix(9, p, 48)
    mean, basis, sv = S.soap_pca_fit(_t(X), _t(omega), k, n_power=2)
    mu_o, basis_o, sv_o = SO.pca(X.astype(np.float64), k)
    np.testing.assert_allclose(mean.cpu().numpy(), mu_o, atol=2e-5)
    np.testing.assert_allclose(sv, sv_o, rtol=2e-3)
    Bg = basis.double().cpu().numpy()
    np.testing.assert_allclose(Bg @ Bg.T, np.eye(k), atol=2e-4)
    # same subspace: the projectors agree
    assert np.abs(Bg.T @ Bg - basis_o.T @ basis_o).max() <= 2e-3
    coef = torch.empty((n, k), dtype=torch.float32, device=DEV)
    S.soap_pca_project(_t(X), mean, basis, coef)
    ref = (X.astype(np.float64) - mean.double().cpu().numpy()) @ Bg.T
    np.testing.assert_allclose(coef.double().cpu().numpy(), ref, atol=2e-3 * np.abs(ref).max())


def test_split_bf16_reconstruction_and_query(S):
    rng = np.random.default_rng(10)
    n, p = 1000, 3000
    basis = np.linalg.qr(rng.normal(size=(p, 128)))[0].T.astype(np.float32)
    mean = rng.normal(0, 1e-3, p).astype(np.float32)
    coef = rng.normal(0, 1e-2, (n, 128)).astype(np.float32)
    s = S.soap_surrogate_create(LO, HI, 128)
    try:
        S.soap_surrogate_set_basis(s, _t(mean), _t(basis))
        out = torch.empty((n, p), dtype=torch.float32, device=DEV)
        S.soap_surrogate_reconstruct(s, _t(coef), out)
        ref = mean + coef.astype(np.float64) @ basis.astype(np.float64)
        bound = np.abs(coef).astype(np.float64) @ np.abs(basis).astype(np.float64)
        assert np.all(np.abs(out.double().cpu().numpy() - ref) <= 3e-5 * bound + 1e-9)
        # query: rows with an input out of range are not accepted; accepted rows equal the
        # reconstruction of the predicted coefficients
        S.soap_surrogate_set_params(s, synth.surrogate_init(11))
        x = synth.surrogate_params(12, 300)
        x[5, 2] = 0.5            # radius above range
        x[7, 6] = 0.1            # vsini below range
        acc = torch.empty(300, dtype=torch.uint8, device=DEV)
        err = torch.empty(300, dtype=torch.float32, device=DEV)
        q = torch.empty((300, p), dtype=torch.float32, device=DEV)
        S.soap_surrogate_query(s, _t(x), 1e30, q, acc, err)
        c = torch.empty((300, 128), dtype=torch.float32, device=DEV)
        S.soap_surrogate_predict(s, _t(x), 1e30, coef=c)
        r = torch.empty_like(q)
        S.soap_surrogate_reconstruct(s, c, r)
        torch.cuda.synchronize()
        a = acc.cpu().numpy()
        assert a[5] == 0 and a[7] == 0 and a.sum() == 298
        assert torch.equal(q, r)
        assert bool(torch.isfinite(err).all())
        S.soap_surrogate_query(s, _t(x), 0.0, q, acc, err)      # nothing passes a zero threshold
        assert int(acc.sum().item()) == 0
    finally:
        S.soap_surrogate_free(s)


def test_surrogate_encode_matches_the_host_statement(S):
    """soap_surrogate_encode (FP32, sincosf) against the FP64 host statement of the network
    inputs (surrogate_pipeline.encode, pinned by test_host_logic): the region centre's y, x, z,
    vsini * x, and the parameters passed through unchanged."""
    from paper_2301_04259_gb300 import surrogate_pipeline as SP
    q = synth.surrogate_params(11, 4099)
    got = SP.encode_dev(q).cpu().numpy().astype(np.float64)
    ref = SP.encode(q.astype(np.float64)).astype(np.float64)
    for k in (2, 3, 6, 7):
        np.testing.assert_array_equal(got[:, k], q[:, k].astype(np.float64))
    np.testing.assert_allclose(got[:, [0, 1, 4]], ref[:, [0, 1, 4]], rtol=0, atol=5e-6)
    np.testing.assert_allclose(got[:, 5], ref[:, 5], rtol=0, atol=5e-5)
    empty = torch.empty((0, 8), dtype=torch.float32, device=DEV)
    S.soap_surrogate_encode(empty, empty)
