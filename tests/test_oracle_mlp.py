"""Pins of the learned-flag oracle: back-propagation against central finite
differences in FP64, BF16 rounding against the format's definition, and the
feature pooling against direct per-cell averages.  CPU only."""
import numpy as np

from oracle import mlp
import synth


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    F = 13
    p = rng.normal(0, 0.4, mlp.n_params(F))
    X = rng.normal(0, 1, (20, F))
    y = rng.integers(0, 3, 20)
    L, g = mlp.gradients(p, X, y)
    assert abs(L - mlp.loss(p, X, y)) < 1e-14
    idx = rng.choice(len(p), 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, X, y) - mlp.loss(p - e, X, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_bf16_rounding_definition():
    # BF16 keeps the top 16 bits of an FP32 value, rounding to nearest even
    vals = np.array([1.0, 1.0 + 2**-8, 1.0 + 2**-7 + 2**-9, 1.0 + 3 * 2**-8, -3.14159, 1e-3], dtype=np.float32)
    r = mlp.to_bf16(vals)
    assert np.all((r.view(np.uint32) & 0xFFFF) == 0)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # exactly half an ulp: ties to even (mantissa ...0)
    assert r[2] == np.float32(1.0 + 2**-7)  # above half: rounds up
    assert r[3] == np.float32(1.0 + 2**-6)  # half an ulp, odd mantissa: rounds up to even
    assert np.all(np.abs(r - vals) <= np.abs(vals) * 2**-8)


def test_gelu_closed_forms():
    z = np.array([0.0, 1.0, -1.0])
    g = mlp.gelu(z)
    assert g[0] == 0.0
    assert abs(g[1] - 0.8413447460685429) < 1e-15       # Phi(1)
    assert abs(g[1] - g[2] - 1.0) < 1e-15                 # gelu(z) - gelu(-z) = z
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(fd, mlp.gelu_prime(z), atol=1e-9)


def test_features_of_uniform_and_pooled_states():
    sp = synth.MeshSpec(ndim=3, N=16, ng=2, ntrees=(1, 1, 1))
    lev, g = np.zeros(1, dtype=np.int32), np.zeros((1, 3), dtype=np.int64)
    rho = np.full((1, 20, 20, 20), 2.0)
    u = synth.primitive_to_state(sp, rho, [0.3 * rho / rho, 0 * rho, 0 * rho], 5.0 * rho / rho)
    f = mlp.block_features(sp, u, lev, 3)
    assert f.shape == (1, 193)
    assert np.allclose(f[0, :128], 0.0, atol=1e-15)           # pooled / mean - 1
    c = np.sqrt(1.4 * 5.0 / 2.0)
    assert np.allclose(f[0, 128:192], 0.3 / c)
    # a density that varies only along x: pooled values are 4-cell averages
    X = synth.cell_centres(sp, lev, g)
    rho = 1.0 + 0.5 * X[0]
    u = synth.primitive_to_state(sp, rho, [0 * rho] * 3, np.ones_like(rho))
    f = mlp.block_features(sp, u, lev, 3)
    x = (np.arange(16) + 0.5) / 16
    r = 1.0 + 0.5 * x
    exp_pool = r.reshape(4, 4).mean(axis=1) / r.mean() - 1.0
    got = f[0, :64].reshape(4, 4, 4)        # (z, y, x) pools
    assert np.allclose(got, exp_pool[None, None, :], atol=1e-14)


def test_adamw_decay_alone_is_geometric():
    """With a zero gradient the moments stay zero and only the decoupled
    decay acts: w_t = w_0 (1 - lr wd)^t."""
    rng = np.random.default_rng(4)
    w0 = rng.normal(0, 1, 50)
    w, m, v = w0.copy(), np.zeros(50), np.zeros(50)
    lr, wd = 1e-2, 0.3
    for t in range(1, 8):
        w, m, v = mlp.adamw_step(w, m, v, np.zeros(50), t, lr, wd)
        np.testing.assert_allclose(w, w0 * (1 - lr * wd) ** t, rtol=1e-14, atol=0)
        assert not m.any() and not v.any()


def test_adamw_bias_correction_is_exact_for_a_constant_gradient():
    """For a constant gradient the bias-corrected moments equal g and g^2 at
    every step, so each step without decay moves w by lr g / (|g| + eps); at
    step 1 that is lr sign(g) up to eps."""
    rng = np.random.default_rng(5)
    g = rng.normal(0, 1e-2, 40)
    w0 = rng.normal(0, 1, 40)
    w, m, v = w0.copy(), np.zeros(40), np.zeros(40)
    lr, eps = 3e-3, 1e-8
    for t in range(1, 12):
        w, m, v = mlp.adamw_step(w, m, v, g, t, lr, 0.0, eps=eps)
        np.testing.assert_allclose(m / (1 - 0.9 ** t), g, rtol=1e-13)
        np.testing.assert_allclose(v / (1 - 0.999 ** t), g * g, rtol=1e-12)
        np.testing.assert_allclose(w, w0 - t * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)
    w1, _, _ = mlp.adamw_step(w0, np.zeros(40), np.zeros(40), g, 1, lr, 0.0, eps=eps)
    assert np.all(np.abs(w1 - (w0 - lr * np.sign(g))) <= 1.01 * lr * eps / np.abs(g))


def test_adamw_decay_uses_the_weights_before_the_step():
    """Decoupled decay: the decay term is lr wd w of the weights before the
    update, added to the Adam step (not folded into the gradient)."""
    w0, g = np.array([2.0, -1.0]), np.array([0.5, 0.5])
    lr, wd = 0.1, 0.2
    w1, _, _ = mlp.adamw_step(w0, np.zeros(2), np.zeros(2), g, 1, lr, wd)
    np.testing.assert_allclose(w1, w0 - lr * (g / (np.abs(g) + 1e-8) + wd * w0), rtol=1e-15)
    # an L2 penalty folded into the gradient would give the same sign step here
    # but a different size for the weight whose gradient it flips
    w0, g = np.array([2.0]), np.array([0.1])
    w1, _, _ = mlp.adamw_step(w0, np.zeros(1), np.zeros(1), g, 1, lr, 1.0)
    assert abs(w1[0] - (2.0 - 0.1 * (1.0 + 2.0))) < 1e-7


def test_bf16_operand_mode_is_within_the_bf16_bound():
    """The BF16-operand forward and gradient (the tensor-core arithmetic)
    differ from the exact FP64 ones by BF16 rounding of the operands only:
    a relative change of at most 2^-8 per operand, so probabilities move by
    far less than 1e-2 and gradients stay within a few per cent of their
    scale; with operands that are BF16-exact and activations forced through
    the same rounding on both sides the two modes agree to FP64 rounding."""
    rng = np.random.default_rng(8)
    F, n = 49, 64
    p = mlp.to_bf16(rng.normal(0, 0.3, mlp.n_params(F)).astype(np.float32)).astype(np.float64)
    X = rng.normal(0, 1, (n, F))
    y = rng.integers(0, 3, n)
    pe, _ = mlp.forward(p, X)
    pb, _ = mlp.forward(p, X, bf16=True)
    assert 0 < np.abs(pe - pb).max() < 1e-2
    _, ge = mlp.gradients(p, X, y)
    _, gb = mlp.gradients(p, X, y, bf16=True)
    for a, b in zip(mlp.unpack(ge, F), mlp.unpack(gb, F)):
        assert np.abs(a - b).max() <= 0.05 * np.abs(a).max()
    # the rounding is applied to the operands, nothing else: an input whose
    # features are BF16-exact and a network with no hidden nonlinearity to
    # round (zero hidden weights: h1 = GELU(b1) = 0, h2 = GELU(b2) = 0 with
    # zero biases) give identical results in both modes
    Xb = mlp.to_bf16(X.astype(np.float32)).astype(np.float64)
    q = p.copy()
    W1, b1, W2, b2, W3, b3 = mlp.unpack(q, F)
    W2[:] = 0.0
    b1[:] = 0.0
    b2[:] = 0.0
    np.testing.assert_array_equal(mlp.forward(q, Xb)[0], mlp.forward(q, Xb, bf16=True)[0])
