"""GPU checks of the learned refinement-flag predictor against its FP64
oracle (features, forward probabilities, gradients), training, the criterion
fallback, and what the trained network gains over evaluating the criterion
of Eq. 12 on every block."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
import synth

pytestmark = pytest.mark.gpu

amr = pytest.importorskip("paper_2605_07612_b300")
torch = pytest.importorskip("torch")

SPEC = dict(ndim=3, N=8, ng=2, ntrees=(4, 4, 4), max_level=2)


def sphere_forest(precision=32, steps=0):
    sp = synth.MeshSpec(**SPEC)
    f = amr.Forest(sp, 0, max_blocks=4096, precision=precision)
    for _ in range(2):
        lev, g = f.blocks()
        f.regrid(synth.ball_flags(sp, lev, g, (0.5, 0.5, 0.5), (0.3, 0.15)))
    lev, g = f.blocks()
    f.set_state(0, synth.over_pressure(sp, lev, g, (0.5, 0.5, 0.5), radius=0.2, p_in=10.0).astype(f.dtype))
    f.compute_dt(0)
    if steps:
        f.step(steps)
    return sp, f


def test_features_match_oracle():
    sp, f = sphere_forest(precision=64, steps=3)
    lev, _ = f.blocks()
    x = f.features(0).cpu().numpy()
    assert x.shape == (193, f.n)
    ref = omlp.block_features(sp, f.get_state(0), lev, sp.max_level).T
    np.testing.assert_allclose(x, ref, rtol=2e-6, atol=2e-6)


@pytest.mark.parametrize("N", [8, 32])
def test_features_match_oracle_fp32(N):
    """FP32 state: per-cell primitives in FP32, pool and block sums in FP64."""
    sp = synth.MeshSpec(ndim=3, N=N, ng=2, ntrees=(2, 2, 2), max_level=1)
    f = amr.Forest(sp, 0, max_blocks=64, precision=32)
    lev, g = f.blocks()
    f.regrid(synth.ball_flags(sp, lev, g, (0.5, 0.5, 0.5), (0.3,)))
    lev, g = f.blocks()
    u = synth.over_pressure(sp, lev, g, (0.5, 0.5, 0.5), radius=0.2, p_in=10.0)
    u[:, 1:4] += 0.3 * synth.fourier3d(sp, lev, g, seed=5)[:, 1:4]
    u = u.astype(np.float32)
    f.set_state(0, u)
    x = f.features(0).cpu().numpy()
    ref = omlp.block_features(sp, u, lev, sp.max_level).T
    np.testing.assert_allclose(x, ref, rtol=2e-5, atol=2e-5)


def test_features_2d_match_oracle():
    sp = synth.MeshSpec(ndim=2, N=16, ng=2, ntrees=(4, 4, 1), max_level=1)
    f = amr.Forest(sp, 0, max_blocks=256, precision=64)
    lev, g = f.blocks()
    u = synth.kelvin_helmholtz(sp, lev, g, seed=3)
    f.set_state(0, u)
    x = f.features(0).cpu().numpy()
    assert x.shape == (49, f.n)
    np.testing.assert_allclose(x, omlp.block_features(sp, u, lev, sp.max_level).T, rtol=2e-6, atol=2e-6)


@pytest.mark.parametrize("F", [193, 49])
@pytest.mark.parametrize("precision", [16, 32])
def test_forward_and_gradient_match_oracle(precision, F):
    """Forward probabilities and every gradient entry against the FP64
    oracle.  precision 32: FP32 activations on CUDA cores, against the exact
    oracle.  precision 16: the BF16 tensor-core passes, against the oracle
    with the same operands rounded to BF16; what remains is FP32
    accumulation order and the rare BF16 rounding of an activation that
    FP32 and FP64 put on opposite sides of a rounding boundary."""
    rng = np.random.default_rng(1)
    n = 300
    m = amr.Mlp(F, seed=7)
    m.set_precision(precision)
    p = m.get_params()
    X = rng.normal(0, 1, (n, F)).astype(np.float32)
    y = rng.integers(0, 3, n).astype(np.int8)
    xd = torch.tensor(X.T.copy(), device="cuda")
    yd = torch.tensor(y, device="cuda")
    prob = m.forward(xd).cpu().numpy()
    pb = omlp.to_bf16(p).astype(np.float64)
    bf16 = precision == 16
    ref, _ = omlp.forward(pb, X.astype(np.float64), bf16=bf16)
    np.testing.assert_allclose(prob, ref, atol=2e-4 if bf16 else 2e-5)
    L, g = m.gradient(xd, yd)
    Lr, gr = omlp.gradients(pb, X.astype(np.float64), y.astype(np.int64), bf16=bf16)
    assert abs(L - Lr) <= (1e-4 if bf16 else 1e-5) * abs(Lr)
    # element by element, per parameter tensor: FP32 accumulation of 300
    # samples against FP64, relative to each tensor's largest entry
    names = ("W1", "b1", "W2", "b2", "W3", "b3")
    for name, a, b in zip(names, omlp.unpack(g.astype(np.float64), F), omlp.unpack(gr, F)):
        scale = np.abs(b).max()
        assert scale > 0, name
        if bf16:
            np.testing.assert_allclose(a, b, rtol=2e-3, atol=2e-3 * scale, err_msg=name)
        else:
            np.testing.assert_allclose(a, b, rtol=1e-4, atol=2e-5 * scale, err_msg=name)


def test_tensor_core_forward_is_bf16_not_fp32():
    """The default passes round operands to BF16: against the exact FP64
    oracle they differ by more than FP32 rounding, against the BF16-operand
    oracle by much less."""
    rng = np.random.default_rng(3)
    F, n = 193, 256
    m = amr.Mlp(F, seed=9)
    pb = omlp.to_bf16(m.get_params()).astype(np.float64)
    X = rng.normal(0, 1, (n, F)).astype(np.float32)
    prob = m.forward(torch.tensor(X.T.copy(), device="cuda")).cpu().numpy()
    exact, _ = omlp.forward(pb, X.astype(np.float64))
    rounded, _ = omlp.forward(pb, X.astype(np.float64), bf16=True)
    assert np.abs(prob - rounded).max() < 0.1 * np.abs(prob - exact).max()


def test_adamw_steps_match_oracle():
    """Three AdamW steps with given gradients (the same FP32 values on both
    sides): FP32 master weights against the FP64 oracle step by step, with
    weight decay, so bias correction, moments and the decoupled decay are all
    checked element by element."""
    rng = np.random.default_rng(6)
    F = 49
    m = amr.Mlp(F, seed=2)
    w = m.get_params().astype(np.float64)
    mo = np.zeros_like(w)
    vo = np.zeros_like(w)
    lr, wd = 2e-3, 0.05
    for t in range(1, 4):
        g = (rng.normal(0, 1e-2, m.P) * rng.choice([1e-3, 1.0, 10.0], m.P)).astype(np.float32)
        m.adamw_step(torch.tensor(g, device="cuda"), lr, wd)
        torch.cuda.synchronize()
        w, mo, vo = omlp.adamw_step(w, mo, vo, g.astype(np.float64), t, lr, wd)
        got = m.get_params().astype(np.float64)
        np.testing.assert_allclose(got, w, rtol=2e-7, atol=1e-5 * lr, err_msg="step %d" % t)
        w = got                      # continue from the FP32 weights, as the GPU does


def test_training_learns_a_separable_rule():
    rng = np.random.default_rng(2)
    F, n = 49, 4000
    X = rng.normal(0, 1, (n, F)).astype(np.float32)
    score = X[:, 0] + 0.5 * X[:, 1]
    y = np.where(score > 0.7, 2, np.where(score < -0.7, 0, 1)).astype(np.int8)
    m = amr.Mlp(F, seed=3)
    xd = torch.tensor(X.T.copy(), device="cuda")
    yd = torch.tensor(y, device="cuda")
    L0, _ = m.gradient(xd, yd)
    L = m.train(xd, yd, epochs=30, batch=256, lr=3e-3)
    acc = (m.forward(xd).argmax(dim=1).cpu().numpy() == y).mean()
    assert L < 0.3 * L0 and acc > 0.95, (L0, L, acc)


def test_fallback_reproduces_the_criterion():
    sp, f = sphere_forest(steps=4)
    m = amr.Mlp(193, seed=0)
    f.fill_ghosts(0)
    plain = f.flag(0)
    flags, nfb = f.mlp_flags(m, 0, tau=1.5)     # nothing is that confident
    assert nfb == f.n
    np.testing.assert_array_equal(flags, plain)
    flags, nfb = f.mlp_flags(m, 0, tau=0.0)     # pure network
    assert nfb == 0 and set(np.unique(flags)) <= {-1, 0, 1}


def test_trained_network_replaces_most_criterion_evaluations():
    """Train on (features, criterion flags) gathered every 3 steps of an
    over-pressure run with regrids; on later, unseen states the network alone
    agrees with the criterion on most blocks, and with the fallback for
    unsure blocks it evaluates the criterion on a minority of them."""
    sp, f = sphere_forest()
    xs, ys, held = [], [], []
    for it in range(12):
        f.step(3)
        f.fill_ghosts(0)
        plain = f.flag(0, c_ref=5e-2, c_deref=6.25e-3)
        x = f.features(0)
        if it < 8:
            xs.append(x)
            ys.append(torch.tensor(plain + 1, dtype=torch.int8, device="cuda"))
        else:
            held.append((x, plain))
        f.regrid(plain)
    X = torch.cat(xs, dim=1).contiguous()
    Y = torch.cat(ys).contiguous()
    m = amr.Mlp(193, seed=4)
    m.train(X, Y, epochs=60, batch=128, lr=3e-3)
    mis = []
    for x, plain in held:
        pred = m.forward(x.contiguous()).argmax(dim=1).cpu().numpy() - 1
        mis.append((pred != plain).mean())
    majority = np.bincount(Y.cpu().numpy()).argmax() - 1
    base = np.mean([(plain != majority).mean() for _, plain in held])
    assert np.mean(mis) < 0.15 and np.mean(mis) < 0.5 * base, (np.mean(mis), base)
    f.fill_ghosts(0)
    plain = f.flag(0)
    flags, nfb = f.mlp_flags(m, 0, tau=0.9)
    assert nfb < 0.5 * f.n
    assert (flags != plain).mean() <= max(np.mean(mis), 0.05)
