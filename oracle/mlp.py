"""FP64 oracle of the learned refinement-flag predictor -- test infrastructure.

The predictor maps per-block features to the three flags of the refinement
criterion of Sec. 3.3 (derefine / keep / refine):

  features  4^d average-pooled density, pressure and speed of each block,
            density and pressure divided by the block mean minus one, speed
            divided by the sound speed of the block-mean state, plus the
            block level over max_level (3 * 4^d + 1 values);
  network   x -> GELU(x W1 + b1) -> GELU(h1 W2 + b2) -> h2 W3 + b3 -> softmax,
            64 hidden units, GELU(z) = z (1 + erf(z / sqrt 2)) / 2;
  loss      mean cross-entropy against the criterion's flags.

The GPU passes use the weights rounded to BF16 (round to nearest even) and
accumulate in FP32; `forward`/`gradients` here take the weights as given
(round them with `to_bf16` to mirror the GPU), in FP64.  With bf16=True they
also round every other operand of a matrix product to BF16, as the GPU's
tensor-core path does: the features, the hidden activations h1 and h2, and in
back-propagation the deltas d1, d2, d3 entering the weight-gradient products
and d2 entering d1 = (d2 W2^T) GELU'(z1); biases, GELU, softmax, the output
delta and the bias gradients (sums of the unrounded deltas) are not rounded.
Parameters are packed as [W1 (F x H), b1, W2 (H x H), b2, W3 (H x 3), b3].
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

H, O = 64, 3


def n_params(F: int) -> int:
    return F * H + H + H * H + H + H * O + O


def unpack(p: np.ndarray, F: int):
    i = 0
    out = []
    for shape in ((F, H), (H,), (H, H), (H,), (H, O), (O,)):
        n = int(np.prod(shape))
        out.append(p[i:i + n].reshape(shape))
        i += n
    return out


def to_bf16(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to BF16 (nearest, ties to even), returned as FP32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_prime(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def _bf16_operand(a):
    """An FP64 operand rounded to BF16 the way the GPU rounds it: to FP32
    first (the GPU holds it in FP32), then to BF16."""
    return to_bf16(np.asarray(a, dtype=np.float32)).astype(np.float64)


def forward(p, X, bf16=False):
    """X [n, F] -> (probabilities [n, 3], cache)."""
    F = X.shape[1]
    W1, b1, W2, b2, W3, b3 = [a.astype(np.float64) for a in unpack(p, F)]
    r = _bf16_operand if bf16 else (lambda a: a)
    z1 = r(X) @ W1 + b1
    h1 = gelu(z1)
    z2 = r(h1) @ W2 + b2
    h2 = gelu(z2)
    z3 = r(h2) @ W3 + b3
    z3 = z3 - z3.max(axis=1, keepdims=True)
    e = np.exp(z3)
    prob = e / e.sum(axis=1, keepdims=True)
    return prob, (X, z1, h1, z2, h2, prob)


def loss(p, X, y):
    prob, _ = forward(p, X)
    return -np.mean(np.log(prob[np.arange(len(y)), y]))


def gradients(p, X, y, bf16=False):
    """Mean cross-entropy and its gradient w.r.t. the packed parameters
    (back-propagation written out layer by layer)."""
    F = X.shape[1]
    W1, b1, W2, b2, W3, b3 = [a.astype(np.float64) for a in unpack(p, F)]
    prob, (X, z1, h1, z2, h2, _) = forward(p, X, bf16=bf16)
    r = _bf16_operand if bf16 else (lambda a: a)
    n = len(y)
    d3 = prob.copy()
    d3[np.arange(n), y] -= 1.0
    d3 /= n
    gW3 = r(h2).T @ r(d3)
    gb3 = d3.sum(axis=0)
    d2 = (d3 @ W3.T) * gelu_prime(z2)
    gW2 = r(h1).T @ r(d2)
    gb2 = d2.sum(axis=0)
    d1 = (r(d2) @ W2.T) * gelu_prime(z1)
    gW1 = r(X).T @ r(d1)
    gb1 = d1.sum(axis=0)
    L = -np.mean(np.log(prob[np.arange(n), y]))
    return L, np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def block_features(spec, u, lev, max_level):
    """Features of every block from a state [nb, V, side^d] (interior cells)."""
    D, N, ng = spec.ndim, spec.N, spec.ng
    nb = u.shape[0]
    shape = (nb, spec.nvar) + (spec.side,) * D
    sl = tuple(slice(ng, ng + N) for _ in range(D))
    U = u.reshape(shape)[(slice(None), slice(None)) + sl].astype(np.float64)
    rho = U[:, 0]
    vel = [U[:, 1 + d] / rho for d in range(D)]
    ke = sum(v * v for v in vel)
    p = (spec.gamma - 1.0) * (U[:, D + 1] - 0.5 * rho * ke)
    speed = np.sqrt(ke)
    q = N // 4
    def pool(a):
        if D == 3:
            return a.reshape(nb, 4, q, 4, q, 4, q).mean(axis=(2, 4, 6)).reshape(nb, -1)
        return a.reshape(nb, 4, q, 4, q).mean(axis=(2, 4)).reshape(nb, -1)
    rm = rho.reshape(nb, -1).mean(axis=1)
    pm = p.reshape(nb, -1).mean(axis=1)
    cm = np.sqrt(spec.gamma * pm / rm)
    f = np.concatenate([pool(rho) / rm[:, None] - 1.0, pool(p) / pm[:, None] - 1.0, pool(speed) / cm[:, None],
                        (np.asarray(lev, dtype=np.float64) / max(1, max_level))[:, None]], axis=1)
    return f


def adamw_step(w, m, v, g, t, lr, weight_decay, beta1=0.9, beta2=0.999, eps=1e-8):
    """One AdamW update (Loshchilov & Hutter, "Decoupled weight decay
    regularization", ICLR 2019, Adam with decoupled weight decay; the
    learning rate scales both the Adam step and the decay) of parameters w
    with moments m, v at step t >= 1 (1-based) from gradient g.  Returns the
    new (w, m, v); FP64.

      m_t = beta1 m + (1 - beta1) g,       v_t = beta2 v + (1 - beta2) g^2
      mhat = m_t / (1 - beta1^t),          vhat = v_t / (1 - beta2^t)
      w_t = w - lr (mhat / (sqrt(vhat) + eps) + weight_decay w)
    """
    w = np.asarray(w, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    w_new = w - lr * (mhat / (np.sqrt(vhat) + eps) + weight_decay * w)
    return w_new, m, v
