"""FP64 reference of the eps-surrogate network and of its training samples.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The network takes the offset d of a cell centre from the sphere centre,
divided by the radius r, and r: 4 -> 32 (ReLU) -> 32 (ReLU) -> 1.  The offset
enters in the orientation fixed by the cube's symmetries (eps does not change
under sign flips and permutations of the components of d): x = (|d/r|
components in decreasing order, r).  The network predicts the correction to
the linear approximation of Sec. 2.3.2 (Eqs. 25-27):
    eps = clamp(eps_lin(|d|, r) + MLP(x), 0, 1).
Parameters are row-major ``W1`` (32x4), ``b1`` (32), ``W2`` (32x32), ``b2``
(32), ``W3`` (1x32), ``b3`` (1).  The loss is the mean squared error of the
correction against (8^3 sub-division sampling label - eps_lin); the optimiser
is Adam (Kingma and Ba, 2015).  ReLU'(0) is taken as 0.

Training samples are drawn from the counter-based generator SplitMix64
(Steele, Lea and Flood, 2014): value k of stream ``seed`` is the SplitMix64
output for state ``seed + (k+1) * 0x9E3779B97F4A7C15``, and a uniform double is
its top 53 bits times 2^-53.  Sample i uses values 5i .. 5i+4:
    r   = 2 + 10 u0
    v   = (2 u1 - 1, 2 u2 - 1, 2 u3 - 1),  nv = sqrt(v.v)   (v = (1,0,0) if nv = 0)
    rho = (r - sqrt(3)/2) + sqrt(3) u4      (a distance inside the partial band)
    t   = rho / nv,  d = (v0 t, v1 t, v2 t)
Every operation is a correctly rounded IEEE operation, so any implementation
of this recipe yields the same bits.
"""
from __future__ import annotations

import numpy as np

from . import eps_linear_batch, supersample_batch

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
HALF_SQRT3 = 0.86602540378443864676
SQRT3 = 1.7320508075688772935


def splitmix64(seed: int, k: np.ndarray) -> np.ndarray:
    """SplitMix64 output number k (0-based) of the stream started at ``seed``."""
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (k + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, k: np.ndarray) -> np.ndarray:
    return (splitmix64(seed, k) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def training_offsets(seed: int, first: int, count: int):
    """Offsets d (count x 3) and radii r of samples first .. first+count-1."""
    i = np.arange(first, first + count, dtype=np.uint64)
    u = [uniform(seed, np.uint64(5) * i + np.uint64(j)) for j in range(5)]
    r = 2.0 + 10.0 * u[0]
    v = np.stack([2.0 * u[1] - 1.0, 2.0 * u[2] - 1.0, 2.0 * u[3] - 1.0], axis=1)
    nv = np.sqrt(v[:, 0] * v[:, 0] + v[:, 1] * v[:, 1] + v[:, 2] * v[:, 2])
    zero = nv == 0.0
    v[zero] = (1.0, 0.0, 0.0)
    nv[zero] = 1.0
    rho = (r - HALF_SQRT3) + SQRT3 * u[4]
    t = rho / nv
    d = v * t[:, None]
    return d, r


def network_inputs(d, r):
    """(|d/r| components in decreasing order, r) for offsets d (m x 3)."""
    a = np.abs(d / r[:, None])
    a = -np.sort(-a, axis=1)
    return np.concatenate([a, r[:, None]], axis=1)


def training_samples(seed: int, first: int, count: int):
    """Network inputs, labels eps = count_8 / 512, offsets and radii."""
    d, r = training_offsets(seed, first, count)
    cnt = supersample_batch(d, r, 8)
    eps = cnt.astype(np.float64) / 512.0
    return network_inputs(d, r), eps, d, r


def linear_eps(d, r):
    """Eqs. 25-27 for offsets d (m x 3) and radii r."""
    dist = np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2])
    return eps_linear_batch(dist, r)


def forward(params, X):
    """Returns (y, cache) for inputs X (m x 4); y has shape (m,)."""
    W1, b1, W2, b2, W3, b3 = params
    a1 = X @ W1.T + b1
    h1 = np.where(a1 > 0.0, a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.where(a2 > 0.0, a2, 0.0)
    y = h2 @ W3.reshape(-1) + b3.reshape(())
    return y, (X, a1, h1, a2, h2)


def loss_and_grads(params, X, t):
    """Mean squared error and its exact gradient by backpropagation."""
    W1, b1, W2, b2, W3, b3 = params
    y, (X, a1, h1, a2, h2) = forward(params, X)
    m = X.shape[0]
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / m
    dW3 = (dy @ h2).reshape(1, -1)
    db3 = np.array([dy.sum()])
    dh2 = np.outer(dy, W3.reshape(-1)) * (a2 > 0.0)
    dW2 = dh2.T @ h1
    db2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (a1 > 0.0)
    dW1 = dh1.T @ X
    db1 = dh1.sum(axis=0)
    return loss, (dW1, db1, dW2, db2, dW3, db3)


def adam_update(params, grads, m_state, v_state, step, lr, beta1=0.9, beta2=0.999,
                eps=1e-8):
    """One Adam step (step counts from 1); returns new params, m, v."""
    out_p, out_m, out_v = [], [], []
    for p, g, m, v in zip(params, grads, m_state, v_state):
        m = beta1 * m + (1.0 - beta1) * g
        v = beta2 * v + (1.0 - beta2) * g * g
        mh = m / (1.0 - beta1 ** step)
        vh = v / (1.0 - beta2 ** step)
        out_p.append(p - lr * mh / (np.sqrt(vh) + eps))
        out_m.append(m)
        out_v.append(v)
    return out_p, out_m, out_v


def eps_from_net(params, d, r):
    """Surrogate eps for offsets d and radii r, clamped to [0, 1]."""
    y, _ = forward(params, network_inputs(d, r))
    return np.clip(linear_eps(d, r) + y, 0.0, 1.0)
