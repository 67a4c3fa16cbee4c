"""Pins of the FP64 reference of the eps surrogate and of its training data."""
import math
import os

import numpy as np

import oracle
from oracle import mlp
from paper_2303_11811_gb300 import inputs


def test_splitmix64_published_vectors():
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.txt")
    want = [int(l, 16) for l in open(path) if l.strip() and not l.startswith("#")]
    # state 0 gives outputs number 0, 1, 2 of the stream seeded with 0
    got = [int(v) for v in mlp.splitmix64(0, np.arange(3))]
    assert got == want


def test_gradients_match_finite_differences():
    params = inputs.mlp_init(3)
    rng = np.random.default_rng(8)
    X = rng.normal(size=(48, 4))
    t = rng.random(48)
    loss, grads = mlp.loss_and_grads(params, X, t)
    h = 1e-6
    for p, g in zip(params, grads):
        flat = p.reshape(-1)
        gflat = g.reshape(-1)
        for k in rng.choice(flat.size, size=min(flat.size, 12), replace=False):
            old = flat[k]
            flat[k] = old + h
            lp, _ = mlp.loss_and_grads(params, X, t)
            flat[k] = old - h
            lm, _ = mlp.loss_and_grads(params, X, t)
            flat[k] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gflat[k]) <= 1e-7 * max(1e-3, abs(gflat[k])) + 1e-10


def test_adam_first_step_moves_each_weight_by_lr():
    """At step 1 the bias-corrected moments are g and g^2, so every parameter
    moves by lr * g / (|g| + eps) (Kingma and Ba, 2015)."""
    params = inputs.mlp_init(1)
    g = [np.full_like(p, 0.3) * np.sign(np.arange(p.size).reshape(p.shape) % 2 - 0.5)
         for p in params]
    z = [np.zeros_like(p) for p in params]
    new, m, v = mlp.adam_update(params, g, z, z, 1, 1e-3)
    for p0, p1, gg in zip(params, new, g):
        assert np.allclose(p1 - p0, -1e-3 * gg / (np.abs(gg) + 1e-8), rtol=1e-12, atol=0)


def test_training_samples_lie_in_the_partial_band():
    d, r = mlp.training_offsets(77, 0, 5000)
    dist = np.sqrt((d * d).sum(axis=1))
    h = math.sqrt(3) / 2
    assert np.all((r >= 2.0) & (r < 12.0))
    assert np.all(dist >= r - h - 1e-12) and np.all(dist <= r + h + 1e-12)
    X, eps, _, _ = mlp.training_samples(77, 0, 5000)
    assert np.all((eps >= 0) & (eps <= 1))
    assert np.all(eps * 512 == np.round(eps * 512))
    a = -np.sort(-np.abs(d / r[:, None]), axis=1)
    assert np.array_equal(X[:, :3], a) and np.all(X[:, 3] == r)
    assert np.all(X[:, 0] >= X[:, 1]) and np.all(X[:, 1] >= X[:, 2])


def test_labels_agree_with_the_linear_approximation():
    """Two independent estimates of the same overlap: 8^3 sampling and the
    closed form of Eqs. 25-27 agree on average to a few hundredths."""
    _, eps, d, r = mlp.training_samples(5, 100, 3000)
    dist = np.sqrt((d * d).sum(axis=1))
    lin = np.array([oracle.eps_linear(a, b) for a, b in zip(dist, r)])
    assert np.mean(np.abs(lin - eps)) < 0.03
    assert np.corrcoef(lin, eps)[0, 1] > 0.98


def test_surrogate_with_zero_network_is_the_linear_approximation():
    """With the network's output fixed at 0 the surrogate is Eqs. 25-27."""
    net = inputs.mlp_init(3)
    net[4] = np.zeros_like(net[4])
    net[5] = np.zeros(1)
    d, r = mlp.training_offsets(3, 0, 500)
    dist = np.sqrt((d * d).sum(axis=1))
    lin = np.array([oracle.eps_linear(a, b) for a, b in zip(dist, r)])
    assert np.array_equal(mlp.eps_from_net(net, d, r), lin)


def test_network_inputs_are_symmetry_invariant():
    """Sign flips and permutations of the offset give the same inputs."""
    d, r = mlp.training_offsets(8, 0, 200)
    X = mlp.network_inputs(d, r)
    Y = mlp.network_inputs(-d[:, [2, 0, 1]], r)
    assert np.array_equal(X, Y)


def test_counter_streams_are_reproducible_and_disjoint():
    a, ra = mlp.training_offsets(9, 0, 100)
    b, rb = mlp.training_offsets(9, 50, 50)
    assert np.array_equal(a[50:], b) and np.array_equal(ra[50:], rb)
    c, _ = mlp.training_offsets(10, 0, 100)
    assert not np.allclose(a, c)
