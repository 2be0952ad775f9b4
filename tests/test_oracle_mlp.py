"""Pins for the float64 MLP reference (no GPU): the analytic gradient agrees
with central finite differences, and a one-layer network is the affine map
computed by numpy's matmul."""
import numpy as np

from oracle import mlp_oracle as mo


def _rand(dims, seed):
    rng = np.random.default_rng(seed)
    n = sum(dims[i + 1] * (dims[i] + 1) for i in range(len(dims) - 1))
    return rng.normal(0, 0.5, size=n)


def test_gradient_matches_finite_differences():
    dims = [5, 7, 6, 3]
    rng = np.random.default_rng(0)
    X = rng.normal(size=(11, 5))
    T = rng.normal(size=(11, 3))
    mask = (rng.random((11, 3)) > 0.3).astype(float)
    p = _rand(dims, 1)
    for m in (None, mask):
        L, g = mo.gradients(p, dims, X, T, m)
        fd = mo.finite_difference(p, dims, X, T, m)
        assert abs(L - mo.loss(p, dims, X, T, m)) < 1e-12
        assert np.max(np.abs(g - fd)) <= 1e-6 * max(1.0, np.max(np.abs(fd)))


def test_single_layer_is_affine():
    dims = [4, 3]
    rng = np.random.default_rng(2)
    X = rng.normal(size=(6, 4))
    p = _rand(dims, 3)
    W = p[:12].reshape(3, 4)
    b = p[12:]
    assert np.allclose(mo.forward(p, dims, X)[-1], np.matmul(X, W.T) + b, rtol=0, atol=1e-12)


def test_relu_blocks_gradient():
    """A hidden unit that is off for every sample passes no gradient to the
    weights feeding it."""
    dims = [2, 2, 1]
    p = np.array([1.0, 0.0, 0.0, 1.0, -5.0, -5.0, 1.0, 1.0, 0.0])  # hidden biases -5: both units off
    X = np.array([[0.1, 0.2], [0.3, -0.1]])
    T = np.array([[1.0], [2.0]])
    _, g = mo.gradients(p, dims, X, T)
    assert np.all(g[:6] == 0.0)
