"""Pins of the FP64 reference of the learned importance sampler (oracle/flow_ref.py):
the map is a bijection of the unit cube, its log-Jacobian equals the log of the
numerical determinant, the sampling density integrates to one (E_u[1] under
y-space reweighting), and the hand-written gradient of the training loss equals
finite differences."""
import numpy as np
import pytest

from oracle import flow_ref as F


@pytest.fixture(scope="module")
def setup():
    d, C = 7, 16
    layers = F.init_params(d, 6, 32, C, seed=3, zero_last=False)
    rng = np.random.default_rng(4)
    return d, C, layers, rng


def test_inverse_and_logdet(setup):
    d, C, layers, rng = setup
    u = rng.uniform(0.02, 0.98, (20, d))
    c = rng.normal(size=(20, C))
    y, lj = F.forward(layers, u, c)
    u2, lj2 = F.inverse(layers, y, c)
    assert np.allclose(u2, u, atol=1e-10)
    assert np.allclose(lj, lj2, atol=1e-9)
    h = 1e-6
    for i in range(5):
        J = np.zeros((d, d))
        for j in range(d):
            up, um = u[i:i + 1].copy(), u[i:i + 1].copy()
            up[0, j] += h
            um[0, j] -= h
            J[:, j] = (F.forward(layers, up, c[i:i + 1])[0] - F.forward(layers, um, c[i:i + 1])[0])[0] / (2 * h)
        assert np.log(abs(np.linalg.det(J))) == pytest.approx(lj[i], abs=1e-6)


def test_density_normalised(setup):
    """int q(y) dy = 1  <=>  E_{y ~ U}[ 1 / |dy/du|(y) ] = 1 (uniform y, inverse map)."""
    d, C, layers, rng = setup
    n = 200000
    y = rng.uniform(size=(n, d))
    c = np.tile(rng.normal(size=(1, C)), (n, 1))
    _, lj = F.inverse(layers, y, c)
    q = np.exp(-lj)
    assert abs(q.mean() - 1.0) < 5 * q.std() / np.sqrt(n)


def test_gradient_matches_finite_differences(setup):
    d, C, layers, rng = setup
    n = 16
    y = rng.uniform(0.05, 0.95, (n, d))
    c = rng.normal(size=(n, C))
    w = rng.uniform(0.1, 1.0, n)
    G = F.grad(layers, y, w, c)
    h = 1e-6
    for k in (0, 3, 5):
        for name in ("W1a", "W1c", "b1", "W2", "b2", "W3", "b3"):
            P = layers[k][name]
            idx = tuple(rng.integers(0, s) for s in P.shape)
            old = P[idx]
            P[idx] = old + h
            lp = F.loss(layers, y, w, c)
            P[idx] = old - h
            lm = F.loss(layers, y, w, c)
            P[idx] = old
            fd = (lp - lm) / (2 * h)
            assert G[k][name][idx] == pytest.approx(fd, rel=1e-5, abs=1e-8), (k, name)
