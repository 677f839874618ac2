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


def _event(rng):
    rec = np.zeros(32, dtype=np.float32)
    for o in range(5):
        rec[4 * o:4 * o + 4] = (rng.uniform(30, 200), rng.uniform(-2.5, 2.5),
                                rng.uniform(-np.pi, np.pi), 4.0 if o == 0 else 5.0)
    rec[24:26] = rng.normal(0, 40, 2)
    return rec


def test_features_closed_form():
    """Lepton along phi = pi/2 and a jet along phi = pi: after the rotation the
    lepton is along +x (py = 0) and the jet along +y."""
    rec = np.zeros(32, dtype=np.float32)
    rec[0:4] = (50.0, 0.0, np.pi / 2, 4.0)
    rec[4:8] = (80.0, np.arcsinh(0.75), np.pi, 5.0)      # pT = 64, pz = 48
    for o in range(2, 5):
        rec[4 * o:4 * o + 4] = (40.0, 0.0, 0.0, 5.0)
    rec[24:26] = (0.0, -30.0)
    f = F.features(rec, 0)
    assert f[0] == pytest.approx(0.5, rel=1e-12, abs=0) and abs(f[1]) < 1e-12
    assert f[2:5] == pytest.approx([0.0, 0.64, 0.48], abs=1e-6)
    assert f[5:8] == pytest.approx([0.0, -0.4, 0.0], abs=1e-6)   # phi = 0 jet -> -y
    assert f[14:16] == pytest.approx([-0.3, 0.0], abs=1e-6)


def test_features_invariances():
    """Rotating the whole event about the beam leaves the features unchanged;
    a permutation only reorders the jet triplets; |p| and pT are preserved."""
    rng = np.random.default_rng(5)
    rec = _event(rng)
    base = F.features(rec, 0)
    rot = rec.copy()
    a = 0.7
    for o in range(5):
        rot[4 * o + 2] = rec[4 * o + 2] + a
    c, s = np.cos(a), np.sin(a)
    rot[24:26] = (c * rec[24] - s * rec[25], s * rec[24] + c * rec[25])
    assert np.allclose(F.features(rot, 0), base, atol=1e-5)
    import itertools
    perms = list(itertools.permutations(range(4)))
    for p in (5, 17, 23):
        f = F.features(rec, p)
        for k in range(4):
            j = perms[p][k]
            assert np.allclose(f[2 + 3 * k:5 + 3 * k], base[2 + 3 * j:5 + 3 * j])
    for k in range(4):
        E, eta = rec[4 * (k + 1)], rec[4 * (k + 1) + 1]
        assert np.linalg.norm(base[2 + 3 * k:5 + 3 * k]) == pytest.approx(E / 100, rel=1e-6, abs=0)
        assert np.hypot(*base[2 + 3 * k:4 + 3 * k]) == pytest.approx(E / np.cosh(eta) / 100, rel=1e-6, abs=0)
    assert np.hypot(base[14], base[15]) == pytest.approx(np.hypot(rec[24], rec[25]) / 100, rel=1e-6, abs=0)
